// Steady heat solve (Eq. 7 discretised as Eq. 16) and the self-consistent
// loop of Fig. 2.  Two methods: the direct separable solve of heat_direct.cu
// (default; any mix of oven-held (Eq. 9) and convective (Eq. 10) faces) and
// red-black successive over-relaxation (below; every face held at T_oven).
//
// The iteration runs in double precision: in FP32 the Jacobi correction of a
// solution of a few kelvin bottoms out near 1e-6 K (rounding of the stencil
// sums), which would make a 1e-6 K stopping test unreachable.
//
// Unknown: dT = T - T_oven on the node grid [hz][hy][hx] spanning the crystal
// [-wx/2, wx/2] x [-wy/2, wy/2] x [0, L], zero on oven-held faces.  Source: the
// heat deposited by the last THERMAL propagation, q_dot = Q / V at each node
// (Q = sum of q_dot dV of the field samples binned to the node, V = dx dy dz,
// halved for each face the node lies on; for the SOR, whose faces are all
// oven-held, only interior nodes matter).
// SOR factor omega = 2 / (1 + sqrt(1 - rho_J^2)) with rho_J the Jacobi
// spectral radius of the anisotropic stencil.  Convergence: the largest Jacobi
// correction over the interior, checked after every kCheckEvery full (red +
// black) sweeps (each check is a reduction and a host synchronisation; the
// sweeps past the first converged one only reduce the error further).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan.h"

namespace shg {

constexpr int kCheckEvery = 8;

struct HeatGeom {
    int hx, hy, hz;
    double ax, ay, az;  // 1/dx^2, 1/dy^2, 1/dz^2
    double invD;        // 1 / (2 (ax + ay + az))
    double qs;          // 1 / (kappa dx dy dz): Q -> q_dot / kappa
    double omega;
};

static HeatGeom heat_geom(const shg_plan* p) {
    HeatGeom g;
    g.hx = p->g.hx;
    g.hy = p->g.hy;
    g.hz = p->g.hz;
    const double dx = p->c.wx / (g.hx - 1), dy = p->c.wy / (g.hy - 1), dz = p->c.L / (g.hz - 1);
    const double ax = 1 / (dx * dx), ay = 1 / (dy * dy), az = 1 / (dz * dz);
    g.ax = ax;
    g.ay = ay;
    g.az = az;
    g.invD = 1.0 / (2.0 * (ax + ay + az));
    g.qs = 1.0 / (p->c.kappa_th * dx * dy * dz);
    const double rho = (ax * std::cos(kPi / (g.hx - 1)) + ay * std::cos(kPi / (g.hy - 1)) +
                        az * std::cos(kPi / (g.hz - 1))) / (ax + ay + az);
    g.omega = 2.0 / (1.0 + std::sqrt(1.0 - rho * rho));
    return g;
}

__device__ __forceinline__ double jacobi_target(const double* T, const double* Q,
                                                const HeatGeom& g, size_t c) {
    const size_t plane = size_t(g.hx) * g.hy;
    const double s = g.ax * (T[c - 1] + T[c + 1]) + g.ay * (T[c - g.hx] + T[c + g.hx]) +
                     g.az * (T[c - plane] + T[c + plane]) + Q[c] * g.qs;
    return s * g.invD;
}

// One colour of a red-black sweep: nodes with (i + j + l) % 2 == colour.
// grid = (ceil((hx - 2 + 1) / 2 / 128), hy - 2, hz - 2), block = 128.
__global__ void k_sor_colour(double* __restrict__ T, const double* __restrict__ Q, HeatGeom g,
                             int colour) {
    const int j = blockIdx.y + 1, l = blockIdx.z + 1;
    const int i0 = 1 + ((colour + 1 + j + l) & 1);  // first interior i of this colour
    const int i = i0 + 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i > g.hx - 2) return;
    const size_t c = (size_t(l) * g.hy + j) * g.hx + i;
    const double t = T[c];
    T[c] = t + g.omega * (jacobi_target(T, Q, g, c) - t);
}

// Largest |Jacobi correction| over the interior (non-negative doubles compare
// as their bit patterns).  grid = (ceil((hx-2)/128), hy - 2, hz - 2).
__global__ void k_max_correction(const double* __restrict__ T, const double* __restrict__ Q,
                                 HeatGeom g, unsigned long long* __restrict__ out) {
    const int j = blockIdx.y + 1, l = blockIdx.z + 1;
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i <= g.hx - 2) {
        const size_t c = (size_t(l) * g.hy + j) * g.hx + i;
        v = fabs(jacobi_target(T, Q, g, c) - T[c]);
    }
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(v)));
}

__global__ void k_max_abs_diff(const double* __restrict__ a, const double* __restrict__ b,
                               size_t n, unsigned long long* __restrict__ out) {
    double v = 0.0;
    for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n;
         k += size_t(gridDim.x) * blockDim.x)
        v = fmax(v, fabs(a[k] - b[k]));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(v)));
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n) {
    for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n;
         k += size_t(gridDim.x) * blockDim.x)
        b[k] = float(a[k]);
}

static shg_status_t max_correction(shg_plan* p, const HeatGeom& g, cudaStream_t st, double* out) {
    auto* d = reinterpret_cast<unsigned long long*>(p->hred);
    SHG_CK(cudaMemsetAsync(d, 0, sizeof(*d), st));
    dim3 grid((g.hx - 2 + 127) / 128, g.hy - 2, g.hz - 2);
    k_max_correction<<<grid, 128, 0, st>>>(p->theat, p->Q, g, d);
    SHG_CK(cudaGetLastError());
    unsigned long long h = 0;
    SHG_CK(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SHG_CK(cudaStreamSynchronize(st));
    memcpy(out, &h, sizeof(double));
    return SHG_OK;
}

static shg_status_t sor(shg_plan* p, int max_sweeps, double tol, double* resid, int* sweeps,
                        cudaStream_t st) {
    const HeatGeom g = heat_geom(p);
    double corr = 0;
    shg_status_t r = max_correction(p, g, st, &corr);
    if (r != SHG_OK) return r;
    int n = 0;
    const int half = (g.hx - 2 + 1) / 2;
    dim3 grid((half + 127) / 128, g.hy - 2, g.hz - 2);
    while (corr >= tol && n < max_sweeps) {
        const int k = std::min(kCheckEvery, max_sweeps - n);
        for (int i = 0; i < k; ++i) {
            k_sor_colour<<<grid, 128, 0, st>>>(p->theat, p->Q, g, 0);
            k_sor_colour<<<grid, 128, 0, st>>>(p->theat, p->Q, g, 1);
        }
        SHG_CK(cudaGetLastError());
        n += k;
        if ((r = max_correction(p, g, st, &corr)) != SHG_OK) return r;
        if (!std::isfinite(corr)) return SHG_ERR_NONFINITE;
    }
    if (resid) *resid = corr;
    if (sweeps) *sweeps = n;
    return SHG_OK;
}

static shg_status_t install_map(shg_plan* p, cudaStream_t st) {
    const size_t nh = size_t(p->g.hx) * p->g.hy * p->g.hz;
    k_to_float<<<256, 256, 0, st>>>(p->theat, p->theat_f, nh);
    SHG_CK(cudaGetLastError());
    return shg_set_temperature(p, p->theat_f, p->g.hx, p->g.hy, p->g.hz, p->c.wx, p->c.wy,
                               reinterpret_cast<shg_stream_t>(st));
}

// The plan's heat solve with its method; max_sweeps bounds the SOR sweeps or
// the refinement passes of the direct solve (at most 50 of those).
static shg_status_t solve(shg_plan* p, int max_sweeps, double tol, double* resid, int* sweeps,
                          cudaStream_t st) {
    if (p->heat_method == SHG_HEAT_SOR)
        return sor(p, max_sweeps, tol, resid, sweeps, st);
    return heat_direct_solve(p, std::min(max_sweeps, 50), tol, resid, sweeps, st);
}

static bool all_oven(const shg_plan* p) {
    for (int k = 0; k < 6; ++k)
        if (p->heat_face[k]) return false;
    return true;
}

}  // namespace shg

using namespace shg;

extern "C" shg_status_t shg_set_heat_boundary(shg_plan_t* p, const int* kinds, const double* h,
                                              double t_inf) {
    if (!p || !kinds || !std::isfinite(t_inf)) return SHG_ERR_INVALID_ARG;
    if (!(p->flags & SHG_FLAG_THERMAL) || !p->Q) return SHG_ERR_STATE;
    bool any_sink = false;
    for (int k = 0; k < 6; ++k) {
        if (kinds[k] != SHG_FACE_OVEN && kinds[k] != SHG_FACE_CONVECTIVE) return SHG_ERR_INVALID_ARG;
        const double hk = (kinds[k] == SHG_FACE_CONVECTIVE) ? (h ? h[k] : 0.0) : 0.0;
        if (!std::isfinite(hk) || hk < 0) return SHG_ERR_INVALID_ARG;
        any_sink |= kinds[k] == SHG_FACE_OVEN || hk > 0;
    }
    // every face insulated: no steady state exists
    if (!any_sink) return SHG_ERR_INVALID_ARG;
    if (p->heat_method == SHG_HEAT_SOR) {
        for (int k = 0; k < 6; ++k)
            if (kinds[k] != SHG_FACE_OVEN) return SHG_ERR_INVALID_ARG;
    }
    if (p->has_result) SHG_CK(cudaStreamSynchronize(p->last_stream));
    for (int k = 0; k < 6; ++k) {
        p->heat_face[k] = kinds[k];
        p->heat_h[k] = kinds[k] == SHG_FACE_CONVECTIVE ? (h ? h[k] : 0.0) : 0.0;
    }
    p->heat_tinf = t_inf;
    // eigenbases of the direct solve for the new boundary (host Jacobi
    // rotations: tens of milliseconds at 128 nodes per axis)
    shg_status_t r = heat_direct_setup(p);
    if (r != SHG_OK) return r;
    // the previous solution belongs to the old boundary (nodes now held at the
    // oven may be non-zero): the next solve starts from dT = 0
    const size_t nh = size_t(p->g.hx) * p->g.hy * p->g.hz;
    SHG_CK(cudaMemset(p->theat, 0, nh * sizeof(double)));
    SHG_CK(cudaMemset(p->theat_prev, 0, nh * sizeof(double)));
    return SHG_OK;
}

extern "C" shg_status_t shg_set_heat_method(shg_plan_t* p, int method) {
    if (!p || (method != SHG_HEAT_DIRECT && method != SHG_HEAT_SOR)) return SHG_ERR_INVALID_ARG;
    if (!(p->flags & SHG_FLAG_THERMAL) || !p->Q) return SHG_ERR_STATE;
    if (method == SHG_HEAT_SOR && !all_oven(p)) return SHG_ERR_INVALID_ARG;
    p->heat_method = method;
    return SHG_OK;
}

extern "C" shg_status_t shg_heat_solve(shg_plan_t* p, int max_sweeps, double tol, double* resid,
                                       int* sweeps, shg_stream_t stream) {
    if (!p || max_sweeps < 0 || !(tol > 0)) return SHG_ERR_INVALID_ARG;
    if (!(p->flags & SHG_FLAG_THERMAL) || !p->Q) return SHG_ERR_STATE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->has_result) SHG_CK(cudaStreamSynchronize(p->last_stream));
    shg_status_t r = solve(p, max_sweeps, tol, resid, sweeps, st);
    if (r != SHG_OK) return r;
    return install_map(p, st);
}

extern "C" shg_status_t shg_get_heat(shg_plan_t* p, double* q_dev, float* dT_dev,
                                     shg_stream_t stream) {
    if (!p) return SHG_ERR_INVALID_ARG;
    if (!(p->flags & SHG_FLAG_THERMAL) || !p->Q) return SHG_ERR_STATE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->has_result && p->last_stream != st) SHG_CK(cudaStreamSynchronize(p->last_stream));
    const size_t nh = size_t(p->g.hx) * p->g.hy * p->g.hz;
    if (q_dev) SHG_CK(cudaMemcpyAsync(q_dev, p->Q, nh * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (dT_dev) {
        k_to_float<<<256, 256, 0, st>>>(p->theat, dT_dev, nh);
        SHG_CK(cudaGetLastError());
    }
    return SHG_OK;
}

extern "C" shg_status_t shg_thermal_loop(shg_plan_t* p, int n_outer, int max_sweeps, double tol,
                                         double* eta_out, double* change_out,
                                         shg_stream_t stream) {
    if (!p || n_outer < 1 || max_sweeps < 0 || !(tol > 0)) return SHG_ERR_INVALID_ARG;
    if (!(p->flags & SHG_FLAG_THERMAL) || !p->Q) return SHG_ERR_STATE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->has_result) SHG_CK(cudaStreamSynchronize(p->last_stream));
    const size_t nh = size_t(p->g.hx) * p->g.hy * p->g.hz;
    // q_dot = 0 before the first pass: dT = 0
    SHG_CK(cudaMemsetAsync(p->theat, 0, nh * sizeof(double), st));
    SHG_CK(cudaMemsetAsync(p->Q, 0, nh * sizeof(double), st));
    for (int it = 0; it < n_outer; ++it) {
        SHG_CK(cudaMemcpyAsync(p->theat_prev, p->theat, nh * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
        shg_status_t r = solve(p, max_sweeps, tol, nullptr, nullptr, st);
        if (r != SHG_OK) return r;
        auto* d = reinterpret_cast<unsigned long long*>(p->hred);
        SHG_CK(cudaMemsetAsync(d, 0, sizeof(*d), st));
        k_max_abs_diff<<<256, 256, 0, st>>>(p->theat, p->theat_prev, nh, d);
        SHG_CK(cudaGetLastError());
        unsigned long long h = 0;
        // into pageable host memory: returns once the value has arrived
        SHG_CK(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
        // stream-ordered on st (same-shape maps after the first iteration)
        if ((r = install_map(p, st)) != SHG_OK) return r;
        double change;
        memcpy(&change, &h, sizeof(double));
        if ((r = shg_propagate(p, stream)) != SHG_OK) return r;
        double eta = 0;
        if ((r = shg_efficiency(p, &eta, nullptr, nullptr)) != SHG_OK) return r;
        if (eta_out) eta_out[it] = eta;
        if (change_out) change_out[it] = change;
    }
    return SHG_OK;
}
