// Three-wave mixing plans (sum/difference-frequency generation): creation,
// tables, initial fields, the propagation of threewave.cuh and the powers.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "launch_passes.cuh"
#include "plan.h"
#include "threewave.cuh"

namespace shg {

// Host-side state of a three-wave plan (shg_plan::w3).
struct ThreeWave {
    shg_crystal3_t c;
    shg_beams3_t b;
    void* q = nullptr;       // device Inst3<R>[1]
    double* red = nullptr;   // device [kRedBlocks][3] partial sums
    double* pw = nullptr;    // device [3] powers
    double pw_host[3] = {0, 0, 0};
};

constexpr int kRed3Threads = 256;

// ------------------------------------------------------------- kernels ----

struct Init3 {
    double x0, dx, y0, dy;
    double w0[3], zf[3], k[3], p[3];
    double cdxdy[3];  // (1/2) eps0 c n_j dx dy
    double* red;
    double* pw;
};

// Eq. (5) at z = 0 for wave j (unnormalised), double precision.
__device__ double2 gauss3(const Init3& d, int j, int m, int n) {
    const double x = d.x0 + d.dx * m, y = d.y0 + d.dy * n;
    const double zr = d.w0[j] * d.w0[j] * d.k[j] * 0.5;
    const double tau = -d.zf[j] / zr;
    const double den = 1.0 + tau * tau;
    const double qr = 1.0 / den, qi = -tau / den;
    const double a = -(x * x + y * y) / (d.w0[j] * d.w0[j]);
    const double mag = exp(a * qr);
    double s, c;
    sincos(a * qi, &s, &c);
    const double er = mag * c, ei = mag * s;
    return make_double2(er * qr - ei * qi, er * qi + ei * qr);
}

__device__ void block_sum3(double (&v)[3]) {
    __shared__ double sh[3][kRed3Threads];
    for (int j = 0; j < 3; ++j) sh[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int w = kRed3Threads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 3; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
        __syncthreads();
    }
    for (int j = 0; j < 3; ++j) v[j] = sh[j][0];
    __syncthreads();
}

// Pass 1: partial sums of |g_j|^2 (fixed order).  grid = kRedBlocks.
__global__ void k_init3_partial(Init3 d, int nx, int ny) {
    double acc[3] = {0, 0, 0};
    const int npts = nx * ny;
    for (int i = blockIdx.x * kRed3Threads + threadIdx.x; i < npts; i += gridDim.x * kRed3Threads)
        for (int j = 0; j < 3; ++j) {
            if (d.p[j] <= 0) continue;
            const double2 g = gauss3(d, j, i % nx, i / nx);
            acc[j] += g.x * g.x + g.y * g.y;
        }
    block_sum3(acc);
    if (threadIdx.x == 0)
        for (int j = 0; j < 3; ++j) d.red[blockIdx.x * 3 + j] = acc[j];
}

// Pass 2: every block sums the partials in the same order, scales and writes.
template <class R>
__global__ void k_init3_write(Init3 d, cx<R>* __restrict__ f, int nx, int ny) {
    using C = cx<R>;
    __shared__ double a0[3];
    if (threadIdx.x < 3) {
        const int j = threadIdx.x;
        double s = 0;
        for (int b = 0; b < kRedBlocks; ++b) s += d.red[b * 3 + j];
        a0[j] = (d.p[j] > 0 && s > 0) ? sqrt(d.p[j] / (d.cdxdy[j] * s)) : 0.0;
    }
    __syncthreads();
    const int npts = nx * ny;
    for (int i = blockIdx.x * kRed3Threads + threadIdx.x; i < npts; i += gridDim.x * kRed3Threads)
        for (int j = 0; j < 3; ++j) {
            if (a0[j] == 0.0) {
                f[size_t(j) * npts + i] = mk<C>(R(0), R(0));
            } else {
                const double2 g = gauss3(d, j, i % nx, i / nx);
                f[size_t(j) * npts + i] = mk<C>(R(a0[j] * g.x), R(a0[j] * g.y));
            }
        }
}

template <class R>
__global__ void k_power3_partial(Init3 d, const cx<R>* __restrict__ f, int nx, int ny) {
    const int npts = nx * ny;
    double acc[3] = {0, 0, 0};
    for (int i = blockIdx.x * kRed3Threads + threadIdx.x; i < npts; i += gridDim.x * kRed3Threads)
        for (int j = 0; j < 3; ++j) {
            const cx<R> u = f[size_t(j) * npts + i];
            acc[j] += double(u.x) * u.x + double(u.y) * u.y;
        }
    block_sum3(acc);
    if (threadIdx.x == 0)
        for (int j = 0; j < 3; ++j) d.red[blockIdx.x * 3 + j] = acc[j];
}

__global__ void k_power3_final(Init3 d) {
    if (threadIdx.x >= 3) return;
    const int j = threadIdx.x;
    double s = 0;
    for (int b = 0; b < kRedBlocks; ++b) s += d.red[b * 3 + j];
    d.pw[j] = d.cdxdy[j] * s;
}

// ------------------------------------------------------------ launchers ----

#define SHG_3W_F32(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)
#define SHG_3W_F64(X) X(8) X(16) X(32) X(64) X(128) X(256)

template <class R, int N> static cudaError_t attr3() {
    cudaError_t e = cudaFuncSetAttribute(k_row3<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(Row3Geom<R, N>::smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_col3<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Col3Geom<R, N>::smem));
    return e;
}

static cudaError_t attrs3() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
#define X(n) if (err == cudaSuccess) err = attr3<float, n>();
        SHG_3W_F32(X)
#undef X
#define X(n) if (err == cudaSuccess) err = attr3<double, n>();
        SHG_3W_F64(X)
#undef X
    });
    return err;
}

template <class R, int N>
static cudaError_t row3(const void* q, int ninst, int ny, int nz, int s, const void* tw,
                        cudaStream_t st) {
    using G = Row3Geom<R, N>;
    dim3 grid((ny + G::ROWS - 1) / G::ROWS, ninst);
    return launch_pdl(k_row3<R, N>, grid, dim3(nth3<R, N>()), G::smem, st,
                      static_cast<const Inst3<R>*>(q), ny, nz, s, static_cast<const pt<R>*>(tw));
}

template <class R, int N>
static cudaError_t col3(const void* q, int ninst, int nx, const void* tw, cudaStream_t st) {
    using G = Col3Geom<R, N>;
    dim3 grid((nx + G::TILE - 1) / G::TILE, ninst);
    return launch_pdl(k_col3<R, N>, grid, dim3(nth3<R, N>()), G::smem, st,
                      static_cast<const Inst3<R>*>(q), nx, static_cast<const pt<R>*>(tw));
}

static cudaError_t launch_row3(bool fp64, int nx, const void* q, int ny, int nz, int s,
                               const void* tw, cudaStream_t st) {
    if (fp64) {
        switch (nx) {
#define X(n) case n: return row3<double, n>(q, 1, ny, nz, s, tw, st);
            SHG_3W_F64(X)
#undef X
        }
    } else {
        switch (nx) {
#define X(n) case n: return row3<float, n>(q, 1, ny, nz, s, tw, st);
            SHG_3W_F32(X)
#undef X
        }
    }
    return cudaErrorInvalidValue;
}

static cudaError_t launch_col3(bool fp64, int ny, const void* q, int nx, const void* tw,
                               cudaStream_t st) {
    if (fp64) {
        switch (ny) {
#define X(n) case n: return col3<double, n>(q, 1, nx, tw, st);
            SHG_3W_F64(X)
#undef X
        }
    } else {
        switch (ny) {
#define X(n) case n: return col3<float, n>(q, 1, nx, tw, st);
            SHG_3W_F32(X)
#undef X
        }
    }
    return cudaErrorInvalidValue;
}

// ----------------------------------------------------------------- host ----

static double lambda3_of(const shg_crystal3_t& c) { return 1.0 / (1.0 / c.lambda1 + 1.0 / c.lambda2); }

static void wave_params(const shg_crystal3_t& c, double lam[3], double n[3]) {
    lam[0] = c.lambda1;
    lam[1] = c.lambda2;
    lam[2] = lambda3_of(c);
    n[0] = c.n1;
    n[1] = c.n2;
    n[2] = c.n3;
}

static Init3 make_init3(const shg_plan* p) {
    const ThreeWave* w = p->w3;
    Init3 d;
    memset(&d, 0, sizeof(d));
    d.dx = p->g.lx / p->g.nx;
    d.dy = p->g.ly / p->g.ny;
    d.x0 = -(p->g.nx / 2) * d.dx;
    d.y0 = -(p->g.ny / 2) * d.dy;
    double lam[3], n[3];
    wave_params(w->c, lam, n);
    for (int j = 0; j < 3; ++j) {
        d.w0[j] = w->b.w0[j];
        d.zf[j] = w->b.z_focus[j];
        d.k[j] = 2 * kPi * n[j] / lam[j];
        d.p[j] = w->b.p[j];
        d.cdxdy[j] = 0.5 * kEps0 * kCLight * n[j] * d.dx * d.dy;
    }
    d.red = w->red;
    d.pw = w->pw;
    return d;
}

// The descriptor of the three-wave passes from the plan's SHG descriptor
// (map, phase table, grid) with the coupling, TPA and lens of the three waves.
template <class R> static void fill_inst3(const shg_plan* p, Inst3<R>* q) {
    memset(q, 0, sizeof(*q));
    if constexpr (sizeof(R) == 8)
        fill_desc_f64(p, &q->d);
    else
        fill_desc_f32(p, &q->d);
    const ThreeWave* w = p->w3;
    double lam[3], n[3];
    wave_params(w->c, lam, n);
    double kap[3], b[3], l[3], psi0[3];
    for (int j = 0; j < 3; ++j) {
        const double cj = 0.5 * kEps0 * kCLight * n[j];
        kap[j] = 2 * kPi * w->c.d_eff / (n[j] * lam[j]);
        b[j] = 0.5 * w->c.beta[j] * cj;
        l[j] = 2 * kPi / lam[j] * w->c.dn_dT;
        psi0[j] = l[j] * w->b.t_oven_offset;
    }
    q->d.kF = R(kap[0]);
    q->d.kS = R(kap[2]);
    q->d.bF = R(b[0]);
    q->d.bS = R(b[2]);
    q->d.lF = R(l[0]);
    q->d.lS = R(l[2]);
    q->d.psi0F = R(psi0[0]);
    q->d.psi0S = R(psi0[2]);
    q->d.undepleted = w->b.undepleted ? 1 : 0;
    q->d.Q = nullptr;
    q->d.mon = nullptr;
    q->k2 = R(kap[1]);
    q->b2 = R(b[1]);
    q->l2 = R(l[1]);
    q->psi02 = R(psi0[1]);
}

shg_status_t upload_desc3(shg_plan* p) {
    std::vector<unsigned char> h(p->fp64 ? sizeof(Inst3<double>) : sizeof(Inst3<float>));
    if (p->fp64)
        fill_inst3<double>(p, reinterpret_cast<Inst3<double>*>(h.data()));
    else
        fill_inst3<float>(p, reinterpret_cast<Inst3<float>*>(h.data()));
    SHG_CK(cudaMemcpy(p->w3->q, h.data(), h.size(), cudaMemcpyHostToDevice));
    return SHG_OK;
}

void free_three_wave(shg_plan* p) {
    ThreeWave* w = p->w3;
    if (!w) return;
    if (w->q) cudaFree(w->q);
    if (w->red) cudaFree(w->red);
    if (w->pw) cudaFree(w->pw);
    delete w;
    p->w3 = nullptr;
}

// K-space factors of the three waves: [3][nx] row factors (diffraction,
// absorption, walk-off, 1/nx) and [3][ny] column factors (diffraction, 1/ny).
shg_status_t build_prop_tables3(shg_plan* p, void* px, void* py) {
    const int nx = p->g.nx, ny = p->g.ny;
    const ThreeWave* w = p->w3;
    double lam[3], n[3];
    wave_params(w->c, lam, n);
    const double dz = w->c.L / p->g.nz;
    std::vector<unsigned char> hx(size_t(3) * nx * 16), hy(size_t(3) * ny * 16);
    auto put = [&](std::vector<unsigned char>& buf, size_t i, double re, double im) {
        if (p->fp64) {
            const double v[2] = {re, im};
            memcpy(buf.data() + i * 16, v, 16);
        } else {
            float v[4];
            v[0] = float(re);
            v[1] = float(im);
            v[2] = float(re - double(v[0]));
            v[3] = float(im - double(v[1]));
            memcpy(buf.data() + i * 16, v, 16);
        }
    };
    auto kvec = [](int k, int m, double len) {
        const int kk = (k < (m + 1) / 2) ? k : k - m;
        return 2.0 * kPi * kk / len;
    };
    for (int j = 0; j < 3; ++j) {
        const double kj = 2 * kPi * n[j] / lam[j];
        const double att = std::exp(-0.5 * w->c.alpha[j] * dz);
        const double tr = std::tan(w->c.walkoff[j]);
        for (int k = 0; k < nx; ++k) {
            const double K = kvec(k, nx, p->g.lx);
            const double ph = -K * K * dz / (2 * kj) - tr * K * dz;
            put(hx, size_t(j) * nx + k, att * std::cos(ph) / nx, att * std::sin(ph) / nx);
        }
        for (int k = 0; k < ny; ++k) {
            const double K = kvec(k, ny, p->g.ly);
            const double ph = -K * K * dz / (2 * kj);
            put(hy, size_t(j) * ny + k, std::cos(ph) / ny, std::sin(ph) / ny);
        }
    }
    SHG_CK(cudaMemcpy(px, hx.data(), hx.size(), cudaMemcpyHostToDevice));
    SHG_CK(cudaMemcpy(py, hy.data(), hy.size(), cudaMemcpyHostToDevice));
    return SHG_OK;
}

shg_status_t three_wave_alloc(shg_plan* p, const shg_crystal3_t* c, const shg_beams3_t* b) {
    ThreeWave* w = new ThreeWave();
    p->w3 = w;
    w->c = *c;
    w->b = *b;
    SHG_CK(cudaMalloc(&w->q, sizeof(Inst3<double>)));
    SHG_CK(cudaMalloc((void**)&w->red, size_t(kRedBlocks) * 3 * sizeof(double)));
    SHG_CK(cudaMalloc((void**)&w->pw, 3 * sizeof(double)));
    const cudaError_t e = attrs3();
    if (e != cudaSuccess) return cuda_fail(e, "three-wave kernel attributes");
    return SHG_OK;
}

// The whole three-wave propagation of one plan on `st`: initial fields, the
// cluster-resident kernel (one launch) or 2 nz + 1 passes, powers.
shg_status_t enqueue_forward3(shg_plan* p, cudaStream_t st) {
    const int nx = p->g.nx, ny = p->g.ny, nz = p->g.nz;
    const Init3 d = make_init3(p);
    k_init3_partial<<<kRedBlocks, kRed3Threads, 0, st>>>(d, nx, ny);
    if (p->fp64)
        k_init3_write<double><<<kRedBlocks, kRed3Threads, 0, st>>>(
            d, static_cast<double2*>(p->field), nx, ny);
    else
        k_init3_write<float><<<kRedBlocks, kRed3Threads, 0, st>>>(
            d, static_cast<float2*>(p->field), nx, ny);
    SHG_CK(cudaGetLastError());
    if (cluster3_path(p)) {
        SHG_CK(launch_cluster3(nx, p->w3->q, nz, p->tw, st));
    } else {
        for (int s = 0; s <= nz; ++s) {
            SHG_CK(launch_row3(p->fp64, nx, p->w3->q, ny, nz, s, p->tw, st));
            if (s < nz) SHG_CK(launch_col3(p->fp64, ny, p->w3->q, nx, p->tw, st));
        }
    }
    if (p->fp64)
        k_power3_partial<double><<<kRedBlocks, kRed3Threads, 0, st>>>(
            d, static_cast<const double2*>(p->field), nx, ny);
    else
        k_power3_partial<float><<<kRedBlocks, kRed3Threads, 0, st>>>(
            d, static_cast<const float2*>(p->field), nx, ny);
    k_power3_final<<<1, 32, 0, st>>>(d);
    SHG_CK(cudaGetLastError());
    return SHG_OK;
}

// Powers of the last propagation (synchronises its stream).
shg_status_t three_wave_powers(shg_plan* p, double out[3]) {
    SHG_CK(cudaStreamSynchronize(p->last_stream));
    SHG_CK(cudaMemcpy(p->w3->pw_host, p->w3->pw, 3 * sizeof(double), cudaMemcpyDeviceToHost));
    for (int j = 0; j < 3; ++j) out[j] = p->w3->pw_host[j];
    return SHG_OK;
}

double three_wave_input_power(const shg_plan* p) {
    return p->w3->b.p[0] + p->w3->b.p[1] + p->w3->b.p[2];
}

}  // namespace shg
