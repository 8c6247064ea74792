// Adjoint sweep orchestration: sqrt(nz) checkpoints, segment recomputation,
// transposed passes, and the gradients with respect to w0, z_focus, T_off and
// the temperature-map nodes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "adjoint.cuh"
#include "plan.h"

namespace shg {

cudaError_t row_adj_f32(int nx, const void* dl, const void* Y, AdjAcc acc, int ny, int nz, int s,
                        const void* tw, cudaStream_t st);
cudaError_t row_adj_f64(int nx, const void* dl, const void* Y, AdjAcc acc, int ny, int nz, int s,
                        const void* tw, cudaStream_t st);

struct Adjoint {
    int K = 0, nck = 0;
    size_t sbytes = 0;         // bytes of one [2][ny][nx] state
    void* ckpt = nullptr;      // [nck] states entering R(cK)
    void* seg = nullptr;       // [K] states entering R(s) of one segment
    void* work = nullptr;
    void* lam = nullptr;       // adjoint field
    float* Gc = nullptr;       // [tz][ny][nx]
    float* Gt = nullptr;
    int gtz = 0;
    double* Gs = nullptr;      // [ny][nx]
    double* red = nullptr;     // reduction scratch
    void* descW = nullptr;     // forward recomputation on `work`
    void* descL = nullptr;     // adjoint field with conjugate tables
    double* nodes = nullptr;   // [2][tz][ty][tx] scratch of the node gather
    float* gdT = nullptr;      // [tz][ty][tx]
    int ntz = 0, nty = 0, ntx = 0;
    bool have_forward = false;
    // the reverse sweep (segment recomputation and transposed passes) as one
    // CUDA graph, reused while the buffers and kernel flavours it baked in hold
    cudaStream_t cap = nullptr;
    cudaGraphExec_t sweep = nullptr;
    const void* sweep_key[2] = {nullptr, nullptr};
    int sweep_vr = -1, sweep_vc = -1;
};

void free_adjoint(shg_plan* p) {
    Adjoint* a = p->adj;
    if (!a) return;
    void* bufs[] = {a->ckpt, a->seg, a->work, a->lam, a->Gc, a->Gt, a->Gs, a->red,
                    a->descW, a->descL, a->nodes, a->gdT};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (a->sweep) cudaGraphExecDestroy(a->sweep);
    if (a->cap) cudaStreamDestroy(a->cap);
    delete a;
    p->adj = nullptr;
}

shg_status_t adjoint_alloc(shg_plan* p) {
    Adjoint* a = new Adjoint();
    p->adj = a;
    const int nz = p->g.nz;
    a->K = std::max(1, int(std::ceil(std::sqrt(double(nz + 1)))));
    a->nck = nz / a->K + 1;
    a->sbytes = size_t(2) * p->g.nx * p->g.ny * p->csize;
    const size_t desc = p->fp64 ? sizeof(InstDesc<double>) : sizeof(InstDesc<float>);
    SHG_CK(cudaMalloc(&a->ckpt, a->nck * a->sbytes));
    SHG_CK(cudaMalloc(&a->seg, a->K * a->sbytes));
    SHG_CK(cudaMalloc(&a->work, a->sbytes));
    SHG_CK(cudaMalloc(&a->lam, a->sbytes));
    SHG_CK(cudaMalloc((void**)&a->Gs, size_t(p->g.nx) * p->g.ny * sizeof(double)));
    SHG_CK(cudaMalloc((void**)&a->red, 8 * 1024 * sizeof(double)));
    SHG_CK(cudaMalloc(&a->descW, desc));
    SHG_CK(cudaMalloc(&a->descL, desc));
    SHG_CK(cudaStreamCreateWithFlags(&a->cap, cudaStreamNonBlocking));
    return SHG_OK;
}

// Called while the forward sweep is enqueued: state entering R(s) -> slot s/K.
shg_status_t adjoint_checkpoint(shg_plan* p, int s, cudaStream_t st) {
    Adjoint* a = p->adj;
    if (!a || s % a->K != 0) return SHG_OK;
    SHG_CK(cudaMemcpyAsync(static_cast<char*>(a->ckpt) + size_t(s / a->K) * a->sbytes, p->field,
                           a->sbytes, cudaMemcpyDeviceToDevice, st));
    a->have_forward = true;
    return SHG_OK;
}

void adjoint_forward_state(shg_plan* p, bool valid) {
    if (p->adj) p->adj->have_forward = valid;
}

// ------------------------------------------------------------ kernels ----

template <class R>
__global__ void k_adj_seed(const cx<R>* __restrict__ field, cx<R>* __restrict__ lam, size_t npts,
                           double scale) {
    using C = cx<R>;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < npts;
         i += size_t(gridDim.x) * blockDim.x) {
        lam[i] = mk<C>(R(0), R(0));
        const C a = field[npts + i];
        lam[npts + i] = mk<C>(R(scale * double(a.x)), R(scale * double(a.y)));
    }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double zre_conj(double2 a, double2 b) {  // Re(conj(a) b)
    return a.x * b.x + a.y * b.y;
}

// Sums for the gradient of the initial pump (Eq. 5 at z = 0, discrete
// normalisation) with respect to w0 and z_focus:
// Re<lam, g>, Re<lam, dg/dw0>, Re<lam, dg/dzf>, Re<g, dg/dw0>, Re<g, dg/dzf>, <g, g>.
template <class R>
__global__ void k_init_vjp(const cx<R>* __restrict__ lamF, int nx, int ny, double x0, double dx,
                           double y0, double dy, double w0, double zf, double kF,
                           double* __restrict__ red) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const double zr = w0 * w0 * kF * 0.5;
    const double tau = -zf / zr;
    const double2 a = make_double2(1.0, tau);
    const double2 u = make_double2(w0 * w0, w0 * w0 * tau);
    const double dtau_dw = -2.0 * tau / w0, dtau_dz = -1.0 / zr;
    const double2 da_dw = make_double2(0.0, dtau_dw), da_dz = make_double2(0.0, dtau_dz);
    const double2 du_dw = make_double2(2 * w0, 2 * w0 * tau + w0 * w0 * dtau_dw);
    const double2 du_dz = make_double2(0.0, w0 * w0 * dtau_dz);
    const int n = nx * ny;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = x0 + dx * (i % nx), y = y0 + dy * (i / nx);
        const double r2 = x * x + y * y;
        // g = exp(-r^2 / u) / a
        const double2 ex = zdiv(make_double2(-r2, 0.0), u);
        const double mag = exp(ex.x);
        double sn, cs;
        sincos(ex.y, &sn, &cs);
        const double2 g = zdiv(make_double2(mag * cs, mag * sn), a);
        const double2 u2 = zmul(u, u);
        const double2 fw = zdiv(zmul(make_double2(r2, 0.0), du_dw), u2);
        const double2 fz = zdiv(zmul(make_double2(r2, 0.0), du_dz), u2);
        const double2 aw = zdiv(da_dw, a), az = zdiv(da_dz, a);
        const double2 gw = zmul(g, make_double2(fw.x - aw.x, fw.y - aw.y));
        const double2 gz = zmul(g, make_double2(fz.x - az.x, fz.y - az.y));
        const cx<R> l = lamF[i];
        const double2 ld = make_double2(double(l.x), double(l.y));
        acc[0] += zre_conj(ld, g);
        acc[1] += zre_conj(ld, gw);
        acc[2] += zre_conj(ld, gz);
        acc[3] += zre_conj(g, gw);
        acc[4] += zre_conj(g, gz);
        acc[5] += g.x * g.x + g.y * g.y;
    }
    __shared__ double sh[6][256];
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 6) red[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_sum_double(const double* __restrict__ v, size_t n, double* __restrict__ out) {
    double a = 0;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x)
        a += v[i];
    __shared__ double sh[256];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// Cell and fraction of every field column / row in the map (as the forward).
template <class R>
__global__ void k_cells(const InstDesc<R>* __restrict__ d, int nx, int ny, int* ix, R* fx,
                        int* iy, R* fy) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nx) lin_cell<R>((d->x0 + d->dx * R(k) - d->tx0) * d->tdx_inv, d->tx, ix[k], fx[k]);
    if (k < ny) lin_cell<R>((d->y0 + d->dy * R(k) - d->ty0) * d->tdy_inv, d->ty, iy[k], fy[k]);
}

// Transposed bilinear interpolation: node (l, j, i) gathers the field-point
// sensitivities of layer l with the weights the forward used.
template <class R>
__global__ void k_gather(const float* __restrict__ Gc, const float* __restrict__ Gt, int nx,
                         int ny, int tx, int ty, int tz, const int* __restrict__ ix,
                         const R* __restrict__ fx, const int* __restrict__ iy,
                         const R* __restrict__ fy, const int* __restrict__ cs,
                         const int* __restrict__ rs, double* __restrict__ outC,
                         double* __restrict__ outT) {
    const size_t nn = size_t(tx) * ty * tz;
    const size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
    if (k >= nn) return;
    const int i = int(k % tx), j = int((k / tx) % ty), l = int(k / (size_t(tx) * ty));
    const int m0 = cs[i > 0 ? i - 1 : 0], m1 = cs[i + 1];
    const int n0 = rs[j > 0 ? j - 1 : 0], n1 = rs[j + 1];
    const size_t plane = size_t(nx) * ny;
    double sc = 0, st = 0;
    for (int n = n0; n < n1; ++n) {
        double wy = iy[n] == j ? 1.0 - double(fy[n]) : (iy[n] + 1 == j ? double(fy[n]) : 0.0);
        if (wy == 0.0) continue;
        for (int m = m0; m < m1; ++m) {
            double wx = ix[m] == i ? 1.0 - double(fx[m]) : (ix[m] + 1 == i ? double(fx[m]) : 0.0);
            if (wx == 0.0) continue;
            const size_t p = size_t(l) * plane + size_t(n) * nx + m;
            sc += wy * wx * Gc[p];
            st += wy * wx * Gt[p];
        }
    }
    outC[k] = sc;
    outT[k] = st;
}

// dT_bar[l'] = T_bar[l'] + f'(dT[l']) dZ/2 (S[l'+1] + [l' >= 1] S[l']), S[l] = sum_{m >= l} C_bar[m]:
// the transpose of the trapezoid cumulative integral C[l] = sum_{m=1..l} dZ/2 (f[m-1] + f[m])
// of the phase integrand f (f = dT, f' = 1 for the linearised model; f = Dk(T_ref + dT) -
// Dk(T_ref), f' = dDk/dT at the node's temperature for Eq. 4).
__global__ void k_trapz_T(const double* __restrict__ Cb, const double* __restrict__ Tb, int tx,
                          int ty, int tz, double dZ, const float* __restrict__ dT, DkModel m,
                          float* __restrict__ g) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= tx * ty) return;
    const size_t plane = size_t(tx) * ty;
    double S_next = 0;  // S[l + 1]
    for (int l = tz - 1; l >= 0; --l) {
        const double S_l = S_next + Cb[l * plane + col];
        const double fp = m.on ? dk_eq4_slope(m, m.t_ref + double(dT[l * plane + col])) : 1.0;
        const double v = Tb[l * plane + col] + fp * 0.5 * dZ * (S_next + (l >= 1 ? S_l : 0.0));
        g[l * plane + col] = float(v);
        S_next = S_l;
    }
}

template <class R> static void fill_adj_descs(shg_plan* p, std::vector<unsigned char>& w,
                                              std::vector<unsigned char>& l) {
    InstDesc<R> d;
    if constexpr (sizeof(R) == 8)
        fill_desc_f64(p, &d);
    else
        fill_desc_f32(p, &d);
    d.Q = nullptr;
    d.mon = nullptr;  // the recomputed segments are not a forward pass to monitor
    InstDesc<R> dw = d, dl = d;
    dw.field = static_cast<cx<R>*>(p->adj->work);
    dl.field = static_cast<cx<R>*>(p->adj->lam);
    dl.px = static_cast<const pt<R>*>(p->pxc);
    dl.py = static_cast<const pt<R>*>(p->pyc);
    w.resize(sizeof(d));
    l.resize(sizeof(d));
    memcpy(w.data(), &dw, sizeof(d));
    memcpy(l.data(), &dl, sizeof(d));
}

}  // namespace shg

using namespace shg;

extern "C" shg_status_t shg_propagate_adjoint(shg_plan_t* p, double d_eta, double* g_w0,
                                              double* g_zf, double* g_toven, float* g_dT_dev,
                                              shg_stream_t stream) {
    if (!p) return SHG_ERR_INVALID_ARG;
    Adjoint* a = p->adj;
    if (!a || !p->has_result || !a->have_forward) return SHG_ERR_STATE;
    if (!(p->b.p1 > 0)) return SHG_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SHG_CK(cudaStreamSynchronize(p->last_stream));
    if (p->ready_pending) SHG_CK(cudaStreamWaitEvent(st, p->ready, 0));
    const int nx = p->g.nx, ny = p->g.ny, nz = p->g.nz;
    const size_t npts = size_t(nx) * ny;
    const bool thermal = p->ttab != nullptr;
    if (thermal && a->gtz != p->tz) {
        if (a->Gc) cudaFree(a->Gc);
        if (a->Gt) cudaFree(a->Gt);
        a->Gc = a->Gt = nullptr;
        SHG_CK(cudaMalloc((void**)&a->Gc, size_t(p->tz) * npts * sizeof(float)));
        SHG_CK(cudaMalloc((void**)&a->Gt, size_t(p->tz) * npts * sizeof(float)));
        a->gtz = p->tz;
    }
    std::vector<unsigned char> hw, hl;
    if (p->fp64)
        fill_adj_descs<double>(p, hw, hl);
    else
        fill_adj_descs<float>(p, hw, hl);
    SHG_CK(cudaMemcpy(a->descW, hw.data(), hw.size(), cudaMemcpyHostToDevice));
    SHG_CK(cudaMemcpy(a->descL, hl.data(), hl.size(), cudaMemcpyHostToDevice));
    if (thermal) {
        SHG_CK(cudaMemsetAsync(a->Gc, 0, size_t(p->tz) * npts * sizeof(float), st));
        SHG_CK(cudaMemsetAsync(a->Gt, 0, size_t(p->tz) * npts * sizeof(float), st));
    }
    SHG_CK(cudaMemsetAsync(a->Gs, 0, npts * sizeof(double), st));
    const double dxdy = (p->g.lx / nx) * (p->g.ly / ny);
    const double cS = 0.5 * kEps0 * kCLight * p->c.n_sh;
    const double scale = 2.0 * cS * dxdy / p->b.p1 * d_eta;
    if (p->fp64)
        k_adj_seed<double><<<256, 256, 0, st>>>(static_cast<const double2*>(p->field),
                                                static_cast<double2*>(a->lam), npts, scale);
    else
        k_adj_seed<float><<<256, 256, 0, st>>>(static_cast<const float2*>(p->field),
                                               static_cast<float2*>(a->lam), npts, scale);
    SHG_CK(cudaGetLastError());
    AdjAcc acc{a->Gc, a->Gt, a->Gs};
    // the same FFT shapes as the forward sweep, to replay its states
    const int vr = fft_variant(p->fp64, nx, 0, row_umap_bit({p}), 1) | row_umap_bit({p});
    const int vc = fft_variant(p->fp64, ny, 1, 0, 1);
    // segments from the last to the first
    auto reverse_sweep = [&](cudaStream_t q) -> shg_status_t {
        for (int c = a->nck - 1; c >= 0; --c) {
            const int sb = c * a->K, se = std::min(sb + a->K, nz + 1);
            if (sb > nz) continue;
            SHG_CK(cudaMemcpyAsync(a->work, static_cast<char*>(a->ckpt) + size_t(c) * a->sbytes,
                                   a->sbytes, cudaMemcpyDeviceToDevice, q));
            for (int s = sb; s < se; ++s) {
                SHG_CK(cudaMemcpyAsync(static_cast<char*>(a->seg) + size_t(s - sb) * a->sbytes,
                                       a->work, a->sbytes, cudaMemcpyDeviceToDevice, q));
                if (s + 1 < se) {
                    SHG_CK(launch_row(p->fp64, nx, a->descW, 1, ny, nz, s, p->tw, 0, q, vr));
                    if (s < nz) SHG_CK(launch_col(p->fp64, ny, a->descW, 1, nx, p->tw, q, vc));
                }
            }
            for (int s = se - 1; s >= sb; --s) {
                if (s < nz) SHG_CK(launch_col(p->fp64, ny, a->descL, 1, nx, p->tw, q));
                const void* Y = static_cast<char*>(a->seg) + size_t(s - sb) * a->sbytes;
                SHG_CK(p->fp64 ? row_adj_f64(nx, a->descL, Y, acc, ny, nz, s, p->tw, q)
                               : row_adj_f32(nx, a->descL, Y, acc, ny, nz, s, p->tw, q));
            }
        }
        return SHG_OK;
    };
    // captured once into a graph (2-3 small operations per step would
    // otherwise be launched one by one from the host)
    if (a->sweep && (a->sweep_key[0] != a->Gc || a->sweep_key[1] != a->Gt ||
                     a->sweep_vr != vr || a->sweep_vc != vc)) {
        cudaGraphExecDestroy(a->sweep);
        a->sweep = nullptr;
    }
    if (!a->sweep) {
        PdlScope pdl(true);  // one instance
        cudaGraph_t graph = nullptr;
        SHG_CK(cudaStreamBeginCapture(a->cap, cudaStreamCaptureModeThreadLocal));
        const shg_status_t r = reverse_sweep(a->cap);
        const cudaError_t e = cudaStreamEndCapture(a->cap, &graph);
        if (r != SHG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(e, "adjoint capture");
        const cudaError_t e2 = cudaGraphInstantiate(&a->sweep, graph, 0);
        cudaGraphDestroy(graph);
        if (e2 != cudaSuccess) return cuda_fail(e2, "adjoint graph");
        a->sweep_key[0] = a->Gc;
        a->sweep_key[1] = a->Gt;
        a->sweep_vr = vr;
        a->sweep_vc = vc;
    }
    SHG_CK(cudaGraphLaunch(a->sweep, st));
    // gradients of the initial pump
    double gw = 0, gz = 0;
    if (!p->custom_init) {
        const int nb = 128;
        const double dx = p->g.lx / nx, dy = p->g.ly / ny;
        const double x0 = -(nx / 2) * dx, y0 = -(ny / 2) * dy;
        const double kF = 2 * kPi * p->c.n_f / p->c.lambda_f;
        if (p->fp64)
            k_init_vjp<double><<<nb, 256, 0, st>>>(static_cast<const double2*>(a->lam), nx, ny, x0,
                                                   dx, y0, dy, p->b.w0, p->b.z_focus, kF, a->red);
        else
            k_init_vjp<float><<<nb, 256, 0, st>>>(static_cast<const float2*>(a->lam), nx, ny, x0,
                                                  dx, y0, dy, p->b.w0, p->b.z_focus, kF, a->red);
        SHG_CK(cudaGetLastError());
        std::vector<double> r(nb * 8);
        SHG_CK(cudaMemcpyAsync(r.data(), a->red, r.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        SHG_CK(cudaStreamSynchronize(st));
        double S[6] = {0, 0, 0, 0, 0, 0};
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < 6; ++k) S[k] += r[b * 8 + k];
        const double cF = 0.5 * kEps0 * kCLight * p->c.n_f * dxdy;
        const double A0 = std::sqrt(p->b.p1 / (cF * S[5]));
        // dJ/dp = A0 Re<lam, dg/dp> + dA0/dp Re<lam, g>,  dA0/dp = -A0 Re<g, dg/dp> / S
        gw = A0 * S[1] - A0 * S[3] / S[5] * S[0];
        gz = A0 * S[2] - A0 * S[4] / S[5] * S[0];
    }
    // oven offset: every stage's dphi/dT_off and dpsi/dT_off
    {
        const int nb = 64;
        k_sum_double<<<nb, 256, 0, st>>>(a->Gs, npts, a->red);
        SHG_CK(cudaGetLastError());
        std::vector<double> r(nb);
        SHG_CK(cudaMemcpyAsync(r.data(), a->red, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        SHG_CK(cudaStreamSynchronize(st));
        double t = 0;
        for (double v : r) t += v;
        if (g_toven) *g_toven = t;
    }
    // temperature-map nodes (also needed for the oven offset under Eq. 4)
    const bool eq4_map = thermal && p->dkm.on;
    if (thermal && (g_dT_dev || eq4_map)) {
        const int tx = p->tx, ty = p->ty, tz = p->tz;
        const size_t nn = size_t(tx) * ty * tz;
        if (a->ntx != tx || a->nty != ty || a->ntz != tz) {
            if (a->nodes) cudaFree(a->nodes);
            if (a->gdT) cudaFree(a->gdT);
            a->nodes = nullptr;
            a->gdT = nullptr;
            SHG_CK(cudaMalloc((void**)&a->nodes, 2 * nn * sizeof(double)));
            SHG_CK(cudaMalloc((void**)&a->gdT, nn * sizeof(float)));
            a->ntx = tx; a->nty = ty; a->ntz = tz;
        }
        const size_t rsz = p->csize / 2;  // bytes of one real
        void* cellbuf = nullptr;
        const size_t cb = (nx + ny) * (sizeof(int) + rsz) + (tx + ty + 4) * sizeof(int);
        SHG_CK(cudaMalloc(&cellbuf, cb));
        char* cp = static_cast<char*>(cellbuf);
        int* ix = reinterpret_cast<int*>(cp);
        int* iy = ix + nx;
        void* fx = cp + (nx + ny) * sizeof(int);
        void* fy = static_cast<char*>(fx) + nx * rsz;
        int* csd = reinterpret_cast<int*>(static_cast<char*>(fy) + ny * rsz);
        int* rsd = csd + tx + 2;
        const int nmax = std::max(nx, ny);
        if (p->fp64)
            k_cells<double><<<(nmax + 127) / 128, 128, 0, st>>>(
                static_cast<const InstDesc<double>*>(a->descL), nx, ny, ix,
                static_cast<double*>(fx), iy, static_cast<double*>(fy));
        else
            k_cells<float><<<(nmax + 127) / 128, 128, 0, st>>>(
                static_cast<const InstDesc<float>*>(a->descL), nx, ny, ix, static_cast<float*>(fx),
                iy, static_cast<float*>(fy));
        std::vector<int> hix(nx), hiy(ny);
        SHG_CK(cudaMemcpyAsync(hix.data(), ix, nx * sizeof(int), cudaMemcpyDeviceToHost, st));
        SHG_CK(cudaMemcpyAsync(hiy.data(), iy, ny * sizeof(int), cudaMemcpyDeviceToHost, st));
        SHG_CK(cudaStreamSynchronize(st));
        // cs[i] = first column whose cell is >= i (cells are non-decreasing in m)
        std::vector<int> cs(tx + 2), rs(ty + 2);
        for (int i = 0; i <= tx + 1; ++i)
            cs[i] = int(std::lower_bound(hix.begin(), hix.end(), i) - hix.begin());
        for (int j = 0; j <= ty + 1; ++j)
            rs[j] = int(std::lower_bound(hiy.begin(), hiy.end(), j) - hiy.begin());
        SHG_CK(cudaMemcpyAsync(csd, cs.data(), cs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        SHG_CK(cudaMemcpyAsync(rsd, rs.data(), rs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        double* Cb = a->nodes;
        double* Tb = a->nodes + nn;
        const int nblk = int((nn + 127) / 128);
        if (p->fp64)
            k_gather<double><<<nblk, 128, 0, st>>>(a->Gc, a->Gt, nx, ny, tx, ty, tz, ix,
                                                   static_cast<double*>(fx), iy,
                                                   static_cast<double*>(fy), csd, rsd, Cb, Tb);
        else
            k_gather<float><<<nblk, 128, 0, st>>>(a->Gc, a->Gt, nx, ny, tx, ty, tz, ix,
                                                  static_cast<float*>(fx), iy,
                                                  static_cast<float*>(fy), csd, rsd, Cb, Tb);
        k_trapz_T<<<(tx * ty + 127) / 128, 128, 0, st>>>(Cb, Tb, tx, ty, tz, p->c.L / (tz - 1),
                                                         p->tmap, plan_dk_model(p), a->gdT);
        SHG_CK(cudaGetLastError());
        if (g_dT_dev)
            SHG_CK(cudaMemcpyAsync(g_dT_dev, a->gdT, nn * sizeof(float), cudaMemcpyDeviceToDevice,
                                   st));
        if (eq4_map && g_toven) {
            // Under Eq. (4) T_off is exactly a uniform shift of every map node (in
            // the phase and in the lens), so dJ/dT_off is the sum of the node gradients.
            std::vector<float> h(nn);
            SHG_CK(cudaMemcpyAsync(h.data(), a->gdT, nn * sizeof(float), cudaMemcpyDeviceToHost, st));
            SHG_CK(cudaStreamSynchronize(st));
            double t = 0;
            for (float v : h) t += double(v);
            *g_toven = t;
        }
        SHG_CK(cudaStreamSynchronize(st));
        cudaFree(cellbuf);
    }
    if (g_w0) *g_w0 = gw;
    if (g_zf) *g_zf = gz;
    SHG_CK(cudaStreamSynchronize(st));
    return SHG_OK;
}
