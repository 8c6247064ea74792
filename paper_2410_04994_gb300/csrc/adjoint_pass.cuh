// Transposed row pass R(s)^T = N_b(s-1)^T N_a(s)^T Lx^H.
#pragma once
#include "adjoint.cuh"
#include "passes.cuh"

namespace shg {

// grid = (ceil(ny / ROWS), 1); block = NTH.  `dl` describes the adjoint field
// (its K-space tables are the conjugates of the forward ones); Y is the state
// that entered the forward row pass R(s).  The adjoint is updated in place.
template <class R, int NX, int NTH = kPassThreads>
__global__ void __launch_bounds__(NTH, 2 * (kPassThreads / NTH))
    k_row_adj(const InstDesc<R>* __restrict__ dl, const cx<R>* __restrict__ Y, AdjAcc acc,
              int ny, int nz, int s, const pt<R>* __restrict__ tw) {
    using C = cx<R>;
    using G = RowGeom<R, NX, 0, NTH>;
    constexpr int E = FftCfg<R, NX>::E, T = G::T, ROWS = G::ROWS, S = G::S;
    constexpr bool WS = T <= 32;  // a row's threads share a warp (as in k_row_pass)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ InstDesc<R> dsh;
    __shared__ StageZ<R> zsh[5];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int lr = threadIdx.x / T, t = threadIdx.x - (threadIdx.x / T) * T;
    const int y = blockIdx.x * ROWS + lr;
    const bool active = y < ny;
    C* sF = smem + lr * S;
    C* sS = smem + (ROWS + lr) * S;
    // shared copies of the twiddles and of the (conjugate) row factors
    pt<R>* twS = reinterpret_cast<pt<R>*>(smem_raw + G::fields);
    pt<R>* pS = twS + NX;
    stage_tables<R, NX>(twS, pS, tw, dl->px);
    if (active) {
        const C* rF = dl->field + size_t(y) * NX;
        const C* rS = dl->field + (size_t(ny) + y) * NX;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            cp_async(&sF[pidx<R>(t + T * m)], &rF[t + T * m]);
            cp_async(&sS[pidx<R>(t + T * m)], &rS[t + T * m]);
        }
    }
    if (threadIdx.x == 0) dsh = *dl;
    if (threadIdx.x < 5) {
        const int q = 4 * s - 2 + threadIdx.x;
        zsh[threadIdx.x] = stage_z(*dl, q < 0 ? 0 : (q > 4 * nz ? 4 * nz : q));
    }
    cp_async_wait_all();
    __syncthreads();
    const InstDesc<R>& d = dsh;
    // Lx^H on each field: the forward transform pair with conjugated factors
    if (s < nz) {
#pragma unroll 1
        for (int f = 0; f < 2; ++f) {
            C* sb = f == 0 ? sF : sS;
            C v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<R>(t + T * m)] : mk<C>(R(0), R(0));
            group_sync<WS>();
            fft_mul_ifft<R, NX, 0, NX, WS>(v, sb, t, twS, pS + f * NX);
            group_sync<WS>();
#pragma unroll
            for (int m = 0; m < E; ++m) sb[pidx<R>(t + T * m)] = v[m];
        }
    }
    const bool thermal = d.ttab != nullptr;
    const MapView<R> mv{d.ttab, d.tx, d.tx * d.ty, 0, 0, 0};
    const R h = R(0.5) * d.dz;
    if (!active) return;
    const C* YF = Y + size_t(y) * NX;
    const C* YS = Y + (size_t(ny) + y) * NX;
    C* lamF = d.field + size_t(y) * NX;
    C* lamS = d.field + (size_t(ny) + y) * NX;
    const size_t plane = size_t(ny) * NX;
    const RowCell<R> rc = thermal ? row_cell(d, y) : RowCell<R>{0, R(0)};
#pragma unroll 1
    for (int m = 0; m < E; ++m) {
        const int xi = t + T * m;
        C lF = sF[pidx<R>(xi)], lS = sS[pidx<R>(xi)];
        const C yF = YF[xi], yS = YS[xi];
        TempSampler<R> ts;
        if (thermal) make_sampler(d, mv, xi, rc, ts);
        Coef<R> c[5];
        StageBar<R> b[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            b[k].phi = b[k].pF = b[k].pS = R(0);
            c[k] = coef_at(d, zsh[k], thermal, ts);
        }
        C xF = yF, xS = yS;
        if (s > 0) rk4(d, xF, xS, c[0], c[1], c[2], h);  // state at z_s
        if (s < nz) rk4_adj(d, xF, xS, c[2], c[3], c[4], h, lF, lS, b[2], b[3], b[4]);
        if (s > 0) rk4_adj(d, yF, yS, c[0], c[1], c[2], h, lF, lS, b[0], b[1], b[2]);
        lamF[xi] = lF;
        lamS[xi] = lS;
        double toff = 0;
        const size_t pix = size_t(y) * NX + xi;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int q = 4 * s - 2 + k;
            if (q < 0 || q > 4 * nz) continue;
            const R gc = d.g * b[k].phi;
            const R gt = d.lF * b[k].pF + d.lS * b[k].pS;
            toff += double(gc) * (double(q) * double(d.dz) * 0.25) + double(gt);
            if (thermal) {
                const int l = zsh[k].l;
                const R tz = zsh[k].t;
                acc.Gc[size_t(l) * plane + pix] += float((R(1) - tz) * gc);
                acc.Gc[size_t(l + 1) * plane + pix] += float(tz * gc);
                acc.Gt[size_t(l) * plane + pix] += float((R(1) - tz) * gt);
                acc.Gt[size_t(l + 1) * plane + pix] += float(tz * gt);
            }
        }
        acc.Gs[pix] += toff;
    }
}

}  // namespace shg
