// The two fused passes of one split step.
//
// The K-space factor of Eq. (A.4) is separable,
//   exp(-i (Kx^2 + Ky^2) dz / 2k) = exp(-i Kx^2 dz / 2k) exp(-i Ky^2 dz / 2k),
// and the 2-D DFT is a product of 1-D DFTs along x and along y, so
// F^{-1} diag(P) F = Lx Ly with Lx = F_x^{-1} diag(px) F_x along every row and
// Ly the same along every column; Lx and Ly commute.  Step s of Eq. (15),
// N_b(s) Lx Ly N_a(s), is therefore marched as
//   row pass R(s):    N_b(s-1) [z_s - dz/2 -> z_s], heat deposit at z_s,
//                     N_a(s) [z_s -> z_s + dz/2], Lx(s)
//   column pass C(s): Ly(s)
// for s = 0..nz-1, followed by a final row pass R(nz) = N_b(nz-1) only.
// Each pass reads and writes both fields once: 2 x (8+8) B of complex64 in
// and out per grid point and pass.
#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "nonlinear.cuh"

namespace shg {

constexpr int kPassThreads = 256;

template <class R, int N> struct RowGeom {
    using F = FftCfg<R, N>;
    static constexpr int T = F::T;
    static constexpr int ROWS = kPassThreads / T;
    static constexpr int S = padded_len<R>(N, T < Bank<R>::W ? T : 1);
    static constexpr size_t smem = size_t(2) * ROWS * S * sizeof(cx<R>);
};

template <class R, int N> struct ColGeom {
    using F = FftCfg<R, N>;
    static constexpr int T = F::T;
    static constexpr int TILE = kPassThreads / T;
    static constexpr int S = padded_len<R>(N, TILE < Bank<R>::W ? Bank<R>::W / TILE : 1);
    static constexpr size_t smem = size_t(2) * TILE * S * sizeof(cx<R>);
};

// Temperature-map sampler for field point (xi, y).
template <class R>
SHG_D void make_sampler(const InstDesc<R>& d, int xi, int y, TempSampler<R>& ts) {
    int ix, iy;
    float fx, fy;
    lin_cell((float(d.x0 + d.dx * R(xi)) - d.tx0) * d.tdx_inv, d.tx, ix, fx);
    lin_cell((float(d.y0 + d.dy * R(y)) - d.ty0) * d.tdy_inv, d.ty, iy, fy);
    ts.base = d.ttab + iy * d.tx + ix;
    ts.tx = d.tx;
    ts.plane = d.tx * d.ty;
    ts.fx = fx;
    ts.fy = fy;
    ts.la = -2;
}

// Per-row heat deposit at z_s: q_dot dV of each point, summed per heat node in
// shared memory, then added to the heat grid in double precision.
template <class R, int N>
SHG_D void deposit_row(const InstDesc<R>& d, const cx<R> (&vF)[FftCfg<R, N>::E],
                       const cx<R> (&vS)[FftCfg<R, N>::E], float* bins, int lr, int t,
                       int y, bool active, int s, int nz) {
    using G = RowGeom<R, N>;
    constexpr int E = FftCfg<R, N>::E, T = G::T, ROWS = G::ROWS;
    const int nb = ROWS * d.hx;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) bins[i] = 0.f;
    __syncthreads();
    const int l = d.hlz[s];
    const int j = active ? d.hiy[y] : -1;
    if (l >= 0 && j >= 0) {
        const R w = d.dxdy * d.dz * ((s == 0 || s == nz) ? R(0.5) : R(1));
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int i = __ldg(&d.hix[t + T * m]);
            if (i < 0) continue;
            const R aF2 = vF[m].x * vF[m].x + vF[m].y * vF[m].y;
            const R aS2 = vS[m].x * vS[m].x + vS[m].y * vS[m].y;
            const R q = aF2 * (d.qaF + d.qbF * aF2) + aS2 * (d.qaS + d.qbS * aS2);
            atomicAdd(&bins[lr * d.hx + i], float(q * w));
        }
    }
    __syncthreads();
    const int y0 = blockIdx.x * ROWS;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const float v = bins[k];
        const int r = k / d.hx, i = k - r * d.hx;
        const int yy = y0 + r;
        if (v != 0.f && l >= 0) {
            const int jj = d.hiy[yy];
            atomicAdd(&d.Q[(size_t(l) * d.hy + jj) * d.hx + i], double(v));
        }
    }
    __syncthreads();
}

// Row pass R(s).  grid = (ceil(ny / ROWS), instances); block = 256.
template <class R, int NX>
__global__ void __launch_bounds__(kPassThreads)
    k_row_pass(const InstDesc<R>* __restrict__ descs, int ny, int nz, int s,
               const pt<R>* __restrict__ tw) {
    using C = cx<R>;
    using G = RowGeom<R, NX>;
    constexpr int E = FftCfg<R, NX>::E, T = G::T, ROWS = G::ROWS, S = G::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const InstDesc<R>& d = descs[blockIdx.y];
    const int lr = threadIdx.x / T, t = threadIdx.x - (threadIdx.x / T) * T;
    const int y = blockIdx.x * ROWS + lr;
    const bool active = y < ny;
    C* rowF = d.field + size_t(y) * NX;
    C* rowS = d.field + (size_t(ny) + y) * NX;
    C vF[E], vS[E];
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            vF[m] = rowF[t + T * m];
            vS[m] = rowS[t + T * m];
        }
    }
    const bool thermal = d.ttab != nullptr;
    const R h = R(0.5) * d.dz;
    // heat deposit needs the state at z_s, i.e. after N_b(s-1)
    if (s > 0 && active) {
#pragma unroll 1
        for (int m = 0; m < E; ++m) {
            TempSampler<R> ts;
            TempSampler<R>* tsp = thermal ? (make_sampler(d, t + T * m, y, ts), &ts) : nullptr;
            const Coef<R> c0 = coef_at(d, 4 * s - 2, tsp);
            const Coef<R> cm = coef_at(d, 4 * s - 1, tsp);
            const Coef<R> c1 = coef_at(d, 4 * s, tsp);
            rk4(d, vF[m], vS[m], c0, cm, c1, h);
        }
    }
    if (d.Q != nullptr) deposit_row<R, NX>(d, vF, vS, reinterpret_cast<float*>(smem), lr, t, y,
                                           active, s, nz);
    if (s < nz && active) {
#pragma unroll 1
        for (int m = 0; m < E; ++m) {
            TempSampler<R> ts;
            TempSampler<R>* tsp = thermal ? (make_sampler(d, t + T * m, y, ts), &ts) : nullptr;
            const Coef<R> c0 = coef_at(d, 4 * s, tsp);
            const Coef<R> cm = coef_at(d, 4 * s + 1, tsp);
            const Coef<R> c1 = coef_at(d, 4 * s + 2, tsp);
            rk4(d, vF[m], vS[m], c0, cm, c1, h);
        }
    }
    if (s < nz) {
        fft_mul_ifft<R, NX>(vF, vS, smem + lr * S, smem + (ROWS + lr) * S, t, tw, d.px,
                            d.px + NX);
    }
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            rowF[t + T * m] = vF[m];
            rowS[t + T * m] = vS[m];
        }
    }
}

// Column pass C(s).  grid = (ceil(nx / TILE), instances); block = 256.
template <class R, int NY>
__global__ void __launch_bounds__(kPassThreads)
    k_col_pass(const InstDesc<R>* __restrict__ descs, int nx, const pt<R>* __restrict__ tw) {
    using C = cx<R>;
    using G = ColGeom<R, NY>;
    constexpr int E = FftCfg<R, NY>::E, T = G::T, TILE = G::TILE, S = G::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const InstDesc<R>& d = descs[blockIdx.y];
    const int c = threadIdx.x % TILE, t = threadIdx.x / TILE;
    const int x = blockIdx.x * TILE + c;
    const bool active = x < nx;
    C* colF = d.field + x;
    C* colS = d.field + size_t(NY) * nx + x;
    C vF[E], vS[E];
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            vF[m] = colF[size_t(t + T * m) * nx];
            vS[m] = colS[size_t(t + T * m) * nx];
        }
    }
    fft_mul_ifft<R, NY>(vF, vS, smem + c * S, smem + (TILE + c) * S, t, tw, d.py, d.py + NY);
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            colF[size_t(t + T * m) * nx] = vF[m];
            colS[size_t(t + T * m) * nx] = vS[m];
        }
    }
}

}  // namespace shg
