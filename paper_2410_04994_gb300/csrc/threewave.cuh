// Three-wave mixing (sum- and difference-frequency generation): the split
// step of Eq. (15) for three fields at omega_3 = omega_1 + omega_2, the
// generalisation of the SHG equations (1)-(2) that the paper names in its
// conclusions.  In the field convention of the SHG kernels:
//   dA1/dz = i k1 A3 conj(A2) e^{-i phi} - b1 |A1|^2 A1 + i psi1 A1
//   dA2/dz = i k2 A3 conj(A1) e^{-i phi} - b2 |A2|^2 A2 + i psi2 A2
//   dA3/dz = i k3 A1 A2 e^{+i phi}       - b3 |A3|^2 A3 + i psi3 A3
// with k_j = 2 pi d / (n_j lambda_j), b_j = beta_j eps0 c n_j / 4 and the
// phase and lens of the SHG path.  Diffraction, absorption and walk-off of
// each wave are its own K-space factor (App. A).  Fields are [3][ny][nx]
// (A1, A2, A3); factor tables [3][nx] and [3][ny].
//
// The passes are those of passes.cuh reduced to one flavour: a row pass
// (both half steps of the nonlinear part, then Lx on each field) and a
// column pass (Ly on each field), the temperature map sampled at its nodes.
#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "nonlinear.cuh"
#include "passes.cuh"

namespace shg {

// Per-instance data: the SHG descriptor carries the shared parts (fields,
// tables, phase table, map and its geometry, grid) with wave 1 in its F slots
// and wave 3 in its SH slots; wave 2's coefficients are added here.
template <class R> struct Inst3 {
    InstDesc<R> d;
    R k2, b2, l2, psi02;
};

template <class R> struct Coef3 {
    R er, ei;   // e^{i phi}
    R p[3];     // lens phase rates of the three waves
};

template <class R, class Sampler>
SHG_D Coef3<R> coef3_at(const Inst3<R>& q, const StageZ<R>& z, bool thermal, Sampler& ts) {
    const InstDesc<R>& d = q.d;
    Coef3<R> k;
    if (!thermal) {
        k.er = z.e.x;
        k.ei = z.e.y;
        k.p[0] = d.psi0F;
        k.p[1] = q.psi02;
        k.p[2] = d.psi0S;
        return k;
    }
    const cx<R> v = ts.at(z.l, z.t);  // (dT, C)
    R s, c;
    sincos_r<R>(d.g * v.y, &s, &c);
    k.er = z.e.x * c - z.e.y * s;
    k.ei = z.e.x * s + z.e.y * c;
    k.p[0] = d.psi0F + d.lF * v.x;
    k.p[1] = q.psi02 + q.l2 * v.x;
    k.p[2] = d.psi0S + d.lS * v.x;
    return k;
}

template <class R>
SHG_D void rhs3(const Inst3<R>& q, const Coef3<R>& k, const cx<R> (&A)[3], cx<R> (&f)[3]) {
    using C = cx<R>;
    const InstDesc<R>& d = q.d;
    const R bj[3] = {d.bF, q.b2, d.bS};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const R g = -bj[j] * (A[j].x * A[j].x + A[j].y * A[j].y);
        f[j] = mk<C>(g * A[j].x - k.p[j] * A[j].y, g * A[j].y + k.p[j] * A[j].x);
    }
    if (!d.undepleted) {
        // v = A3 e^{-i phi}; A3 conj(A2) e^{-i phi} = v conj(A2)
        const C v = mk<C>(A[2].x * k.er + A[2].y * k.ei, A[2].y * k.er - A[2].x * k.ei);
        const C c1 = cmulc(v, A[1]), c2 = cmulc(v, A[0]);
        f[0].x -= d.kF * c1.y;
        f[0].y += d.kF * c1.x;
        f[1].x -= q.k2 * c2.y;
        f[1].y += q.k2 * c2.x;
    }
    const C w = cmul(A[0], A[1]);
    const C we = mk<C>(w.x * k.er - w.y * k.ei, w.x * k.ei + w.y * k.er);  // A1 A2 e^{+i phi}
    f[2].x -= d.kS * we.y;
    f[2].y += d.kS * we.x;
}

// One classical RK4 step of size h from the stage coefficients at z0, z0 + h/2, z0 + h.
template <class R>
SHG_D void rk4_3(const Inst3<R>& q, cx<R> (&A)[3], const Coef3<R>& c0, const Coef3<R>& cm,
                 const Coef3<R>& c1, R h) {
    using C = cx<R>;
    C k[3], acc[3], y[3];
    rhs3(q, c0, A, k);
    const R hh = R(0.5) * h;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        acc[j] = k[j];
        y[j] = mk<C>(A[j].x + hh * k[j].x, A[j].y + hh * k[j].y);
    }
    rhs3(q, cm, y, k);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        acc[j] = mk<C>(acc[j].x + R(2) * k[j].x, acc[j].y + R(2) * k[j].y);
        y[j] = mk<C>(A[j].x + hh * k[j].x, A[j].y + hh * k[j].y);
    }
    rhs3(q, cm, y, k);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        acc[j] = mk<C>(acc[j].x + R(2) * k[j].x, acc[j].y + R(2) * k[j].y);
        y[j] = mk<C>(A[j].x + h * k[j].x, A[j].y + h * k[j].y);
    }
    rhs3(q, c1, y, k);
    const R h6 = h * (R(1) / R(6));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        A[j].x += h6 * (acc[j].x + k[j].x);
        A[j].y += h6 * (acc[j].y + k[j].y);
    }
}

// Block size of the three-wave passes: 64 threads for transform groups of at
// most 16 threads, so that a single instance spreads over four times as many
// CTAs as with 256 (a 128^2 instance: 16 instead of 4) while a column tile
// still spans a whole 32-byte sector per row (TILE >= 4); else 256.
template <class R, int N> constexpr int nth3() {
    return FftCfg<R, N, 0>::T <= 16 ? 64 : kPassThreads;
}

template <class R, int N, int NTH = nth3<R, N>()> struct Row3Geom {
    using F = FftCfg<R, N, 0>;
    static constexpr int T = F::T;
    static constexpr int ROWS = NTH / T;
    static constexpr int S = padded_len<R>(N, T < Bank<R>::W ? T : 1);
    static constexpr size_t fields = size_t(3) * ROWS * S * sizeof(cx<R>);
    static constexpr size_t smem = fields + size_t(4) * N * sizeof(pt<R>);  // twiddles + 3 rows
};

// Row pass R(s) of the three fields.  grid = (ceil(ny / ROWS), instances).
template <class R, int NX, int NTH = nth3<R, NX>()>
__global__ void __launch_bounds__(NTH, 1)
    k_row3(const Inst3<R>* __restrict__ qs, int ny, int nz, int s, const pt<R>* __restrict__ tw) {
    using C = cx<R>;
    using G = Row3Geom<R, NX, NTH>;
    constexpr int E = FftCfg<R, NX, 0>::E, T = G::T, ROWS = G::ROWS, S = G::S;
    constexpr bool WS = T <= 32;  // a row's threads share a warp (see k_row_pass)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Inst3<R> qsh;
    __shared__ StageZ<R> zsh[5];
    C* smem = reinterpret_cast<C*>(smem_raw);
    pt<R>* twS = reinterpret_cast<pt<R>*>(smem_raw + G::fields);
    pt<R>* pS = twS + NX;  // [3][NX]
    const int lr = threadIdx.x / T, t = threadIdx.x - lr * T;
    const int y = blockIdx.x * ROWS + lr;
    const bool active = y < ny;
    const Inst3<R>& qg = qs[blockIdx.y];
    for (int k = threadIdx.x; k < 4 * NX; k += NTH) {
        if (k < NX)
            cp_async(&twS[tw_pos<NX>(k)], &tw[k * (1024 / NX)]);
        else
            cp_async(&pS[k - NX], &qg.d.px[k - NX]);
    }
    if (threadIdx.x == 0) qsh = qg;
    if (threadIdx.x < 5) {
        const int q = 4 * s - 2 + threadIdx.x;
        zsh[threadIdx.x] = stage_z(qg.d, q < 0 ? 0 : (q > 4 * nz ? 4 * nz : q));
    }
    pdl_wait();  // the fields are the previous pass's output
    pdl_trigger();
    if (active) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const C* row = qg.d.field + (size_t(f) * ny + y) * NX;
#pragma unroll
            for (int m = 0; m < E; ++m)
                cp_async(&smem[(f * ROWS + lr) * S + pidx<R>(t + T * m)], &row[t + T * m]);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const Inst3<R>& q = qsh;
    const InstDesc<R>& d = q.d;
    const bool thermal = d.ttab != nullptr;
    const MapView<R> mv{d.ttab, d.tx, d.tx * d.ty, 0, 0, 0};
    const RowCell<R> rc = thermal ? row_cell(d, y) : RowCell<R>{0, R(0)};
    const R h = R(0.5) * d.dz;
    if (active) {
#pragma unroll 1
        for (int m = 0; m < E; ++m) {
            const int xi = t + T * m;
            C A[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) A[f] = smem[(f * ROWS + lr) * S + pidx<R>(xi)];
            TempSampler<R> ts;
            if (thermal) make_sampler(d, mv, xi, rc, ts);
            const Coef3<R> cz = coef3_at(q, zsh[2], thermal, ts);
            if (s > 0) {
                const Coef3<R> c0 = coef3_at(q, zsh[0], thermal, ts);
                const Coef3<R> cm = coef3_at(q, zsh[1], thermal, ts);
                rk4_3(q, A, c0, cm, cz, h);
            }
            if (s < nz) {
                const Coef3<R> cm = coef3_at(q, zsh[3], thermal, ts);
                const Coef3<R> c1 = coef3_at(q, zsh[4], thermal, ts);
                rk4_3(q, A, cz, cm, c1, h);
            }
#pragma unroll
            for (int f = 0; f < 3; ++f) smem[(f * ROWS + lr) * S + pidx<R>(xi)] = A[f];
        }
    }
    group_sync<WS>();  // the transforms read points that other threads of the row advanced
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        C* sb = smem + (f * ROWS + lr) * S;
        C* row = d.field + (size_t(f) * ny + y) * NX;
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<R>(t + T * m)] : mk<C>(R(0), R(0));
        if (s < nz) {
            group_sync<WS>();
            fft_mul_ifft<R, NX, 0, NX, WS>(v, sb, t, twS, pS + f * NX);
        }
        if (active) {
#pragma unroll
            for (int m = 0; m < E; ++m) row[t + T * m] = v[m];
        }
    }
}

template <class R, int N, int NTH = nth3<R, N>()> struct Col3Geom {
    using F = FftCfg<R, N, 0>;
    static constexpr int T = F::T;
    static constexpr int TILE = NTH / T;
    static constexpr int S = padded_len<R>(N, TILE < Bank<R>::W ? Bank<R>::W / TILE : 1);
    static constexpr size_t fields = size_t(3) * TILE * S * sizeof(cx<R>);
    static constexpr size_t smem = fields + size_t(4) * N * sizeof(pt<R>);
};

// Column pass C(s) of the three fields.  grid = (ceil(nx / TILE), instances).
template <class R, int NY, int NTH = nth3<R, NY>()>
__global__ void __launch_bounds__(NTH, 1)
    k_col3(const Inst3<R>* __restrict__ qs, int nx, const pt<R>* __restrict__ tw) {
    using C = cx<R>;
    using G = Col3Geom<R, NY, NTH>;
    constexpr int E = FftCfg<R, NY, 0>::E, T = G::T, TILE = G::TILE, S = G::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    pt<R>* twS = reinterpret_cast<pt<R>*>(smem_raw + G::fields);
    pt<R>* pS = twS + NY;  // [3][NY]
    const InstDesc<R>& d = qs[blockIdx.y].d;
    C* field = d.field;
    const int c = threadIdx.x % TILE, t = threadIdx.x / TILE;
    const int x = blockIdx.x * TILE + c;
    const bool active = x < nx;
    for (int k = threadIdx.x; k < 4 * NY; k += NTH) {
        if (k < NY)
            cp_async(&twS[tw_pos<NY>(k)], &tw[k * (1024 / NY)]);
        else
            cp_async(&pS[k - NY], &d.py[k - NY]);
    }
    pdl_wait();  // the fields are the previous pass's output
    pdl_trigger();
    if (active) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const C* col = field + size_t(f) * NY * nx + x;
#pragma unroll
            for (int m = 0; m < E; ++m)
                cp_async(&smem[(f * TILE + c) * S + pidx<R>(t + T * m)], col + size_t(t + T * m) * nx);
        }
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        C* sb = smem + (f * TILE + c) * S;
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<R>(t + T * m)] : mk<C>(R(0), R(0));
        __syncthreads();
        fft_mul_ifft<R, NY, 0, NY>(v, sb, t, twS, pS + f * NY);
        if (active) {
            C* col = field + size_t(f) * NY * nx + x;
#pragma unroll
            for (int m = 0; m < E; ++m) col[size_t(t + T * m) * nx] = v[m];
        }
    }
}

}  // namespace shg
