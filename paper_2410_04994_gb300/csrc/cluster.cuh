// Cluster-resident propagation of one small instance (FP32, N x N, N = 64 or
// 128): the whole z-march of Eq. (15) in one launch, with the fields held in
// the shared memory of a thread-block cluster instead of making two round
// trips through global memory per step.
//
// The K CTAs of a cluster split the N x N grid of both fields: CTA c holds
// rows [cR, cR + R) in its row buffer and columns [cR, cR + R) in its column
// buffer (R = N / K).  Step s applies N_b(s-1), N_a(s) (pointwise, in
// whatever layout holds the fields) and L = Lx Ly.  Lx and Ly are diagonal
// in separable spectra and commute exactly, so their order alternates and
// one transpose per step suffices:
//   s even (rows):    RK4 on the rows, Lx, barrier, gather the columns, Ly
//   s odd (columns):  RK4 on the columns, Ly, barrier, gather the rows, Lx
// A gather reads the other CTAs' buffers through distributed shared memory.
// One cluster barrier per step is enough: a CTA rewrites its row buffer (RK4,
// Lx, or the row gather that fills it) only after a barrier that every other
// CTA reached after its last read of that buffer (the column gather of the
// step before, in which the other CTAs read it), and the same holds for the
// column buffer.  A last barrier keeps every CTA resident until the final
// gather has read it.
// The barriers are the hardware cluster barrier (every CTA executes the same
// sequence of them; there is no spin-wait).  The arithmetic per point is that
// of the streaming passes: the packed-FP32 RK4 of nonlinear.cuh and the
// register FFT of fft.cuh.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"
#include "fft.cuh"
#include "nonlinear.cuh"

namespace shg {

template <int N, int K> struct ClusterGeom {
    static constexpr int R = N / K;          // rows (and columns) per CTA
    static constexpr int V = 1;              // 8 points per thread per transform
    using F = FftCfg<float, N, V>;
    static constexpr int E = F::E, T = F::T;
    static constexpr int NT = 2 * R * T;     // one group of T threads per transform (2 fields x R)
    static constexpr int S = padded_len<float>(N, T < Bank<float>::W ? T : 1);
    static constexpr int PAIRS = R * N / 2;  // point pairs per CTA
    static_assert(PAIRS % NT == 0, "whole pairs per thread");
    static_assert(2 * R * N == E * NT, "each gather moves E points per thread");
    static constexpr size_t buf = size_t(2) * R * S * sizeof(float2);  // one of Rbuf, Cbuf
    static constexpr size_t smem = 2 * buf + size_t(5) * N * sizeof(float4);
};

template <int N, int K>
__global__ void __launch_bounds__(ClusterGeom<N, K>::NT, 1)
    k_cluster_prop(const InstDesc<float>* __restrict__ descs, int nz, const float4* __restrict__ tw) {
    namespace cg = cooperative_groups;
    using G = ClusterGeom<N, K>;
    constexpr int R = G::R, V = G::V, E = G::E, T = G::T, NT = G::NT, S = G::S;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ InstDesc<float> dsh;
    __shared__ StageZ<float> zsh[2][5];  // stage data of step s in zsh[s & 1]
    float2* Rbuf = reinterpret_cast<float2*>(smem_raw);              // [2][R][S] rows
    float2* Cbuf = reinterpret_cast<float2*>(smem_raw + G::buf);     // [2][R][S] columns
    float4* twS = reinterpret_cast<float4*>(smem_raw + 2 * G::buf);  // [N]
    float4* pxS = twS + N;                                           // [2][N]
    float4* pyS = pxS + 2 * N;                                       // [2][N]
    const int tid = threadIdx.x;
    const int cid = int(cluster.block_rank());
    const int y0 = cid * R;
    const InstDesc<float>& dg = descs[blockIdx.y];
    // constant tables and this CTA's rows of both fields
    stage_tables<float, N>(twS, pxS, tw, dg.px);
    for (int k = tid; k < 2 * N; k += NT) cp_async(&pyS[k], &dg.py[k]);
    for (int e = tid; e < 2 * R * N; e += NT) {
        const int x = e % N, r = (e / N) % R, f = e / (R * N);
        cp_async(&Rbuf[(f * R + r) * S + pidx<float>(x)], &dg.field[(size_t(f) * N + y0 + r) * N + x]);
    }
    if (tid == 0) dsh = dg;
    cp_async_wait_all();
    __syncthreads();
    const InstDesc<float>& d = dsh;
    const bool thermal = d.ttab != nullptr;   // the launcher admits only the per-point table then
    const float4* __restrict__ umap4 = reinterpret_cast<const float4*>(d.umap);
    const float h = 0.5f * d.dz;
    // transform group of this thread
    const int g = tid / T, t = tid - g * T;
    const int gf = g / R;
    // Stage data of step s (5 stage points) into zsh[s & 1].
    auto stage = [&](int s) {
        if (tid < 5) {
            const int q = 4 * s - 2 + tid;
            zsh[s & 1][tid] = stage_z(d, q < 0 ? 0 : (q > 4 * nz ? 4 * nz : q));
        }
    };
    // The layout of step s: rows (s even: Rbuf[f][r][x], this CTA's rows
    // y0 + r) or columns (s odd: Cbuf[f][c][y], this CTA's columns y0 + c).
    // Pair p of this thread: in rows, the points (2j, 2j + 1) of row y0 + r;
    // in columns, the columns (y0 + 2jj, y0 + 2jj + 1) of row y.  Either way
    // the pair is one entry [l][row][pair] of the per-point table.
    constexpr int PPT = G::PAIRS / NT;
    auto pair_of = [&](bool rows_l, int p, float2*& e0, float2*& e1, int& row, int& jg) {
        if (rows_l) {
            const int r = p / (N / 2), j = p - r * (N / 2);
            e0 = Rbuf + r * S + pidx<float>(2 * j);
            e1 = Rbuf + r * S + pidx<float>(2 * j + 1);
            row = y0 + r;
            jg = j;
        } else {
            const int y = p / (R / 2), jj = p - y * (R / 2);
            e0 = Cbuf + (2 * jj) * S + pidx<float>(y);
            e1 = Cbuf + (2 * jj + 1) * S + pidx<float>(y);
            row = y;
            jg = y0 / 2 + jj;
        }
    };
    // Per-point table entries of this thread's pairs for the map layers that
    // step s's stage points fall between (at most three: the launcher admits
    // the table path only when one step spans less than one layer), loaded
    // into registers one step ahead, so that their latency is hidden behind
    // the transforms and the cluster barrier of the step before.  Layers past
    // the span are not read.
    float4 tv[PPT][3];
#pragma unroll
    for (int i = 0; i < PPT; ++i) tv[i][0] = tv[i][1] = tv[i][2] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto load_tables = [&](int s) {
        if (!thermal) return;
        const int q0 = 4 * s - 2, q4 = 4 * s + 2;
        const int l0 = stage_z(d, q0 < 0 ? 0 : q0).l;
        const int l4 = stage_z(d, q4 > 4 * nz ? 4 * nz : q4).l;
        const int span = l4 + 2 - l0;
        if (span > 3 && tid == 0 && d.status) atomicExch(d.status, int(SHG_ERR_STATE));
        const int nl = span < 3 ? span : 3;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            float2 *e0, *e1;
            int row, jg;
            pair_of((s & 1) == 0, tid + NT * i, e0, e1, row, jg);
            const float4* src = umap4 + (size_t(l0) * N + row) * (N / 2) + jg;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (k < nl) tv[i][k] = __ldg(src + size_t(k) * N * (N / 2));
        }
    };
    // F^-1 diag(p) F along the rows (Lx, factors pxS) or the columns (Ly,
    // pyS) held in buf: group g transforms field gf, row or column g - gf R.
    auto transform = [&](float2* buf, const float4* fac) {
        float2* line = buf + g * S;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = line[pidx<float>(t + T * m)];
        group_sync<true>();  // the exchanges reuse the line (a line's threads share a warp)
        fft_mul_ifft<float, N, V, N, true>(v, line, t, twS, fac + gf * N);
#pragma unroll
        for (int m = 0; m < E; ++m) line[pidx<float>(t + T * m)] = v[m];
    };
    // Transposes through distributed shared memory.  All E remote loads of a
    // thread are issued before its local stores (a store could alias a remote
    // load for all the compiler knows, which would serialise the loads).
    // Columns: Cbuf[f][c][y] = element y0 + c of row y, held by CTA y / R.
    auto gather_columns = [&] {
        float2 gv[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = tid + NT * m;
            const int c = e % R, y = (e / R) % N, f = e / (R * N);
            const float2* src = cluster.map_shared_rank(Rbuf, y / R);
            gv[m] = src[(f * R + y % R) * S + pidx<float>(y0 + c)];
        }
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = tid + NT * m;
            const int c = e % R, y = (e / R) % N, f = e / (R * N);
            Cbuf[(f * R + c) * S + pidx<float>(y)] = gv[m];
        }
    };
    // Rows: Rbuf[f][r][x] = element y0 + r of column x, held by CTA x / R.
    auto gather_rows = [&] {
        float2 gv[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = tid + NT * m;
            const int r = e % R, x = (e / R) % N, f = e / (R * N);
            const float2* src = cluster.map_shared_rank(Cbuf, x / R);
            gv[m] = src[(f * R + x % R) * S + pidx<float>(y0 + r)];
        }
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int e = tid + NT * m;
            const int r = e % R, x = (e / R) % N, f = e / (R * N);
            Rbuf[(f * R + r) * S + pidx<float>(x)] = gv[m];
        }
    };
    stage(0);
    load_tables(0);
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s <= nz; ++s) {
        const bool rows_l = (s & 1) == 0;
        const StageZ<float>* zs = zsh[s & 1];
        const int lmin = zs[0].l;
        // ---- nonlinear half steps on this CTA's points (two per thread pass)
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            float2 *e0, *e1;
            int row, jg;
            pair_of(rows_l, tid + NT * i, e0, e1, row, jg);
            float2 aF0 = e0[0], aF1 = e1[0];
            float2 aS0 = e0[R * S], aS1 = e1[R * S];
            const RegPairSampler ps{tv[i][0], tv[i][1], tv[i][2], lmin};
            auto cq = [&](int q) { return coef2_at(d, zs[q], thermal, ps); };
            Cx2 F{pk2(aF0.x, aF1.x), pk2(aF0.y, aF1.y)}, Sx{pk2(aS0.x, aS1.x), pk2(aS0.y, aS1.y)};
            const Coef2 z2 = cq(2);
            if (s > 0) {
                const Coef2 c0 = cq(0);
                const Coef2 cm = cq(1);
                rk4_2(d, F, Sx, c0, cm, z2, h);
            }
            if (s < nz) {
                const Coef2 cm = cq(3);
                const Coef2 c1 = cq(4);
                rk4_2(d, F, Sx, z2, cm, c1, h);
            }
            up2(F.r, aF0.x, aF1.x);
            up2(F.i, aF0.y, aF1.y);
            up2(Sx.r, aS0.x, aS1.x);
            up2(Sx.i, aS0.y, aS1.y);
            e0[0] = aF0;
            e1[0] = aF1;
            e0[R * S] = aS0;
            e1[R * S] = aS1;
        }
        // the next step's stage data and table entries, in flight during the
        // transforms (zsh[(s + 1) & 1] was last read in step s - 1)
        if (s < nz) {
            stage(s + 1);
            load_tables(s + 1);
        }
        __syncthreads();
        if (s == nz) break;  // the last row pass is N_b alone
        // ---- L = Lx Ly, in the order that needs one transpose: the layout
        // this step starts in, the barrier, the transpose, the other layout
        if (rows_l) {
            transform(Rbuf, pxS);
            cluster.sync();
            gather_columns();
            __syncthreads();
            transform(Cbuf, pyS);
        } else {
            transform(Cbuf, pyS);
            cluster.sync();
            gather_rows();
            __syncthreads();
            transform(Rbuf, pxS);
        }
        __syncthreads();  // the next step's pairs were transformed by other groups
    }
    // the final state to global memory, from the layout of step nz
    if ((nz & 1) == 0) {
        for (int e = tid; e < 2 * R * N; e += NT) {
            const int x = e % N, r = (e / N) % R, f = e / (R * N);
            d.field[(size_t(f) * N + y0 + r) * N + x] = Rbuf[(f * R + r) * S + pidx<float>(x)];
        }
    } else {
        for (int e = tid; e < 2 * R * N; e += NT) {
            const int c = e % R, y = (e / R) % N, f = e / (R * N);
            d.field[(size_t(f) * N + y) * N + y0 + c] = Cbuf[(f * R + c) * S + pidx<float>(y)];
        }
    }
    // no CTA leaves while another may still read its buffers (the transpose
    // of step nz - 1 has no barrier after it)
    cluster.sync();
}

}  // namespace shg
