// Cluster-resident propagation of one small three-wave instance (FP32, N x N,
// N = 64 or 128): the z-march of the three coupled fields of threewave.cuh in
// one launch, with the fields held in the shared memory of a thread-block
// cluster (the scheme of cluster.cuh with three fields instead of two).
//
// The K CTAs of a cluster split the grid: CTA c holds rows [cR, cR + R) of
// the three fields in its row buffer and columns [cR, cR + R) in its column
// buffer (R = N / K).  Step s applies N_b(s-1) and N_a(s) pointwise in the
// layout that holds the fields, then L = Lx Ly; the two factors are diagonal
// in separable spectra and commute exactly, so their order alternates and
// each step needs one transpose through distributed shared memory:
//   s even (rows):    RK4 on the rows, Lx, barrier, gather the columns, Ly
//   s odd (columns):  RK4 on the columns, Ly, barrier, gather the rows, Lx
// The buffer-reuse argument of cluster.cuh holds unchanged: a CTA rewrites a
// buffer only after a cluster barrier that every other CTA reached after its
// last read of it, and a final barrier keeps every CTA resident until the
// last gather has read it.  The only synchronisation is the hardware cluster
// barrier (no spin-wait).
//
// Transforms run one group of T threads per line (3 fields x R lines), so a
// CTA has 3 R T threads; its R N points are walked with that stride, two or
// three per thread.  The temperature map enters through the per-point table
// ((dT, C) of every field point at every map layer), whose entries for the
// next step are loaded into registers during the current step's transforms.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"
#include "fft.cuh"
#include "nonlinear.cuh"
#include "threewave.cuh"

namespace shg {

template <int N, int K> struct Cluster3Geom {
    static constexpr int R = N / K;          // rows (and columns) per CTA
    static constexpr int V = 1;              // 8 points per thread per transform
    using F = FftCfg<float, N, V>;
    static constexpr int E = F::E, T = F::T;
    static constexpr int NT = 3 * R * T;     // one group of T threads per line (3 fields x R)
    static constexpr int S = padded_len<float>(N, T < Bank<float>::W ? T : 1);
    static constexpr int PTS = R * N;        // points per CTA
    static constexpr int PPT = (PTS + NT - 1) / NT;
    static_assert(3 * R * N == E * NT, "each gather moves E points per thread");
    static constexpr size_t buf = size_t(3) * R * S * sizeof(float2);  // one of Rbuf, Cbuf
    static constexpr size_t smem = 2 * buf + size_t(7) * N * sizeof(float4);
};

// The (dT, C) of one point at map layers lmin, lmin + 1, lmin + 2, in
// registers; stage points fall between lmin and lmin + 2.
struct RegPointSampler {
    float2 v0, v1, v2;
    int lmin;
    SHG_D float2 at(int l, float t) const {
        const bool up = l != lmin;
        const float2 a = up ? v1 : v0, b = up ? v2 : v1;
        return make_float2(a.x + t * (b.x - a.x), a.y + t * (b.y - a.y));
    }
};

template <int N, int K>
__global__ void __launch_bounds__(Cluster3Geom<N, K>::NT, 1)
    k_cluster3(const Inst3<float>* __restrict__ qs, int nz, const float4* __restrict__ tw) {
    namespace cg = cooperative_groups;
    using G = Cluster3Geom<N, K>;
    constexpr int R = G::R, V = G::V, E = G::E, T = G::T, NT = G::NT, S = G::S, PPT = G::PPT;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Inst3<float> qsh;
    __shared__ StageZ<float> zsh[2][5];  // stage data of step s in zsh[s & 1]
    float2* Rbuf = reinterpret_cast<float2*>(smem_raw);              // [3][R][S] rows
    float2* Cbuf = reinterpret_cast<float2*>(smem_raw + G::buf);     // [3][R][S] columns
    float4* twS = reinterpret_cast<float4*>(smem_raw + 2 * G::buf);  // [N]
    float4* pxS = twS + N;                                           // [3][N]
    float4* pyS = pxS + 3 * N;                                       // [3][N]
    const int tid = threadIdx.x;
    const int cid = int(cluster.block_rank());
    const int y0 = cid * R;
    const Inst3<float>& qg = qs[blockIdx.y];
    // constant tables and this CTA's rows of the three fields
    for (int k = tid; k < 7 * N; k += NT) {
        if (k < N)
            cp_async(&twS[tw_pos<N>(k)], &tw[k * (1024 / N)]);
        else if (k < 4 * N)
            cp_async(&pxS[k - N], &qg.d.px[k - N]);
        else
            cp_async(&pyS[k - 4 * N], &qg.d.py[k - 4 * N]);
    }
    for (int e = tid; e < 3 * R * N; e += NT) {
        const int x = e % N, r = (e / N) % R, f = e / (R * N);
        cp_async(&Rbuf[(f * R + r) * S + pidx<float>(x)],
                 &qg.d.field[(size_t(f) * N + y0 + r) * N + x]);
    }
    if (tid == 0) qsh = qg;
    cp_async_wait_all();
    __syncthreads();
    const Inst3<float>& q = qsh;
    const InstDesc<float>& d = q.d;
    const bool thermal = d.ttab != nullptr;  // the launcher admits only the per-point table then
    const float* __restrict__ umapf = reinterpret_cast<const float*>(d.umap);
    const float h = 0.5f * d.dz;
    // transform group of this thread: line g of the buffer, field g / R
    const int g = tid / T, t = tid - g * T;
    const int gf = g / R;
    auto stage = [&](int s) {
        if (tid < 5) {
            const int qz = 4 * s - 2 + tid;
            zsh[s & 1][tid] = stage_z(d, qz < 0 ? 0 : (qz > 4 * nz ? 4 * nz : qz));
        }
    };
    // Point p of this thread in the layout of step s: in rows (s even) point x
    // of row y0 + r at Rbuf[f][r][x]; in columns (s odd) row y of column
    // y0 + c at Cbuf[f][c][y], the R columns of one row on consecutive threads.
    auto point_of = [&](bool rows_l, int p, float2*& e, int& x, int& y) {
        if (rows_l) {
            const int r = p / N;
            x = p - r * N;
            y = y0 + r;
            e = Rbuf + r * S + pidx<float>(x);
        } else {
            const int c = p % R;
            y = p / R;
            x = y0 + c;
            e = Cbuf + c * S + pidx<float>(y);
        }
    };
    // Table entries of this thread's points for the (at most three) map
    // layers that step s's stage points fall between, one step ahead.  The
    // table is pair-interleaved: (dT_2j, dT_2j+1, C_2j, C_2j+1) at [l][y][j].
    float2 tv[PPT][3];
#pragma unroll
    for (int i = 0; i < PPT; ++i) tv[i][0] = tv[i][1] = tv[i][2] = make_float2(0.f, 0.f);
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
            const int p = tid + NT * i;
            if (p < G::PTS) {
                float2* e;
                int x, y;
                point_of((s & 1) == 0, p, e, x, y);
                const float* src = umapf + ((size_t(l0) * N + y) * (N / 2) + (x >> 1)) * 4 + (x & 1);
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (k < nl) {
                        const float* sk = src + size_t(k) * 2 * N * N;
                        tv[i][k] = make_float2(__ldg(sk), __ldg(sk + 2));
                    }
            }
        }
    };
    // F^-1 diag(p) F along the rows (Lx, factors pxS) or the columns (Ly,
    // pyS) held in buf.
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
    // Transposes through distributed shared memory, all remote loads of a
    // thread before its local stores.  Columns: Cbuf[f][c][y] = element
    // y0 + c of row y, held by CTA y / R.
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
        // ---- nonlinear half steps on this CTA's points
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            const int p = tid + NT * i;
            if (p < G::PTS) {
                float2* e;
                int x, y;
                point_of(rows_l, p, e, x, y);
                float2 A[3];
#pragma unroll
                for (int f = 0; f < 3; ++f) A[f] = e[f * R * S];
                RegPointSampler ps{tv[i][0], tv[i][1], tv[i][2], lmin};
                const Coef3<float> cz = coef3_at(q, zs[2], thermal, ps);
                if (s > 0) {
                    const Coef3<float> c0 = coef3_at(q, zs[0], thermal, ps);
                    const Coef3<float> cm = coef3_at(q, zs[1], thermal, ps);
                    rk4_3(q, A, c0, cm, cz, h);
                }
                if (s < nz) {
                    const Coef3<float> cm = coef3_at(q, zs[3], thermal, ps);
                    const Coef3<float> c1 = coef3_at(q, zs[4], thermal, ps);
                    rk4_3(q, A, cz, cm, c1, h);
                }
#pragma unroll
                for (int f = 0; f < 3; ++f) e[f * R * S] = A[f];
            }
        }
        // the next step's stage data and table entries, in flight during the
        // transforms (zsh[(s + 1) & 1] was last read in step s - 1)
        if (s < nz) {
            stage(s + 1);
            load_tables(s + 1);
        }
        __syncthreads();
        if (s == nz) break;  // the last pass is N_b alone
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
        __syncthreads();  // the next step's points were transformed by other groups
    }
    // the final state to global memory, from the layout of step nz
    if ((nz & 1) == 0) {
        for (int e = tid; e < 3 * R * N; e += NT) {
            const int x = e % N, r = (e / N) % R, f = e / (R * N);
            d.field[(size_t(f) * N + y0 + r) * N + x] = Rbuf[(f * R + r) * S + pidx<float>(x)];
        }
    } else {
        for (int e = tid; e < 3 * R * N; e += NT) {
            const int c = e % R, y = (e / R) % N, f = e / (R * N);
            d.field[(size_t(f) * N + y) * N + y0 + c] = Cbuf[(f * R + c) * S + pidx<float>(y)];
        }
    }
    cluster.sync();  // no CTA leaves while another may still read its buffers
}

}  // namespace shg
