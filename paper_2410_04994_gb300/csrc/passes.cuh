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
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"
#include "nonlinear.cuh"
#include "tma.cuh"

namespace shg {

constexpr int kPassThreads = 256;

// Resident CTAs per SM the launch is compiled for (register budget).
template <int V> struct MinBlocks { static constexpr int value = V == 0 ? 2 : 3; };

// Per-thread prefetch slots of the per-point temperature table (FP32): two
// buffers x up to three map layers x one float4 (the point pair of one loop
// iteration).
constexpr int kSlotLayers = 3;
template <class R, int NTH = kPassThreads> constexpr size_t slot_bytes() {
    return sizeof(R) == 4 ? size_t(2) * kSlotLayers * NTH * sizeof(float4) : 0;
}

template <class R, int N, int V = 0, int NTH = kPassThreads> struct RowGeom {
    using F = FftCfg<R, N, V>;
    static constexpr int T = F::T;
    static constexpr int ROWS = NTH / T;  // rows per CTA of NTH threads
    static constexpr int S = padded_len<R>(N, T < Bank<R>::W ? T : 1);
    static constexpr size_t fields = size_t(2) * ROWS * S * sizeof(cx<R>);
    static constexpr size_t tables = size_t(3) * N * sizeof(pt<R>);  // twiddles + 2 factor rows
};


template <class R, int N, int V = 0, int NTH = kPassThreads> struct ColGeom {
    using F = FftCfg<R, N, V>;
    static constexpr int T = F::T;
    static constexpr int TILE = NTH / T;  // columns per CTA of NTH threads
    static constexpr int S = padded_len<R>(N, TILE < Bank<R>::W ? Bank<R>::W / TILE : 1);
    static constexpr size_t fields = size_t(2) * TILE * S * sizeof(cx<R>);
    static constexpr size_t smem = fields + size_t(3) * N * sizeof(pt<R>);  // + twiddles, factors
};

// Where the row pass reads the temperature map from ([tz][ty][tx] storage with
// the given strides, node (l0, iy0, ix0) at `base`).
template <class R> struct MapView {
    const cx<R>* base;
    int stride, plane, l0, iy0, ix0;
};

// Map row cell of field row y (the same for every point of the row).
template <class R> struct RowCell {
    int iy;
    R fy;
};
template <class R> SHG_D RowCell<R> row_cell(const InstDesc<R>& d, int y) {
    RowCell<R> rc;
    lin_cell<R>((d.y0 + d.dy * R(y) - d.ty0) * d.tdy_inv, d.ty, rc.iy, rc.fy);
    return rc;
}

// Temperature-map sampler for field point (xi, y).
template <class R>
SHG_D void make_sampler(const InstDesc<R>& d, const MapView<R>& mv, int xi, const RowCell<R>& rc,
                        TempSampler<R>& ts) {
    int ix;
    R fx;
    lin_cell<R>((d.x0 + d.dx * R(xi) - d.tx0) * d.tdx_inv, d.tx, ix, fx);
    const int iy = rc.iy;
    const R fy = rc.fy;
    ts.base = mv.base + (iy - mv.iy0) * mv.stride + (ix - mv.ix0);
    ts.tx = mv.stride;
    ts.plane = mv.plane;
    ts.l0 = mv.l0;
    ts.fx = fx;
    ts.fy = fy;
    ts.la = -2;
}

// Copy (cp.async, one group, L2 evict-first) the per-point table entries of
// map layers lmin .. lmin + nl - 1 for the point pair (2j, 2j + 1) of row y
// into the calling thread's slots: layer k at slots[k * NTH + thread].
template <int NX, int NTH>
SHG_D void prefetch_slots(float4* slots, const float4* umap, int lmin, int nl, int ny, int y, int j) {
    const uint64_t pol = l2_evict_first_policy();
#pragma unroll 1
    for (int k = 0; k < nl; ++k) {
        const int o = ((lmin + k) * ny + y) * (NX / 2) + j;  // < 2^31: the table is <= 4 GiB
        cp_async_stream(slots + k * NTH + threadIdx.x, umap + o, pol);
    }
    cp_async_commit();
}

// Row pass R(s).  grid = (ceil(ny / ROWS), instances); block = NTH (256, or
// 128 for half as many rows per CTA).
//
// The CTA's rows of both fields are copied into padded shared buffers with
// cp.async (all copies in flight at once).  The nonlinear part runs on the
// shared copy in a rolled loop, so that no register array is indexed
// dynamically: iteration i of thread t advances the adjacent points 2j and
// 2j + 1, j = t + T*i (in FP32 together, in packed arithmetic).  The
// transforms then run field by field from the same buffers, each thread on
// the points x = t + T*m.  With a
// per-point temperature table (FP32), the (dT, C) of the map layers that this
// step's stage points fall between are streamed from it by cp.async into
// per-thread slots one loop iteration ahead (UM: the launcher has checked
// that every instance with a map has that table and that one step spans less
// than one map layer, so at most three layers are touched); otherwise each
// point samples the node table bilinearly.  The heat deposit at z_s (THERMAL plans) is binned
// per CTA in shared memory and added to the heat grid with one
// double-precision atomic per touched node.
// ZS = false: the instantiation for groups without power monitors (the
// monitor's code at z_s is compiled out; the heat deposit stays a runtime
// branch: removing it too made the compiler spill in the 256-point kernel).
// PRE = true: the row-layout pass of the one-pass-per-step schedule
// (k_col_step below), which applies Lx to the staged rows before the
// nonlinear part as well: the second half of L(s-1) = Ly Lx, then N_b(s-1),
// N_a(s), then the first half of L(s) = Lx Ly.
template <class R, int NX, int V = 0, bool UM = false, int NTH = kPassThreads, bool ZS = true,
          bool PRE = false>
__global__ void __launch_bounds__(NTH, MinBlocks<V>::value * (kPassThreads / NTH))
    k_row_pass(const InstDesc<R>* __restrict__ descs, int ny, int nz, int s,
               const pt<R>* __restrict__ tw) {
    using C = cx<R>;
    using G = RowGeom<R, NX, V, NTH>;
    constexpr int E = FftCfg<R, NX, V>::E, T = G::T, ROWS = G::ROWS, S = G::S;
    // A row's T threads are consecutive: with T <= 32 they share a warp, and
    // everything that passes between them (staged points, transform
    // exchanges, the nonlinear part's pairs) needs only the warp barrier.
    constexpr bool WS = T <= 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ InstDesc<R> dsh;
    __shared__ StageZ<R> zsh[5];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int lr = threadIdx.x / T, t = threadIdx.x - (threadIdx.x / T) * T;
    const int y = blockIdx.x * ROWS + lr;
    const bool active = y < ny;
    C* sF = smem + lr * S;
    C* sS = smem + (ROWS + lr) * S;
    // shared copies of the twiddles and of the row factors of both fields
    pt<R>* twS = reinterpret_cast<pt<R>*>(smem_raw + G::fields + (UM ? slot_bytes<R, NTH>() : 0));
    pt<R>* pS = twS + NX;
    {
        // constant tables first: they do not depend on the previous kernel
        const InstDesc<R>& dg = descs[blockIdx.y];
        stage_tables<R, NX>(twS, pS, tw, dg.px);
        if (threadIdx.x == 0) dsh = dg;
        if (threadIdx.x < 5) {
            const int q = 4 * s - 2 + threadIdx.x;
            zsh[threadIdx.x] = stage_z(dg, q < 0 ? 0 : (q > 4 * nz ? 4 * nz : q));
        }
        pdl_wait();  // the fields are the previous pass's output
        pdl_trigger();
        C* rowF = dg.field + size_t(y) * NX;
        C* rowS = dg.field + (size_t(ny) + y) * NX;
        if (active) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                cp_async(&sF[pidx<R>(t + T * m)], &rowF[t + T * m]);
                cp_async(&sS[pidx<R>(t + T * m)], &rowS[t + T * m]);
            }
        }
    }
    const bool dep = descs[blockIdx.y].Q != nullptr;
    float4* slots = reinterpret_cast<float4*>(smem_raw + G::fields);
    const float4* umap4 = reinterpret_cast<const float4*>(descs[blockIdx.y].umap);
    float* bins = reinterpret_cast<float*>(pS + 2 * NX);
    const int nb = dep ? ROWS * descs[blockIdx.y].hx : 0;
    for (int i = threadIdx.x; i < nb; i += NTH) bins[i] = 0.f;
    __syncthreads();
    const InstDesc<R>& d = dsh;
    const bool thermal = d.ttab != nullptr;
    const MapView<R> mv{d.ttab, d.tx, d.tx * d.ty, 0, 0, 0};
    // Layers lmin .. lmin + nl - 1 hold every stage point of this pass (the
    // stage layers are non-decreasing in q).
    const int lmin = zsh[0].l, nl = zsh[4].l + 2 - zsh[0].l;
    const bool um = UM && thermal;
    if (um && (d.umap == nullptr || nl > kSlotLayers)) {  // excluded by the launcher
        cp_async_wait_all();
        if (threadIdx.x == 0 && d.status) atomicExch(d.status, int(SHG_ERR_STATE));
        return;
    }
    bool staged = false;
    if constexpr (UM) {
        if (um && active) {
            cp_async_commit();  // the field rows
            prefetch_slots<NX, NTH>(slots, umap4, lmin, nl, ny, y, t);
            cp_async_wait_group<1>();
            staged = true;
        }
    }
    if (!staged) cp_async_wait_all();
    __syncthreads();
    if constexpr (PRE) {
        // Lx on both staged rows (the rows of inactive threads are zeros)
#pragma unroll 1
        for (int f = 0; f < 2; ++f) {
            C* sb = f == 0 ? sF : sS;
            C v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<R>(t + T * m)] : mk<C>(R(0), R(0));
            group_sync<WS>();  // the transform's exchanges reuse the buffer
            fft_mul_ifft<R, NX, V, NX, WS>(v, sb, t, twS, pS + f * NX);
            if (active) {
#pragma unroll
                for (int m = 0; m < E; ++m) sb[pidx<R>(t + T * m)] = v[m];
            }
        }
        group_sync<WS>();  // the nonlinear part reads points other threads of the row transformed
    }
    const R h = R(0.5) * d.dz;
    const int l_dep = dep ? d.hlz[s] : -1;
    const int j_dep = (dep && active) ? d.hiy[y] : -1;
    const R w_dep = dep ? d.dxdy * d.dz * ((s == 0 || s == nz) ? R(0.5) : R(1)) : R(0);
    const RowCell<R> rc = thermal ? row_cell(d, y) : RowCell<R>{0, R(0)};
    // Heat deposit of one point at z_s.
    auto deposit = [&](int xi, const C& aF, const C& aS) {
        const int i = __ldg(&d.hix[xi]);
        if (i >= 0) {
            const R aF2 = aF.x * aF.x + aF.y * aF.y;
            const R aS2 = aS.x * aS.x + aS.y * aS.y;
            const R q = aF2 * (d.qaF + d.qbF * aF2) + aS2 * (d.qaS + d.qbS * aS2);
            atomicAdd(&bins[lr * d.hx + i], float(q * w_dep));
        }
    };
    // Power monitor: this thread's share of sum |A_F|^2, sum |A_SH|^2 at z_s.
    const bool mon = ZS && d.mon != nullptr && (s % d.mon_every == 0 || s == nz);
    R monF = R(0), monS = R(0);
    auto monitor = [&](const C& aF, const C& aS) {
        monF += aF.x * aF.x + aF.y * aF.y;
        monS += aS.x * aS.x + aS.y * aS.y;
    };
    // One point: N_b(s-1) [z_s - dz/2 -> z_s], deposit at z_s, N_a(s).
    auto point = [&](int xi, C& aF, C& aS, auto& ts) {
        const Coef<R> cz = coef_at(d, zsh[2], thermal, ts);  // z_s, shared by both halves
        if (s > 0) {
            const Coef<R> c0 = coef_at(d, zsh[0], thermal, ts);
            const Coef<R> cm = coef_at(d, zsh[1], thermal, ts);
            rk4(d, aF, aS, c0, cm, cz, h);
        }
        if (l_dep >= 0 && j_dep >= 0) deposit(xi, aF, aS);
        if (mon) monitor(aF, aS);
        if (s < nz) {
            const Coef<R> cm = coef_at(d, zsh[3], thermal, ts);
            const Coef<R> c1 = coef_at(d, zsh[4], thermal, ts);
            rk4(d, aF, aS, cz, cm, c1, h);
        }
    };
    // The same for two points at once in packed FP32 arithmetic, with the
    // stage coefficients of stage point q from cq(q) (the body exists for
    // FP32 only).
    auto pair_t = [&](auto tpa, int xa, int xb, auto& aF0, auto& aS0, auto& aF1, auto& aS1,
                      auto&& cq) {
        constexpr bool TPA = decltype(tpa)::value;
        if constexpr (sizeof(R) == 4) {
            const Coef2 z2 = cq(2);  // z_s, shared by both halves
            Cx2 F{pk2(aF0.x, aF1.x), pk2(aF0.y, aF1.y)}, S{pk2(aS0.x, aS1.x), pk2(aS0.y, aS1.y)};
            if (s > 0) {
                const Coef2 c0 = cq(0);
                const Coef2 cm = cq(1);
                rk4_2<TPA>(dsh, F, S, c0, cm, z2, h);
            }
            if ((l_dep >= 0 && j_dep >= 0) || mon) {
                up2(F.r, aF0.x, aF1.x);
                up2(F.i, aF0.y, aF1.y);
                up2(S.r, aS0.x, aS1.x);
                up2(S.i, aS0.y, aS1.y);
                if (l_dep >= 0 && j_dep >= 0) {
                    deposit(xa, aF0, aS0);
                    deposit(xb, aF1, aS1);
                }
                if (mon) {
                    monitor(aF0, aS0);
                    monitor(aF1, aS1);
                }
            }
            if (s < nz) {
                const Coef2 cm = cq(3);
                const Coef2 c1 = cq(4);
                rk4_2<TPA>(dsh, F, S, z2, cm, c1, h);
            }
            up2(F.r, aF0.x, aF1.x);
            up2(F.i, aF0.y, aF1.y);
            up2(S.r, aS0.x, aS1.x);
            up2(S.i, aS0.y, aS1.y);
        }
    };
    // the pump-TPA-free form where bF = 0 (uniform over the CTA's instance)
    auto pair = [&](int xa, int xb, auto& aF0, auto& aS0, auto& aF1, auto& aS1, auto&& cq) {
        if (dsh.bF != R(0))
            pair_t(std::true_type{}, xa, xb, aF0, aS0, aF1, aS1, cq);
        else
            pair_t(std::false_type{}, xa, xb, aF0, aS0, aF1, aS1, cq);
    };
    if (active) {
        // two adjacent points per iteration: in FP32 they advance together in
        // packed arithmetic; in FP64 they give the scheduler two RK4
        // dependency chains to interleave
#pragma unroll 1
        for (int i = 0; i < E / 2; ++i) {
            const int j = t + T * i, x0 = 2 * j, x1 = x0 + 1;
            C aF0 = sF[pidx<R>(x0)], aS0 = sS[pidx<R>(x0)];
            C aF1 = sF[pidx<R>(x1)], aS1 = sS[pidx<R>(x1)];
            if constexpr (UM) {
                const int buf = i & 1;
                if (um) {
                    if (i + 1 < E / 2) {
                        prefetch_slots<NX, NTH>(slots + (buf ^ 1) * kSlotLayers * NTH, umap4,
                                                lmin, nl, ny, y, j + T);
                        cp_async_wait_group<1>();
                    } else {
                        cp_async_wait_group<0>();
                    }
                }
                const PairSampler ps{slots + buf * kSlotLayers * NTH + threadIdx.x, NTH, lmin};
                pair(x0, x1, aF0, aS0, aF1, aS1,
                     [&](int q) { return coef2_at(dsh, zsh[q], thermal, ps); });
            } else if constexpr (sizeof(R) == 4) {
                TempSampler<R> s0, s1;
                if (thermal) {
                    make_sampler(d, mv, x0, rc, s0);
                    make_sampler(d, mv, x1, rc, s1);
                }
                pair(x0, x1, aF0, aS0, aF1, aS1, [&](int q) {
                    return pack2(coef_at(d, zsh[q], thermal, s0), coef_at(d, zsh[q], thermal, s1));
                });
            } else {
                {
                    TempSampler<R> s0;
                    if (thermal) make_sampler(d, mv, x0, rc, s0);
                    point(x0, aF0, aS0, s0);
                }
                {
                    TempSampler<R> s1;
                    if (thermal) make_sampler(d, mv, x1, rc, s1);
                    point(x1, aF1, aS1, s1);
                }
            }
            sF[pidx<R>(x0)] = aF0;
            sS[pidx<R>(x0)] = aS0;
            sF[pidx<R>(x1)] = aF1;
            sS[pidx<R>(x1)] = aS1;
        }
    }
    group_sync<WS>();  // the transforms read points that other threads of the row advanced
    if (mon) {
        // per-warp FP64 sums, one atomic pair per warp
        double vF = double(monF), vS = double(monS);
        for (int o = 16; o > 0; o >>= 1) {
            vF += __shfl_xor_sync(0xffffffffu, vF, o);
            vS += __shfl_xor_sync(0xffffffffu, vS, o);
        }
        if ((threadIdx.x & 31) == 0) {
            const int slot = (s % d.mon_every == 0) ? s / d.mon_every : d.mon_last;
            atomicAdd(&d.mon[2 * slot], vF);
            atomicAdd(&d.mon[2 * slot + 1], vS);
        }
    }
    if (dep) {
        __syncthreads();
        const int y0 = blockIdx.x * ROWS;
        for (int k = threadIdx.x; k < nb; k += NTH) {
            const float v = bins[k];
            if (v != 0.f && l_dep >= 0) {
                const int r = k / d.hx, i = k - r * d.hx;
                const int jj = d.hiy[y0 + r];
                atomicAdd(&d.Q[(size_t(l_dep) * d.hy + jj) * d.hx + i], double(v));
            }
        }
    }
    // Lx on each field in turn (none in the last pass); results to global.
#pragma unroll 1
    for (int f = 0; f < 2; ++f) {
        C* sb = f == 0 ? sF : sS;
        C* row = d.field + (size_t(f) * ny + y) * NX;
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<R>(t + T * m)] : mk<C>(R(0), R(0));
        if (s < nz) {
            group_sync<WS>();  // the transform's first stores reuse the staging buffer
            fft_mul_ifft<R, NX, V, NX, WS>(v, sb, t, twS, pS + f * NX);
        }
        if (active) {
#pragma unroll
            for (int m = 0; m < E; ++m) row[t + T * m] = v[m];
        }
    }
}

// Column pass C(s).  grid = (ceil(nx / TILE), instances); block = NTH (256;
// 128 or 64 for fewer columns per CTA and more resident CTAs; 512 at the
// lengths 512 and 1024 for twice the columns per CTA, so that each row
// segment a warp reads is a whole 32-byte sector).
// The TILE columns of both fields are staged into padded shared buffers with
// cp.async, one commit group per field, transformed field by field (the
// second field is still landing while the first is transformed), and written
// back from registers.
template <class R, int NY, int V = 0, int NTH = kPassThreads>
__global__ void __launch_bounds__(NTH, MinBlocks<V>::value * kPassThreads / NTH)
    k_col_pass(const InstDesc<R>* __restrict__ descs, int nx, const pt<R>* __restrict__ tw) {
    using C = cx<R>;
    using G = ColGeom<R, NY, V, NTH>;
    constexpr int E = FftCfg<R, NY, V>::E, T = G::T, TILE = G::TILE, S = G::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    pt<R>* twS = reinterpret_cast<pt<R>*>(smem_raw + G::fields);
    pt<R>* pS = twS + NY;
    C* field = descs[blockIdx.y].field;
    const int c = threadIdx.x % TILE, t = threadIdx.x / TILE;
    const int x = blockIdx.x * TILE + c;
    const bool active = x < nx;
    stage_tables<R, NY>(twS, pS, tw, descs[blockIdx.y].py);  // independent of the previous pass
    pdl_wait();
    pdl_trigger();
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        if (active) {
            const C* col = field + size_t(f) * NY * nx + x;
            C* sb = smem + (f * TILE + c) * S;
#pragma unroll
            for (int m = 0; m < E; ++m)
                cp_async(&sb[pidx<R>(t + T * m)], col + size_t(t + T * m) * nx);
        }
        cp_async_commit();
    }
#pragma unroll 1
    for (int f = 0; f < 2; ++f) {
        if (f == 0)
            cp_async_wait_group<1>();
        else
            cp_async_wait_group<0>();
        C* sb = smem + (f * TILE + c) * S;
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<R>(t + T * m)] : mk<C>(R(0), R(0));
        __syncthreads();  // all staged values read before the transform's stores
        fft_mul_ifft<R, NY, V, NY>(v, sb, t, twS, pS + f * NY);
        if (active) {
            C* col = field + size_t(f) * NY * nx + x;
#pragma unroll
            for (int m = 0; m < E; ++m) col[size_t(t + T * m) * nx] = v[m];
        }
    }
}

// Column-layout pass of the one-pass-per-step schedule.  Lx and Ly commute
// exactly (diagonal factors of a separable spectrum), so step s may apply
// L(s) as Lx Ly or as Ly Lx, and the nonlinear part, being pointwise, may run
// in either layout.  Pass s of the schedule applies the second half of
// L(s-1), then N_b(s-1) and N_a(s), then the first half of L(s): in the row
// layout for even s (k_row_pass with PRE: Lx, N, Lx) and in the column layout
// for odd s (here: Ly, N, Ly; no Ly after the last step).  That is nz + 1
// passes per propagation, each reading and writing both fields once, instead
// of 2 nz + 1.  FP32; per-point temperature table or uniform temperature; no
// monitor (the launcher checks).  The heat deposit at z_s (THERMAL plans) is
// binned per CTA in shared memory, [TILE][hy] (the heat-grid column of each
// field column is fixed, its row varies), and added to the heat grid with one
// double-precision atomic per touched node.  The TILE columns of both
// fields are staged as in k_col_pass.  Pair i of a thread is the columns
// (x0 + 2 jj, x0 + 2 jj + 1) of row y, whose table entry is
// [l][y][x0 / 2 + jj]; it is streamed into the thread's slots one iteration
// ahead, as in the row pass.  V: the transform shape (0: 16 elements per
// thread; 1: 8, in CTAs of which three fit per SM, with half the columns).
template <int NY, int NTH = kPassThreads, int V = 0>
__global__ void __launch_bounds__(NTH, MinBlocks<V>::value * kPassThreads / NTH)
    k_col_step(const InstDesc<float>* __restrict__ descs, int nx, int nz, int s,
               const pt<float>* __restrict__ tw) {
    using C = cx<float>;
    using G = ColGeom<float, NY, V, NTH>;
    constexpr int E = FftCfg<float, NY, V>::E, T = G::T, TILE = G::TILE, S = G::S;
    constexpr int NP = E / 2;  // pairs per thread
    static_assert((TILE / 2) * NY == NP * NTH, "whole pairs per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ InstDesc<float> dsh;
    __shared__ StageZ<float> zsh[5];
    C* smem = reinterpret_cast<C*>(smem_raw);                         // [2][TILE][S]
    float4* slots = reinterpret_cast<float4*>(smem_raw + G::fields);  // [2][layers][NTH]
    pt<float>* twS = reinterpret_cast<pt<float>*>(smem_raw + G::fields + slot_bytes<float, NTH>());
    pt<float>* pS = twS + NY;  // [2][NY]
    float* bins = reinterpret_cast<float*>(pS + 2 * NY);  // [TILE][hy] heat deposits
    const int c = threadIdx.x % TILE, t = threadIdx.x / TILE;
    const int x0 = blockIdx.x * TILE, x = x0 + c;
    const bool active = x < nx;
    const bool dep = descs[blockIdx.y].Q != nullptr;
    const int nb = dep ? TILE * descs[blockIdx.y].hy : 0;
    for (int i = threadIdx.x; i < nb; i += NTH) bins[i] = 0.f;
    {
        const InstDesc<float>& dg = descs[blockIdx.y];
        stage_tables<float, NY>(twS, pS, tw, dg.py);
        if (threadIdx.x == 0) dsh = dg;
        if (threadIdx.x < 5) {
            const int q = 4 * s - 2 + threadIdx.x;
            zsh[threadIdx.x] = stage_z(dg, q < 0 ? 0 : (q > 4 * nz ? 4 * nz : q));
        }
        pdl_wait();  // the fields are the previous pass's output
        pdl_trigger();
        if (active) {
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const C* col = dg.field + size_t(f) * NY * nx + x;
                C* sb = smem + (f * TILE + c) * S;
#pragma unroll
                for (int m = 0; m < E; ++m)
                    cp_async(&sb[pidx<float>(t + T * m)], col + size_t(t + T * m) * nx);
            }
        }
    }
    cp_async_commit();  // the field columns and the constant tables
    __syncthreads();    // dsh, zsh
    const InstDesc<float>& d = dsh;
    const bool thermal = d.ttab != nullptr;
    const float4* umap4 = reinterpret_cast<const float4*>(d.umap);
    const int lmin = zsh[0].l, nl = zsh[4].l + 2 - zsh[0].l;
    if (thermal && (d.umap == nullptr || nl > kSlotLayers)) {  // excluded by the launcher
        cp_async_wait_all();
        if (threadIdx.x == 0 && d.status) atomicExch(d.status, int(SHG_ERR_STATE));
        return;
    }
    // pair i of this thread: the columns x0 + 2 jj, x0 + 2 jj + 1 of row y
    auto pair_at = [&](int i, int& y, int& jj) {
        const int p = threadIdx.x + NTH * i;
        y = p / (TILE / 2);
        jj = p - y * (TILE / 2);
    };
    // the table entries of pair i (layers lmin .. lmin + nl - 1) into slot
    // buffer b, as one commit group
    auto prefetch = [&](int i, int b) {
        int y, jj;
        pair_at(i, y, jj);
        if (x0 + 2 * jj < nx) {
            const uint64_t pol = l2_evict_first_policy();
#pragma unroll 1
            for (int k = 0; k < nl; ++k) {
                const size_t o = (size_t(lmin + k) * NY + y) * size_t(nx / 2) + x0 / 2 + jj;
                cp_async_stream(slots + (b * kSlotLayers + k) * NTH + threadIdx.x, umap4 + o, pol);
            }
        }
        cp_async_commit();
    };
    if (thermal) {
        prefetch(0, 0);
        cp_async_wait_group<1>();
    } else {
        cp_async_wait_all();
    }
    __syncthreads();
    // Ly: the second half of L(s-1) (s >= 1 for every pass of this kernel)
#pragma unroll 1
    for (int f = 0; f < 2; ++f) {
        C* sb = smem + (f * TILE + c) * S;
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<float>(t + T * m)] : mk<C>(0.f, 0.f);
        __syncthreads();  // the transform's exchanges reuse the buffer
        fft_mul_ifft<float, NY, V, NY>(v, sb, t, twS, pS + f * NY);
        if (active) {
#pragma unroll
            for (int m = 0; m < E; ++m) sb[pidx<float>(t + T * m)] = v[m];
        }
    }
    __syncthreads();  // the pairs were transformed by other threads
    // N_b(s-1), the heat deposit at z_s, N_a(s), two adjacent columns per
    // iteration in packed FP32
    const float h = 0.5f * d.dz;
    const int l_dep = dep ? d.hlz[s] : -1;
    const float w_dep = dep ? d.dxdy * d.dz * ((s == 0 || s == nz) ? 0.5f : 1.f) : 0.f;
    auto deposit = [&](int xi, int y, const C& aF, const C& aS) {
        const int i = __ldg(&d.hix[xi]), j = __ldg(&d.hiy[y]);
        if (i >= 0 && j >= 0) {
            const float aF2 = aF.x * aF.x + aF.y * aF.y;
            const float aS2 = aS.x * aS.x + aS.y * aS.y;
            const float q = aF2 * (d.qaF + d.qbF * aF2) + aS2 * (d.qaS + d.qbS * aS2);
            atomicAdd(&bins[(xi - x0) * d.hy + j], q * w_dep);
        }
    };
#pragma unroll 1
    for (int i = 0; i < NP; ++i) {
        const int b = i & 1;
        if (thermal) {
            if (i + 1 < NP) {
                prefetch(i + 1, b ^ 1);
                cp_async_wait_group<1>();
            } else {
                cp_async_wait_group<0>();
            }
        }
        int y, jj;
        pair_at(i, y, jj);
        if (x0 + 2 * jj >= nx) continue;
        C* e0 = smem + (2 * jj) * S + pidx<float>(y);
        C* e1 = smem + (2 * jj + 1) * S + pidx<float>(y);
        C aF0 = e0[0], aF1 = e1[0], aS0 = e0[TILE * S], aS1 = e1[TILE * S];
        const PairSampler ps{slots + b * kSlotLayers * NTH + threadIdx.x, NTH, lmin};
        auto cq = [&](int q) { return coef2_at(dsh, zsh[q], thermal, ps); };
        Cx2 F{pk2(aF0.x, aF1.x), pk2(aF0.y, aF1.y)}, Sx{pk2(aS0.x, aS1.x), pk2(aS0.y, aS1.y)};
        const Coef2 z2 = cq(2);
        if (s > 0) {
            const Coef2 c0 = cq(0);
            const Coef2 cm = cq(1);
            rk4_2(dsh, F, Sx, c0, cm, z2, h);
        }
        if (l_dep >= 0) {
            up2(F.r, aF0.x, aF1.x);
            up2(F.i, aF0.y, aF1.y);
            up2(Sx.r, aS0.x, aS1.x);
            up2(Sx.i, aS0.y, aS1.y);
            deposit(x0 + 2 * jj, y, aF0, aS0);
            deposit(x0 + 2 * jj + 1, y, aF1, aS1);
        }
        if (s < nz) {
            const Coef2 cm = cq(3);
            const Coef2 c1 = cq(4);
            rk4_2(dsh, F, Sx, z2, cm, c1, h);
        }
        up2(F.r, aF0.x, aF1.x);
        up2(F.i, aF0.y, aF1.y);
        up2(Sx.r, aS0.x, aS1.x);
        up2(Sx.i, aS0.y, aS1.y);
        e0[0] = aF0;
        e1[0] = aF1;
        e0[TILE * S] = aS0;
        e1[TILE * S] = aS1;
    }
    __syncthreads();  // the transforms read points that other threads advanced
    if (l_dep >= 0) {
        // one double atomic per touched heat node
        for (int k = threadIdx.x; k < nb; k += NTH) {
            const float v = bins[k];
            if (v != 0.f) {
                const int cc = k / d.hy, j = k - cc * d.hy;
                const int i = __ldg(&d.hix[x0 + cc]);
                atomicAdd(&d.Q[(size_t(l_dep) * d.hy + j) * d.hx + i], double(v));
            }
        }
    }
    // Ly: the first half of L(s) (none after the last step); results to global
#pragma unroll 1
    for (int f = 0; f < 2; ++f) {
        C* sb = smem + (f * TILE + c) * S;
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = active ? sb[pidx<float>(t + T * m)] : mk<C>(0.f, 0.f);
        if (s < nz) {
            __syncthreads();
            fft_mul_ifft<float, NY, V, NY>(v, sb, t, twS, pS + f * NY);
        }
        if (active) {
            C* col = d.field + size_t(f) * NY * nx + x;
#pragma unroll
            for (int m = 0; m < E; ++m) col[size_t(t + T * m) * nx] = v[m];
        }
    }
}

// Column pass staged by TMA (FP32).  One elected thread issues 3-D box copies
// of the CTA's TILE columns of both fields ([field][row][column] boxes of up
// to 256 rows) from the instance's tensor map into a dense shared buffer, one
// mbarrier per field; before each field the block waits on its barrier with
// a bounded number of polls (on expiry it records SHG_ERR_TIMEOUT in the
// instance status, lets the issued copies land and returns).  Each field is
// then transformed from that buffer through one padded exchange buffer and
// written back from registers.  grid = (ceil(nx / TILE), instances).
template <int NY> struct ColTma {
    using G = ColGeom<float, NY, 0>;
    static constexpr int TILE = G::TILE, S = G::S, BY = NY < 256 ? NY : 256;
    static constexpr size_t stage_bytes = size_t(2) * NY * TILE * sizeof(float2);
    static constexpr size_t tables = size_t(3) * NY * sizeof(float4);
    static constexpr size_t smem = 128 + stage_bytes + size_t(TILE) * S * sizeof(float2) + tables + 16;
};

constexpr unsigned kTmaMaxPolls = 1u << 20;

template <int NY>
__global__ void __launch_bounds__(kPassThreads, 2)
    k_col_tma(const CUtensorMap* __restrict__ tmaps, const InstDesc<float>* __restrict__ descs,
              int nx, const pt<float>* __restrict__ tw) {
    using K = ColTma<NY>;
    using G = typename K::G;
    constexpr int E = FftCfg<float, NY, 0>::E, T = G::T, TILE = K::TILE, S = K::S, BY = K::BY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                              ~uintptr_t(127));
    float2* exch = stage + 2 * NY * TILE;
    float4* twS = reinterpret_cast<float4*>(exch + TILE * S);
    float4* pS = twS + NY;
    uint64_t* bar = reinterpret_cast<uint64_t*>(pS + 2 * NY);
    const InstDesc<float>& d = descs[blockIdx.y];
    const int x0 = blockIdx.x * TILE;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    stage_tables<float, NY>(twS, pS, tw, d.py);  // independent of the previous pass
    __syncthreads();
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) {
        // one barrier per field, so that field 0 is transformed while field 1 lands
        const CUtensorMap* tm = tmaps + blockIdx.y;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            mbar_arrive_expect_tx(&bar[f], unsigned(K::stage_bytes / 2));
#pragma unroll
            for (int yb = 0; yb < NY; yb += BY)
                tma_load_3d(stage + (size_t(f) * NY + yb) * TILE, tm, x0, yb, f, &bar[f]);
        }
    }
    cp_async_wait_all();
    const int c = threadIdx.x % TILE, t = threadIdx.x / TILE;
    const int x = x0 + c;
    const bool active = x < nx;
#pragma unroll 1
    for (int f = 0; f < 2; ++f) {
        const bool ok = mbar_wait_bounded(&bar[f], 0, d.wait_polls);
        if (__syncthreads_or(!ok)) {
            // Give up on this tile: report, then let the copies already issued
            // land (bounded again) before the CTA's shared memory is released.
            if (threadIdx.x == 0) {
                if (d.status) atomicExch(d.status, int(SHG_ERR_TIMEOUT));
                for (int g = f; g < 2; ++g) mbar_wait_bounded(&bar[g], 0, kTmaMaxPolls);
            }
            return;
        }
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = stage[(size_t(f) * NY + t + T * m) * TILE + c];
        fft_mul_ifft<float, NY, 0, NY>(v, exch + c * S, t, twS, pS + f * NY);
        if (active) {
            float2* col = d.field + size_t(f) * NY * nx + x;
#pragma unroll
            for (int m = 0; m < E; ++m) col[size_t(t + T * m) * nx] = v[m];
        }
    }
}

}  // namespace shg
