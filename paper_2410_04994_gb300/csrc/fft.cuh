// Batched complex FFTs for the split-step passes, held in registers.
//
// A length-N transform is spread over T = N/E threads that each hold E
// elements; thread t holds positions t + T*m, m = 0..E-1.  The transform is
// the Stockham autosort formulation (Govindaraju et al., "High performance
// discrete Fourier transforms on graphics processors", SC 2008): stage s of
// radix R and stride Ns takes butterfly j from positions j + r N/R, multiplies
// by W_{Ns R}^{(j mod Ns) r}, does an R-point DFT in registers and writes to
// (j/Ns) Ns R + (j mod Ns) + r Ns.  The first stage's inputs and the last
// stage's outputs are exactly the thread's own positions t + T*m, so a
// transform needs (stages - 1) shared-memory exchanges and its result stays
// in registers in natural order, ready for the K-space multiply and the
// inverse transform.
//
// Stage twiddles come from one table W_1024^k = exp(-2 pi i k / 1024),
// computed in double precision on the host and kept as (hi, lo) float pairs
// (plainly rounded entries still left a measurable power drift over
// thousands of steps).
#pragma once
#include "common.cuh"

namespace shg {

// Sizes handled per thread and the radix sequence of each transform length.
// Variant V = 0 is the default shape; V = 1 is an alternative with 8 elements
// per thread (fewer registers, more resident CTAs) that the launcher's
// autotuner may pick per size and pass.
template <class R, int N, int V = 0> struct FftCfg;
#define SHG_FFT_CFG_V(RT, NN, VV, EE, R0_, R1_, R2_, R3_)                              \
    template <> struct FftCfg<RT, NN, VV> {                                            \
        static constexpr int E = EE, T = NN / EE, R0 = R0_, R1 = R1_, R2 = R2_, R3 = R3_; \
        static constexpr int NST = 1 + (R1_ > 1) + (R2_ > 1) + (R3_ > 1);              \
        static_assert(R0_ * R1_ * R2_ * R3_ == NN, "radices must multiply to N");      \
    };
#define SHG_FFT_CFG(RT, NN, EE, R0_, R1_, R2_, R3_) SHG_FFT_CFG_V(RT, NN, 0, EE, R0_, R1_, R2_, R3_)
SHG_FFT_CFG(float, 8, 8, 8, 1, 1, 1)
SHG_FFT_CFG(float, 16, 16, 16, 1, 1, 1)
SHG_FFT_CFG(float, 32, 16, 16, 2, 1, 1)
SHG_FFT_CFG(float, 64, 16, 16, 4, 1, 1)
SHG_FFT_CFG(float, 128, 16, 16, 8, 1, 1)
SHG_FFT_CFG(float, 256, 16, 16, 16, 1, 1)
SHG_FFT_CFG(float, 512, 8, 8, 8, 8, 1)
SHG_FFT_CFG(float, 1024, 8, 8, 8, 8, 2)
SHG_FFT_CFG(double, 8, 8, 8, 1, 1, 1)
SHG_FFT_CFG(double, 16, 8, 8, 2, 1, 1)
SHG_FFT_CFG(double, 32, 8, 8, 4, 1, 1)
SHG_FFT_CFG(double, 64, 8, 8, 8, 1, 1)
SHG_FFT_CFG(double, 128, 8, 8, 8, 2, 1)
SHG_FFT_CFG(double, 256, 8, 8, 8, 4, 1)
SHG_FFT_CFG_V(float, 64, 1, 8, 8, 8, 1, 1)
SHG_FFT_CFG_V(float, 128, 1, 8, 8, 8, 2, 1)
SHG_FFT_CFG_V(float, 256, 1, 8, 8, 8, 4, 1)
#undef SHG_FFT_CFG
#undef SHG_FFT_CFG_V

// Shared-memory padding: one spare element per bank row so that the strided
// Stockham stores spread over all banks (16 float2 or 8 double2 per 128 B).
template <class R> struct Bank;
template <> struct Bank<float> { static constexpr int SH = 4, W = 16; };
template <> struct Bank<double> { static constexpr int SH = 3, W = 8; };
template <class R> SHG_HD int pidx(int a) { return a + (a >> Bank<R>::SH); }

// Length of one transform's padded buffer, congruent to `lanes_mod` modulo
// the bank width so that neighbouring groups in a half-warp use other banks.
template <class R> constexpr int padded_len(int n, int lanes_mod) {
    int s = n + (n >> Bank<R>::SH) + 1;
    int w = Bank<R>::W;
    int want = ((lanes_mod % w) + w) % w;
    while (s % w != want) ++s;
    return s;
}

// Products by the DFT constants.  In single precision every non-trivial
// constant is applied as an unevaluated (hi + lo) float pair, so that the
// product is rounded once from the exact value: rounding the constant itself
// to FP32 would change |W| by up to ~6e-8 (1/sqrt(2) -> |W|^2 = 1 - 6e-8),
// a bias that the split-step march would accumulate linearly, step after step.
SHG_D float2 pmulc(float2 a, float4 p) {  // a * conj(p_hi + p_lo)
    float2 r;
    r.x = fmaf(a.x, p.x, fmaf(a.y, p.y, fmaf(a.x, p.z, a.y * p.w)));
    r.y = fmaf(a.y, p.x, fmaf(-a.x, p.y, fmaf(a.y, p.z, -a.x * p.w)));
    return r;
}
SHG_D double2 pmulc(double2 a, double2 p) {
    return make_double2(a.x * p.x + a.y * p.y, a.y * p.x - a.x * p.y);
}

template <class R> struct W16K;
template <> struct W16K<float> {
    static constexpr double H = 0.70710678118654752440, C1 = 0.92387953251128675613,
                            S1 = 0.38268343236508977173;
    static constexpr float Hh = float(H), Hl = float(H - double(float(H)));
    static constexpr float C1h = float(C1), C1l = float(C1 - double(float(C1)));
    static constexpr float S1h = float(S1), S1l = float(S1 - double(float(S1)));
};

SHG_D float scale_h(float u) { return fmaf(u, W16K<float>::Hh, u * W16K<float>::Hl); }
SHG_D double scale_h(double u) { return u * 0.70710678118654752440; }

// d * exp(dir * 2 pi i k / 16), dir = -1 forward, +1 inverse.
template <int DIR, class C> SHG_D C mul_w16(C d, int k) {
    using R = decltype(C::x);
    k &= 15;
    if (k == 0) return d;
    if (k == 4) return DIR < 0 ? mk<C>(d.y, -d.x) : mk<C>(-d.y, d.x);
    if (k == 8) return mk<C>(-d.x, -d.y);
    if (k == 12) return DIR < 0 ? mk<C>(-d.y, d.x) : mk<C>(d.y, -d.x);
    if ((k & 1) == 0) {
        // k = 2, 6, 10, 14: |cos| = |sin| = 1/sqrt(2)
        const R sc = (k == 2 || k == 14) ? R(1) : R(-1);           // sign of cos
        R ss = (k == 2 || k == 6) ? R(1) : R(-1);                  // sign of sin
        if (DIR < 0) ss = -ss;
        return mk<C>(scale_h(sc * d.x - ss * d.y), scale_h(ss * d.x + sc * d.y));
    }
    // odd k: (|cos|, |sin|) = (cos pi/8, sin pi/8) or swapped
    const bool big_c = (k == 1 || k == 7 || k == 9 || k == 15);
    const R sc = (k <= 4 || k >= 12) ? R(1) : R(-1);
    R ss = (k < 8) ? R(1) : R(-1);
    if (DIR < 0) ss = -ss;
    if constexpr (sizeof(R) == 4) {
        using K = W16K<float>;
        const float ch = big_c ? K::C1h : K::S1h, cl = big_c ? K::C1l : K::S1l;
        const float sh = big_c ? K::S1h : K::C1h, sl = big_c ? K::S1l : K::C1l;
        return pmul(d, make_float4(sc * ch, ss * sh, sc * cl, ss * sl));
    } else {
        const double c = big_c ? 0.92387953251128675613 : 0.38268343236508977173;
        const double s = big_c ? 0.38268343236508977173 : 0.92387953251128675613;
        return pmul(d, make_double2(sc * c, ss * s));
    }
}

// In-register R-point DFT (R = 2, 4, 8, 16), natural order in and out:
// radix-2 decimation in frequency, then a register renaming by bit reversal.
template <int R, int DIR, class C> SHG_D void dft_reg(C (&u)[R]) {
#pragma unroll
    for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * half) {
#pragma unroll
            for (int i = 0; i < half; ++i) {
                C a = u[b + i], c = u[b + i + half];
                u[b + i] = cadd(a, c);
                u[b + i + half] = mul_w16<DIR>(csub(a, c), i * (16 / (2 * half)));
            }
        }
    }
    C o[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        int r = 0;
#pragma unroll
        for (int bit = 1, rb = R >> 1; bit < R; bit <<= 1, rb >>= 1)
            if (k & bit) r |= rb;
        o[k] = u[r];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) u[k] = o[k];
}

// Where the constant tables of a transform live.  TL = 0: the plan's tables
// in global memory, twiddles W_1024^k (read through the read-only cache).
// TL = N > 0: copies in shared memory, twiddles W_N^k, k < N (so that
// streamed tiles cannot evict them from L1).
template <int TL> constexpr int tab_len() { return TL == 0 ? 1024 : TL; }

// Position of twiddle k in a shared table (TL > 0).  A stage reads entries
// jm r (times a stride) with jm = 0 .. NS-1 across the lanes of a row group;
// for even r those fall into a few of the eight 16-byte bank groups of a
// 128-byte shared-memory row ((hi, lo) pairs are 16 bytes), up to 8 ways for
// r = 8.  XOR-ing bits 0-2 of k with bits 3-5 spreads every such run over all
// eight groups.  It permutes each aligned block of 64 entries (or the whole
// table when N < 64), so the table keeps its size.
template <int TL> SHG_HD int tw_pos(int k) { return TL == 0 ? k : (k ^ ((k >> 3) & 7)); }
template <int TL, class P> SHG_D P ld_tab(const P* p) {
    if constexpr (TL == 0)
        return __ldg(p);
    else
        return *p;
}

// One Stockham stage on the thread's E registers.
template <int N, int E, int T, int R, int NS, bool LAST, int DIR, int TL, class C>
SHG_D void stage(C (&v)[E], C* sm, int t, const pt<decltype(C::x)>* __restrict__ tw) {
    using RT = decltype(C::x);
    constexpr int B = E / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + T * b;
        C u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = v[b + r * B];
        const int jm = j & (NS - 1);
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const auto w = ld_tab<TL>(&tw[tw_pos<TL>(jm * r * (tab_len<TL>() / (NS * R)))]);
                u[r] = DIR < 0 ? pmul(u[r], w) : pmulc(u[r], w);
                // bound the number of (hi, lo) twiddles the compiler keeps in
                // flight: without this it hoists them all and spills
                if ((r & 3) == 3) asm volatile("" ::: "memory");
            }
        }
        dft_reg<R, DIR>(u);
        if (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * B] = u[r];
        } else {
            const int base = (j / NS) * NS * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[pidx<RT>(base + r * NS)] = u[r];
        }
    }
}

template <int E, int T, class C> SHG_D void reload(C (&v)[E], const C* sm, int t) {
    using RT = decltype(C::x);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = sm[pidx<RT>(t + T * m)];
}

// Barrier between the exchanges of a transform group.  WS: the group's
// threads are consecutive and lie within one warp (T <= 32, group = thread
// index / T), so the warp barrier orders its shared-memory exchanges;
// otherwise (groups strided across warps) the block barrier.
template <bool WS> SHG_D void group_sync() {
    if constexpr (WS)
        __syncwarp();
    else
        __syncthreads();
}

// Forward (DIR = -1) or inverse (DIR = +1, unnormalised) transform of one
// sequence held as E registers per thread.  Every thread of the block (WS:
// of the warp) must call this (it contains the barriers of group_sync).
template <class RT, int N, int V, int DIR, int TL = 0, bool WS = false, class C>
SHG_D void fft1(C (&a)[FftCfg<RT, N, V>::E], C* sa, int t, const pt<RT>* __restrict__ tw) {
    using F = FftCfg<RT, N, V>;
    constexpr int E = F::E, T = F::T;
    constexpr int R0 = F::R0, R1 = F::R1, R2 = F::R2, R3 = F::R3;
    constexpr bool L0 = (F::NST == 1), L1 = (F::NST == 2), L2 = (F::NST == 3);
    static_assert(!WS || T <= 32, "a warp-synchronous group lies within one warp");
    stage<N, E, T, R0, 1, L0, DIR, TL>(a, sa, t, tw);
    if constexpr (F::NST >= 2) {
        group_sync<WS>();
        reload<E, T>(a, sa, t);
        group_sync<WS>();
        stage<N, E, T, (R1 > 1 ? R1 : 2), R0, L1, DIR, TL>(a, sa, t, tw);
    }
    if constexpr (F::NST >= 3) {
        group_sync<WS>();
        reload<E, T>(a, sa, t);
        group_sync<WS>();
        stage<N, E, T, (R2 > 1 ? R2 : 2), R0 * R1, L2, DIR, TL>(a, sa, t, tw);
    }
    if constexpr (F::NST >= 4) {
        group_sync<WS>();
        reload<E, T>(a, sa, t);
        group_sync<WS>();
        stage<N, E, T, (R3 > 1 ? R3 : 2), R0 * R1 * R2, true, DIR, TL>(a, sa, t, tw);
    }
}

// FFT -> multiply by the per-bin factors p[k] -> inverse FFT, i.e. the 1-D
// linear operator F^{-1} diag(p) F along the thread group's axis.  The 1/N of
// the inverse is folded into the factor table.  No barrier is needed between
// the two transforms: every thread has passed the barrier that follows the
// forward transform's last reload before any inverse store happens.  With
// TL = N the twiddles (W_N^k) and the factors p are read from shared memory.
template <class RT, int N, int V = 0, int TL = 0, bool WS = false, class C>
SHG_D void fft_mul_ifft(C (&a)[FftCfg<RT, N, V>::E], C* sa, int t, const pt<RT>* __restrict__ tw,
                        const pt<RT>* __restrict__ p) {
    using F = FftCfg<RT, N, V>;
    constexpr int E = F::E, T = F::T;
    fft1<RT, N, V, -1, TL, WS>(a, sa, t, tw);
#pragma unroll
    for (int m = 0; m < E; ++m) a[m] = pmul(a[m], ld_tab<TL>(&p[t + T * m]));
    fft1<RT, N, V, +1, TL, WS>(a, sa, t, tw);
}

// Copy the twiddles W_N^k (every (1024/N)-th entry of the plan's table) and
// the 2N factors of both fields into shared memory (cp.async, 16 B each; the
// caller commits and waits, then synchronises the block).
template <class RT, int N>
SHG_D void stage_tables(pt<RT>* twS, pt<RT>* pS, const pt<RT>* tw, const pt<RT>* p) {
    for (int k = threadIdx.x; k < 3 * N; k += blockDim.x) {
        if (k < N)
            cp_async(&twS[tw_pos<N>(k)], &tw[k * (1024 / N)]);
        else
            cp_async(&pS[k - N], &p[k - N]);
    }
}

}  // namespace shg
