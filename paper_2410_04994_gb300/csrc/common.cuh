// Shared device-side definitions of the SHG split-step kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/shg.h"

#define SHG_HD __host__ __device__ __forceinline__
#define SHG_D __device__ __forceinline__

// ----------------------------------------------------------- complex ----
template <class R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <class R> using cx = typename Cx<R>::T;

// K-space factor entries: in single precision a (hi, lo) pair of float2 packed
// in a float4, so that the multiply is exact to rounding (no per-step bias
// from representing the factor in FP32); in double precision plain double2.
template <class R> struct PropT;
template <> struct PropT<float> { using T = float4; };
template <> struct PropT<double> { using T = double2; };
template <class R> using pt = typename PropT<R>::T;

SHG_HD float2 pmul(float2 a, float4 p) {
    float2 r;
    r.x = fmaf(a.x, p.x, fmaf(-a.y, p.y, fmaf(a.x, p.z, -a.y * p.w)));
    r.y = fmaf(a.x, p.y, fmaf(a.y, p.x, fmaf(a.x, p.w, a.y * p.z)));
    return r;
}
SHG_HD double2 pmul(double2 a, double2 p) {
    double2 r;
    r.x = a.x * p.x - a.y * p.y;
    r.y = a.x * p.y + a.y * p.x;
    return r;
}

template <class C> SHG_HD C mk(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <class C> SHG_HD C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <class C> SHG_HD C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
// Single precision: on the device both components in one packed f32x2
// instruction (rounded exactly as the two scalar ones).
template <> SHG_HD float2 cadd<float2>(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    float2 r;
    asm("{\n .reg .b64 a, b, r;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
        " add.rn.f32x2 r, a, b;\n mov.b64 {%0, %1}, r;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
#else
    return mk<float2>(a.x + b.x, a.y + b.y);
#endif
}
template <> SHG_HD float2 csub<float2>(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    float2 r;
    asm("{\n .reg .b64 a, b, r;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
        " sub.rn.f32x2 r, a, b;\n mov.b64 {%0, %1}, r;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
#else
    return mk<float2>(a.x - b.x, a.y - b.y);
#endif
}
template <class C> SHG_HD C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <class C> SHG_HD C cmulc(C a, C b) {
    return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <class C> SHG_HD C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
template <class C> SHG_HD C cconj(C a) { return mk<C>(a.x, -a.y); }

// ------------------------------------------------ phase-mismatch model ----
// Eq. (4): Dk(T) = (4 pi / lambda_F) (n_SH(T) - n_F(T)) - 2 pi / Lambda(T),
// Lambda(T) = Lambda(25 C) (1 + a (T - 25) + b (T - 25)^2), n_j(T) cubic
// polynomials in (T - 25 C).  `on` = 0 selects the linearised dk0 + g dT.
struct DkModel {
    int on;
    double t_oven;         // oven temperature (deg C)
    double t_ref;          // T_oven + T_off (deg C): the uniform part of the temperature
    double k_mat;          // 4 pi / lambda_F
    double lam25, a, b;    // grating period at 25 C and its expansion
    double nF[4], nS[4];   // index polynomial coefficients
};
SHG_HD double dk_eq4(const DkModel& m, double T) {
    const double u = T - 25.0;
    const double nF = m.nF[0] + u * (m.nF[1] + u * (m.nF[2] + u * m.nF[3]));
    const double nS = m.nS[0] + u * (m.nS[1] + u * (m.nS[2] + u * m.nS[3]));
    const double lam = m.lam25 * (1.0 + m.a * u + m.b * u * u);
    return m.k_mat * (nS - nF) - 6.283185307179586477 / lam;
}
// dDk/dT of Eq. (4) at T.
SHG_HD double dk_eq4_slope(const DkModel& m, double T) {
    const double u = T - 25.0;
    const double dF = m.nF[1] + u * (2.0 * m.nF[2] + 3.0 * u * m.nF[3]);
    const double dS = m.nS[1] + u * (2.0 * m.nS[2] + 3.0 * u * m.nS[3]);
    const double lam = m.lam25 * (1.0 + m.a * u + m.b * u * u);
    return m.k_mat * (dS - dF) + 6.283185307179586477 * m.lam25 * (m.a + 2.0 * m.b * u) / (lam * lam);
}
// The integrand of the map table's C channel at a node of temperature offset dT:
// dT itself (linearised model), or Dk(T_ref + dT) - Dk(T_ref) (Eq. 4).
SHG_HD double phase_integrand(const DkModel& m, double dT) {
    return m.on ? dk_eq4(m, m.t_ref + dT) - dk_eq4(m, m.t_ref) : dT;
}

// ------------------------------------------------------ per-instance ----
// Everything one pass needs about one instance; built on the host by the plan.
// Launch-variant bit of the row pass: read the per-point temperature table.
constexpr int kRowUmap = 8;  // above every flavour number (0-5)
// Launch bit of the row pass (with kRowUmap only): no instance of the group
// monitors its power, so the kernel is instantiated without that code.
constexpr int kRowLean = 16;

template <class R> struct InstDesc {
    cx<R>* field;          // [2][ny][nx]: A_F then A_SH
    const pt<R>* px;       // [2][nx] row factor exp(-i Kx^2 dz/2k_j) exp(-alpha_j dz/2) / nx
    const pt<R>* py;       // [2][ny] column factor exp(-i Ky^2 dz/2k_j) / ny
    const cx<R>* eph;      // [4 nz + 1] e^{i theta(q dz/4)}, theta = (dk0 + g T_off) z mod 2 pi
    const cx<R>* ttab;     // [tz][ty][tx] (dT, C) or nullptr for a uniform temperature
    const cx<R>* umap;     // FP32: every map layer bilinearly sampled at every field
                           // point, [tz][ny][nx/2] of (dT_2j, dT_2j+1, C_2j, C_2j+1),
                           // or nullptr (sample ttab in the pass)
    int tx, ty, tz;
    R tx0, tdx_inv, ty0, tdy_inv, tdz_inv;  // node 0 position and 1/spacing of the map
    R x0, dx, y0, dy;      // field sample positions x_m = x0 + m dx
    R kF, kS;              // coupling constants (1/V)
    R bF, bS;              // (1/2) beta_j (eps0 c n_j / 2): TPA factor per |A|^2
    R lF, lS;              // (2 pi / lambda_j) dn/dT: lens phase per kelvin
    R psi0F, psi0S;        // lens phase rate of the uniform offset T_off
    R g;                   // dDk/dT
    R dz;
    int undepleted;
    // heat deposits (THERMAL plans only)
    double* Q;             // [hz][hy][hx] sum of q_dot dV
    const int* hix;        // [nx] heat node of each column or -1
    const int* hiy;        // [ny]
    const int* hlz;        // [nz + 1] heat layer of each z_s or -1
    int hx, hy, hz;
    R qaF, qaS, qbF, qbS;  // alpha_j I-coefficient and beta_j I^2-coefficient per |A|^2, |A|^4
    R dxdy;
    int* status;           // set to a non-zero shg_status_t by a kernel that gave up
    unsigned wait_polls;   // bound on the polls of a device-side wait (0: give up at once)
    // power monitor: sum |A_F|^2, sum |A_SH|^2 (times eps0 c n_j dx dy / 2 on the
    // host) at z_s for s % mon_every == 0 and at s = nz, into mon[2 * slot]
    double* mon;           // [2 * n_slots] or nullptr
    int mon_every;         // sampling interval in steps (>= 1)
    int mon_last;          // slot of s = nz when nz % mon_every != 0
};

// Asynchronous global -> shared copies (LDGSTS), so that a whole tile is in
// flight at once without holding registers.
template <class C> SHG_D void cp_async(C* smem_dst, const C* gsrc) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    if constexpr (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc));
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
// 8-byte cp.async whose L2 lines are the first to be evicted (data streamed
// once per pass, so that it does not push re-read data such as the fields out
// of L2).
SHG_D uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
template <class C> SHG_D void cp_async_stream(C* smem_dst, const C* gsrc, uint64_t pol) {
    static_assert(sizeof(C) == 8 || sizeof(C) == 16, "8- or 16-byte elements");
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    if constexpr (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(s),
                     "l"(gsrc), "l"(pol));
    else
        asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s),
                     "l"(gsrc), "l"(pol));
}
// Programmatic dependent launch (sm_90 and later).  pdl_trigger lets the
// next kernel of the stream be scheduled now (its prologue overlaps this
// kernel's tail); pdl_wait blocks until the previous kernel of the stream has
// completed and its writes are visible.  Both are no-ops for a kernel
// launched without the programmatic-serialisation attribute.  The passes
// stage their constant tables, wait, and trigger only then, so that at most
// the next pass's CTAs sit resident and waiting: a trigger at kernel entry lets
// the CTAs of several later passes pile up on the SMs.
SHG_D void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
SHG_D void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

SHG_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> SHG_D void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
SHG_D void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Error flag word shared by the kernels of one launch sequence.
struct DevStatus {
    int code;
    int where;
};
