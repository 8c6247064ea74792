// Reverse (adjoint) sweep of the discrete split-step map.
//
// Convention: for a real objective J and a complex state y, the adjoint
// lambda satisfies dJ = Re sum conj(lambda) dy.  A real-differentiable map
// dy_o = P dy_i + Q conj(dy_i) (Wirtinger parts P = df/dy, Q = df/dconj(y))
// then pulls back as lambda_i = sum_o conj(P_oi) lambda_o + Q_oi conj(lambda_o).
//
// Wirtinger derivatives of the right-hand side of Eqs. (1)-(2) (E = e^{i phi},
// bj = beta_j eps0 c n_j / 4, the coupling of the pump absent when undepleted):
//   df_F/dA_F  = -2 bF |A_F|^2 + i psi_F      df_F/dconj(A_F) = -bF A_F^2 + i kF A_SH E*
//   df_F/dA_SH = i kF conj(A_F) E*            df_F/dconj(A_SH) = 0
//   df_SH/dA_F = 2 i kS A_F E                 df_SH/dconj(A_F) = 0
//   df_SH/dA_SH = -2 bS |A_SH|^2 + i psi_SH   df_SH/dconj(A_SH) = -bS A_SH^2
// and with respect to the real stage parameters
//   df_F/dphi = kF A_SH conj(A_F) E*,  df_SH/dphi = -kS A_F^2 E,
//   df_j/dpsi_j = i A_j.
#pragma once
#include "nonlinear.cuh"

namespace shg {

template <class R> struct StageBar {
    R phi, pF, pS;  // dJ/dphi, dJ/dpsi_F, dJ/dpsi_SH accumulated at one stage point
};

// (gF, gS) += J_f(a)^T (mF, mS); parameter sensitivities added to sb.
template <class R>
SHG_D void rhs_adj(const InstDesc<R>& d, const Coef<R>& k, cx<R> aF, cx<R> aS, cx<R> mF,
                   cx<R> mS, cx<R>& gF, cx<R>& gS, StageBar<R>& sb) {
    using C = cx<R>;
    const C E = mk<C>(k.er, k.ei);
    const C Ec = mk<C>(k.er, -k.ei);
    const R aF2 = aF.x * aF.x + aF.y * aF.y;
    const R aS2 = aS.x * aS.x + aS.y * aS.y;
    // pump row: (-2 bF |A_F|^2 - i psi_F) mF + Q_FF conj(mF) - 2 i kS conj(A_F) E* mS
    C t1 = cmul(mk<C>(-R(2) * d.bF * aF2, -k.pF), mF);
    C qFF = cscale(cmul(aF, aF), -d.bF);
    C cplF = mk<C>(R(0), R(0));  // A_SH conj(A_F) E* (pump coupling, also its dphi)
    if (!d.undepleted) {
        const C iaSE = cmul(mk<C>(R(0), d.kF), cmul(aS, Ec));  // i kF A_SH E*
        qFF = cadd(qFF, iaSE);
        cplF = cmul(cmulc(aS, aF), Ec);
    }
    C t2 = cmulc(qFF, mF);  // qFF * conj(mF)
    const C caFEc = cmulc(Ec, aF);  // conj(A_F) E*
    C t3 = cmul(mk<C>(R(0), -R(2) * d.kS), cmul(caFEc, mS));
    gF = cadd(gF, cadd(t1, cadd(t2, t3)));
    // SH row: -i kF A_F E mF (depleted only) + (-2 bS |A_SH|^2 - i psi_SH) mS - bS A_SH^2 conj(mS)
    C u = cadd(cmul(mk<C>(-R(2) * d.bS * aS2, -k.pS), mS),
               cmulc(cscale(cmul(aS, aS), -d.bS), mS));
    if (!d.undepleted) u = cadd(u, cmul(mk<C>(R(0), -d.kF), cmul(cmul(aF, E), mF)));
    gS = cadd(gS, u);
    // Re(conj(m) df/dp) for the stage parameters
    const C dSdphi = cscale(cmul(cmul(aF, aF), E), -d.kS);
    R ph = mF.x * (d.kF * cplF.x) + mF.y * (d.kF * cplF.y);  // Re(conj(mF) kF cplF)
    ph += mS.x * dSdphi.x + mS.y * dSdphi.y;
    sb.phi += ph;
    sb.pF += mF.y * aF.x - mF.x * aF.y;  // Re(conj(mF) i A_F)
    sb.pS += mS.y * aS.x - mS.x * aS.y;
}

// Transposed RK4 step.  Forward: y1 = y0 + h/6 (k1 + 2k2 + 2k3 + k4) with
// stages at c0, cm, cm, c1.  On entry (lF, lS) is the adjoint of y1; on exit
// that of y0.  The stage states are recomputed from y0.
template <class R>
SHG_D void rk4_adj(const InstDesc<R>& d, cx<R> y0F, cx<R> y0S, const Coef<R>& c0,
                   const Coef<R>& cm, const Coef<R>& c1, R h, cx<R>& lF, cx<R>& lS,
                   StageBar<R>& b0, StageBar<R>& bm, StageBar<R>& b1) {
    using C = cx<R>;
    const R hh = R(0.5) * h;
    C kF, kS;
    rhs(d, c0, y0F.x, y0F.y, y0S.x, y0S.y, kF.x, kF.y, kS.x, kS.y);
    const C Y2F = mk<C>(y0F.x + hh * kF.x, y0F.y + hh * kF.y);
    const C Y2S = mk<C>(y0S.x + hh * kS.x, y0S.y + hh * kS.y);
    rhs(d, cm, Y2F.x, Y2F.y, Y2S.x, Y2S.y, kF.x, kF.y, kS.x, kS.y);
    const C Y3F = mk<C>(y0F.x + hh * kF.x, y0F.y + hh * kF.y);
    const C Y3S = mk<C>(y0S.x + hh * kS.x, y0S.y + hh * kS.y);
    rhs(d, cm, Y3F.x, Y3F.y, Y3S.x, Y3S.y, kF.x, kF.y, kS.x, kS.y);
    const C Y4F = mk<C>(y0F.x + h * kF.x, y0F.y + h * kF.y);
    const C Y4S = mk<C>(y0S.x + h * kS.x, y0S.y + h * kS.y);

    const R h6 = h * (R(1) / R(6)), h3 = h * (R(1) / R(3));
    C k4bF = cscale(lF, h6), k4bS = cscale(lS, h6);
    C k3bF = cscale(lF, h3), k3bS = cscale(lS, h3);
    C k2bF = k3bF, k2bS = k3bS;
    C k1bF = k4bF, k1bS = k4bS;
    C ybF = lF, ybS = lS;
    C gF, gS;
    // stage 4 (c1)
    gF = mk<C>(R(0), R(0)); gS = gF;
    rhs_adj(d, c1, Y4F, Y4S, k4bF, k4bS, gF, gS, b1);
    ybF = cadd(ybF, gF); ybS = cadd(ybS, gS);
    k3bF = cadd(k3bF, cscale(gF, h)); k3bS = cadd(k3bS, cscale(gS, h));
    // stage 3 (cm)
    gF = mk<C>(R(0), R(0)); gS = gF;
    rhs_adj(d, cm, Y3F, Y3S, k3bF, k3bS, gF, gS, bm);
    ybF = cadd(ybF, gF); ybS = cadd(ybS, gS);
    k2bF = cadd(k2bF, cscale(gF, hh)); k2bS = cadd(k2bS, cscale(gS, hh));
    // stage 2 (cm)
    gF = mk<C>(R(0), R(0)); gS = gF;
    rhs_adj(d, cm, Y2F, Y2S, k2bF, k2bS, gF, gS, bm);
    ybF = cadd(ybF, gF); ybS = cadd(ybS, gS);
    k1bF = cadd(k1bF, cscale(gF, hh)); k1bS = cadd(k1bS, cscale(gS, hh));
    // stage 1 (c0)
    gF = mk<C>(R(0), R(0)); gS = gF;
    rhs_adj(d, c0, y0F, y0S, k1bF, k1bS, gF, gS, b0);
    lF = cadd(ybF, gF);
    lS = cadd(ybS, gS);
}

// Buffers receiving the parameter sensitivities of the reverse sweep.
struct AdjAcc {
    float* Gc;   // [tz][ny][nx]: g dJ/dphi, by z-interpolation weight per map layer
    float* Gt;   // [tz][ny][nx]: l_F dJ/dpsi_F + l_SH dJ/dpsi_SH, same weights
    double* Gs;  // [ny][nx]: dJ/dT_off per field point (summed over all stages)
};

}  // namespace shg
