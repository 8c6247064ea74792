"""Pins of the three-wave (sum/difference-frequency) oracle, oracle/threewave.py.

* Degenerate limit: with lambda1 = lambda2 = lambda_F, n1 = n2 = n_F, n3 = n_SH
  and A1 = A2 = A_F / sqrt(2), the three-wave equations are exactly the SHG
  equations of Eqs. (1)-(2) (k3 = 2 k_SH, and k_F (A_F/sqrt2)* sqrt2 = k_F A_F*),
  so A3 = A_SH and A1 = A2 = A_F / sqrt(2) at every z: compared with the SHG
  oracle (itself pinned in test_oracle_pins.py) on a focused, absorbing,
  phase-mismatched run with a temperature map.  (Two-photon absorption of
  the inputs is left out there: splitting A_F into two waves halves each
  one's intensity, so that term has no degenerate counterpart.)
* Plane waves, phase matched, equal photon fluxes: the normalised amplitudes
  u_j = a_j sqrt(n_j / omega_j) obey du1/dz = -G u2 u3, du2/dz = -G u1 u3,
  du3/dz = G u1 u2 with G = (d/c) sqrt(w1 w2 w3 / (n1 n2 n3)), so
  u3(L) = u0 tanh(G u0 L): the generated power follows tanh^2.
* Undepleted inputs, phase mismatch Dk: P3(L) = P3_0 sinc^2(Dk L / 2) L^2 scaling
  against the phase-matched run (RK4 on this quadrature is Simpson's rule).
* Manley-Rowe: without losses the photon fluxes obey N1 - N2 = const and
  N1 + N3 = const (N_j = P_j / omega_j), to the RK4 error.
* Each wave alone diffracts as the Gaussian beam of its own wavenumber.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import ssfm
from oracle import threewave as T3
from tests import pins

EPS0C = 8.8541878128e-12 * 299792458.0


def _degenerate(w3):
    """The SHG workload equivalent to a degenerate three-wave workload."""
    return W.Workload(name="shg_equiv", nx=w3.nx, ny=w3.ny, nz=w3.nz, lx=w3.lx, ly=w3.ly,
                      L=w3.L, lambda_f=w3.lambda1, n_f=w3.n1, n_sh=w3.n3, d_eff=w3.d_eff,
                      alpha_f=w3.alpha[0], alpha_sh=w3.alpha[2], beta_f=w3.beta[0],
                      beta_sh=w3.beta[2], dk0=w3.dk0, ddk_dT=w3.ddk_dT, dn_dT=w3.dn_dT,
                      p1=w3.p[0] + w3.p[1], w0=w3.w0[0], z_focus=w3.z_focus[0], t_off=w3.t_off,
                      dT=w3.dT, t_lx=w3.t_lx, t_ly=w3.t_ly)


def test_degenerate_limit_is_the_shg_oracle():
    base = W.depleted_absorbing(n=32, nz=60, tgrid=(8, 8, 12), p1=300.0)
    w3 = W.ThreeWave(name="deg", nx=32, ny=32, nz=60, lx=base.lx, ly=base.ly,
                     lambda1=base.lambda_f, lambda2=base.lambda_f, n1=base.n_f, n2=base.n_f,
                     n3=base.n_sh, alpha=(base.alpha_f, base.alpha_f, base.alpha_sh),
                     beta=(0.0, 0.0, 7e-11), dk0=40.0, ddk_dT=-3.0, dn_dT=2e-5,
                     p=(150.0, 150.0, 0.0), w0=(base.w0,) * 3, z_focus=(0.4 * base.L,) * 3,
                     t_off=0.5, dT=base.dT, t_lx=base.t_lx, t_ly=base.t_ly)
    A, P = T3.run(w3)
    AF, AS, eta = ssfm.run(_degenerate(w3))
    s2 = math.sqrt(2.0)
    assert float((A[0] - AF / s2).abs().max()) < 1e-12 * float(AF.abs().max())
    assert float((A[1] - AF / s2).abs().max()) < 1e-12 * float(AF.abs().max())
    assert float((A[2] - AS).abs().max()) < 1e-12 * float(AS.abs().max())
    assert float(eta) > 0.05


def _plane(w3, amps):
    p = T3.params_from(w3)
    return [torch.full((p.ny, p.nx), complex(a), dtype=torch.complex128) for a in amps]


def _plane_case(nz, dk0=0.0):
    return W.sfg_case(n=8, nz=nz, with_map=False).with_(
        alpha=(0.0, 0.0, 0.0), beta=(0.0, 0.0, 0.0), ddk_dT=0.0, dn_dT=0.0, dk0=dk0)


def test_equal_photon_fluxes_follow_tanh():
    w3 = _plane_case(400)
    p = T3.params_from(w3)
    om = [2 * math.pi * 299792458.0 / lam for lam in p.lambdas]
    G = (p.d_eff / 299792458.0) * math.sqrt(om[0] * om[1] * om[2] / (p.n1 * p.n2 * p.n3))
    u0 = 1.1 / (G * p.L)                     # G u0 L = 1.1: strong conversion
    a1, a2 = u0 / math.sqrt(p.n1 / om[0]), u0 / math.sqrt(p.n2 / om[1])
    A, P = T3.run(w3, A0=_plane(w3, (a1, a2, 0.0)))
    u3 = float(A[2].abs().mean()) * math.sqrt(p.n3 / om[2])
    assert abs(u3 / (u0 * math.tanh(G * u0 * p.L)) - 1) < 1e-9
    assert float(A[2].abs().std()) < 1e-12 * float(A[2].abs().mean())


def test_undepleted_sfg_follows_sinc2():
    a = (3e6, 2e6, 0.0)
    ref = _plane_case(400).with_(undepleted=True)
    A0, _ = T3.run(ref, A0=_plane(ref, a))
    for dkL in (1.0, 2.5 * math.pi):
        w3 = ref.with_(dk0=dkL / ref.L)
        A, _ = T3.run(w3, A0=_plane(w3, a))
        ratio = float(A[2].abs().mean() ** 2 / A0[2].abs().mean() ** 2)
        sinc2 = (math.sin(dkL / 2) / (dkL / 2)) ** 2
        assert abs(ratio - sinc2) < 1e-8, (dkL, ratio, sinc2)


def test_manley_rowe_photon_fluxes():
    """Focused beams without losses: the photon fluxes N1 - N2 and N1 + N3
    are conserved to the RK4 error, which falls as dz^4."""
    errs = []
    for nz in (100, 200):
        w3 = W.sfg_case(n=32, nz=nz, with_map=False).with_(alpha=(0.0, 0.0, 0.0),
                                                           beta=(0.0, 0.0, 0.0), p=(200.0, 300.0, 0.0))
        p = T3.params_from(w3)
        A, P = T3.run(w3)
        om = [1.0 / lam for lam in p.lambdas]
        N0 = [w3.p[0] / om[0], w3.p[1] / om[1], 0.0]
        N = [P[j] / om[j] for j in range(3)]
        assert N[2] > 0.05 * N0[0]
        errs.append(max(abs((N[0] - N[1]) - (N0[0] - N0[1])), abs((N[0] + N[2]) - N0[0])) / N0[0])
    assert errs[1] < 1e-10
    assert errs[0] / errs[1] > 8.0


@pytest.mark.parametrize("j", [0, 1, 2])
def test_each_wave_alone_diffracts_with_its_own_wavenumber(j):
    """One input only (no coupling partner): wave j propagates as the
    analytic Gaussian beam of Eq. (5) with k_j, to the aliasing error."""
    w3 = W.sfg_case(n=128, nz=40, with_map=False).with_(
        alpha=(0.0, 0.0, 0.0), beta=(0.0, 0.0, 0.0), dn_dT=0.0,
        p=tuple(5.0 if k == j else 0.0 for k in range(3)),
        w0=(40e-6, 40e-6, 40e-6), z_focus=(0.6 * W.L_CRYSTAL,) * 3)
    p = T3.params_from(w3)
    A, P = T3.run(w3)
    x = ssfm.axis(p.nx, p.lx).numpy()
    y = ssfm.axis(p.ny, p.ly).numpy()
    lam = (w3.lambda1, w3.lambda2, 1.0 / (1.0 / w3.lambda1 + 1.0 / w3.lambda2))[j]
    k = 2.0 * math.pi * (w3.n1, w3.n2, w3.n3)[j] / lam      # from the inputs, not the oracle
    g = pins.gaussian_beam(x, y, p.L, 40e-6, 0.6 * W.L_CRYSTAL, k)
    a0 = T3.gaussian(p, j, 5.0, 40e-6, 0.6 * W.L_CRYSTAL).numpy()
    g0 = pins.gaussian_beam(x, y, 0.0, 40e-6, 0.6 * W.L_CRYSTAL, k)
    scale = a0[p.ny // 2, p.nx // 2] / g0[p.ny // 2, p.nx // 2]
    err = np.abs(A[j].numpy() - scale * g).max() / np.abs(scale * g).max()
    assert err < 1e-6, err
    for k in range(3):
        if k != j:
            assert float(A[k].abs().max()) == 0.0


# ----------------------------------------------------------- planted mistakes ----
# Each mistake is planted in the oracle (monkeypatch, CPU only) and must make
# at least one of the pins above fail.

def _kappa3_with_lambda1(monkeypatch):
    # the generated wave's coupling with lambda_1 instead of lambda_3
    orig = T3.Params3.kappa.fget

    def kappa(self):
        k = orig(self)
        return (k[0], k[1], 2.0 * math.pi * self.d_eff / (self.n3 * self.lambda1))
    monkeypatch.setattr(T3.Params3, "kappa", property(kappa))


def _kappa2_with_n1(monkeypatch):
    # wave 2's coupling with wave 1's index
    orig = T3.Params3.kappa.fget

    def kappa(self):
        k = orig(self)
        return (k[0], 2.0 * math.pi * self.d_eff / (self.n1 * self.lambda2), k[2])
    monkeypatch.setattr(T3.Params3, "kappa", property(kappa))


def _rhs_mutant(kind):
    def rhs(self, A, coef):
        p = self.p
        phi, psi = coef
        e = torch.exp(1j * phi)
        k1, k2, k3 = p.kappa
        out = [-0.5 * p.beta[j] * self.c[j] * A[j].abs() ** 2 * A[j] + 1j * psi[j] * A[j]
               for j in range(3)]
        a2 = A[1] if kind == "no_conj" else torch.conj(A[1])
        e3 = torch.conj(e) if kind == "phase_sign" else e
        out[0] = out[0] + 1j * k1 * A[2] * a2 * torch.conj(e)
        out[1] = out[1] + 1j * k2 * A[2] * torch.conj(A[0]) * torch.conj(e)
        out[2] = out[2] + 1j * k3 * A[0] * A[1] * e3
        return out
    return lambda mp: mp.setattr(T3.Nonlinear3, "rhs", rhs)


def _wave2_with_k1(monkeypatch):
    # wave 2 diffracting with wave 1's wavenumber
    orig = T3.Params3.k.fget
    monkeypatch.setattr(T3.Params3, "k",
                        property(lambda self: (orig(self)[0], orig(self)[0], orig(self)[2])))


MUTANTS = {
    "kappa3 with lambda1": (_kappa3_with_lambda1, [test_degenerate_limit_is_the_shg_oracle]),
    "kappa2 with n1": (_kappa2_with_n1, [test_manley_rowe_photon_fluxes]),
    "wave 1 coupling without conj": (_rhs_mutant("no_conj"),
                                     [test_degenerate_limit_is_the_shg_oracle]),
    "generated wave phase sign": (_rhs_mutant("phase_sign"),
                                  [test_degenerate_limit_is_the_shg_oracle]),
    "wave 2 with k1": (_wave2_with_k1,
                       [lambda: test_each_wave_alone_diffracts_with_its_own_wavenumber(1)]),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_three_wave_mistake_fails_a_pin(name, monkeypatch):
    plant, checks = MUTANTS[name]
    plant(monkeypatch)
    failed = 0
    for check in checks:
        try:
            check()
        except AssertionError:
            failed += 1
    assert failed > 0, f"planted mistake '{name}' passed every pin"
