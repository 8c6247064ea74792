"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, for the duration of
the test only, by monkeypatching) and runs the pins that should notice it:
at least one of them must fail. The planted mistakes are the kinds a
restatement of the paper can make:
- a dropped factor or term;
- a flipped sign;
- a wrong wavelength or index;
- a transposed operand;
- a lower-order step.

A mistake that no pin catches shows a gap in the pins.
"""
import math

import pytest
import torch

from oracle import heat, ssfm
from tests import test_oracle_pins as P


# ------------------------------------------------------------ the mistakes ----

def _wrap_linear_init(extra):
    """Linear.__init__ followed by extra(self, p): a changed K-space factor."""
    orig = ssfm.Linear.__init__

    def init(self, p):
        orig(self, p)
        extra(self, p)
    return init


def _k(p):
    Kx = ssfm.wavenumbers(p.nx, p.lx)
    Ky = ssfm.wavenumbers(p.ny, p.ly)
    return Kx, Ky, Kx[None, :] ** 2 + Ky[:, None] ** 2


def diffraction_sign(self, p):
    # exp(+i K^2 dz / 2k): App. A's printed sign instead of reading 1
    _, _, K2 = _k(p)
    self.PF = self.PF * torch.exp(2j * K2 * p.dz / (2 * p.k_f))
    self.PS = self.PS * torch.exp(2j * K2 * p.dz / (2 * p.k_sh))


def absorption_on_intensity(self, p):
    # exp(-alpha dz) on the amplitude: alpha taken as an amplitude rate
    self.PF = self.PF * math.exp(-0.5 * p.alpha_f * p.dz)
    self.PS = self.PS * math.exp(-0.5 * p.alpha_sh * p.dz)


def walkoff_sign(self, p):
    # the beam drifts toward -x
    Kx, _, _ = _k(p)
    self.PS = self.PS * torch.exp(2j * math.tan(p.walkoff_sh) * Kx[None, :] * p.dz)
    self.PF = self.PF * torch.exp(2j * math.tan(p.walkoff_f) * Kx[None, :] * p.dz)


def walkoff_along_y(self, p):
    # the walk-off factor applied along y instead of x
    Kx, Ky, _ = _k(p)
    for name, rho in (("PF", p.walkoff_f), ("PS", p.walkoff_sh)):
        t = math.tan(rho) * p.dz
        f = torch.exp(1j * t * Kx[None, :]) * torch.exp(-1j * t * Ky[:, None])
        setattr(self, name, getattr(self, name) * f)


def no_negative_frequencies(monkeypatch):
    # K = 2 pi m / L for every bin m, without the negative half of fftfreq
    monkeypatch.setattr(ssfm, "wavenumbers",
                        lambda n, length: 2 * math.pi * torch.arange(n, dtype=torch.float64) / length)


def kappa_sh_with_sh_wavelength(monkeypatch):
    # Eq. 2 as printed: 2 pi d / (n_SH lambda_SH)
    monkeypatch.setattr(ssfm.Params, "kappa_sh",
                        property(lambda self: 2 * math.pi * self.d_eff / (self.n_sh * self.lambda_sh)))


def _wrap_rhs(change):
    orig = ssfm.Nonlinear.rhs

    def rhs(self, AF, AS, coef):
        fF, fS = orig(self, AF, AS, coef)
        return change(self, AF, AS, coef, fF, fS)
    return rhs


def tpa_without_half(self, AF, AS, coef, fF, fS):
    # -beta I A instead of -(1/2) beta I A
    p = self.p
    IF = self.cF * AF.abs() ** 2
    IS = self.cS * AS.abs() ** 2
    return fF - 0.5 * p.beta_f * IF * AF, fS - 0.5 * p.beta_sh * IS * AS


def pump_coupling_without_conjugate(self, AF, AS, coef, fF, fS):
    # i kappa_F A_SH A_F e^{-i phi}: the conjugate of A_F dropped
    p = self.p
    e = torch.exp(1j * coef[0])
    if not p.undepleted:
        fF = (fF - 1j * p.kappa_f * AS * torch.conj(AF) * torch.conj(e)
              + 1j * p.kappa_f * AS * AF * torch.conj(e))
    return fF, fS


def undepleted_drops_the_sh_drive(self, AF, AS, coef, fF, fS):
    # the undepleted switch removes the SH equation's drive instead of the pump's
    p = self.p
    e = torch.exp(1j * coef[0])
    if p.undepleted:
        fF = fF + 1j * p.kappa_f * AS * torch.conj(AF) * torch.conj(e)
        fS = fS - 1j * p.kappa_sh * AF * AF * e
    return fF, fS


def _wrap_coefficients(change):
    orig = ssfm.Nonlinear.coefficients

    def coefficients(self, z):
        self._z = z
        return change(self, *orig(self, z))
    return coefficients


def phase_sign(self, phi, psiF, psiS):
    # e^{+i phi} on the pump and e^{-i phi} on the SH: Dk of the opposite sign
    return -phi, psiF, psiS


def lens_with_sh_wavelength(self, phi, psiF, psiS):
    # psi_F computed with 2 pi / lambda_SH
    return phi, psiF * (self.k0S / self.k0F), psiS


def rk4_wrong_third_stage(self, AF, AS, z0, h):
    # the third stage re-uses the first slope: k3 = f(y + h/2 k1)
    c0 = self.coefficients(z0)
    cm = self.coefficients(z0 + 0.5 * h)
    c1 = self.coefficients(z0 + h)
    k1F, k1S = self.rhs(AF, AS, c0)
    k2F, k2S = self.rhs(AF + 0.5 * h * k1F, AS + 0.5 * h * k1S, cm)
    k3F, k3S = self.rhs(AF + 0.5 * h * k1F, AS + 0.5 * h * k1S, cm)
    k4F, k4S = self.rhs(AF + h * k3F, AS + h * k3S, c1)
    return (AF + (h / 6.0) * (k1F + 2 * k2F + 2 * k3F + k4F),
            AS + (h / 6.0) * (k1S + 2 * k2S + 2 * k3S + k4S))


def rk4_frozen_coefficients(self, AF, AS, z0, h):
    # the stage coefficients of z0 used at every stage of the step
    c0 = self.coefficients(z0)
    k1F, k1S = self.rhs(AF, AS, c0)
    k2F, k2S = self.rhs(AF + 0.5 * h * k1F, AS + 0.5 * h * k1S, c0)
    k3F, k3S = self.rhs(AF + 0.5 * h * k2F, AS + 0.5 * h * k2S, c0)
    k4F, k4S = self.rhs(AF + h * k3F, AS + h * k3S, c0)
    return (AF + (h / 6.0) * (k1F + 2 * k2F + 2 * k3F + k4F),
            AS + (h / 6.0) * (k1S + 2 * k2S + 2 * k3S + k4S))


def power_without_half(monkeypatch):
    # P = eps0 c n sum |A|^2 dx dy: the 1/2 of the intensity dropped
    monkeypatch.setattr(ssfm, "power", lambda A, n_j, dx, dy: EPS0C * n_j * (A.abs() ** 2).sum() * dx * dy)


EPS0C = ssfm.EPS0 * ssfm.C_LIGHT


def pump_curvature_sign(monkeypatch):
    # tau0 = +f / z_R: the beam starts diverging instead of converging
    orig = ssfm.initial_pump
    monkeypatch.setattr(ssfm, "initial_pump",
                        lambda p, p1, w0, z_focus: orig(p, p1, w0, -ssfm._t(z_focus)))


def focus_at_the_centre(monkeypatch):
    # the focus taken at L/2 whatever z_focus says
    orig = ssfm.initial_pump
    monkeypatch.setattr(ssfm, "initial_pump",
                        lambda p, p1, w0, z_focus: orig(p, p1, w0, 0.5 * p.L + 0 * ssfm._t(z_focus)))


def cumulative_left_sum(monkeypatch):
    # C by the left Riemann sum instead of the trapezoid rule
    def cum(dT, L):
        dZ = L / (dT.shape[0] - 1)
        rows = [torch.zeros_like(dT[0])]
        for l in range(1, dT.shape[0]):
            rows.append(rows[-1] + dZ * dT[l - 1])
        return torch.stack(rows, 0)
    monkeypatch.setattr(ssfm, "cumulative_dT", cum)


def bilinear_transposed(monkeypatch):
    # the x and y fractions swapped in the transverse interpolation
    def bil(self, t):
        ix, fx, iy, fy = self.ix, self.fx, self.iy, self.fy
        n = min(len(fx), len(fy))
        fx2 = fx.clone()
        fy2 = fy.clone()
        fx2[:n], fy2[:n] = fy[:n], fx[:n]
        t00 = t[iy][:, ix]
        t01 = t[iy][:, ix + 1]
        t10 = t[iy + 1][:, ix]
        t11 = t[iy + 1][:, ix + 1]
        fxr, fyc = fx2[None, :], fy2[:, None]
        return (1 - fyc) * ((1 - fxr) * t00 + fxr * t01) + fyc * ((1 - fxr) * t10 + fxr * t11)
    monkeypatch.setattr(ssfm.TemperatureField, "_bilinear", bil)


def map_extrapolated(monkeypatch):
    # no clamp at the map's edge: linear extrapolation outside it
    def lin_index(coord, origin, spacing, n):
        u = (coord - origin) / spacing
        i = torch.floor(u).clamp(0, n - 2)
        return i.long(), u - i
    monkeypatch.setattr(ssfm, "_lin_index", lin_index)


def deposit_full_weight_at_entrance(monkeypatch):
    # the trapezoid's half weight dropped at z = 0
    orig = ssfm.HeatDeposit.add

    def add(self, AF, AS, z, wz):
        return orig(self, AF, AS, z, 2 * wz if z == 0 else wz)
    monkeypatch.setattr(ssfm.HeatDeposit, "add", add)


def deposit_without_tpa(monkeypatch):
    # q_dot without the two-photon terms beta_j I_j^2
    def qdot(self, AF, AS):
        p = self.p
        return p.alpha_f * self.cF * AF.abs() ** 2 + p.alpha_sh * self.cS * AS.abs() ** 2
    monkeypatch.setattr(ssfm.HeatDeposit, "qdot", qdot)


def deposit_floor_node(monkeypatch):
    # floor instead of round: the node below rather than the nearest one
    orig = ssfm.HeatDeposit.__init__

    def init(self, p, hx, hy, hz, wx, wy):
        orig(self, p, hx, hy, hz, wx, wy)
        x = ssfm.axis(p.nx, p.lx)
        y = ssfm.axis(p.ny, p.ly)
        self.ix = torch.floor((x + wx / 2) / self.hdx).long()
        self.iy = torch.floor((y + wy / 2) / self.hdy).long()
        self.okx = (self.ix >= 0) & (self.ix < hx)
        self.oky = (self.iy >= 0) & (self.iy < hy)
    monkeypatch.setattr(ssfm.HeatDeposit, "__init__", init)


def stencil_spacings_swapped(monkeypatch):
    # 1/dy^2 on the x neighbours and 1/dx^2 on the y neighbours
    orig = heat.jacobi_target
    monkeypatch.setattr(heat, "jacobi_target",
                        lambda T, q, kappa, dx, dy, dz, bc=heat.DIRICHLET:
                        orig(T, q, kappa, dy, dx, dz, bc))


def source_without_conductivity(monkeypatch):
    # q_dot not divided by kappa
    orig = heat.jacobi_target
    monkeypatch.setattr(heat, "jacobi_target",
                        lambda T, q, kappa, dx, dy, dz, bc=heat.DIRICHLET:
                        orig(T, q, 1.0, dx, dy, dz, bc))


def sh_diffraction_with_kf(self, p):
    # the SH diffracts with the pump's wavenumber
    _, _, K2 = _k(p)
    self.PS = (self.PS * torch.exp(1j * K2 * p.dz / (2 * p.k_sh))
               * torch.exp(-1j * K2 * p.dz / (2 * p.k_f)))


def sh_intensity_with_nf(monkeypatch):
    # I_SH = eps0 c n_F |A_SH|^2 / 2
    orig = ssfm.Nonlinear.__init__

    def init(self, p, temp):
        orig(self, p, temp)
        self.cS = self.cF
    monkeypatch.setattr(ssfm.Nonlinear, "__init__", init)


def undepleted_ignored(self, AF, AS, coef, fF, fS):
    # the undepleted switch has no effect
    p = self.p
    if p.undepleted:
        fF = fF + 1j * p.kappa_f * AS * torch.conj(AF) * torch.conj(torch.exp(1j * coef[0]))
    return fF, fS


def lens_without_offset(self, phi, psiF, psiS):
    # psi_j from dT alone, without the oven offset T_off
    t = self.temp.t_off
    return phi, psiF - self.k0F * self.p.dn_dT * t, psiS - self.k0S * self.p.dn_dT * t


def cumulative_without_slope(self, phi, psiF, psiS):
    # phi = ... + C instead of ... + g C
    _, c = self.temp.at(self._z)
    return phi + (1 - self.p.ddk_dT) * c, psiF, psiS


def no_deposit_at_exit(monkeypatch):
    # the trapezoid's last sample, at z = L, left out
    orig = ssfm.HeatDeposit.add

    def add(self, AF, AS, z, wz):
        if z != self.p.L:
            orig(self, AF, AS, z, wz)
    monkeypatch.setattr(ssfm.HeatDeposit, "add", add)


def deposits_never_reset(monkeypatch):
    # every outer iteration adds its deposits to the previous ones
    orig = ssfm.HeatDeposit.__init__
    shared = {}

    def init(self, p, hx, hy, hz, wx, wy):
        orig(self, p, hx, hy, hz, wx, wy)
        self.Q = shared.setdefault((hx, hy, hz), self.Q)
    monkeypatch.setattr(ssfm.HeatDeposit, "__init__", init)


def loop_map_over_the_window(monkeypatch):
    # the loop installs dT over the field window instead of the crystal
    def loop(w, n_outer, tol=1e-6, max_sweeps=100000, nsteps=None):
        p = ssfm.params_from_workload(w)
        q = torch.zeros((w.hz, w.hy, w.hx), dtype=torch.float64)
        dT_prev = torch.zeros_like(q)
        history = []
        for _ in range(n_outer):
            dT, sweeps, _ = heat.sor_solve(q, w.kappa_th, w.wx, w.wy, w.L, tol, max_sweeps,
                                           T0=dT_prev)
            change = float((dT - dT_prev).abs().max())
            dep = ssfm.HeatDeposit(p, w.hx, w.hy, w.hz, w.wx, w.wy)
            temp = ssfm.TemperatureField(p, dT, w.lx, w.ly, w.t_off)
            AF0 = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus)
            AF, AS = ssfm.propagate(p, AF0, torch.zeros_like(AF0), temp, dep)
            eta = float(ssfm.power(AS, p.n_sh, p.dx, p.dy) / w.p1)
            q = dep.qdot_nodes()
            history.append(dict(eta=eta, dT=dT, change=change, sweeps=sweeps))
            dT_prev = dT
        return history
    monkeypatch.setattr(heat, "thermal_loop", loop)


def heat_source_sign(monkeypatch):
    # kappa lap T = +q_dot: the source cools
    orig = heat.jacobi_target
    monkeypatch.setattr(heat, "jacobi_target",
                        lambda T, q, kappa, dx, dy, dz, bc=heat.DIRICHLET:
                        orig(T, -q, kappa, dx, dy, dz, bc))


def ghost_without_doubling(monkeypatch):
    # the convective face's ghost node taken as 0 instead of T_inner - ...
    def nsum(T, axis):
        n = T.shape[axis]
        S = torch.zeros_like(T)
        sl = lambda a, b: tuple(slice(a, b) if k == axis else slice(None) for k in range(3))  # noqa: E731
        S[sl(1, n - 1)] = T[sl(2, n)] + T[sl(0, n - 2)]
        S[sl(0, 1)] = T[sl(1, 2)]
        S[sl(n - 1, n)] = T[sl(n - 2, n - 1)]
        return S
    monkeypatch.setattr(heat, "_neighbour_sum", nsum)


def convection_heats(monkeypatch):
    # -kappa dT/dn = -h (T - T_inf): the sign of Eq. (10) flipped
    orig = heat._face_terms
    monkeypatch.setattr(heat, "_face_terms", lambda *a: tuple(-x for x in orig(*a)))


def convection_without_spacing(monkeypatch):
    # the ghost node's offset without the spacing d (h / kappa instead of d h / kappa)
    def terms(shape, dx, dy, dz, kappa, bc):
        diag = torch.zeros(shape, dtype=torch.float64)
        for k, (axis, d) in enumerate(((2, dx), (2, dx), (1, dy), (1, dy), (0, dz), (0, dz))):
            if not bc.convective(k):
                continue
            layer = [slice(None)] * 3
            layer[axis] = 0 if k % 2 == 0 else shape[axis] - 1
            diag[tuple(layer)] += 2.0 * (1.0 / d ** 2) * bc.h_of(k) / kappa
        return diag, diag * bc.t_inf
    monkeypatch.setattr(heat, "_face_terms", terms)


def face_cells_full_volume(monkeypatch):
    # a face node's source density over a whole cell instead of its half cell
    monkeypatch.setattr(ssfm.HeatDeposit, "qdot_nodes",
                        lambda self: self.Q / (self.hdx * self.hdy * self.hdz))


def _qpm_dk(mutate):
    def dk(self, lambda_f, T):
        u = T - 25.0
        nF = sum(c * u ** k for k, c in enumerate(self.n_f_t))
        nS = sum(c * u ** k for k, c in enumerate(self.n_sh_t))
        return mutate(self, lambda_f, T, u, nF, nS)
    return dk


def grating_b_sign(self, lambda_f, T, u, nF, nS):
    # Lambda(T) with the quadratic term's sign flipped
    lam = self.lambda25 * (1.0 + self.a_lambda * u - self.b_lambda * u * u)
    return 4.0 * math.pi / lambda_f * (nS - nF) - 2.0 * math.pi / lam


def grating_about_the_oven(self, lambda_f, T, u, nF, nS):
    # the grating expanded about the oven temperature instead of 25 C
    v = T - self.t_oven
    lam = self.lambda25 * (1.0 + self.a_lambda * v + self.b_lambda * v * v)
    return 4.0 * math.pi / lambda_f * (nS - nF) - 2.0 * math.pi / lam


def material_term_2pi(self, lambda_f, T, u, nF, nS):
    # 2 pi / lambda_F instead of 4 pi / lambda_F on the index difference
    lam = self.lambda25 * (1.0 + self.a_lambda * u + self.b_lambda * u * u)
    return 2.0 * math.pi / lambda_f * (nS - nF) - 2.0 * math.pi / lam


def eq4_without_offset(monkeypatch):
    # the local temperature of Eq. (4) taken without the oven offset
    orig = ssfm.Nonlinear.coefficients

    def coefficients(self, z):
        p = self.p
        if p.qpm is None:
            return orig(self, z)
        d, c = self.temp.at(z)
        t_off = self.temp.t_off
        phi = p.qpm.dk(p.lambda_f, p.qpm.t_oven) * z + c
        dT_eff = d + t_off
        return phi, self.k0F * p.dn_dT * dT_eff, self.k0S * p.dn_dT * dT_eff
    monkeypatch.setattr(ssfm.Nonlinear, "coefficients", coefficients)


def eq4_integrand_not_relative(monkeypatch):
    # C' integrates Dk(T_ref + dT) instead of Dk(T_ref + dT) - Dk(T_ref)
    orig = ssfm.TemperatureField.__init__

    def init(self, p, dT, t_lx, t_ly, t_off=0.0):
        orig(self, p, dT, t_lx, t_ly, t_off)
        if p.qpm is not None:
            t_ref = p.qpm.t_oven + self.t_off
            self.C = ssfm.cumulative_dT(p.qpm.dk(p.lambda_f, t_ref + self.dT), p.L)
    monkeypatch.setattr(ssfm.TemperatureField, "__init__", init)


# ------------------------------------------------------------------ cases ----

def _attr(obj, name, value):
    return lambda mp: mp.setattr(obj, name, value)


BK = [lambda: P.test_boyd_kleinman_undepleted(2.84, 0.5736),
      lambda: P.test_boyd_kleinman_undepleted(2.84, -0.5736)]


def TPA():
    for wave in ("sh", "f"):
        P.test_two_photon_absorption_closed_form(wave)


def pump_tpa_with_sh_intensity(self, AF, AS, coef, fF, fS):
    # the pump's two-photon loss driven by I_SH
    p = self.p
    IF = self.cF * AF.abs() ** 2
    IS = self.cS * AS.abs() ** 2
    return fF + 0.5 * p.beta_f * IF * AF - 0.5 * p.beta_f * IS * AF, fS


def pump_tpa_dropped(self, AF, AS, coef, fF, fS):
    # beta_F left out of the pump equation
    return fF + 0.5 * self.p.beta_f * self.cF * AF.abs() ** 2 * AF, fS


def DIFFRACTION():
    for f in (0.5, 0.3):
        P.test_diffraction_reproduces_gaussian_beam(f)


def PUMP():
    for f in (0.5, 0.3):
        P.test_initial_pump_is_eq5_with_discrete_power(f)

CASES = {
    "diffraction sign": (_attr(ssfm.Linear, "__init__", _wrap_linear_init(diffraction_sign)),
                         [DIFFRACTION]),
    "absorption doubled": (_attr(ssfm.Linear, "__init__", _wrap_linear_init(absorption_on_intensity)),
                           [P.test_beer_lambert_decay_of_both_waves]),
    "walk-off sign": (_attr(ssfm.Linear, "__init__", _wrap_linear_init(walkoff_sign)),
                      [P.test_walkoff_is_an_exact_translation,
                       P.test_walkoff_moves_the_beam_centroid_at_tan_rho]),
    "walk-off along y": (_attr(ssfm.Linear, "__init__", _wrap_linear_init(walkoff_along_y)),
                         [P.test_walkoff_is_an_exact_translation]),
    "no negative frequencies": (no_negative_frequencies,
                                [DIFFRACTION]),
    "axis spacing L/(n-1)": (_attr(ssfm, "axis", lambda n, length: (
        torch.arange(n, dtype=torch.float64) - n // 2) * (length / (n - 1))),
                             [P.test_wavenumber_bins_match_plane_waves]),
    "kappa_SH with lambda_SH": (kappa_sh_with_sh_wavelength,
                                [P.test_plane_wave_conversion_follows_tanh_squared,
                                 P.test_manley_rowe_without_losses]),
    "TPA without the 1/2": (_attr(ssfm.Nonlinear, "rhs", _wrap_rhs(tpa_without_half)),
                            [TPA]),
    "pump TPA with I_SH": (_attr(ssfm.Nonlinear, "rhs", _wrap_rhs(pump_tpa_with_sh_intensity)), [TPA]),
    "pump TPA dropped": (_attr(ssfm.Nonlinear, "rhs", _wrap_rhs(pump_tpa_dropped)), [TPA]),
    "pump coupling without conjugate": (
        _attr(ssfm.Nonlinear, "rhs", _wrap_rhs(pump_coupling_without_conjugate)),
        [P.test_manley_rowe_without_losses, P.test_plane_wave_conversion_follows_tanh_squared]),
    "undepleted drops the SH drive": (
        _attr(ssfm.Nonlinear, "rhs", _wrap_rhs(undepleted_drops_the_sh_drive)), BK),
    "phase sign": (_attr(ssfm.Nonlinear, "coefficients", _wrap_coefficients(phase_sign)), BK),
    "lens with lambda_SH": (_attr(ssfm.Nonlinear, "coefficients",
                                  _wrap_coefficients(lens_with_sh_wavelength)),
                            [P.test_uniform_lens_phase_rotates_fields]),
    "RK4 third stage": (_attr(ssfm.Nonlinear, "rk4", rk4_wrong_third_stage),
                        [P.test_manley_rowe_without_losses]),
    "RK4 frozen coefficients": (_attr(ssfm.Nonlinear, "rk4", rk4_frozen_coefficients),
                                [P.test_phase_mismatched_plane_wave_follows_sinc_squared]),
    "power without the 1/2": (power_without_half,
                              [PUMP]),
    "pump curvature sign": (pump_curvature_sign,
                            [PUMP]),
    "focus at the centre": (focus_at_the_centre, [PUMP, DIFFRACTION]),
    "cumulative left sum": (cumulative_left_sum, [P.test_trilinear_tables_exact_for_affine_maps]),
    "bilinear transposed": (bilinear_transposed, [P.test_trilinear_tables_exact_for_affine_maps]),
    "map extrapolated": (map_extrapolated,
                         [P.test_temperature_map_is_clamped_outside_its_extent]),
    "deposit full weight at z = 0": (deposit_full_weight_at_entrance,
                                     [P.test_heat_deposits_balance_absorbed_power]),
    "deposit without TPA": (deposit_without_tpa, [P.test_heat_deposits_balance_absorbed_power]),
    "deposit on the node below": (deposit_floor_node,
                                  [P.test_heat_deposit_lands_on_the_nearest_node]),
    "stencil spacings swapped": (stencil_spacings_swapped, [P.test_sor_matches_direct_sparse_solve]),
    "SH diffraction with k_F": (_attr(ssfm.Linear, "__init__", _wrap_linear_init(sh_diffraction_with_kf)),
                                BK + [P.test_manley_rowe_without_losses]),
    "SH intensity with n_F": (sh_intensity_with_nf, [TPA]),
    "undepleted switch ignored": (_attr(ssfm.Nonlinear, "rhs", _wrap_rhs(undepleted_ignored)),
                                  [P.test_phase_mismatched_plane_wave_follows_sinc_squared]),
    "lens without T_off": (_attr(ssfm.Nonlinear, "coefficients",
                                 _wrap_coefficients(lens_without_offset)),
                           [P.test_uniform_lens_phase_rotates_fields]),
    "C without dDk/dT": (_attr(ssfm.Nonlinear, "coefficients",
                               _wrap_coefficients(cumulative_without_slope)),
                         [P.test_uniform_temperature_equals_shifted_mismatch]),
    "no deposit at the exit": (no_deposit_at_exit, [P.test_heat_deposits_balance_absorbed_power]),
    "deposits never reset": (deposits_never_reset, [P.test_thermal_loop_fixed_point_behaviour]),
    "loop map over the window": (loop_map_over_the_window,
                                 [P.test_thermal_loop_fixed_point_behaviour]),
    "node density without hdz": (_attr(ssfm.HeatDeposit, "qdot_nodes",
                                       lambda self: self.Q / (self.hdx * self.hdy)),
                                 [P.test_thermal_loop_fixed_point_behaviour]),
    "cell-centred heat grid": (_attr(heat, "spacings",
                                     lambda hx, hy, hz, wx, wy, L: (wx / hx, wy / hy, L / hz)),
                               [P.test_sor_matches_direct_sparse_solve,
                                P.test_sor_recovers_discrete_eigenmode]),
    "heat source sign": (heat_source_sign, [P.test_thermal_loop_fixed_point_behaviour]),
    "grating b sign": (_attr(ssfm.QPM, "dk", _qpm_dk(grating_b_sign)),
                       [P.test_eq4_zero_crossing_at_the_constructed_phase_matching_temperature]),
    "grating about the oven": (_attr(ssfm.QPM, "dk", _qpm_dk(grating_about_the_oven)),
                               [P.test_eq4_zero_crossing_at_the_constructed_phase_matching_temperature]),
    "material term 2 pi": (_attr(ssfm.QPM, "dk", _qpm_dk(material_term_2pi)),
                           [P.test_eq4_with_linear_indices_and_rigid_grating_is_the_linearised_model]),
    "Eq. 4 without the offset": (eq4_without_offset,
                                 [P.test_eq4_with_linear_indices_and_rigid_grating_is_the_linearised_model]),
    "Eq. 4 integrand absolute": (eq4_integrand_not_relative,
                                 [P.test_eq4_with_linear_indices_and_rigid_grating_is_the_linearised_model]),
    "convective ghost not doubled": (ghost_without_doubling,
                                     [P.test_all_convective_faces_balance_the_source_exactly]),
    "convection heats": (convection_heats,
                         [P.test_all_convective_faces_balance_the_source_exactly]),
    "convective offset without spacing": (convection_without_spacing,
                                          [P.test_all_convective_faces_balance_the_source_exactly]),
    "face cells of full volume": (face_cells_full_volume,
                                  [P.test_loop_with_convective_faces_conserves_energy]),
    "source not divided by kappa": (source_without_conductivity,
                                    [P.test_sor_matches_direct_sparse_solve,
                                     P.test_sor_recovers_discrete_eigenmode]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    plant, pins = CASES[name]
    plant(monkeypatch)
    caught = None
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught = pin
            break
    assert caught is not None, f"no pin caught the planted mistake: {name}"
