"""Pins of the FP64 oracle against results fixed by the paper and by mathematics.

Each test targets one piece of the oracle so that a dropped term, a wrong sign
or a transposed operand fails at least one of them:

* FFT step and K convention        -> brute-force DFT, plane-wave bin
* initial pump (Eq. 5/6)           -> analytic Gaussian, discrete power = P1
* diffraction (App. A, reading 1)  -> analytic Gaussian beam at z, w(z) law
* linear absorption in L           -> Beer-Lambert
* walk-off term in L (Sec. 6)      -> exact integer-cell translation,
                                      centroid drift tan(rho) z
* coupling terms (Eq. 1/2, kappa)  -> plane-wave tanh^2 law, Manley-Rowe,
                                      Boyd-Kleinman h(sigma, xi)
* phase sign and Dk (Eq. 3/4)      -> Boyd-Kleinman at sigma = +-0.57,
                                      plane-wave sinc^2 at Dk L = 3 pi
* TPA terms                        -> closed-form plane-wave decay of each wave
* temperature tables / lens phase  -> exact trilinear of affine maps,
                                      uniform dT == shifted dk0, e^{i psi z}
* heat solve (Eq. 16)              -> direct sparse solve, discrete eigenmode
* self-consistent loop (Fig. 2)    -> lossless special case, maximum principle,
                                      contraction
* heat source deposits (Eq. 8)     -> energy balance
* gradients (autograd of the map)  -> central finite differences
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import heat, ssfm
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _p(w):
    return ssfm.params_from_workload(w)


# ------------------------------------------------------------------ FFT ----

@pytest.mark.parametrize("shape", [(8, 8), (16, 8), (2, 4), (1, 1)])
def test_fft_step_matches_brute_force_dft(shape):
    """The oracle's own radix-2 DFT (oracle/fft.c) against the O(N^4) sum of
    the DFT's definition, and its inverse back to the input."""
    from oracle import fft as dft
    rng = np.random.default_rng(3)
    a = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    ref = pins.brute_dft2(a)
    got = dft.fft2(torch.tensor(a)).numpy()
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    back = dft.ifft2(torch.tensor(got)).numpy()
    assert np.max(np.abs(back - a)) < 1e-13


@pytest.mark.parametrize("shape", [(128, 256), (2, 1024), (1024, 4)])
def test_fft_matches_a_library_fft_at_every_stage_count(shape):
    """Large lengths (up to the 10 stages of 1024) against numpy's FFT, a
    library routine that shares nothing with the oracle's code."""
    from oracle import fft as dft
    rng = np.random.default_rng(4)
    a = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    got = dft.fft2(torch.tensor(a)).numpy()
    ref = np.fft.fft2(a)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(dft.ifft2(torch.tensor(a)).numpy() - np.fft.ifft2(a))) < 1e-15 * np.abs(a).sum()


def test_fft_gradient_is_the_adjoint_map():
    """The DFT's vector-Jacobian products (used by the oracle's autograd
    gradients) against numerical differentiation."""
    from oracle import fft as dft
    x = torch.randn(4, 8, dtype=torch.complex128, requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: dft.fft2(t), (x,))
    assert torch.autograd.gradcheck(lambda t: dft.ifft2(t * t), (x,))


def test_oracle_uses_no_library_fft():
    """The oracle's sources call no library FFT (torch.fft, numpy.fft, scipy)."""
    import glob
    import re
    root = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle")
    for f in glob.glob(os.path.join(root, "*.py")) + glob.glob(os.path.join(root, "*.c")):
        code = open(f).read()
        assert not re.search(r"torch\.fft|np\.fft|numpy\.fft|scipy\.fft|fftpack|fftw", code,
                             re.I), f


def test_wavenumber_bins_match_plane_waves():
    n, L = 16, 1e-3
    x = ssfm.axis(n, L).numpy()
    K = ssfm.wavenumbers(n, L).numpy()
    for b in (0, 1, 5, 8, 9, 15):
        wave = np.exp(1j * K[b] * x)
        spec = pins.brute_dft2(wave[None, :])[0]
        assert np.argmax(np.abs(spec)) == b
        assert abs(abs(spec[b]) - n) < 1e-9


# ----------------------------------------------------------------- init ----

@pytest.mark.parametrize("focus", [0.5, 0.3])
def test_initial_pump_is_eq5_with_discrete_power(focus):
    """Eq. 5 at the entrance for a focus at the centre and off it (f = 0.3 L)."""
    w = W.plain_focused(n=64, nz=10)
    w = w.with_(z_focus=focus * w.L)
    p = _p(w)
    A = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus).numpy()
    x = ssfm.axis(p.nx, p.lx).numpy()
    y = ssfm.axis(p.ny, p.ly).numpy()
    g = pins.gaussian_beam(x, y, 0.0, w.w0, w.z_focus, p.k_f)
    ratio = A / g
    assert np.allclose(ratio, ratio[0, 0], rtol=1e-13, atol=0)
    assert abs(ratio[0, 0].imag) < 1e-12 * abs(ratio[0, 0])
    P = 0.5 * pins.EPS0 * pins.C_LIGHT * p.n_f * np.sum(np.abs(A) ** 2) * p.dx * p.dy
    assert abs(P / w.p1 - 1) < 1e-13


# ----------------------------------------------------------- diffraction ----

def _free_run(w):
    p = _p(w)
    AF0 = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus)
    AS0 = torch.zeros_like(AF0)
    temp = ssfm.TemperatureField(p, None, 0, 0, 0.0)
    AF, AS = ssfm.propagate(p, AF0, AS0, temp)
    return p, AF0, AF


@pytest.mark.parametrize("focus", [0.5, 0.3])
def test_diffraction_reproduces_gaussian_beam(focus):
    w = W.plain_focused(n=128, nz=20, xi=2.84).with_(d_eff=0.0)
    zf = focus * w.L
    # a window of ten radii at whichever end the beam is wider
    lw = 10 * max(W.beam_radius(0.0, w.w0, zf), W.beam_radius(w.L, w.w0, zf))
    w = w.with_(z_focus=zf, lx=lw, ly=lw)
    p, AF0, AF = _free_run(w)
    x = ssfm.axis(p.nx, p.lx).numpy()
    y = ssfm.axis(p.ny, p.ly).numpy()
    g0 = pins.gaussian_beam(x, y, 0.0, w.w0, w.z_focus, p.k_f)
    a0 = (AF0.numpy() / g0)[p.ny // 2, p.nx // 2]
    ref = a0 * pins.gaussian_beam(x, y, p.L, w.w0, w.z_focus, p.k_f)
    err = np.linalg.norm(AF.numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-9
    # second-moment radius w(z)^2 = 2 <r^2>
    I = np.abs(AF.numpy()) ** 2
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    wz = math.sqrt(2 * np.sum(r2 * I) / np.sum(I))
    z_r = w.w0 ** 2 * p.k_f / 2
    assert abs(wz / (w.w0 * math.sqrt(1 + ((p.L - w.z_focus) / z_r) ** 2)) - 1) < 1e-6
    # unitary propagator
    P0 = ssfm.power(AF0, p.n_f, p.dx, p.dy)
    P1 = ssfm.power(AF, p.n_f, p.dx, p.dy)
    assert abs(float(P1 / P0) - 1) < 1e-13


def test_beer_lambert_decay_of_both_waves():
    w = W.plain_focused(n=32, nz=40).with_(d_eff=0.0, alpha_f=7.0, alpha_sh=19.0)
    p = _p(w)
    AF0 = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus)
    AS0 = 0.3 * AF0.roll(3, 1)
    temp = ssfm.TemperatureField(p, None, 0, 0, 0.0)
    AF, AS = ssfm.propagate(p, AF0, AS0, temp)
    for A0, A, n, a in ((AF0, AF, p.n_f, p.alpha_f), (AS0, AS, p.n_sh, p.alpha_sh)):
        ratio = float(ssfm.power(A, n, p.dx, p.dy) / ssfm.power(A0, n, p.dx, p.dy))
        assert abs(ratio / math.exp(-a * p.L) - 1) < 1e-12


# -------------------------------------------------------------- coupling ----

def _uniform_run(w, AF0, AS0):
    p = _p(w)
    temp = ssfm.TemperatureField(p, None, 0, 0, w.t_off)
    return p, ssfm.propagate(p, AF0, AS0, temp)


def test_walkoff_is_an_exact_translation():
    """With tan(rho) dz equal to m grid cells, the walk-off factor is the
    shift theorem for an m-cell translation toward +x: the step with walk-off
    equals the step without it followed by a circular roll of m cells (SH
    only, the pump untouched)."""
    n, m = 32, 3
    base = W.plain_focused(n=n, nz=50)
    dx, dz = base.lx / n, base.L / base.nz
    w = base.with_(walkoff_sh=math.atan(m * dx / dz))
    rng = np.random.default_rng(5)
    AF = torch.tensor(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    AS = torch.tensor(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    f1, s1 = ssfm.Linear(_p(w))(AF, AS)
    f0, s0 = ssfm.Linear(_p(base))(AF, AS)
    assert torch.max(torch.abs(f1 - f0)) < 1e-12
    assert torch.max(torch.abs(s1 - torch.roll(s0, m, dims=1))) < 1e-11


def test_walkoff_moves_the_beam_centroid_at_tan_rho():
    """Linear propagation of the pump alone (no coupling, no losses) with a
    walk-off angle: the centroid of |A_F|^2 moves along x by tan(rho) z, while
    diffraction alone leaves it in place."""
    rho = 1e-3  # a 2-cell drift over L, so that the beam stays clear of the window edge
    w = W.plain_focused(n=64, nz=40).with_(d_eff=0.0, walkoff_f=rho)
    p = _p(w)
    AF0 = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus)
    AF, _, _ = ssfm.run(w)
    x = ssfm.axis(w.nx, w.lx)
    def cx(a):
        I = (a.abs() ** 2).sum(dim=0)
        return float((I * x).sum() / I.sum())
    assert abs(cx(AF0)) < 1e-12 * w.lx
    assert abs(cx(AF) - math.tan(rho) * w.L) < 1e-8 * (w.lx / w.nx)


def test_plane_wave_conversion_follows_tanh_squared():
    w = W.plain_focused(n=8, nz=1000)
    p = _p(w)
    gamma_L = 1.5
    a0 = gamma_L / (p.L * math.sqrt(p.kappa_f * p.kappa_sh))
    AF0 = torch.full((8, 8), a0, dtype=torch.complex128)
    AS0 = torch.zeros_like(AF0)
    p, (AF, AS) = _uniform_run(w, AF0, AS0)
    eta = float(ssfm.power(AS, p.n_sh, p.dx, p.dy) / ssfm.power(AF0, p.n_f, p.dx, p.dy))
    assert abs(eta - math.tanh(gamma_L) ** 2) < 1e-10


def test_phase_mismatched_plane_wave_follows_sinc_squared():
    """Undepleted uniform pump, no losses, Dk L = 3 pi: the SH equation is the
    quadrature A_SH(L) = i kappa_SH A_F^2 int_0^L e^{i Dk z} dz, so
    eta = (n_SH / n_F) kappa_SH^2 |A_F|^2 L^2 sinc^2(Dk L / 2).  RK4 on a
    quadrature is Simpson's rule, and the stage points' z enter through phi,
    so the rule must hold to 1e-8 at nz = 200."""
    w = W.plain_focused(n=8, nz=200, undepleted=True)
    dk = 3 * math.pi / w.L
    w = w.with_(dk0=dk)
    a0 = 1e6
    AF0 = torch.full((8, 8), a0, dtype=torch.complex128)
    AS0 = torch.zeros_like(AF0)
    p, (AF, AS) = _uniform_run(w, AF0, AS0)
    kappa_sh = 2 * math.pi * w.d_eff / (w.n_sh * w.lambda_f)
    x = dk * w.L / 2
    ref = (w.n_sh / w.n_f) * (kappa_sh * a0 * w.L * math.sin(x) / x) ** 2
    eta = float(ssfm.power(AS, p.n_sh, p.dx, p.dy) / ssfm.power(AF0, p.n_f, p.dx, p.dy))
    assert 1e-5 < ref < 1e-1
    assert abs(eta / ref - 1) < 1e-8
    assert float((AF - AF0).abs().max()) < 1e-9 * a0   # the pump stays put


def test_manley_rowe_without_losses():
    """P_F + P_SH is conserved up to the RK4 error, which falls as dz^4."""
    def defect(w):
        AF, AS, eta = ssfm.run(w)
        p = _p(w)
        tot = float(ssfm.power(AF, p.n_f, p.dx, p.dy) + ssfm.power(AS, p.n_sh, p.dx, p.dy))
        assert float(eta) > 0.01
        return abs(tot / w.p1 - 1)

    assert defect(W.plain_focused(n=32, nz=100)) < 1e-10
    lossless = W.depleted_absorbing(n=32, nz=100, tgrid=(16, 16, 24)).with_(
        alpha_f=0.0, alpha_sh=0.0, beta_sh=0.0)
    e100 = defect(lossless)
    e200 = defect(lossless.with_(nz=200))
    assert e200 < 1e-10
    assert e100 / e200 > 10.0


@pytest.mark.parametrize("xi,sigma", [(2.84, 0.0), (2.84, 0.5736), (2.84, -0.5736),
                                      (1.0, 0.5736)])
def test_boyd_kleinman_undepleted(xi, sigma):
    """Eq. (17) with h(sigma, xi) from independent quadrature.  BK assume the
    harmonic diffracts like the driving polarisation (k_SH = 2 k_F), so the pin
    uses n_SH = n_F; sigma = b Dk / 2 with b = L / xi."""
    w = W.plain_focused(n=128, nz=100, xi=xi, undepleted=True).with_(n_sh=W.N_F)
    b = w.L / xi
    w = w.with_(dk0=2 * sigma / b)
    _, _, eta = ssfm.run(w)
    ref = pins.bk_constant(w.d_eff, w.L, w.n_f, w.n_sh, w.lambda_f) * w.p1 * pins.bk_h(sigma, xi)
    assert abs(float(eta) / ref - 1) < 5e-4


def test_paper_optimum_focusing_from_bk_quadrature():
    """The paper's optimum xi = 2.84 (Sec. 5.1) and 29 um waist pin the BK
    reference and the xi = L/(2 z_R) convention."""
    gold = json.load(open(GOLDEN))
    from scipy.optimize import minimize_scalar

    def hmax(xi):
        r = minimize_scalar(lambda s: -pins.bk_h(s, xi), bounds=(0, 2), method="bounded",
                            options={"xatol": 1e-7})
        return -r.fun

    r = minimize_scalar(lambda xi: -hmax(xi), bounds=(1.5, 4.5), method="bounded",
                        options={"xatol": 1e-4})
    assert abs(r.x - gold["xi_opt"]["value"]) < 0.01
    assert abs(-r.fun - 1.068) < 1e-3
    w0 = W.waist_for_xi(gold["xi_opt"]["value"], gold["crystal_length_m"]["value"])
    assert abs(w0 * 1e6 - gold["w_F_at_xi_opt_um"]["value"]) < 0.5
    # h(0, xi) = arctan(xi)^2 / xi in closed form
    assert abs(pins.bk_h(0.0, 2.84) - math.atan(2.84) ** 2 / 2.84) < 1e-10


@pytest.mark.parametrize("wave", ["sh", "f"])
def test_two_photon_absorption_closed_form(wave):
    """One uniform wave alone (no coupling) with alpha_j and beta_j:
    second-order convergence to I0 e^{-a z} / (1 + b I0 (1 - e^{-a z}) / a)."""
    errs = []
    for nz in (50, 100):
        w = W.plain_focused(n=8, nz=nz).with_(d_eff=0.0)
        if wave == "sh":
            w = w.with_(alpha_sh=20.0, beta_sh=2e-12)
        else:
            w = w.with_(alpha_f=20.0, beta_f=2e-12)
        p = _p(w)
        a = 3e7
        full = torch.full((8, 8), a, dtype=torch.complex128)
        none = torch.zeros_like(full)
        AF0, AS0 = (none, full) if wave == "sh" else (full, none)
        p, (AF, AS) = _uniform_run(w, AF0, AS0)
        n, A, alpha, beta = ((p.n_sh, AS, p.alpha_sh, p.beta_sh) if wave == "sh"
                             else (p.n_f, AF, p.alpha_f, p.beta_f))
        I0 = 0.5 * ssfm.EPS0 * ssfm.C_LIGHT * n * a * a
        I = 0.5 * ssfm.EPS0 * ssfm.C_LIGHT * n * float(A[0, 0].abs() ** 2)
        ref = pins.tpa_plane_wave(I0, alpha, beta, p.L)
        assert ref < 0.5 * I0   # strong absorption regime
        errs.append(abs(I / ref - 1))
    assert errs[1] < 1e-5
    assert 3.5 < errs[0] / errs[1] < 4.5


# ------------------------------------------------------------ temperature ----

def test_trilinear_tables_exact_for_affine_maps():
    w = W.plain_focused(n=16, nz=10)
    p = _p(w)
    tx, ty, tz = 5, 6, 7
    t_lx, t_ly = 1.5 * p.lx, 1.5 * p.ly
    X = -t_lx / 2 + np.arange(tx) * t_lx / (tx - 1)
    Y = -t_ly / 2 + np.arange(ty) * t_ly / (ty - 1)
    Z = np.arange(tz) * p.L / (tz - 1)
    a, bx, cy, dz = 0.3, 1.7e3, -2.1e3, 40.0
    dT = a + bx * X[None, None, :] + cy * Y[None, :, None] + dz * Z[:, None, None]
    temp = ssfm.TemperatureField(p, torch.tensor(dT), t_lx, t_ly, 0.0)
    x = ssfm.axis(p.nx, p.lx).numpy()
    y = ssfm.axis(p.ny, p.ly).numpy()
    for z in (0.0, 0.3 * p.L, Z[3], p.L):
        d, c = temp.at(z)
        ref = a + bx * x[None, :] + cy * y[:, None] + dz * z
        assert np.max(np.abs(d.numpy() - ref)) < 1e-12
    # the trapezoid cumulative integral of a linear-in-z map is exact at nodes
    d, c = temp.at(Z[4])
    refc = (a + bx * x[None, :] + cy * y[:, None]) * Z[4] + dz * Z[4] ** 2 / 2
    assert np.max(np.abs(c.numpy() - refc)) < 1e-12


def test_temperature_map_is_clamped_outside_its_extent():
    """A map narrower than the field window: field points beyond its edge take
    the edge value (reading 7), so an affine map evaluates to the affine
    function at the coordinates clipped to the map's extent."""
    w = W.plain_focused(n=16, nz=10)
    p = _p(w)
    tx, ty, tz = 5, 4, 3
    t_lx, t_ly = 0.5 * p.lx, 0.4 * p.ly
    X = -t_lx / 2 + np.arange(tx) * t_lx / (tx - 1)
    Y = -t_ly / 2 + np.arange(ty) * t_ly / (ty - 1)
    Z = np.arange(tz) * p.L / (tz - 1)
    a, bx, cy, dz = -0.4, 2.3e3, 1.1e3, 25.0
    dT = a + bx * X[None, None, :] + cy * Y[None, :, None] + dz * Z[:, None, None]
    temp = ssfm.TemperatureField(p, torch.tensor(dT), t_lx, t_ly, 0.0)
    x = np.clip(ssfm.axis(p.nx, p.lx).numpy(), -t_lx / 2, t_lx / 2)
    y = np.clip(ssfm.axis(p.ny, p.ly).numpy(), -t_ly / 2, t_ly / 2)
    assert np.sum(np.abs(ssfm.axis(p.nx, p.lx).numpy()) > t_lx / 2) >= 4  # points outside
    for z in (0.0, 0.45 * p.L, p.L):
        d, _ = temp.at(z)
        ref = a + bx * x[None, :] + cy * y[:, None] + dz * z
        assert np.max(np.abs(d.numpy() - ref)) < 1e-12


def test_uniform_temperature_equals_shifted_mismatch():
    base = W.plain_focused(n=32, nz=30).with_(ddk_dT=-0.6 * 300, dn_dT=0.0)
    c = 1.7
    m = np.full((3, 4, 5), c)
    with_map = base.with_(dT=m, t_lx=base.lx, t_ly=base.ly)
    shifted = base.with_(dk0=base.dk0 + base.ddk_dT * c, ddk_dT=0.0)
    offset = base.with_(t_off=c)
    _, AS1, e1 = ssfm.run(with_map)
    _, AS2, e2 = ssfm.run(shifted)
    _, AS3, e3 = ssfm.run(offset)
    assert abs(float(e1) / float(e2) - 1) < 1e-12
    assert abs(float(e3) / float(e2) - 1) < 1e-12
    assert abs(float(e2) / float(ssfm.run(base)[2]) - 1) > 1e-3   # the shift matters


def test_uniform_lens_phase_rotates_fields():
    w = W.plain_focused(n=32, nz=100).with_(d_eff=0.0, dn_dT=1e-5)
    c = 2.0
    _, AF_free = _free_run(w)[0], _free_run(w)[2]
    AF, _, _ = ssfm.run(w.with_(t_off=c))
    k0 = 2 * math.pi / w.lambda_f
    ref = AF_free * np.exp(1j * k0 * w.dn_dT * c * w.L)
    err = float((AF - ref).abs().max() / ref.abs().max())
    assert err < 1e-8


# ------------------------------------------------------------------ heat ----

def _assemble(hx, hy, hz, dx, dy, dz):
    import scipy.sparse as sp
    n = (hz - 2) * (hy - 2) * (hx - 2)
    idx = -np.ones((hz, hy, hx), dtype=np.int64)
    idx[1:-1, 1:-1, 1:-1] = np.arange(n).reshape(hz - 2, hy - 2, hx - 2)
    rows, cols, vals = [], [], []
    for l in range(1, hz - 1):
        for j in range(1, hy - 1):
            for i in range(1, hx - 1):
                r = idx[l, j, i]
                rows.append(r); cols.append(r)
                vals.append(-2 / dx ** 2 - 2 / dy ** 2 - 2 / dz ** 2)
                for (ll, jj, ii, d) in ((l, j, i + 1, dx), (l, j, i - 1, dx), (l, j + 1, i, dy),
                                        (l, j - 1, i, dy), (l + 1, j, i, dz), (l - 1, j, i, dz)):
                    if idx[ll, jj, ii] >= 0:
                        rows.append(r); cols.append(idx[ll, jj, ii]); vals.append(1 / d ** 2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n)), idx


def test_sor_matches_direct_sparse_solve():
    from scipy.sparse.linalg import spsolve
    hx, hy, hz = 10, 8, 12
    wx, wy, L, kappa = 2e-3, 1e-3, 0.03, 8.4
    dx, dy, dz = wx / (hx - 1), wy / (hy - 1), L / (hz - 1)   # node-centred, faces included
    rng = np.random.default_rng(5)
    q = rng.uniform(0, 1e8, size=(hz, hy, hx))
    T, sweeps, corr = heat.sor_solve(torch.tensor(q), kappa, wx, wy, L, tol=1e-13)
    A, idx = _assemble(hx, hy, hz, dx, dy, dz)
    sol = spsolve(A.tocsc(), -q[1:-1, 1:-1, 1:-1].ravel() / kappa)
    ref = np.zeros_like(q)
    ref[1:-1, 1:-1, 1:-1] = sol.reshape(hz - 2, hy - 2, hx - 2)
    assert np.max(np.abs(T.numpy() - ref)) < 1e-9 * np.max(np.abs(ref))
    assert 1 < sweeps < 5000


def test_sor_recovers_discrete_eigenmode():
    hx, hy, hz = 17, 9, 33
    wx, wy, L, kappa = 2e-3, 1e-3, 0.03, 8.4
    dx, dy, dz = wx / (hx - 1), wy / (hy - 1), L / (hz - 1)   # node-centred, faces included
    X = np.arange(hx) * dx
    Y = np.arange(hy) * dy
    Z = np.arange(hz) * dz
    mode = (np.sin(np.pi * Z / L)[:, None, None] * np.sin(np.pi * Y / wy)[None, :, None]
            * np.sin(np.pi * X / wx)[None, None, :])
    lam = pins.discrete_laplacian_eigen(hx, hy, hz, dx, dy, dz)
    q = -kappa * lam * 3.0 * mode       # kappa lap T + q = 0 for T = 3 * mode
    T, _, _ = heat.sor_solve(torch.tensor(q), kappa, wx, wy, L, tol=1e-12)
    assert np.max(np.abs(T.numpy() - 3.0 * mode)) < 1e-9


def _slab_profile(coord, length, q, kappa, h, t_inf):
    """Steady 1-D profile of kappa T'' + q = 0 with T(0) = 0 and the
    convective end -kappa T'(length) = h (T(length) - t_inf): a quadratic,
    T = -q s^2 / (2 kappa) + A s."""
    A = (q * length + h * q * length ** 2 / (2 * kappa) + h * t_inf) / (kappa + h * length)
    return -q * coord ** 2 / (2 * kappa) + A * coord


@pytest.mark.parametrize("axis", ["z", "y"])
def test_convective_face_slab_closed_form(axis):
    """Eq. (10) on one face, Eq. (9) on the opposite one, insulated sides
    (h = 0) and a uniform source: the solution is the quadratic slab profile,
    and the ghost-node scheme is exact for quadratics, so the discrete
    solution equals it at the nodes.  axis z: oven at the entrance face,
    convection at the exit face; axis y: the bottom-oven configuration of
    Sec. 4.2 reduced to one dimension."""
    hx, hy, hz = 5, 6, 17
    # a short crystal keeps the z spacing near the transverse ones (the
    # profile is exact at any length; a 30 mm one only slows the SOR down)
    wx, wy, L, kappa = 2e-3, 1e-3, 4e-3, 8.4
    q0 = 3e6 if axis == "z" else 3e5
    if axis == "z":
        faces, hs, length, h = ("C", "C", "C", "C", "D", "C"), (0, 0, 0, 0, 0, 350.0), L, 350.0
    else:
        faces, hs, length, h = ("C", "C", "D", "C", "C", "C"), (0, 0, 0, 800.0, 0, 0), wy, 800.0
    bc = heat.HeatBC(faces, hs, -3.0)
    q = torch.full((hz, hy, hx), q0, dtype=torch.float64)
    T, sweeps, _ = heat.sor_solve(q, kappa, wx, wy, L, tol=1e-13, max_sweeps=200000, bc=bc)
    dx, dy, dz = heat.spacings(hx, hy, hz, wx, wy, L)
    if axis == "z":
        ref = _slab_profile(np.arange(hz) * dz, L, q0, kappa, h, -3.0)[:, None, None]
    else:
        ref = _slab_profile(np.arange(hy) * dy, wy, q0, kappa, h, -3.0)[None, :, None]
    ref = np.broadcast_to(ref, T.shape)
    assert np.max(np.abs(T.numpy() - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(ref)) > 0.1


def test_all_convective_faces_balance_the_source_exactly():
    """With every face convective (no oven), summing the node equations over
    the node cells (halved on each face) telescopes to the discrete energy
    balance sum q_i V_i = sum over face nodes of h (T_i - T_inf) A_i, A_i the
    face cell's area; it holds to the solver's tolerance for any source, and
    covers the edges and corners where two or three faces meet."""
    hx, hy, hz = 7, 6, 9
    wx, wy, L, kappa, h, t_inf = 2e-3, 1e-3, 0.03, 8.4, 2e3, 0.7
    bc = heat.HeatBC(("C",) * 6, h, t_inf)
    rng = np.random.default_rng(8)
    q = rng.uniform(0, 1e7, size=(hz, hy, hx))
    T, _, _ = heat.sor_solve(torch.tensor(q), kappa, wx, wy, L, tol=1e-14, max_sweeps=500000,
                             bc=bc)
    T = T.numpy()
    dx, dy, dz = heat.spacings(hx, hy, hz, wx, wy, L)
    wgt = [np.ones(n) for n in (hz, hy, hx)]
    for w_ in wgt:
        w_[0] = w_[-1] = 0.5
    V = dx * dy * dz * wgt[0][:, None, None] * wgt[1][None, :, None] * wgt[2][None, None, :]
    gen = float((q * V).sum())
    out = 0.0
    for axis, (d, n) in enumerate(((dz, hz), (dy, hy), (dx, hx))):
        others = [k for k in range(3) if k != axis]
        area = dx * dy * dz / d
        for end in (0, n - 1):
            sl = [slice(None)] * 3
            sl[axis] = end
            wf = np.ones_like(T[tuple(sl)])
            shape2 = [T.shape[k] for k in others]
            wf = wgt[others[0]][:, None] * wgt[others[1]][None, :]
            out += float((h * (T[tuple(sl)] - t_inf) * area * wf.reshape(shape2)).sum())
    assert abs(out / gen - 1) < 1e-9, (out, gen)


def test_convective_sor_matches_direct_sparse_solve():
    """A mixed configuration (oven on y- and z-, convection elsewhere, with
    different h per face) against scipy's sparse direct solve of the same
    node equations."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve
    hx, hy, hz = 6, 5, 7
    wx, wy, L, kappa = 2e-3, 1e-3, 0.03, 8.4
    hs = (400.0, 900.0, 0.0, 1500.0, 0.0, 250.0)
    bc = heat.HeatBC(("C", "C", "D", "C", "D", "C"), hs, 1.5)
    dx, dy, dz = heat.spacings(hx, hy, hz, wx, wy, L)
    rng = np.random.default_rng(9)
    q = rng.uniform(0, 1e7, size=(hz, hy, hx))
    T, _, _ = heat.sor_solve(torch.tensor(q), kappa, wx, wy, L, tol=1e-14, max_sweeps=500000,
                             bc=bc)
    unknown = heat.unknown_mask((hz, hy, hx), bc).numpy()
    idx = -np.ones((hz, hy, hx), dtype=int)
    idx[unknown] = np.arange(int(unknown.sum()))
    rows, cols, vals, rhs = [], [], [], []
    dims = (hz, hy, hx)
    sp_of = (dz, dy, dx)
    face = {(2, 0): 0, (2, 1): 1, (1, 0): 2, (1, 1): 3, (0, 0): 4, (0, 1): 5}
    for node in zip(*np.nonzero(unknown)):
        r = idx[node]
        b = -q[node] / kappa
        diag = 0.0
        for axis in range(3):
            a = 1.0 / sp_of[axis] ** 2
            diag -= 2 * a
            for step, side in ((-1, 0), (1, 1)):
                nb = list(node)
                nb[axis] += step
                if 0 <= nb[axis] < dims[axis]:
                    target = [tuple(nb)]
                else:
                    # ghost beyond a convective face: 2 x the inner neighbour,
                    # and -2 d (h / kappa) (T - T_inf)
                    hk = hs[face[(axis, side)]]
                    inner = list(node)
                    inner[axis] -= step
                    target = [tuple(inner)]
                    diag -= 2 * a * sp_of[axis] * hk / kappa
                    b -= 2 * a * sp_of[axis] * hk / kappa * 1.5
                for t in target:
                    if idx[t] >= 0:
                        rows.append(r); cols.append(idx[t]); vals.append(a)
        rows.append(r); cols.append(r); vals.append(diag)
        rhs.append(b)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(len(rhs), len(rhs)))
    sol = spsolve(A.tocsc(), np.array(rhs))
    ref = np.zeros((hz, hy, hx))
    ref[unknown] = sol
    assert np.max(np.abs(T.numpy() - ref)) < 1e-9 * np.max(np.abs(ref))


def test_heat_deposits_balance_absorbed_power():
    """P_in - P_out = sum of deposited q_dot dV, to the trapezoid rule's O(dz^2)."""
    errs = []
    for nz in (40, 80):
        w = W.plain_focused(n=32, nz=nz, p1=2e3).with_(alpha_f=5.0, alpha_sh=30.0,
                                                      beta_sh=5e-12, beta_f=1e-12)
        p = _p(w)
        dep = ssfm.HeatDeposit(p, 9, 9, 11, p.lx, p.ly)
        AF, AS, eta = ssfm.run(w, deposit=dep)
        lost = w.p1 - float(ssfm.power(AF, p.n_f, p.dx, p.dy) + ssfm.power(AS, p.n_sh, p.dx, p.dy))
        assert float(eta) > 1e-3 and lost > 0.05 * w.p1
        errs.append(abs(float(dep.Q.sum()) / lost - 1))
    assert errs[1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 5.0


def test_heat_deposit_lands_on_the_nearest_node():
    """One field sample at a time: its q_dot dV (Eq. 8) goes to the heat node
    nearest to it in x, y and z, found here by brute-force distance; a sample
    more than half a cell beyond the heat grid deposits nothing."""
    w = W.plain_focused(n=16, nz=10).with_(alpha_f=3.0)
    p = _p(w)
    hx, hy, hz = 7, 5, 4
    wx, wy = 0.8 * p.lx, 0.6 * p.ly
    dep = ssfm.HeatDeposit(p, hx, hy, hz, wx, wy)
    x = ssfm.axis(p.nx, p.lx).numpy()
    y = ssfm.axis(p.ny, p.ly).numpy()
    X = -wx / 2 + np.arange(hx) * wx / (hx - 1)
    Y = -wy / 2 + np.arange(hy) * wy / (hy - 1)
    Zn = np.arange(hz) * p.L / (hz - 1)
    a, wz = 1e6, 1e-3
    q_ref = p.alpha_f * 0.5 * pins.EPS0 * pins.C_LIGHT * p.n_f * a * a * p.dx * p.dy * wz
    inside_seen = outside_seen = 0
    for (m, k, z) in ((3, 5, 0.37 * p.L), (8, 8, 0.9 * p.L), (12, 2, 0.1 * p.L),
                      (0, 7, 0.5 * p.L), (10, 15, 0.62 * p.L), (13, 11, 0.0)):
        AF = torch.zeros((p.ny, p.nx), dtype=torch.complex128)
        AF[k, m] = a
        dep.Q.zero_()
        dep.add(AF, torch.zeros_like(AF), z, wz)
        i, j, l = (int(np.argmin(np.abs(X - x[m]))), int(np.argmin(np.abs(Y - y[k]))),
                   int(np.argmin(np.abs(Zn - z))))
        inside = (abs(X[i] - x[m]) < 0.5 * wx / (hx - 1)
                  and abs(Y[j] - y[k]) < 0.5 * wy / (hy - 1))
        if inside:
            inside_seen += 1
            assert abs(float(dep.Q[l, j, i]) / q_ref - 1) < 1e-12
            assert abs(float(dep.Q.sum()) - float(dep.Q[l, j, i])) == 0.0
        else:
            outside_seen += 1
            assert float(dep.Q.abs().sum()) == 0.0
    assert inside_seen >= 3 and outside_seen >= 2


def test_thermal_loop_fixed_point_behaviour():
    """The self-consistent loop of Fig. 2 on a small grid (100 W, 2 x 1 x 30 mm
    crystal):
    - without absorption nothing is deposited: dT stays 0 and every iteration
      repeats the plain propagation's eta exactly;
    - with absorption the first iteration starts from q_dot = 0 (the plain
      eta again);
    - every solve gives dT >= 0 with zero faces (maximum principle for a
      non-negative source and Dirichlet faces);
    - the iteration contracts: the second change is under a fifth of the first."""
    w = W.thermal_loop(n=16, nz=40, heat=(9, 9, 11), n_outer=3, p1=100.0)
    lossless = w.with_(alpha_f=0.0, alpha_sh=0.0, beta_f=0.0, beta_sh=0.0)
    eta_plain = float(ssfm.run(lossless.with_(dT=None))[2])
    for it in heat.thermal_loop(lossless, 3):
        assert float(it["dT"].abs().max()) == 0.0
        assert abs(it["eta"] / eta_plain - 1) < 1e-13
    h = heat.thermal_loop(w, 3)
    assert abs(h[0]["eta"] / float(ssfm.run(w.with_(dT=None))[2]) - 1) < 1e-13
    assert h[0]["change"] == 0.0
    for it in h[1:]:
        dT = it["dT"]
        assert float(dT.min()) >= 0.0 and float(dT.max()) > 0.1
        faces = (dT[0], dT[-1], dT[:, 0], dT[:, -1], dT[:, :, 0], dT[:, :, -1])
        assert all(float(f.abs().max()) == 0.0 for f in faces)
    assert h[1]["change"] > 1.0
    assert h[2]["change"] < 0.2 * h[1]["change"]
    # each iteration propagates through its solved dT as a map over the
    # crystal cross-section wx x wy (reading 12), nothing else
    for it in h[1:]:
        ref = ssfm.run(w.with_(dT=it["dT"].numpy(), t_lx=w.wx, t_ly=w.wy))[2]
        assert abs(it["eta"] / float(ref) - 1) < 1e-13


def test_loop_with_convective_faces_conserves_energy():
    """Every face convective (no oven): in steady state all the heat the beams
    deposit (Eq. 8) leaves through the faces by convection (Eq. 10).  The
    second iteration's dT, solved from the first pass's deposits, carries
    exactly that heat out; this holds only if a face node's source density
    uses its half-size cell (the entrance and exit facets receive deposits)."""
    w = W.thermal_loop(n=16, nz=40, heat=(9, 9, 11), n_outer=2, p1=100.0)
    w = w.with_(heat_faces=("C",) * 6, h_conv=4e3, t_inf=0.0)
    hist = heat.thermal_loop(w, 2, tol=1e-13, max_sweeps=500000)
    deposited = float(hist[0]["Q"].sum())
    assert deposited > 0.01 * w.p1
    T = hist[1]["dT"].numpy()
    hx, hy, hz = w.hx, w.hy, w.hz
    dx, dy, dz = heat.spacings(hx, hy, hz, w.wx, w.wy, w.L)
    wgt = [np.ones(n) for n in (hz, hy, hx)]
    for w_ in wgt:
        w_[0] = w_[-1] = 0.5
    out = 0.0
    for axis, d in enumerate((dz, dy, dx)):
        others = [k for k in range(3) if k != axis]
        for end in (0, T.shape[axis] - 1):
            sl = [slice(None)] * 3
            sl[axis] = end
            wf = wgt[others[0]][:, None] * wgt[others[1]][None, :]
            out += float((w.h_conv * T[tuple(sl)] * (dx * dy * dz / d) * wf).sum())
    assert abs(out / deposited - 1) < 1e-8, (out, deposited)


# ------------------------------------------------- Eq. (4) phase mismatch ----

def _eq4_case():
    w = W.depleted_absorbing(n=32, nz=60, tgrid=(8, 8, 12), p1=300.0)
    return w.with_(ddk_dT=0.0, dk0=0.0, t_off=1.5)


def test_eq4_with_linear_indices_and_rigid_grating_is_the_linearised_model():
    """With n_j(T) linear in T and a rigid grating (a = b = 0), Eq. (4) is
    exactly Dk(T_oven) + g (T - T_oven), g = (4 pi / lambda_F) (n_SH' - n_F').
    With the period chosen for phase matching at T_oven (Dk(T_oven) = 0), the
    Eq. (4) run must reproduce the linearised run (dk0 = 0, dDk/dT = g) with
    the same map and oven offset, to rounding."""
    w = _eq4_case()
    lam = w.lambda_f
    nF0, sF, nS0, sS, t_oven = 2.14, 3e-5, 2.18, 9e-5, 48.0
    dn = (nS0 - nF0) + (sS - sF) * (t_oven - 25.0)
    period = lam / (2.0 * dn)              # 2 pi / period = (4 pi / lambda) dn
    g = 4.0 * math.pi / lam * (sS - sF)
    q = W.Qpm(t_oven=t_oven, lambda25=period, a_lambda=0.0, b_lambda=0.0,
              n_f_t=(nF0, sF), n_sh_t=(nS0, sS))
    AF, AS, eta = ssfm.run(w.with_(qpm=q))
    AF2, AS2, eta2 = ssfm.run(w.with_(ddk_dT=g))
    # rounding: Dk(T_ref + dT) - Dk(T_ref) cancels two terms of ~5e5 / m
    assert abs(float(eta) / float(eta2) - 1) < 1e-10
    assert float((AS - AS2).norm() / AS2.norm()) < 1e-9
    # and the slope matters at this size: without it the result differs
    assert abs(float(ssfm.run(w)[2]) / float(eta2) - 1) > 1e-3


def test_eq4_zero_crossing_at_the_constructed_phase_matching_temperature():
    """The paper's grating expansion (a_Lambda, b_Lambda of MgO:sPPLT) and
    temperature-dependent indices; the period at 25 C is chosen so that the
    quasi-phase-matching condition 2 pi / Lambda(T_pm) = (4 pi / lambda_F)
    (n_SH - n_F)(T_pm) holds at T_pm = 60 C.  At T_oven + T_off = T_pm the
    uniform-temperature run equals the phase-matched run (Dk = 0) to rounding;
    3 K away it does not."""
    w = _eq4_case().with_(dT=None, dn_dT=0.0)
    lam = w.lambda_f
    a, b, t_pm = 2.2e-6, -5.9e-9, 60.0
    nF, nS = (2.14, 2e-5, 3e-8), (2.18, 7e-5, -4e-8)
    u = t_pm - 25.0
    dn = sum(c * u ** k for k, c in enumerate(nS)) - sum(c * u ** k for k, c in enumerate(nF))
    lam25 = lam / (2.0 * dn) / (1.0 + a * u + b * u * u)
    q = W.Qpm(t_oven=55.0, lambda25=lam25, a_lambda=a, b_lambda=b, n_f_t=nF, n_sh_t=nS)
    AF, AS, eta = ssfm.run(w.with_(qpm=q, t_off=5.0))
    AF0, AS0, eta0 = ssfm.run(w.with_(t_off=0.0))        # dk0 = 0: phase matched
    assert abs(float(eta) / float(eta0) - 1) < 1e-10
    assert float((AS - AS0).norm() / AS0.norm()) < 1e-9
    eta_off = float(ssfm.run(w.with_(qpm=q, t_off=8.0))[2])
    assert eta_off < (1 - 1e-3) * float(eta0)


# ------------------------------------------------------------- gradients ----

def _grad_case():
    w = W.depleted_absorbing(n=16, nz=12, tgrid=(5, 6, 7), xi=2.0, p1=400.0)
    return w.with_(t_off=0.3, ddk_dT=-60.0, dn_dT=3e-4)


def _eta(w, w0, zf, toff, dT):
    return ssfm.run(w, w0=w0, z_focus=zf, t_off=toff, dT=dT)[2]


def test_autograd_gradients_match_central_differences():
    w = _grad_case()
    dT0 = torch.tensor(w.dT, dtype=torch.float64)
    w0 = torch.tensor(w.w0, dtype=torch.float64, requires_grad=True)
    zf = torch.tensor(w.z_focus, dtype=torch.float64, requires_grad=True)
    to = torch.tensor(w.t_off, dtype=torch.float64, requires_grad=True)
    dT = dT0.clone().requires_grad_(True)
    eta = _eta(w, w0, zf, to, dT)
    g_w0, g_zf, g_to, g_dT = torch.autograd.grad(eta, (w0, zf, to, dT))
    # invariant: the oven offset enters as a uniform dT
    assert abs(float(g_to) - float(g_dT.sum())) < 1e-10 * float(g_dT.abs().sum())

    def fd(fun, x, h):
        return (float(fun(x + h)) - float(fun(x - h))) / (2 * h)

    with torch.no_grad():
        cases = [
            (g_w0, fd(lambda v: _eta(w, v, w.z_focus, w.t_off, dT0), w.w0, 1e-4 * w.w0)),
            (g_zf, fd(lambda v: _eta(w, w.w0, v, w.t_off, dT0), w.z_focus, 1e-4 * w.z_focus)),
            (g_to, fd(lambda v: _eta(w, w.w0, w.z_focus, v, dT0), w.t_off, 1e-4)),
        ]
        rng = np.random.default_rng(7)
        d = torch.tensor(rng.normal(size=tuple(dT0.shape)))
        cases.append(((g_dT * d).sum(),
                      fd(lambda s: _eta(w, w.w0, w.z_focus, w.t_off, dT0 + s * d), 0.0, 1e-4)))
    for g, ref in cases:
        assert abs(float(g) - ref) <= 1e-6 * abs(ref) + 1e-12
