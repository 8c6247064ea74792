"""GPU parity of the forward split-step path (C ABI) against the FP64 oracle.

Element-by-element comparison of both fields and of eta on the same seeded
inputs.  Bars: FP64 fields agree to 1e-9; FP32 fields to a relative L2 error
of 1e-4 and eta to a relative error of 1e-4.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from tests.helpers import ETA_TOL, FIELD_TOL, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _compare(w, eta_tol, field_tol, fields=None):
    eta, a_f, a_sh = gpu_run(w, fields)
    eta_ref, AF, AS = oracle_run(w, fields)
    e_eta = abs(eta / eta_ref - 1) if eta_ref != 0 else abs(eta)
    e_f = rel_l2(a_f, AF)
    e_s = rel_l2(a_sh, AS) if float(AS.norm()) > 0 else float(a_sh.abs().max())
    assert math.isfinite(eta)
    assert e_eta <= eta_tol, (w.name, eta, eta_ref, e_eta)
    assert e_f <= field_tol, (w.name, e_f)
    assert e_s <= field_tol, (w.name, e_s)
    return eta, eta_ref


@pytest.mark.parametrize("undepleted", [False, True])
def test_plain_fp64_32x32(undepleted):
    """Plain SSFM, 32 x 32, nz = 100, FP64 throughout (undepleted and depleted)."""
    w = W.plain_focused(n=32, nz=100, undepleted=undepleted)
    _compare(w, 1e-9, 1e-9)


def test_depleted_absorbing_fp32_128x128_full():
    """Depleted pump with alpha, TPA, seeded dT map and lens, 128 x 128, nz = 1000."""
    w = W.depleted_absorbing()
    _compare(w, ETA_TOL, FIELD_TOL)


@pytest.mark.parametrize("n", [8, 16, 32, 64, 128, 256, 512, 1024])
def test_every_transform_length_fp32(n):
    """Square grids of every supported size, thermal map on, a few steps."""
    nz = {8: 20, 16: 20, 32: 20, 64: 12, 128: 8, 256: 4, 512: 2, 1024: 1}[n]
    w = W.depleted_absorbing(n=n, nz=nz, tgrid=(9, 7, 5), p1=400.0)
    _compare(w, ETA_TOL, FIELD_TOL)


@pytest.mark.parametrize("nx,ny", [(64, 16), (16, 128), (8, 1024), (256, 32)])
def test_rectangular_grids_fp32(nx, ny):
    base = W.depleted_absorbing(n=64, nz=6, tgrid=(6, 9, 4), p1=300.0)
    w = base.with_(nx=nx, ny=ny, ly=base.ly * ny / max(nx, ny), lx=base.lx * nx / max(nx, ny))
    _compare(w, ETA_TOL, FIELD_TOL)


@pytest.mark.parametrize("n", [8, 16, 64, 256])
def test_fp64_transform_lengths(n):
    """FP64 fields with a temperature map (stored and sampled in double)."""
    w = W.depleted_absorbing(n=n, nz=6, tgrid=(5, 5, 5), p1=300.0).with_(precision="f64")
    _compare(w, 1e-9, 1e-9)


@pytest.mark.parametrize("n", [8, 64, 256])
def test_fp64_without_map(n):
    w = W.depleted_absorbing(n=n, nz=6, tgrid=(5, 5, 5), p1=300.0).with_(
        precision="f64", dT=None, t_off=0.4)
    _compare(w, 1e-9, 1e-9)


def test_plane_wave_custom_fields_tanh_law():
    """Uniform fields set through shg_set_fields: eta follows tanh^2 and the oracle."""
    w = W.plain_focused(n=16, nz=400, precision="f32")
    from oracle.ssfm import params_from_workload
    p = params_from_workload(w)
    gl = 1.2
    a0 = gl / (p.L * math.sqrt(p.kappa_f * p.kappa_sh))
    AF0 = torch.full((16, 16), a0, dtype=torch.complex128)
    AS0 = torch.zeros_like(AF0)
    eps0c = 8.8541878128e-12 * 299792458.0
    p1 = 0.5 * eps0c * p.n_f * a0 * a0 * p.lx * p.ly
    w = w.with_(p1=p1)
    eta, eta_ref = _compare(w, ETA_TOL, FIELD_TOL, fields=(AF0, AS0))
    assert abs(eta - math.tanh(gl) ** 2) < 1e-5


def test_zero_power_and_zero_coupling():
    w = W.depleted_absorbing(n=32, nz=10, tgrid=(5, 5, 5))
    eta, a_f, a_sh = gpu_run(w.with_(p1=0.0))
    assert eta == 0.0 and float(a_f.abs().max()) == 0.0
    w2 = w.with_(d_eff=0.0)
    eta2, a_f2, a_sh2 = gpu_run(w2)
    assert eta2 == 0.0 and float(a_sh2.abs().max()) == 0.0
    eta_ref, AF, AS = oracle_run(w2)
    assert rel_l2(a_f2, AF) < FIELD_TOL


def test_single_step():
    w = W.depleted_absorbing(n=64, nz=1, tgrid=(5, 5, 5), p1=500.0)
    _compare(w, ETA_TOL, FIELD_TOL)


def test_undepleted_fp32_matches_oracle():
    w = W.plain_focused(n=64, nz=50, undepleted=True, precision="f32")
    _compare(w, ETA_TOL, FIELD_TOL)


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4", "5"])
@pytest.mark.parametrize("n", [32, 64, 128, 256, 512, 1024])
def test_every_kernel_flavour_of_the_autotuner(n, variant, monkeypatch):
    """Each kernel flavour the autotuner can pick, forced through
    SHG_FFT_VARIANT (0/1: the two FFT shapes with cp.async staging, 2: the
    TMA-staged column pass, 3/4: both passes in 128-/64-thread CTAs, 5: the
    column pass in 512-thread CTAs at 512 and 1024), matches the oracle on its
    own (single plans kept on the streaming passes).  A flavour a length does
    not have falls back to flavour 0."""
    monkeypatch.setenv("SHG_FFT_VARIANT", variant)
    monkeypatch.setenv("SHG_CLUSTER", "0")
    w = W.depleted_absorbing(n=n, nz=6 if n < 512 else (2 if n == 512 else 1), tgrid=(9, 7, 5),
                             p1=400.0)
    _compare(w, ETA_TOL, FIELD_TOL)


def test_wide_column_flavour_over_several_steps_and_rectangular(monkeypatch):
    """Flavour 5 (4 columns per CTA at 1024, 8 at 512) over several steps, with
    nx != ny, so that a CTA's tile is not the whole row (ny = 1024 columns of
    length 1024, nx = 256 columns per row for ny = 512)."""
    monkeypatch.setenv("SHG_FFT_VARIANT", "5")
    monkeypatch.setenv("SHG_CLUSTER", "0")
    w = W.depleted_absorbing(n=256, nz=8, tgrid=(9, 7, 5), p1=400.0)
    _compare(w.with_(ny=512, ly=2 * w.ly), ETA_TOL, FIELD_TOL)
    _compare(w.with_(nx=128, lx=w.lx / 2, ny=1024, ly=4 * w.ly, nz=3), ETA_TOL, FIELD_TOL)


def test_bounded_wait_reports_timeout_and_context_survives(monkeypatch):
    """A device-side wait that runs out (the TMA column pass with a poll
    limit of 0, so every mbarrier wait gives up at once) is reported as
    SHG_ERR_TIMEOUT by the next efficiency call; the CTAs drain their copies
    before returning, and the same plan with the default limit afterwards
    matches the oracle."""
    import paper_2410_04994_gb300 as pkg
    monkeypatch.setenv("SHG_FFT_VARIANT", "2")
    monkeypatch.setenv("SHG_CLUSTER", "0")   # the TMA column pass is a streaming pass
    w = W.plain_focused(n=64, nz=4, precision="f32")
    plan = pkg.Plan(w)
    pkg.shg_set_wait_limit(plan.handle, 0)
    plan.propagate()
    with pytest.raises(pkg.ShgError) as ei:
        plan.efficiency()
    assert ei.value.status == pkg.SHG_ERR_TIMEOUT
    pkg.shg_set_wait_limit(plan.handle, 1 << 20)
    plan.propagate()
    eta, _, _ = plan.efficiency()
    eta_ref, _, _ = oracle_run(w)
    assert abs(eta / eta_ref - 1) < ETA_TOL
    with pytest.raises(pkg.ShgError):
        pkg.shg_set_wait_limit(None, 0)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_walkoff_of_both_waves(precision):
    """Walk-off of both waves (opposite directions), with coupling, losses and
    a seeded temperature map, against the oracle."""
    w = W.depleted_absorbing(n=64, nz=40, tgrid=(9, 7, 5), p1=400.0).with_(
        walkoff_f=2e-3, walkoff_sh=-5e-3, precision=precision)
    if precision == "f64":
        _compare(w, 1e-9, 1e-9)
    else:
        _compare(w, ETA_TOL, FIELD_TOL)
