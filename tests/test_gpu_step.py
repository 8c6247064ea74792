"""The one-pass-per-step schedule against the oracle and against the two-pass
schedule.

FP32 plans on the per-point temperature table without monitors, heat deposits
or adjoint state run nz + 1 passes: even passes in the row layout (Lx, N, Lx),
odd passes in the column layout (Ly, N, Ly), which applies L = Lx Ly in
alternating order (the two factors commute exactly).  Bars: eta and field L2
1e-4 against the oracle (the FP32 bar), 2e-5 against the two-pass schedule
(the same arithmetic in another rounding order).
"""
import pytest
import torch

import workloads as W
from tests.helpers import ETA_TOL, FIELD_TOL, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _check(w):
    eta, a_f, a_sh = gpu_run(w)
    eta_ref, AF, AS = oracle_run(w)
    assert abs(eta / eta_ref - 1) <= ETA_TOL, (w.name, eta, eta_ref)
    assert rel_l2(a_f, AF) <= FIELD_TOL and rel_l2(a_sh, AS) <= FIELD_TOL, w.name
    return eta, a_f, a_sh


@pytest.mark.parametrize("n,nz", [(16, 7), (32, 8), (64, 9), (128, 6), (256, 5), (512, 4),
                                  (1024, 3)])
def test_step_schedule_matches_oracle(n, nz, monkeypatch):
    monkeypatch.setenv("SHG_CLUSTER", "0")
    _check(W.depleted_absorbing(n=n, nz=nz, tgrid=(9, 7, 5), p1=400.0))


@pytest.mark.parametrize("nz", [2, 3, 4])
def test_shortest_schedules(nz, monkeypatch):
    """nz = 2 ends on a row pass with the transform before the nonlinear part
    (and no transform after it), nz = 3 on a column pass.  (nz = 1 never takes
    this schedule: a map of two layers spans more than one step then, so the
    per-point table path is not admitted.)"""
    monkeypatch.setenv("SHG_CLUSTER", "0")
    eta, _, _ = _check(W.depleted_absorbing(n=64, nz=nz, tgrid=(5, 5, 2), p1=60.0))
    assert 0.1 < eta < 0.5   # a physical conversion at this coarse step


@pytest.mark.parametrize("nx,ny", [(256, 64), (64, 256), (32, 1024)])
def test_rectangular_grids(nx, ny, monkeypatch):
    monkeypatch.setenv("SHG_CLUSTER", "0")
    w = W.depleted_absorbing(n=64, nz=6, tgrid=(9, 7, 5), p1=400.0)
    _check(w.with_(nx=nx, ny=ny, lx=w.lx * nx / 64, ly=w.ly * ny / 64))


@pytest.mark.parametrize("variant", ["0", "1", "3", "4"])
def test_each_row_flavour(variant, monkeypatch):
    monkeypatch.setenv("SHG_CLUSTER", "0")
    monkeypatch.setenv("SHG_FFT_VARIANT", variant)
    _check(W.depleted_absorbing(n=128, nz=7, tgrid=(9, 7, 5), p1=400.0))


def test_step_schedule_equals_the_two_pass_schedule(monkeypatch):
    """The same plan through both schedules (fresh plans: the schedule is
    fixed when a plan's graph is captured)."""
    monkeypatch.setenv("SHG_CLUSTER", "0")
    w = W.depleted_absorbing(n=256, nz=40, tgrid=(16, 16, 20), p1=200.0)
    eta_s, af_s, ash_s = gpu_run(w)
    monkeypatch.setenv("SHG_STEP_PASSES", "0")
    eta_t, af_t, ash_t = gpu_run(w)
    assert abs(eta_s / eta_t - 1) < 2e-5
    assert rel_l2(af_s, af_t.to(torch.complex128)) < 2e-5
    assert rel_l2(ash_s, ash_t.to(torch.complex128)) < 2e-5


def test_step_schedule_in_a_mixed_batch():
    """A batch of three grid groups (one graph launch, one branch per group),
    against the oracle for every instance."""
    import paper_2410_04994_gb300 as pkg
    insts = W.sweep_instances(nz=9, groups=((64, 2), (128, 2), (256, 1)), tgrid=(9, 9, 6))
    plans = [pkg.Plan(w) for w in insts]
    for p, w in zip(plans, insts):
        p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for p, w, e in zip(plans, insts, etas):
        eta_ref, AF, AS = oracle_run(w)
        assert abs(e / eta_ref - 1) <= ETA_TOL, (w.name, e, eta_ref)
        a_f, a_sh = p.fields()
        assert rel_l2(a_f.cpu(), AF) <= FIELD_TOL and rel_l2(a_sh.cpu(), AS) <= FIELD_TOL


def test_pass_times_report_the_step_kernels():
    """shg_pass_times times the row- and column-layout step passes for a
    group on this schedule; both take about as long as a row pass."""
    import paper_2410_04994_gb300 as pkg
    insts = W.sweep_instances(nz=9, groups=((256, 4),), tgrid=(9, 9, 6))
    plans = [pkg.Plan(w) for w in insts]
    for p, w in zip(plans, insts):
        p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    g = pkg.shg_pass_times([p.handle for p in plans], nsteps=3)[0]
    assert g["nx"] == 256 and g["instances"] == 4 and g["passes_per_step"] == 1
    assert g["row_ms"] > 0 and g["col_ms"] > 0
    assert 0.3 < g["col_ms"] / g["row_ms"] < 3


@pytest.mark.parametrize("variant", [None, "1"])
def test_heat_deposits_agree_between_the_schedules(variant, monkeypatch):
    """A THERMAL plan with a map deposits q_dot dV at every z_s in whichever
    layout the pass runs; the heat grid and eta agree with the two-pass
    schedule (deposit order differs: float bins, double atomics).  Variant
    "1": both step passes in the 8-element shape."""
    import numpy as np
    if variant is not None:
        monkeypatch.setenv("SHG_FFT_VARIANT", variant)
    import paper_2410_04994_gb300 as pkg
    w = W.thermal_loop(n=128, nz=60, heat=(32, 24, 40), p1=100.0, n_outer=1)
    dT = np.asarray(W.depleted_absorbing(n=128, nz=60, tgrid=(12, 12, 20)).dT)

    def run():
        plan = pkg.Plan(w, thermal=True)
        plan.set_temperature(torch.as_tensor(dT), w.t_lx, w.t_ly)
        plan.propagate()
        eta = plan.efficiency()[0]
        q = torch.empty((w.hz, w.hy, w.hx), dtype=torch.float64, device="cuda")
        pkg.shg_get_heat(plan.handle, q, None)
        return eta, q.cpu().numpy()

    eta_s, q_s = run()
    monkeypatch.setenv("SHG_STEP_PASSES", "0")
    eta_t, q_t = run()
    assert abs(eta_s / eta_t - 1) < 2e-5
    assert q_s.sum() > 0
    assert np.abs(q_s - q_t).max() <= 2e-5 * np.abs(q_t).max()
    assert abs(q_s.sum() / q_t.sum() - 1) < 1e-5


@pytest.mark.parametrize("n", [16, 64, 256, 512])
def test_column_layout_pass_in_128_thread_ctas(n, monkeypatch):
    """SHG_FFT_VARIANT=3 forces the column-layout pass in 128-thread CTAs (half
    the columns per CTA; lengths up to 512), which the tuner may also pick."""
    monkeypatch.setenv("SHG_CLUSTER", "0")
    monkeypatch.setenv("SHG_FFT_VARIANT", "3")
    _check(W.depleted_absorbing(n=n, nz=5, tgrid=(9, 7, 4), p1=400.0))


@pytest.mark.parametrize("n,nz", [(512, 4), (1024, 3)])
def test_column_layout_pass_in_512_thread_ctas(n, nz, monkeypatch):
    """SHG_FFT_VARIANT=5 forces the column-layout pass in 512-thread CTAs
    (lengths 512 and 1024: twice the columns per CTA)."""
    monkeypatch.setenv("SHG_CLUSTER", "0")
    monkeypatch.setenv("SHG_FFT_VARIANT", "5")
    _check(W.depleted_absorbing(n=n, nz=nz, tgrid=(9, 7, 3), p1=400.0))


@pytest.mark.parametrize("n,nz", [(64, 6), (256, 5)])
def test_column_layout_pass_in_the_8_element_shape(n, nz, monkeypatch):
    """SHG_FFT_VARIANT=1 forces the 8-element shape for both step passes
    (lengths 64 to 256; 256-thread CTAs, three per SM), which the tuner may
    also pick; a rectangular grid takes it along y alone."""
    monkeypatch.setenv("SHG_CLUSTER", "0")
    monkeypatch.setenv("SHG_FFT_VARIANT", "1")
    w = W.depleted_absorbing(n=n, nz=nz, tgrid=(9, 7, 4), p1=400.0)
    _check(w)
    _check(w.with_(nx=32, ny=n, lx=w.lx * 32 / n))
