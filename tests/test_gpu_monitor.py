"""Power monitor (shg_set_monitor / shg_get_monitor) against the oracle.

The monitor records P_F(z_s), P_SH(z_s) (Eq. 17's discrete powers) every k
steps inside the row pass, at the point of the step where the state is at
z_s.  The oracle's state after s whole steps is that same state, so its
powers must agree: to 1e-12 in FP64, to 1e-5 (relative to P1) in FP32.
Without losses the total P_F + P_SH is conserved by Eqs. (1)-(2)
(Manley-Rowe): its drift in FP32 stays within 1e-5 of P1.
"""
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _oracle_powers(w, steps):
    from oracle import ssfm
    p = ssfm.params_from_workload(w)
    temp = ssfm.TemperatureField(p, None if w.dT is None else torch.as_tensor(w.dT), w.t_lx,
                                 w.t_ly, w.t_off)
    out = []
    for s in steps:
        AF0 = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus)
        AF, AS = ssfm.propagate(p, AF0, torch.zeros_like(AF0), temp, nsteps=s)
        out.append((float(ssfm.power(AF, p.n_f, p.dx, p.dy)),
                    float(ssfm.power(AS, p.n_sh, p.dx, p.dy))))
    return out


def _gpu_monitor(w, every):
    import paper_2410_04994_gb300 as pkg
    plan = pkg.Plan(w)
    if w.dT is not None:
        plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    pkg.shg_set_monitor(plan.handle, every)
    plan.propagate()
    eta, p_f, p_sh = plan.efficiency()
    z, pf, psh = pkg.shg_get_monitor(plan.handle)
    return plan, (eta, p_f, p_sh), z, pf, psh


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_monitor_matches_oracle_powers(precision, tol):
    """Absorbing workload with a map, nz = 60 sampled every 7 steps (so the
    last sample, s = nz, is off the regular grid)."""
    w = W.depleted_absorbing(n=32, nz=60, tgrid=(8, 8, 8), p1=300.0).with_(precision=precision)
    plan, (eta, p_f, p_sh), z, pf, psh = _gpu_monitor(w, 7)
    steps = list(range(0, 60, 7)) + [60]
    assert len(z) == len(steps)
    assert all(abs(zz - s * w.L / w.nz) < 1e-15 for zz, s in zip(z, steps))
    ref = _oracle_powers(w, steps)
    for (rf, rs), gf, gs in zip(ref, pf, psh):
        assert abs(gf - rf) <= tol * w.p1, (gf, rf)
        assert abs(gs - rs) <= tol * w.p1, (gs, rs)
    # the last sample is the propagation's own result (its FP64 reduction; the
    # monitor adds up to 16 points per thread in the field precision first)
    same = 1e-12 if precision == "f64" else 1e-6
    assert abs(pf[-1] / p_f - 1) < same and abs(psh[-1] - p_sh) <= same * w.p1
    # absorption only removes power
    tot = [a + b for a, b in zip(pf, psh)]
    assert all(b < a for a, b in zip(tot, tot[1:]))


def test_manley_rowe_drift_without_losses_fp32():
    """Lossless depleted SHG at 128 x 128, nz = 400, 200 W (strong conversion,
    then back-conversion of the focused beams): P_F + P_SH stays at P1 to
    1e-5 at every sample while the SH power rises to a sizeable fraction."""
    w = W.plain_focused(n=128, nz=400, p1=200.0, precision="f32")
    plan, (eta, _, _), z, pf, psh = _gpu_monitor(w, 20)
    for a, b in zip(pf, psh):
        assert abs((a + b) / w.p1 - 1) < 1e-5, (a + b) / w.p1 - 1
    assert psh[0] == 0.0 and max(psh) > 0.2 * w.p1


def test_monitor_in_a_batch_and_off_again():
    import paper_2410_04994_gb300 as pkg
    insts = [W.depleted_absorbing(n=n, nz=30, tgrid=(6, 6, 6), p1=300.0) for n in (16, 32)]
    plans = [pkg.Plan(w) for w in insts]
    for p, w in zip(plans, insts):
        p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
        pkg.shg_set_monitor(p.handle, 10)
    pkg.shg_batch_submit([p.handle for p in plans])
    for p, w in zip(plans, insts):
        z, pf, psh = pkg.shg_get_monitor(p.handle)
        ref = _oracle_powers(w, [0, 10, 20, 30])
        assert len(z) == 4
        for (rf, rs), gf, gs in zip(ref, pf, psh):
            assert abs(gf - rf) <= 1e-5 * w.p1 and abs(gs - rs) <= 1e-5 * w.p1
    pkg.shg_set_monitor(plans[0].handle, 0)
    plans[0].propagate()
    with pytest.raises(pkg.ShgError) as ei:
        pkg.shg_get_monitor(plans[0].handle)
    assert ei.value.status == pkg.SHG_ERR_STATE
