"""Three-wave mixing plans (shg_plan_create_3w) against the three-wave oracle.

Sum-frequency generation (1550 + 1064 -> 631 nm) and difference-frequency
generation (631 - 1064 -> 1550 nm) with the absorbing workloads' losses and a
seeded temperature map; the degenerate case against the SHG path; the
undepleted switch.  Bars: FP32 powers and field L2 1e-4 (relative to the
largest power and field), FP64 1e-9.
"""
import math

import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(w):
    import paper_2410_04994_gb300 as pkg
    plan = pkg.Plan3(w)
    if w.dT is not None:
        plan.set_temperature(w.dT, w.t_lx, w.t_ly)
    plan.propagate()
    P = plan.powers()
    A = [a.cpu().to(torch.complex128) for a in plan.fields()]
    return plan, P, A


def _check(w, tol):
    from oracle import threewave as T3
    plan, P, A = _gpu(w)
    Ao, Po = T3.run(w)
    pmax = max(Po)
    for j in range(3):
        assert abs(P[j] - Po[j]) <= tol * pmax, (w.name, j, P[j], Po[j])
        if float(Ao[j].norm()) > 0:
            ref = max(float(a.norm()) for a in Ao)
            assert float((A[j] - Ao[j]).norm()) <= tol * ref, (w.name, j)
    return plan, P, Po


@pytest.mark.parametrize("precision,tol", [("f32", 1e-4), ("f64", 1e-9)])
def test_sfg_matches_oracle(precision, tol):
    n = 64 if precision == "f32" else 32
    plan, P, Po = _check(W.sfg_case(n=n, nz=120).with_(precision=precision), tol)
    assert Po[2] > 0.01 * (20.0 + 30.0)
    import paper_2410_04994_gb300 as pkg
    eta, p1, p3 = pkg.shg_efficiency(plan.handle)
    assert abs(eta - P[2] / 50.0) < 1e-12 and p1 == P[0] and p3 == P[2]


@pytest.mark.parametrize("precision,tol", [("f32", 1e-4), ("f64", 1e-9)])
def test_dfg_matches_oracle(precision, tol):
    n = 64 if precision == "f32" else 32
    plan, P, Po = _check(W.dfg_case(n=n, nz=120).with_(precision=precision), tol)
    assert Po[0] > 1e-3 and Po[1] > 2.0   # the idler appears, the seed is amplified


def test_sfg_every_size_and_walkoff():
    for n in (16, 128, 256):
        w = W.sfg_case(n=n, nz={16: 40, 128: 30, 256: 8}[n]).with_(
            walkoff=(1e-3, -2e-3, 3e-3), dk0=30.0, t_off=0.3)
        _check(w, 1e-4)


def test_undepleted_switch():
    _check(W.sfg_case(n=32, nz=40).with_(undepleted=True, precision="f64"), 1e-9)


def test_degenerate_three_wave_plan_reproduces_the_shg_plan():
    """lambda1 = lambda2, n1 = n2, equal inputs: the three-wave plan's A3 is
    the SHG plan's A_SH and A1 = A2 = A_F / sqrt(2) (FP64, same map)."""
    import paper_2410_04994_gb300 as pkg
    base = W.depleted_absorbing(n=32, nz=40, tgrid=(8, 8, 12), p1=300.0).with_(precision="f64")
    w3 = W.ThreeWave(name="deg", nx=32, ny=32, nz=40, lx=base.lx, ly=base.ly,
                     lambda1=base.lambda_f, lambda2=base.lambda_f, n1=base.n_f, n2=base.n_f,
                     n3=base.n_sh, alpha=(base.alpha_f, base.alpha_f, base.alpha_sh),
                     beta=(0.0, 0.0, base.beta_sh), ddk_dT=base.ddk_dT, dn_dT=base.dn_dT,
                     p=(150.0, 150.0, 0.0), w0=(base.w0,) * 3, z_focus=(base.z_focus,) * 3,
                     dT=base.dT, t_lx=base.t_lx, t_ly=base.t_ly, precision="f64")
    _, P3, A3 = _gpu(w3)
    shg = pkg.Plan(base)
    shg.set_temperature(torch.as_tensor(base.dT), base.t_lx, base.t_ly)
    shg.propagate()
    eta, p_f, p_sh = shg.efficiency()
    a_f, a_sh = [a.cpu() for a in shg.fields()]
    s2 = math.sqrt(2.0)
    assert float((A3[0] - a_f / s2).abs().max()) <= 1e-10 * float(a_f.abs().max())
    assert float((A3[2] - a_sh).abs().max()) <= 1e-10 * float(a_sh.abs().max())
    assert abs(P3[2] / p_sh - 1) < 1e-10


def test_three_wave_plans_refuse_shg_only_calls():
    import paper_2410_04994_gb300 as pkg
    w = W.sfg_case(n=16, nz=4)
    plan = pkg.Plan3(w)
    with pytest.raises(pkg.ShgError):
        pkg.shg_batch_submit([plan.handle])
    with pytest.raises(pkg.ShgError):
        pkg.shg_set_monitor(plan.handle, 1)
    with pytest.raises(pkg.ShgError):
        pkg.shg_plan_create_3w(*pkg.structs3_from(w.with_(p=(0.0, 0.0, 0.0))))
    with pytest.raises(pkg.ShgError):
        pkg.shg_plan_create_3w(*pkg.structs3_from(w), pkg.SHG_FLAG_THERMAL)


@pytest.mark.parametrize("case,n,nz", [("sfg", 64, 41), ("sfg", 128, 40), ("dfg", 128, 33),
                                       ("dfg", 64, 48)])
def test_cluster_resident_path_matches_oracle(case, n, nz):
    """Single FP32 plans of 64^2 and 128^2 whose map layers one step does not
    outrun (nz >= tz) run the whole z-march in one cluster launch; odd and
    even nz end in either layout.  Walk-off, a phase offset and the map."""
    mk = W.sfg_case if case == "sfg" else W.dfg_case
    w = mk(n=n, nz=nz).with_(walkoff=(1e-3, -2e-3, 3e-3), dk0=30.0, t_off=0.3)
    _check(w, 1e-4)


@pytest.mark.parametrize("n", [64, 128])
def test_cluster_resident_path_without_map_and_undepleted(n):
    _check(W.sfg_case(n=n, nz=25, with_map=False), 1e-4)
    _check(W.sfg_case(n=n, nz=25, with_map=False).with_(undepleted=True), 1e-4)


def test_cluster_resident_path_equals_the_passes(monkeypatch):
    """The same plan through the cluster kernel and through the row and
    column passes (SHG_CLUSTER=0): the same arithmetic in another rounding
    order (L applied as Lx Ly or Ly Lx; the map through the per-point table
    or sampled at its nodes)."""
    w = W.sfg_case(n=128, nz=200)
    _, P_c, A_c = _gpu(w)
    monkeypatch.setenv("SHG_CLUSTER", "0")
    _, P_p, A_p = _gpu(w)
    for j in range(3):
        assert abs(P_c[j] / P_p[j] - 1) < 2e-5, (j, P_c[j], P_p[j])
        assert float((A_c[j] - A_p[j]).norm()) <= 2e-5 * float(A_p[j].norm())
