"""GPU parity of the Eq. (4) phase-mismatch model against the oracle.

Synthetic index polynomials (cubic in T - 25 C) and the paper's MgO:sPPLT
grating expansion; the grating period is chosen so that quasi-phase matching
holds at 60 C.  The map adds a seeded dT(x,y,z) on top of T_oven + T_off, so
the nonlinear Dk(T) is integrated node by node (the table's C channel).
Bars: FP32 eta and fields 1e-4; FP64 1e-9; FP64 adjoint: scalar gradients
1e-7, map-node gradients 1e-6 (accumulated in FP32 buffers).
"""
import numpy as np
import pytest
import torch

import workloads as W
from tests.helpers import ETA_TOL, FIELD_TOL, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

T_PM = 60.0
# index slopes of a few 1e-6 / K: dDk/dT ~ 24 / (m K), so the 6 K of the map
# dephase the 30 mm crystal by a few radians
N_F = (2.14, 2e-6, 3e-9, -1e-11)
N_SH = (2.18, 4e-6, -4e-9, 2e-11)


def _qpm(t_oven):
    a, b, u = 2.2e-6, -5.9e-9, T_PM - 25.0
    dn = sum(c * u ** k for k, c in enumerate(N_SH)) - sum(c * u ** k for k, c in enumerate(N_F))
    lam25 = W.LAMBDA_F / (2.0 * dn) / (1.0 + a * u + b * u * u)
    return W.Qpm(t_oven=t_oven, lambda25=lam25, a_lambda=a, b_lambda=b, n_f_t=N_F, n_sh_t=N_SH)


def _case(n=64, nz=120, t_oven=58.0, t_off=1.5, precision="f32", amp=3.0):
    w = W.depleted_absorbing(n=n, nz=nz, tgrid=(12, 12, 16), p1=80.0)
    # a stronger map (amp x the recipe's 2 K) so that Dk's curvature matters
    w = w.with_(dT=(w.dT * amp).astype(np.float32))
    return w.with_(qpm=_qpm(t_oven), t_off=t_off, precision=precision)


def _compare(w, eta_tol, field_tol):
    eta, a_f, a_sh = gpu_run(w)
    eta_ref, AF, AS = oracle_run(w)
    assert abs(eta / eta_ref - 1) <= eta_tol, (eta, eta_ref)
    assert rel_l2(a_f, AF) <= field_tol and rel_l2(a_sh, AS) <= field_tol
    return eta_ref


@pytest.mark.parametrize("precision,tol", [("f32", ETA_TOL), ("f64", 1e-9)])
def test_eq4_with_map_matches_oracle(precision, tol):
    n = 64 if precision == "f32" else 32
    _compare(_case(n=n, precision=precision), tol, tol if precision == "f64" else FIELD_TOL)


def test_eq4_uniform_temperature_matches_oracle():
    w = _case().with_(dT=None)
    _compare(w, ETA_TOL, FIELD_TOL)


def test_temperature_scan_in_one_batch():
    """A temperature-tuning scan (Sec. 5.1's Fig. 4a, with these synthetic
    indices): oven offsets around the phase-matching temperature, as one
    batch.  The offsets are set through shg_set_beams on existing plans, so
    each plan rebuilds its Eq. (4) tables for its own T_oven + T_off."""
    import paper_2410_04994_gb300 as pkg
    offs = [-6.0, -2.0, 0.0, 2.0, 5.0]
    insts = [_case(n=32, nz=80, t_oven=T_PM, t_off=0.0) for _ in offs]
    plans = [pkg.Plan(w) for w in insts]
    for p, w in zip(plans, insts):
        p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    for p, o in zip(plans, offs):
        p.set_beams(t_off=o)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    refs = [oracle_run(w.with_(t_off=o))[0] for w, o in zip(insts, offs)]
    for e, r in zip(etas, refs):
        assert abs(e / r - 1) <= ETA_TOL, (e, r)
    assert len(set(np.round(refs, 6))) == len(refs)   # the scan resolves the offsets


def test_switching_back_to_the_linear_model():
    import paper_2410_04994_gb300 as pkg
    w = _case(n=32, nz=40)
    plan = pkg.Plan(w)
    plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    pkg.shg_set_phase_model(plan.handle, None)
    plan.propagate()
    eta, _, _ = plan.efficiency()
    ref = oracle_run(w.with_(qpm=None))[0]
    assert abs(eta / ref - 1) <= ETA_TOL
    with pytest.raises(pkg.ShgError):
        pkg.shg_set_phase_model(plan.handle, _qpm(40.0).__class__(40.0, -1.0))


def test_eq4_adjoint_matches_oracle_autograd():
    """The reverse sweep under Eq. (4): dDk/dT at each node's temperature in
    the map gradient, and dJ/dT_off as the sum of the node gradients."""
    from oracle import ssfm
    import paper_2410_04994_gb300 as pkg
    from paper_2410_04994_gb300.autograd import efficiency
    w = _case(n=16, nz=24, precision="f64")
    dT = torch.tensor(w.dT, dtype=torch.float64, requires_grad=True)
    w0 = torch.tensor(w.w0, dtype=torch.float64, requires_grad=True)
    zf = torch.tensor(w.z_focus, dtype=torch.float64, requires_grad=True)
    to = torch.tensor(w.t_off, dtype=torch.float64, requires_grad=True)
    eta_o = ssfm.run(w, w0=w0, z_focus=zf, t_off=to, dT=dT)[2]
    go = torch.autograd.grad(eta_o, (w0, zf, to, dT))
    plan = pkg.Plan(w, adjoint=True)
    dTg = torch.tensor(w.dT, dtype=torch.float64, device="cuda", requires_grad=True)
    w0g = torch.tensor(w.w0, dtype=torch.float64, requires_grad=True)
    zfg = torch.tensor(w.z_focus, dtype=torch.float64, requires_grad=True)
    tog = torch.tensor(w.t_off, dtype=torch.float64, requires_grad=True)
    eta = efficiency(plan, w0g, zfg, tog, dTg)
    eta.backward()
    assert abs(float(eta.detach()) / float(eta_o.detach()) - 1) < 1e-9
    for got, ref in ((w0g.grad, go[0]), (zfg.grad, go[1]), (tog.grad, go[2])):
        assert abs(float(got) - float(ref)) <= 1e-7 * abs(float(ref)), (float(got), float(ref))
    # the per-node sensitivities are accumulated and returned in FP32 buffers
    gT, rT = dTg.grad.cpu().numpy(), go[3].numpy()
    assert np.abs(gT - rT).max() <= 1e-6 * np.abs(rT).max()
    assert abs(float(tog.grad) - gT.sum()) <= 1e-6 * np.abs(gT).sum()
