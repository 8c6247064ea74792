"""GPU heat solve (direct separable solve and SOR) and convective faces against
the oracle.

Each side runs the whole chain from the same workload: its own propagation
deposits q_dot (Eq. 8), its own solver solves Eq. (16) with the faces of
Eqs. (9)-(10).  The oracle's SOR stops at a Jacobi correction below 1e-10 K
here, so both sides sit at the discrete solution; the bar is 1e-4 of the
largest |dT| (the deposits of FP32 fields agree to ~1e-6).
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

CONFIGS = {
    "all_oven": ("all", 0.0, 0.0),
    "surrounded": ("surrounded", 2e3, 0.0),       # end facets in air
    "bottom": ("bottom", 2e3, -1.0),              # one oven under y-, ambient 1 K below it
}


def _case(name, n=64, nz=100, heat=(16, 12, 24)):
    oven, h, t_inf = CONFIGS[name]
    w = W.thermal_loop(n=n, nz=nz, heat=heat, p1=100.0, n_outer=3)
    return W.with_oven(w, oven, h_conv=h, t_inf=t_inf)


def _gpu_solve(w, method=None):
    import paper_2410_04994_gb300 as pkg
    plan = pkg.Plan(w, thermal=True)
    if method is not None:
        pkg.shg_set_heat_method(plan.handle, method)
    plan.propagate()
    plan.efficiency()
    resid, passes = pkg.shg_heat_solve(plan.handle, 200000, 1e-9)
    dT = torch.empty((w.hz, w.hy, w.hx), dtype=torch.float32, device="cuda")
    q = torch.empty((w.hz, w.hy, w.hx), dtype=torch.float64, device="cuda")
    pkg.shg_get_heat(plan.handle, q, dT)
    torch.cuda.synchronize()
    return dT.cpu().numpy(), q.cpu().numpy(), resid, passes


def _oracle_solve(w):
    from oracle import heat, ssfm
    p = ssfm.params_from_workload(w)
    dep = ssfm.HeatDeposit(p, w.hx, w.hy, w.hz, w.wx, w.wy)
    ssfm.run(w.with_(dT=None), deposit=dep)
    T, sweeps, corr = heat.sor_solve(dep.qdot_nodes(), w.kappa_th, w.wx, w.wy, w.L, tol=1e-10,
                                     max_sweeps=2000000, bc=heat.bc_of(w))
    return T.numpy(), dep.Q.numpy()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_direct_solve_matches_oracle(name):
    w = _case(name)
    dT, Q, resid, passes = _gpu_solve(w)
    dTo, Qo = _oracle_solve(w)
    assert np.linalg.norm(Q - Qo) <= 1e-4 * np.linalg.norm(Qo)
    scale = np.abs(dTo).max()
    assert scale > 0.05
    assert np.abs(dT - dTo).max() <= 1e-4 * scale, (name, np.abs(dT - dTo).max() / scale)
    assert resid < 1e-9 and 1 <= passes <= 6
    if name != "all_oven":   # the convective faces are unknowns that carry heat
        assert np.abs(dTo[:, :, 0]).max() > 0 or np.abs(dTo[0]).max() > 0


def test_direct_and_sor_reach_the_same_solution():
    """All faces in the oven: the SOR (FP64 sweeps) and the direct solve
    (FP32 transforms, FP64 refinement) give the same dT."""
    import paper_2410_04994_gb300 as pkg
    w = _case("all_oven")
    d_direct, _, _, passes = _gpu_solve(w)
    d_sor, _, _, sweeps = _gpu_solve(w, pkg.SHG_HEAT_SOR)
    assert sweeps > 10 * passes
    assert np.abs(d_direct - d_sor).max() <= 1e-6 * np.abs(d_sor).max()


def test_thermal_loop_with_convective_end_facets_matches_oracle():
    """Fig. 2's loop with the surrounded oven (end facets cooled by
    convection): eta and the change of dT of every iteration."""
    import paper_2410_04994_gb300 as pkg
    from oracle import heat
    w = _case("surrounded")
    plan = pkg.Plan(w, thermal=True)
    etas, changes = pkg.shg_thermal_loop(plan.handle, 3, 200000, 1e-9)
    hist = heat.thermal_loop(w, 3, tol=1e-10, max_sweeps=2000000)
    for k, h in enumerate(hist):
        assert abs(etas[k] / h["eta"] - 1) < 1e-4, (k, etas[k], h["eta"])
        assert abs(changes[k] - h["change"]) <= 1e-4 * max(h["change"], 1e-6) + 1e-6


def test_full_heat_grid_cold_start():
    """The 128 x 128 x 256 grid of the thermal workload: a cold-start direct
    solve agrees with the SOR on the same deposits and takes a few passes."""
    import paper_2410_04994_gb300 as pkg
    w = W.thermal_loop(n=256, nz=200)
    d_direct, _, resid, passes = _gpu_solve(w)
    d_sor, _, _, sweeps = _gpu_solve(w, pkg.SHG_HEAT_SOR)
    scale = np.abs(d_sor).max()
    assert passes <= 6 and resid < 1e-9
    # the SOR stops at a correction of 1e-9 K: within a few 1e-8 K of the solution
    assert np.abs(d_direct - d_sor).max() <= 1e-6 * scale + 1e-7


def test_heat_boundary_and_method_refusals():
    import paper_2410_04994_gb300 as pkg
    w = _case("all_oven")
    plan = pkg.Plan(w, thermal=True)
    bad = [(["D", "D", "D", "D", "D", 7], 0.0),            # unknown kind
           (["C"] * 6, 0.0),                                 # insulated everywhere
           (["C", "D", "D", "D", "D", "D"], -1.0),          # negative h
           (["C", "D", "D", "D", "D", "D"], float("nan"))]
    for kinds, h in bad:
        with pytest.raises(pkg.ShgError) as ei:
            pkg.shg_set_heat_boundary(plan.handle, kinds, h)
        assert ei.value.status == pkg.SHG_ERR_INVALID_ARG
    pkg.shg_set_heat_boundary(plan.handle, ["D", "D", "D", "D", "C", "C"], 10.0)
    with pytest.raises(pkg.ShgError):
        pkg.shg_set_heat_method(plan.handle, pkg.SHG_HEAT_SOR)   # SOR: oven faces only
    plain = pkg.Plan(W.plain_focused(n=16, nz=4, precision="f32"))
    with pytest.raises(pkg.ShgError) as ei:
        pkg.shg_set_heat_boundary(plain.handle, ["D"] * 6, 0.0)
    assert ei.value.status == pkg.SHG_ERR_STATE
