"""Full-size parity of the adjoint and thermal workloads against stored
FP64-oracle values.

The oracle needs tens of minutes for these sizes, so ``tests/golden/
make_golden.py`` (which calls only ``oracle/``) ran it once and stored the
values; the GPU runs the same seeded inputs through the C ABI here.

* Adjoint workload (256 x 256, nz = 2000, 64 x 64 x 128 map): the FP32 reverse
  sweep against central finite differences of the FP64 oracle for w0, z_focus,
  T_off and three seeded directions in the map's node space (bar 1e-3; for
  T_off and the directions relative to the larger of the derivative and the
  gradient's l1 scale, because the phase-matching slope is tiny).
* Thermal workload, first pass at full length (1024 x 1024, nz = 8000, heat grid
  128 x 128 x 256): eta, P_F, P_SH, the heat deposited per heat-grid layer, and
  the output fields on a stride-16 subgrid and the central 32 x 32 block.
* Thermal loop, two iterations at 1024 x 1024 with nz = 100 on the full heat
  grid: eta, the change of dT and the deposits per iteration, dT on a subgrid,
  and the second pass's fields.
Bars: eta and powers 1e-4 relative, fields 1e-4 relative L2, deposits 1e-4
relative L2, dT 1e-3 of its maximum.
"""
import math
import os

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.fail(f"stored oracle values {name} are missing (tests/golden/make_golden.py)")
    if path.endswith(".json"):
        import json
        return json.load(open(path))
    return dict(np.load(path))


def _rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def _field_checks(a_f, a_sh, g):
    """Stride and centre samples of the GPU fields against the stored ones."""
    s, c = int(g["stride"]), int(g["centre"])
    for a, sub, cen in ((a_f, g["af_sub"], g["af_centre"]), (a_sh, g["ash_sub"], g["ash_centre"])):
        a = a.cpu().numpy()
        ny, nx = a.shape
        c0, c1 = ny // 2 - c // 2, nx // 2 - c // 2
        assert _rel_l2(a[::s, ::s], sub) <= 1e-4, _rel_l2(a[::s, ::s], sub)
        assert _rel_l2(a[c0:c0 + c, c1:c1 + c], cen) <= 1e-4


def test_adjoint_full_size_fp32_vs_oracle_finite_differences():
    import paper_2410_04994_gb300 as pkg
    fd = _load("adjoint_fd_256_nz2000.json")
    w = W.adjoint_case()
    plan = pkg.Plan(w, adjoint=True)
    dT = torch.as_tensor(w.dT).cuda()
    plan.set_temperature(dT, w.t_lx, w.t_ly)
    plan.propagate()
    eta, _, _ = plan.efficiency()
    assert abs(eta / fd["eta"] - 1) <= 1e-4, (eta, fd["eta"])
    g_dT = torch.empty_like(dT)
    gw, gz, gt = pkg.shg_propagate_adjoint(plan.handle, 1.0, g_dT)
    gT = g_dT.double().cpu().numpy()
    l1 = float(np.abs(gT).sum())   # sensitivity to 1 K on every node
    assert abs(gw - fd["d_w0"]["value"]) <= 1e-3 * abs(fd["d_w0"]["value"]), (gw, fd["d_w0"])
    assert abs(gz - fd["d_zf"]["value"]) <= 1e-3 * abs(fd["d_zf"]["value"]), (gz, fd["d_zf"])
    ref_t = fd["d_toff"]["value"]
    assert abs(gt - ref_t) <= 1e-3 * max(abs(ref_t), l1), (gt, ref_t, l1)
    # the oven offset is a uniform dT: its derivative is the sum over the nodes
    assert abs(gt - gT.sum()) <= 1e-3 * l1
    rng = np.random.default_rng(fd["d_map_directions"][0]["seed"])
    for d in fd["d_map_directions"]:
        v = rng.normal(size=gT.shape)
        got = float((gT * v).sum())
        scale = max(abs(d["value"]), float(np.abs(gT * v).sum()) * 1e-2)
        assert abs(got - d["value"]) <= 1e-3 * scale, (d["index"], got, d["value"])


def test_thermal_first_pass_full_length_vs_oracle():
    import paper_2410_04994_gb300 as pkg
    g = _load("thermal_pass_1024_nz8000.npz")
    w = W.thermal_loop()
    plan = pkg.Plan(w, thermal=True)
    etas, changes = pkg.shg_thermal_loop(plan.handle, 1, 1000, 1e-6)
    eta, p_f, p_sh = plan.efficiency()
    assert etas[0] == eta and changes[0] == 0.0
    assert abs(eta / float(g["eta"]) - 1) <= 1e-4, (eta, float(g["eta"]))
    assert abs(p_f / float(g["p_f"]) - 1) <= 1e-4
    assert abs(p_sh / float(g["p_sh"]) - 1) <= 1e-4
    q = torch.empty((w.hz, w.hy, w.hx), dtype=torch.float64, device="cuda")
    pkg.shg_get_heat(plan.handle, q, None)
    ql = q.sum(dim=(1, 2)).cpu().numpy()
    assert np.linalg.norm(ql - g["q_layers"]) <= 1e-4 * np.linalg.norm(g["q_layers"])
    assert abs(float(q.sum()) / float(g["q_total"]) - 1) <= 1e-4
    a_f, a_sh = plan.fields()
    _field_checks(a_f, a_sh, g)


def test_thermal_loop_two_iterations_full_heat_grid_vs_oracle():
    import paper_2410_04994_gb300 as pkg
    g = _load("thermal_loop2_1024_nz100.npz")
    w = W.thermal_loop(nz=100, n_outer=2)
    plan = pkg.Plan(w, thermal=True)
    etas, changes = pkg.shg_thermal_loop(plan.handle, 2, 200000, 1e-6)
    for k in range(2):
        assert abs(etas[k] / float(g[f"eta{k}"]) - 1) <= 1e-4, (k, etas[k], float(g[f"eta{k}"]))
        ref = float(g[f"change{k}"])
        assert abs(changes[k] - ref) <= 1e-3 * max(ref, 1e-6) + 2e-5, (k, changes[k], ref)
    assert math.isfinite(etas[1]) and etas[1] != etas[0]   # the feedback is active
    q = torch.empty((w.hz, w.hy, w.hx), dtype=torch.float64, device="cuda")
    dT = torch.empty((w.hz, w.hy, w.hx), dtype=torch.float32, device="cuda")
    pkg.shg_get_heat(plan.handle, q, dT)
    ql = q.sum(dim=(1, 2)).cpu().numpy()
    assert np.linalg.norm(ql - g["q_layers1"]) <= 1e-4 * np.linalg.norm(g["q_layers1"])
    dT = dT.cpu().numpy()
    dmax = float(g["dT_max"])
    assert dmax > 1e-3
    assert np.abs(dT[::8, ::4, ::4] - g["dT_sub"]).max() <= 1e-3 * dmax + 1e-5
    assert abs(float(np.abs(dT).max()) - dmax) <= 1e-3 * dmax
    a_f, a_sh = plan.fields()
    _field_checks(a_f, a_sh, g)


def test_extension_workloads_vs_stored_oracle_values():
    """The measured extension workloads at their bench sizes: the Eq. (4)
    phase model on the depleted workload (128^2 x 1000, the cluster-resident
    path) and sum- and difference-frequency generation (128^2 x 1000),
    against stored oracle values (extensions.json).  Bars: eta and powers
    1e-4 (three-wave: relative to the largest power)."""
    import paper_2410_04994_gb300 as pkg
    g = _load("extensions.json")
    w = W.eq4_case()
    plan = pkg.Plan(w)
    plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    plan.propagate()
    eta, p_f, p_sh = plan.efficiency()
    ref = g["eq4"]
    assert abs(eta / ref["eta"] - 1) <= 1e-4, (eta, ref["eta"])
    assert abs(p_f / ref["p_f"] - 1) <= 1e-4 and abs(p_sh / ref["p_sh"] - 1) <= 1e-4
    for key, w3 in (("sfg", W.sfg_case(n=128, nz=1000)), ("dfg", W.dfg_case(n=128, nz=1000))):
        p3 = pkg.Plan3(w3)
        p3.set_temperature(w3.dT, w3.t_lx, w3.t_ly)
        p3.propagate()
        P = p3.powers()
        ref = g[key]["powers"]
        assert max(abs(a - b) for a, b in zip(P, ref)) <= 1e-4 * max(ref), (key, P, ref)
