"""The two ways the row pass reads the temperature map, against the oracle and
against each other.

- The per-point table (the FP32 default): every map layer sampled bilinearly at
  every field point once, when the map is set. The pass then streams the
  layers it needs.
- The node sampler: the same bilinear sample taken in the pass from the node
  table. It is used with SHG_FLAG_NODE_SAMPLER, or automatically when one
  z-step spans a map layer or more.

Both evaluate the same trilinear temperature, so they must agree with each
other to rounding and with the oracle to the FP32 bars.
"""
import math

import pytest
import torch

import workloads as W
from tests.helpers import ETA_TOL, FIELD_TOL, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _streaming_passes(monkeypatch):
    """These tests are about the streaming passes' temperature lookup: keep
    single plans off the cluster-resident path."""
    monkeypatch.setenv("SHG_CLUSTER", "0")


def _run(w, node_sampler=False):
    import paper_2410_04994_gb300 as pkg
    plan = pkg.Plan(w, node_sampler=node_sampler)
    plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    plan.propagate()
    eta, _, _ = plan.efficiency()
    a_f, a_sh = plan.fields()
    torch.cuda.synchronize()
    return eta, a_f.cpu(), a_sh.cpu()


def _check(w, eta, a_f, a_sh):
    eta_ref, AF, AS = oracle_run(w)
    assert math.isfinite(eta)
    assert abs(eta / eta_ref - 1) <= ETA_TOL, (w.name, eta, eta_ref)
    assert rel_l2(a_f, AF) <= FIELD_TOL
    assert rel_l2(a_sh, AS) <= FIELD_TOL


@pytest.mark.parametrize("n", [32, 64, 128, 256, 512, 1024])
def test_table_and_node_sampler_agree_and_match_oracle(n):
    """nz = 6 over 4 map intervals: the table path is taken; the flag forces
    the node sampler on the same inputs."""
    w = W.depleted_absorbing(n=n, nz=6, tgrid=(9, 7, 5), p1=400.0)
    eta_t, af_t, as_t = _run(w)
    eta_n, af_n, as_n = _run(w, node_sampler=True)
    _check(w, eta_t, af_t, as_t)
    _check(w, eta_n, af_n, as_n)
    assert abs(eta_t / eta_n - 1) < 1e-6
    assert rel_l2(as_t, as_n) < 1e-6 and rel_l2(af_t, af_n) < 1e-6


def test_steps_spanning_several_layers_use_the_node_sampler():
    """nz = 4 over 15 map intervals: each pass touches up to five layers, more
    than the table path holds, so the launcher takes the node sampler."""
    w = W.depleted_absorbing(n=64, nz=4, tgrid=(9, 7, 16), p1=400.0)
    _check(w, *_run(w))


def test_batch_recaptures_when_a_new_map_changes_the_row_path():
    """A batch captured with the table path; then one plan gets a map with 15
    intervals over nz = 12 steps, which needs the node sampler, and the next
    submit must rebuild its graph (a stale table-path graph would stop with
    SHG_ERR_STATE)."""
    import paper_2410_04994_gb300 as pkg
    ws = [W.depleted_absorbing(n=64, nz=12, tgrid=(9, 7, 5), p1=300.0, seed=s) for s in (0, 1)]
    plans = [pkg.Plan(w) for w in ws]
    for p, w in zip(plans, ws):
        p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for e, w in zip(etas, ws):
        assert abs(e / oracle_run(w)[0] - 1) <= ETA_TOL
    fine = W.depleted_absorbing(n=64, nz=12, tgrid=(9, 7, 16), p1=300.0, seed=2)
    ws[0] = ws[0].with_(dT=fine.dT)
    plans[0].set_temperature(torch.as_tensor(ws[0].dT), ws[0].t_lx, ws[0].t_ly)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for p, e, w in zip(plans, etas, ws):
        eta_ref, AF, AS = oracle_run(w)
        assert abs(e / eta_ref - 1) <= ETA_TOL, (w.name, e, eta_ref)
        assert rel_l2(p.fields()[1].cpu(), AS) <= FIELD_TOL


def test_same_shape_map_update_is_stream_ordered():
    """A second map of the same shape takes the asynchronous path of
    shg_set_temperature. It is enqueued on stream b, after the propagation
    still running on stream a. A propagation on a must wait for that rebuild,
    and a batch on a must too; both see the new map."""
    import paper_2410_04994_gb300 as pkg
    w1 = W.depleted_absorbing(n=64, nz=12, tgrid=(9, 7, 5), p1=300.0, seed=0)
    w2 = w1.with_(dT=W.depleted_absorbing(n=64, nz=12, tgrid=(9, 7, 5), p1=300.0, seed=3).dT)
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    plan = pkg.Plan(w1)
    plan.set_temperature(torch.as_tensor(w1.dT), w1.t_lx, w1.t_ly, stream=a)
    plan.propagate(stream=a)
    m2 = torch.as_tensor(w2.dT).cuda()
    torch.cuda.synchronize()
    plan.set_temperature(m2, w2.t_lx, w2.t_ly, stream=b)
    plan.propagate(stream=a)
    eta, _, _ = plan.efficiency()
    eta_ref, _, AS = oracle_run(w2)
    assert abs(eta / eta_ref - 1) <= ETA_TOL, (eta, eta_ref, oracle_run(w1)[0])
    # back to map 1 on b, then a batch on a
    m1 = torch.as_tensor(w1.dT).cuda()
    torch.cuda.synchronize()
    plan.set_temperature(m1, w1.t_lx, w1.t_ly, stream=b)
    e1 = pkg.shg_batch_submit([plan.handle], stream=a)[0]
    assert abs(e1 / oracle_run(w1)[0] - 1) <= ETA_TOL


def test_batched_map_update_equals_single_updates():
    """shg_set_temperature_batch over a mixed set: two grids, and one plan
    without a map yet, which takes the single-plan path. Afterwards every plan
    propagates bit-identically to the same plan updated by
    shg_set_temperature."""
    import paper_2410_04994_gb300 as pkg
    base = W.sweep_instances(nz=12, groups=((64, 3), (128, 2)), tgrid=(9, 9, 12))
    new = W.sweep_instances(nz=12, groups=((64, 3), (128, 2)), tgrid=(9, 9, 12), seed=7)
    pa, pb = [pkg.Plan(w) for w in base], [pkg.Plan(w) for w in base]
    for pl in (pa, pb):
        for p, w in zip(pl[1:], base[1:]):     # plan 0 starts without a map
            p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
        pkg.shg_batch_submit([p.handle for p in pl])
    maps = [torch.as_tensor(w.dT).cuda() for w in new]
    pkg.shg_set_temperature_batch([p.handle for p in pa], maps, [w.t_lx for w in new],
                                  [w.t_ly for w in new])
    for p, m, w in zip(pb, maps, new):
        p.set_temperature(m, w.t_lx, w.t_ly)
    ea = pkg.shg_batch_submit([p.handle for p in pa])
    eb = pkg.shg_batch_submit([p.handle for p in pb])
    assert ea == eb
    # the plans keep their beams (from `base`); only the maps changed
    assert abs(ea[3] / oracle_run(base[3].with_(dT=new[3].dT))[0] - 1) <= ETA_TOL
