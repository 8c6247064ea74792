"""The cluster-resident single-instance path (one launch per propagation, the
fields in distributed shared memory) against the oracle and against the
streaming passes.

It is taken by single FP32 plans with nx = ny in {64, 128}, a uniform
temperature or a map with the per-point table, no heat grid, no adjoint
checkpoints and no power monitor; SHG_CLUSTER=0 turns it off.  Bars as for
the other FP32 parity tests: eta 1e-4 and field L2 1e-4 against the oracle.
"""
import pytest
import torch

import workloads as W
from tests.helpers import ETA_TOL, FIELD_TOL, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _check(w, fields=None):
    eta, a_f, a_sh = gpu_run(w, fields)
    eta_ref, AF, AS = oracle_run(w, fields)
    assert abs(eta / eta_ref - 1) <= ETA_TOL, (w.name, eta, eta_ref)
    assert rel_l2(a_f, AF) <= FIELD_TOL and rel_l2(a_sh, AS) <= FIELD_TOL
    return eta, a_f, a_sh


@pytest.mark.parametrize("n", [64, 128])
def test_cluster_path_with_map_matches_oracle(n, monkeypatch):
    monkeypatch.setenv("SHG_CLUSTER", "1")
    _check(W.depleted_absorbing(n=n, nz=60, tgrid=(16, 16, 20), p1=200.0))


@pytest.mark.parametrize("n", [64, 128])
def test_cluster_path_uniform_temperature_and_walkoff(n, monkeypatch):
    monkeypatch.setenv("SHG_CLUSTER", "1")
    w = W.depleted_absorbing(n=n, nz=40, tgrid=(8, 8, 8), p1=300.0).with_(
        dT=None, t_off=0.4, walkoff_f=2e-3, walkoff_sh=-4e-3, beta_f=1e-10)
    _check(w)


def test_cluster_path_custom_fields(monkeypatch):
    monkeypatch.setenv("SHG_CLUSTER", "1")
    w = W.depleted_absorbing(n=64, nz=20, tgrid=(8, 8, 8), p1=300.0)
    from oracle import ssfm
    p = ssfm.params_from_workload(w)
    AF0 = ssfm.initial_pump(p, w.p1, 0.8 * w.w0, 0.3 * w.L)
    AS0 = 0.1 * torch.roll(AF0, 3, 1)
    _check(w, fields=(AF0, AS0))


def test_cluster_path_full_depleted_workload(monkeypatch):
    """The depleted workload at full size (128 x 128, nz = 1000, 64 x 64 x 128
    map) on the cluster path, and the streaming path on the same plan data:
    both match the oracle, and each other to FP32 rounding."""
    w = W.depleted_absorbing()
    monkeypatch.setenv("SHG_CLUSTER", "1")
    eta_c, af_c, as_c = _check(w)
    monkeypatch.setenv("SHG_CLUSTER", "0")
    eta_s, af_s, as_s = gpu_run(w)
    assert abs(eta_c / eta_s - 1) < 2e-5
    assert rel_l2(af_c, af_s.to(torch.complex128)) < 2e-5


def test_cluster_path_is_taken_and_repeatable(monkeypatch):
    """Two propagations of the same plan give bit-identical results (no
    atomics or reductions whose order could vary on this path)."""
    import paper_2410_04994_gb300 as pkg
    monkeypatch.setenv("SHG_CLUSTER", "1")
    w = W.depleted_absorbing(n=128, nz=30, tgrid=(16, 16, 20), p1=200.0)
    plan = pkg.Plan(w)
    plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    plan.propagate()
    a1 = [x.clone() for x in plan.fields()]
    plan.propagate()
    a2 = plan.fields()
    assert all(bool((x == y).all()) for x, y in zip(a1, a2))
