"""Batched sweep (shg_batch_submit) against single-plan propagation and the
oracle: the graph-launched batch gives bit-identical eta to the same plans
propagated one by one, runs are deterministic, and sampled instances of the
384-instance sweep match the FP64 oracle at full length (nz = 2000)."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from tests.helpers import ETA_TOL, FIELD_TOL, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _plans(insts):
    import paper_2410_04994_gb300 as pkg
    plans = [pkg.Plan(w) for w in insts]
    for p, w in zip(plans, insts):
        if w.dT is not None:
            p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    return plans


def _mixed(nz=30):
    return W.sweep_instances(nz=nz, groups=((16, 3), (32, 4), (64, 2)), tgrid=(9, 9, 12))


def test_batch_equals_single_plan_propagation():
    import paper_2410_04994_gb300 as pkg
    insts = _mixed()
    plans = _plans(insts)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for p, e in zip(plans, etas):
        p.propagate()
        e1, _, _ = p.efficiency()
        assert e1 == e          # same kernels, same data: bit-identical
    # and the efficiency call after a batch reports the batch's result
    etas2 = pkg.shg_batch_submit([p.handle for p in plans])
    assert etas2 == etas
    assert plans[0].efficiency()[0] == etas[0]


def test_batch_matches_oracle_per_instance():
    import paper_2410_04994_gb300 as pkg
    insts = _mixed()
    plans = _plans(insts)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for p, w, e in zip(plans, insts, etas):
        eta_ref, AF, AS = oracle_run(w)
        assert abs(e / eta_ref - 1) < ETA_TOL, (w.name, e, eta_ref)
        a_f, a_sh = p.fields()
        assert rel_l2(a_f.cpu(), AF) < FIELD_TOL
        assert rel_l2(a_sh.cpu(), AS) < FIELD_TOL


def test_batch_rejects_bad_input():
    import paper_2410_04994_gb300 as pkg
    with pytest.raises(pkg.ShgError) as ei:
        pkg.shg_batch_submit([])
    assert ei.value.status == pkg.SHG_ERR_INVALID_ARG


@pytest.mark.slow
@pytest.mark.parametrize("n", [64, 128])
def test_sweep_instances_full_length(n):
    """The first instance of a size group of the 384-instance sweep (seeded
    map, losses, oven offset), propagated inside the full-size mixed batch at
    nz = 2000, against the oracle."""
    import paper_2410_04994_gb300 as pkg
    insts = W.sweep_instances()
    k = next(i for i, w in enumerate(insts) if w.nx == n)
    plans = _plans(insts)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    assert all(math.isfinite(e) and 0 <= e < 1 for e in etas)
    eta_ref, AF, AS = oracle_run(insts[k])
    assert abs(etas[k] / eta_ref - 1) < ETA_TOL
    a_f, a_sh = plans[k].fields()
    assert rel_l2(a_sh.cpu(), AS) < FIELD_TOL
    assert rel_l2(a_f.cpu(), AF) < FIELD_TOL


@pytest.mark.parametrize("variant", ["1", "2", "3"])
def test_batch_with_each_forced_kernel_flavour(variant, monkeypatch):
    """The batch path with the alternative FFT shape (1), the TMA-staged
    column pass over the group's tensor-map array (2) or the 128-thread column
    pass (3) forced, against the oracle per instance."""
    import paper_2410_04994_gb300 as pkg
    monkeypatch.setenv("SHG_FFT_VARIANT", variant)
    insts = W.sweep_instances(nz=12, groups=((64, 2), (128, 2), (256, 1)), tgrid=(9, 9, 12))
    plans = _plans(insts)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for p, w, e in zip(plans, insts, etas):
        eta_ref, AF, AS = oracle_run(w)
        assert abs(e / eta_ref - 1) < ETA_TOL, (w.name, e, eta_ref)
        a_f, a_sh = p.fields()
        assert rel_l2(a_sh.cpu(), AS) < FIELD_TOL
