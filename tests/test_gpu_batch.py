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


def test_batch_equals_single_plan_propagation(monkeypatch):
    import paper_2410_04994_gb300 as pkg
    # the same streaming kernels on both sides (single small plans would
    # otherwise take the cluster-resident path)
    monkeypatch.setenv("SHG_CLUSTER", "0")
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
@pytest.mark.parametrize("n", [64, 128, 256])
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


@pytest.mark.parametrize("tz", [12, 16])
@pytest.mark.parametrize("variant", ["1", "2", "3", "4"])
def test_batch_with_each_forced_kernel_flavour(variant, tz, monkeypatch):
    """The batch path with the alternative FFT shape (1), the TMA-staged
    column pass over the group's tensor-map array (2) or the passes in 128- or
    64-thread CTAs (3, 4) forced, against the oracle per instance. With 12 map
    layers over nz = 12 the rows take the per-point table, with 16 layers the
    node sampler."""
    import paper_2410_04994_gb300 as pkg
    monkeypatch.setenv("SHG_FFT_VARIANT", variant)
    insts = W.sweep_instances(nz=12, groups=((64, 2), (128, 2), (256, 1)), tgrid=(9, 9, tz))
    plans = _plans(insts)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for p, w, e in zip(plans, insts, etas):
        eta_ref, AF, AS = oracle_run(w)
        assert abs(e / eta_ref - 1) < ETA_TOL, (w.name, e, eta_ref)
        a_f, a_sh = p.fields()
        assert rel_l2(a_sh.cpu(), AS) < FIELD_TOL


def test_tuner_cache_file_records_and_replays_decisions(tmp_path):
    """SHG_TUNE_CACHE: a fresh process records one decision per (size, pass)
    of the batch; a second process that reads a doctored file (every column
    pass forced to the TMA flavour) uses it without re-timing and still
    matches the first process's result to FP32 rounding."""
    import json
    import os
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    script = (
        "import json, torch, workloads as W, paper_2410_04994_gb300 as pkg\n"
        "insts = W.sweep_instances(nz=8, groups=((64, 2), (128, 2)), tgrid=(9, 9, 12))\n"
        "plans = [pkg.Plan(w) for w in insts]\n"
        "[p.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly) for p, w in zip(plans, insts)]\n"
        "print(json.dumps(pkg.shg_batch_submit([p.handle for p in plans])))\n")
    env = dict(os.environ, SHG_TUNE_CACHE=str(cache))
    env.pop("SHG_FFT_VARIANT", None)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r1 = subprocess.run([sys.executable, "-c", script], env=env, cwd=root,
                        capture_output=True, text=True)
    assert r1.returncode == 0, r1.stderr[-2000:]
    out1 = r1.stdout
    lines = [tuple(map(int, l.split())) for l in cache.read_text().splitlines()]
    # one column decision (key 1, or 5 for a group of few instances) and one
    # row decision per size
    cols = {n for _, n, p, _ in lines if p % 4 == 1}
    assert cols == {64, 128} and len(lines) == 4, lines
    cache.write_text("".join(f"{f} {n} {p} {2 if p % 4 == 1 else v}\n" for f, n, p, v in lines))
    r2 = subprocess.run([sys.executable, "-c", script], env=env, cwd=root,
                        capture_output=True, text=True)
    assert r2.returncode == 0, r2.stderr[-2000:]
    out2 = r2.stdout
    assert len(cache.read_text().splitlines()) == 4      # nothing re-timed
    e1, e2 = json.loads(out1.strip().splitlines()[-1]), json.loads(out2.strip().splitlines()[-1])
    for a, b in zip(e1, e2):
        assert abs(a / b - 1) < 1e-5
    # decisions that do not apply (the TMA flavour for a row pass, an unknown
    # length) are read, ignored for what they do not fit, and change nothing
    cache.write_text("".join(f"{f} {n} {p} {2 if p % 4 != 1 else 4}\n" for f, n, p, v in lines)
                     + "0 48 1 3\n")
    r3 = subprocess.run([sys.executable, "-c", script], env=env, cwd=root,
                        capture_output=True, text=True)
    assert r3.returncode == 0, r3.stderr[-2000:]
    e3 = json.loads(r3.stdout.strip().splitlines()[-1])
    for a, b in zip(e1, e3):
        assert abs(a / b - 1) < 1e-5


def test_pass_times_of_a_mixed_batch():
    """shg_pass_times on two grid groups (it tunes them first): one entry per
    group with its sizes, instance count and positive row and column times;
    a second call gives the same shape of answer."""
    import paper_2410_04994_gb300 as pkg
    insts = W.sweep_instances(nz=8, groups=((64, 3), (128, 2)), tgrid=(9, 9, 12))
    plans = _plans(insts)
    for _ in range(2):
        t = pkg.shg_pass_times([p.handle for p in plans], nsteps=3)
        assert [(g["nx"], g["ny"], g["instances"]) for g in t] == [(64, 64, 3), (128, 128, 2)]
        assert all(0 < g["row_ms"] < 100 and 0 < g["col_ms"] < 100 for g in t)


@pytest.mark.slow
def test_full_sweep_power_budget_of_every_instance():
    """All 384 instances of the benchmark sweep at nz = 2000, in the batch the
    benchmark times: every eta is finite and in (0, 1), and no instance ends
    with more power than it started with (losses only remove power; the
    coupling conserves it)."""
    import paper_2410_04994_gb300 as pkg
    insts = W.sweep_instances()
    plans = _plans(insts)
    etas = pkg.shg_batch_submit([p.handle for p in plans])
    for p, w, e in zip(plans, insts, etas):
        eta, p_f, p_sh = p.efficiency()
        assert eta == e and 0 < e < 1
        assert p_f + p_sh <= w.p1 * (1 + 1e-5), (w.name, p_f, p_sh, w.p1)
