"""The benchmark's reference arm on the CPU: the FP64 oracle timed on a tiny
sample, and the one JSON line it prints (keys, units, and the rules that rank
0 alone runs it and that its e2e moves no bytes)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--steps", "1", "--warmup", "1", "--ref-zsteps", "2"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_arm_prints_one_complete_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "grid-point-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 1)
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == "sweep_384_mixed_nz2000"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "2 z-steps" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_plain_comparison_form_is_the_oracle_map():
    """The plain PyTorch form that the benchmark times as its FP64 GPU
    comparison (its own code, unfused, torch.fft) computes the oracle's map:
    run here on the CPU over the full length, its eta matches the oracle's to
    1e-10 in complex128 and to the FP32 bar in complex64."""
    import math

    import torch

    import bench
    import workloads as W
    from tests.helpers import ETA_TOL, oracle_run
    w = W.depleted_absorbing(n=32, nz=40, tgrid=(9, 7, 5), p1=400.0).with_(t_off=0.4)
    eta_ref = oracle_run(w)[0]
    eps0c = 8.8541878128e-12 * 299792458.0
    for real, tol in ((torch.float64, 1e-10), (torch.float32, ETA_TOL)):
        a, s, step = bench.plain_form(w, "cpu", real)
        for k in range(w.nz):
            a, s = step(a, s, k * w.L / w.nz)
        p_sh = 0.5 * eps0c * w.n_sh * float((s.abs() ** 2).sum()) * (w.lx / w.nx) * (w.ly / w.ny)
        assert math.isfinite(p_sh)
        assert abs(p_sh / w.p1 / eta_ref - 1) < tol, (real, p_sh / w.p1, eta_ref)
