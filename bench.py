"""Throughput benchmark of the fused FP32 split-step SHG path on GB300.

Workload (default): the batched focusing / power / oven sweep: 384
independent instances on mixed grids (128 x 64^2, 192 x 128^2, 64 x 256^2),
nz = 2000 each, seeded 64 x 64 x 128 temperature maps, all propagated by one
CUDA-graph launch of the C ABI's shg_batch_submit per step.  One step = one
full propagation of every instance (1.573e10 grid-point-steps).

Metric: grid-point-steps per second, sum over instances of nx ny nz / time.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "SSFM grid-point-steps/s (Nx*Ny*Nz/s) vs plain FP64 GPU form; eta rel err vs oracle"
UNIT = "grid-point-steps/s"
FP32_LANES_PER_SM = 128
N_SM = 152


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "_fallback": True}


def row_flops_per_point(n: int, thermal: bool) -> float:
    """Algorithmic FP32 flops of one row pass per grid point.  Two RK4 half
    steps: 4 right-hand sides of 51 flops, 3 stage vectors (8), the weighted
    sum (24) and the update (8) each; with a temperature map 5 stage points of
    coefficients (trilinear dT and C, e^{i g C}, psi: ~20 flops each); two
    fields x (forward + inverse 1-D FFT at 5 n log2 n / n per point + a complex
    multiply)."""
    rk4 = 2 * (4 * 51 + 3 * 8 + 24 + 8)
    coef = 5 * 20 if thermal else 0
    fft = 2 * (2 * 5 * math.log2(n) + 6)
    return rk4 + coef + fft


def step_flops_per_point(n: int, thermal: bool) -> float:
    """Algorithmic FP32 flops per grid point of one pass of the one-pass-per-
    step schedule (passes_per_step == 1 in shg_pass_times): a whole step, the
    nonlinear part of row_flops_per_point and the transforms along the pass's
    axis twice (the second half of L(s-1) and the first half of L(s))."""
    fft = 2 * (2 * 5 * math.log2(n) + 6)
    return row_flops_per_point(n, thermal) + fft


def threewave_flops_per_point_step(n: int, thermal: bool) -> float:
    """Algorithmic FP32 flops per grid point and z-step of a three-wave plan:
    two RK4 half steps of the three coupled fields (4 right-hand sides of 69
    flops: TPA and lens of each wave 3 x 9, the two difference-frequency
    couplings 26, the sum-frequency coupling 16; stage vectors 3 x 12; the
    weighted sums 30; the update 12); stage coefficients at 5 points (about
    42 flops each with a map); Lx and Ly of the three fields (forward and
    inverse 1-D FFT at 5 n log2 n / n per point, and a complex multiply)."""
    rk4 = 2 * (4 * 69 + 36 + 30 + 12)
    coef = 5 * 42 if thermal else 0
    fft = 2 * 3 * (2 * 5 * math.log2(n) + 6)
    return rk4 + coef + fft


def col_bytes_per_point() -> float:
    """Column pass: read and write both complex64 fields once."""
    return 2 * 2 * 8.0


class Clocks:
    """nvidia-smi sampler for the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------- plain GPU forms (comparisons) ----

def plain_group_form(ws, dev: str = "cuda", real=torch.float64):
    """The same split step written plainly in PyTorch for B instances of one
    grid: complex fields [B, ny, nx], torch.fft over the last two axes (cuFFT
    on the GPU) and unfused elementwise operations, in the real type `real`
    (complex the matching type).  This is the design the paper describes
    (Sec. 4: cuFFT plus separate elementwise kernels), batched.
    Returns (A_F(0), A_SH(0), step); step(a, s, z) advances one z-step from z
    (a float, or a 0-d float64 tensor on `dev` so that a CUDA graph can
    replay the step)."""
    cdt = torch.complex128 if real == torch.float64 else torch.complex64
    f64 = torch.float64
    w = ws[0]
    for v in ws:
        assert (v.nx, v.ny, v.nz, v.L, v.lambda_f, v.n_f, v.n_sh, v.d_eff) == \
            (w.nx, w.ny, w.nz, w.L, w.lambda_f, w.n_f, w.n_sh, w.d_eff)
        assert (v.alpha_f, v.alpha_sh, v.beta_f, v.beta_sh, v.dk0, v.ddk_dT, v.dn_dT) == \
            (w.alpha_f, w.alpha_sh, w.beta_f, w.beta_sh, w.dk0, w.ddk_dT, w.dn_dT)
    B = len(ws)
    eps0c = 8.8541878128e-12 * 299792458.0
    nx, ny, dz = w.nx, w.ny, w.L / w.nz

    def col(vals, dt=f64):
        return torch.tensor([float(v) for v in vals], dtype=dt, device=dev)

    lx, ly = col(v.lx for v in ws), col(v.ly for v in ws)
    x = (torch.arange(nx, dtype=f64, device=dev) - nx // 2)[None, :] * (lx / nx)[:, None]
    y = (torch.arange(ny, dtype=f64, device=dev) - ny // 2)[None, :] * (ly / ny)[:, None]
    kF = 2 * math.pi * w.n_f / w.lambda_f
    kS = 2 * math.pi * w.n_sh / (w.lambda_f / 2)
    w0 = col(v.w0 for v in ws)[:, None, None]
    zr = w0 ** 2 * kF / 2
    q = torch.complex(torch.ones_like(zr), -col(v.z_focus for v in ws)[:, None, None] / zr)
    r2 = (x[:, None, :] ** 2 + y[:, :, None] ** 2).to(torch.complex128)
    AF = torch.exp(-r2 / (w0 ** 2 * q)) / q
    dxdy = (lx / nx) * (ly / ny)
    pw = 0.5 * eps0c * w.n_f * (AF.abs() ** 2).sum(dim=(1, 2)) * dxdy
    AF = (AF * torch.sqrt(col(v.p1 for v in ws) / pw)[:, None, None]).to(cdt)
    AS = torch.zeros_like(AF)

    def freq(n, length):
        b = torch.arange(n, dtype=f64, device=dev)
        m = torch.where(b < (n + 1) // 2, b, b - n)
        return 2 * math.pi * m[None, :] / length[:, None]

    Kx, Ky = freq(nx, lx), freq(ny, ly)
    K2 = Kx[:, None, :] ** 2 + Ky[:, :, None] ** 2
    PF = (torch.exp(-1j * K2 * dz / (2 * kF)) * math.exp(-w.alpha_f * dz / 2)).to(cdt)
    PS = (torch.exp(-1j * K2 * dz / (2 * kS)) * math.exp(-w.alpha_sh * dz / 2)).to(cdt)
    dT = torch.stack([torch.as_tensor(v.dT, dtype=f64) for v in ws]).to(dev)
    _, tz, ty, tx = dT.shape
    dZ = w.L / (tz - 1)
    C = torch.cumsum(torch.cat([torch.zeros_like(dT[:, :1]),
                                0.5 * dZ * (dT[:, 1:] + dT[:, :-1])], 1), 1)
    dT, C = dT.to(real), C.to(real)

    def cell(coord, length, n):
        u = ((coord + length[:, None] / 2) / (length[:, None] / (n - 1))).clamp(0, n - 1)
        i = torch.floor(u).clamp(max=n - 2)
        return i.long(), (u - i).to(real)

    ix, fx = cell(x, col(v.t_lx for v in ws), tx)
    iy, fy = cell(y, col(v.t_ly for v in ws), ty)
    bidx = torch.arange(B, device=dev)[:, None, None]
    fxr, fyc = fx[:, None, :], fy[:, :, None]

    def bil(t2):
        a = t2[bidx, iy[:, :, None], ix[:, None, :]]
        b = t2[bidx, iy[:, :, None], ix[:, None, :] + 1]
        c = t2[bidx, iy[:, :, None] + 1, ix[:, None, :]]
        d = t2[bidx, iy[:, :, None] + 1, ix[:, None, :] + 1]
        return (1 - fyc) * ((1 - fxr) * a + fxr * b) + fyc * ((1 - fxr) * c + fxr * d)

    cF, cS = 0.5 * eps0c * w.n_f, 0.5 * eps0c * w.n_sh
    kapF = 2 * math.pi * w.d_eff / (w.n_f * w.lambda_f)
    kapS = 2 * math.pi * w.d_eff / (w.n_sh * w.lambda_f)
    k0F, k0S = 2 * math.pi / w.lambda_f, 4 * math.pi / w.lambda_f
    toff = col([v.t_off for v in ws], real)[:, None, None]

    def coef(z):
        zt = torch.as_tensor(z, dtype=f64, device=dev)
        u = (zt / dZ).clamp(0.0, tz - 1.0)
        l = torch.floor(u).clamp(max=tz - 2)
        t = (u - l).to(real)
        li = l.long().reshape(1)
        d0, d1 = dT.index_select(1, li)[:, 0], dT.index_select(1, li + 1)[:, 0]
        c0, c1 = C.index_select(1, li)[:, 0], C.index_select(1, li + 1)[:, 0]
        d = (1 - t) * bil(d0) + t * bil(d1) + toff
        c = (1 - t) * bil(c0) + t * bil(c1)
        phi = (w.dk0 + w.ddk_dT * toff) * zt.to(real) + w.ddk_dT * c
        return torch.exp(1j * phi), k0F * w.dn_dT * d, k0S * w.dn_dT * d

    def rhs(a, s, cf):
        e, pF, pS = cf
        fF = -0.5 * w.beta_f * cF * a.abs() ** 2 * a + 1j * pF * a
        fF = fF + 1j * kapF * s * a.conj() * e.conj()
        fS = 1j * kapS * a * a * e - 0.5 * w.beta_sh * cS * s.abs() ** 2 * s + 1j * pS * s
        return fF, fS

    def rk4(a, s, z0, h):
        c0, cm, c1 = coef(z0), coef(z0 + h / 2), coef(z0 + h)
        k1 = rhs(a, s, c0)
        k2 = rhs(a + h / 2 * k1[0], s + h / 2 * k1[1], cm)
        k3 = rhs(a + h / 2 * k2[0], s + h / 2 * k2[1], cm)
        k4 = rhs(a + h * k3[0], s + h * k3[1], c1)
        return (a + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
                s + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))

    def step(a, s, z):
        a, s = rk4(a, s, z, dz / 2)
        a = torch.fft.ifft2(PF * torch.fft.fft2(a))
        s = torch.fft.ifft2(PS * torch.fft.fft2(s))
        return rk4(a, s, z + dz / 2, dz / 2)

    return AF, AS, step


def plain_form(w, dev: str = "cuda", real=torch.float64):
    """plain_group_form for one instance, fields [ny, nx]."""
    AF, AS, step = plain_group_form([w], dev, real)

    def step1(a, s, z):
        a2, s2 = step(a[None], s[None], z)
        return a2[0], s2[0]

    return AF[0], AS[0], step1


def plain_gpu_rate(ws, nsteps: int, real=torch.float64):
    """plain_group_form on the GPU with one z-step captured in a CUDA graph
    and replayed (so the timing is of the kernels, not of Python dispatch).
    Returns (grid-point-steps/s over `nsteps` z-steps, how it ran)."""
    AF, AS, step = plain_group_form(ws, "cuda", real)
    nx, ny, dz = ws[0].nx, ws[0].ny, ws[0].L / ws[0].nz
    zt = torch.zeros((), dtype=torch.float64, device="cuda")
    a_buf, s_buf = AF.clone(), AS.clone()

    def body():
        a, s = step(a_buf, s_buf, zt)
        a_buf.copy_(a)
        s_buf.copy_(s)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            body()
    torch.cuda.current_stream().wait_stream(side)
    how = "one z-step captured in a CUDA graph, replayed"
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            body()
        run = graph.replay
    except Exception as e:  # capture refused: time the same step eagerly
        how = f"eager (graph capture failed: {type(e).__name__})"
        run = body
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(nsteps):
        zt.fill_(k * dz)
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    return len(ws) * nx * ny * nsteps / (e0.elapsed_time(e1) * 1e-3), how


# ------------------------------------------------------------------ oracle ----

def oracle_sample_rate(instances, nsteps: int):
    """FP64 CPU oracle (as it stands) on `nsteps` z-steps of each instance."""
    from oracle import ssfm
    pts = 0
    t0 = time.perf_counter()
    for w in instances:
        p = ssfm.params_from_workload(w)
        temp = ssfm.TemperatureField(p, torch.as_tensor(w.dT), w.t_lx, w.t_ly, w.t_off)
        AF0 = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus)
        ssfm.propagate(p, AF0, torch.zeros_like(AF0), temp, nsteps=nsteps)
        pts += w.nx * w.ny * nsteps
    dt = time.perf_counter() - t0
    return pts / dt, dt


def oracle_threads(n: int = 0) -> int:
    """Set (n > 0) and return the oracle's thread count: PyTorch's CPU ops
    and the OpenMP loop of its C DFT use the same number."""
    from oracle import fft as oracle_fft
    if n > 0:
        torch.set_num_threads(n)
        oracle_fft.set_threads(n)
    else:
        oracle_fft.set_threads(torch.get_num_threads())
    return torch.get_num_threads()


def oracle_baseline(sample, nsteps: int, single_steps: int):
    """Best of three timed runs on all host threads, plus one run on one
    thread (per-core context)."""
    cores = oracle_threads()
    runs = [oracle_sample_rate(sample, nsteps) for _ in range(3)]
    rate = max(r for r, _ in runs)
    out = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
           "nproc": os.cpu_count(),
           "sample": f"best of 3 runs of {nsteps} z-steps of one instance per grid size "
                     f"({', '.join(f'{w.nx}^2' for w in sample)}), "
                     f"{sum(dt for _, dt in runs):.1f} s of CPU work"}
    if single_steps > 0:
        oracle_threads(1)
        r1, dt1 = oracle_sample_rate(sample, single_steps)
        oracle_threads(cores)
        out["single_core"] = {"value": r1, "unit": UNIT,
                              "sample": f"{single_steps} z-steps per instance, 1 thread, "
                                        f"{dt1:.1f} s"}
    return out


def sample_instances(insts):
    """First instance of every grid size of the sweep."""
    seen, out = set(), []
    for w in insts:
        if w.nx not in seen:
            seen.add(w.nx)
            out.append(w)
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    insts = W.sweep_instances(seed=1)
    sample = sample_instances(insts)
    nsteps = args.ref_zsteps
    cores = oracle_threads()
    for _ in range(args.warmup):
        oracle_sample_rate(sample, nsteps)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = oracle_sample_rate(sample, nsteps)
        rates.append(r)
        times.append(dt)
    value = float(np.mean(rates))
    desc = (f"{nsteps} z-steps of one instance of each grid ({', '.join(f'{w.nx}^2' for w in sample)})"
            " of the 384-instance sweep per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sweep_384_mixed_nz2000", "sample": desc},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT,
                             "cores": cores, "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- multi-rank ----

def rank_instances(rank: int, nz: int = 2000, groups=W.SWEEP_GROUPS):
    """Instances of one rank: an independent seeded sweep (seed 1 + rank), so
    per-rank work is fixed as ranks are added (weak scaling) and no data moves
    between ranks."""
    return W.sweep_instances(seed=1 + rank, nz=nz, groups=groups)


def aggregate_rate(point_steps_local: float, seconds_local: float, world: int, device=None):
    """Whole-job throughput: point-steps summed over ranks / the slowest
    rank's time (the only collective of the benchmark; not on the data path)."""
    if world == 1:
        return point_steps_local / seconds_local, seconds_local
    t = torch.tensor([seconds_local], dtype=torch.float64, device=device)
    n = torch.tensor([point_steps_local], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
    return float(n) / float(t), float(t)


# ------------------------------------------------------------ every config ----

GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden(name):
    """Stored oracle values (written by tests/golden/make_golden.py, which
    calls only the FP64 oracle), or None if that file is absent."""
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        return None
    if path.endswith(".json"):
        return json.load(open(path))
    return dict(np.load(path))


def _rel(a, b):
    return abs(a / b - 1) if b else abs(a)


def _event_ms(fn, reps, stream):
    """CUDA-event time of fn() (which may synchronise) on `stream`, per call."""
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _pass_roof(pkg, plan, w, stream, fp32_peak, fp64_peak, l2_gbs, hbm_gbs, thermal):
    """Row and column launch times of one plan (CUDA events) and their
    fractions of the binding roofs."""
    t = min((pkg.shg_pass_times([plan.handle], nsteps=10, stream=stream)[0] for _ in range(3)),
            key=lambda g: g["row_ms"] + g["col_ms"])
    npts = w.nx * w.ny
    fp64 = getattr(w, "precision", "f32") == "f64"
    peak = fp64_peak if fp64 else fp32_peak
    one = t.get("passes_per_step", 2) == 1
    row_flops = (step_flops_per_point if one else row_flops_per_point)(w.nx, thermal) * npts
    col_bytes = col_bytes_per_point() * (2 if fp64 else 1) * npts
    out = {"row_ms": t["row_ms"], "col_ms": t["col_ms"], "passes_per_step": t.get("passes_per_step", 2),
            "row_alu_frac": row_flops / (t["row_ms"] * 1e-3) / (peak * 1e12),
            "row_alu_peak_tflops": peak,
            "col_gbs": col_bytes / (t["col_ms"] * 1e-3) / 1e9,
            "col_hbm_frac": col_bytes / (t["col_ms"] * 1e-3) / 1e9 / hbm_gbs,
            "col_l2_frac": col_bytes / (t["col_ms"] * 1e-3) / 1e9 / l2_gbs}
    if one:
        out["col_alu_frac"] = (step_flops_per_point(w.ny, thermal) * npts / (t["col_ms"] * 1e-3)
                               / (peak * 1e12))
    return out


def time_configs(pkg, stream, mp, hbm_gbs):
    """Every workload at full size, timed through the C ABI with CUDA events
    on `stream`, with its error against stored FP64-oracle values."""
    fp32, fp64, l2 = mp["fp32_peak_tflops"], mp["fp64_tflops"], mp["l2_read_gbs"]
    out = {}
    cfg_eta = golden("configs_eta.json") or {}

    # plain: 32^2, nz = 100, FP64, single instance
    w = W.plain_focused()
    plan = pkg.Plan(w)
    run = lambda: (plan.propagate(stream), plan.efficiency())  # noqa: E731
    run()
    ms = statistics.median(_event_ms(run, 20, stream))
    eta = plan.efficiency()[0]
    e = {"workload": "plain_32x32_nz100_fp64", "value": w.point_steps / (ms * 1e-3),
         "unit": UNIT, "ms_per_propagation": ms, "dtype": "f64"}
    if "plain" in cfg_eta:
        e["eta_rel_err_vs_oracle"] = _rel(eta, cfg_eta["plain"]["eta"])
    e["passes"] = _pass_roof(pkg, plan, w, stream, fp32, fp64, l2, hbm_gbs, False)
    out["plain"] = e
    del plan

    # depleted: 128^2, nz = 1000, FP32, seeded map, single instance
    w = W.depleted_absorbing()
    plan = pkg.Plan(w)
    plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    run = lambda: (plan.propagate(stream), plan.efficiency())  # noqa: E731
    run()
    ms = statistics.median(_event_ms(run, 10, stream))
    eta = plan.efficiency()[0]
    e = {"workload": "depleted_128x128_nz1000", "value": w.point_steps / (ms * 1e-3),
         "unit": UNIT, "ms_per_propagation": ms, "us_per_z_step": 1e3 * ms / w.nz,
         "dtype": "f32"}
    if "depleted" in cfg_eta:
        e["eta_rel_err_vs_oracle"] = _rel(eta, cfg_eta["depleted"]["eta"])
    e["passes"] = _pass_roof(pkg, plan, w, stream, fp32, fp64, l2, hbm_gbs, True)
    out["depleted"] = e
    del plan

    # adjoint: 256^2, nz = 2000, FP32, forward + reverse sweep
    w = W.adjoint_case()
    plan = pkg.Plan(w, adjoint=True)
    dT = torch.as_tensor(w.dT).cuda()
    plan.set_temperature(dT, w.t_lx, w.t_ly)
    g_dT = torch.empty_like(dT)
    fwd = lambda: (plan.propagate(stream), plan.efficiency())  # noqa: E731
    bwd = lambda: pkg.shg_propagate_adjoint(plan.handle, 1.0, g_dT, stream)  # noqa: E731
    fwd()
    bwd()
    f_ms = statistics.median(_event_ms(fwd, 3, stream))
    b_ms = statistics.median(_event_ms(lambda: (fwd(), bwd()), 3, stream)) - f_ms
    eta = plan.efficiency()[0]
    gw, gz, gt = bwd()
    e = {"workload": "adjoint_256x256_nz2000", "value": w.point_steps / (f_ms * 1e-3),
         "unit": UNIT, "forward_ms": f_ms, "backward_ms": b_ms,
         "forward_plus_backward_point_steps_per_s": w.point_steps / ((f_ms + b_ms) * 1e-3),
         "dtype": "f32"}
    fd = golden("adjoint_fd_256_nz2000.json")
    if fd is not None:
        e["eta_rel_err_vs_oracle"] = _rel(eta, fd["eta"])
        gT = g_dT.double().cpu().numpy()
        scale_t = float(np.abs(gT).sum())   # 1 K applied to every node
        errs = {"w0": _rel(gw, fd["d_w0"]["value"]), "z_focus": _rel(gz, fd["d_zf"]["value"]),
                "t_off": abs(gt - fd["d_toff"]["value"]) / max(abs(fd["d_toff"]["value"]),
                                                               scale_t)}
        rng = np.random.default_rng(fd["d_map_directions"][0]["seed"])
        for d in fd["d_map_directions"]:
            v = rng.normal(size=gT.shape)
            got = float((gT * v).sum())
            errs[f"map_direction_{d['index']}"] = abs(got - d["value"]) / max(
                abs(d["value"]), float(np.abs(gT * v).sum()) * 1e-2)
        e["gradient_rel_err_vs_oracle_fd"] = errs
    e["passes"] = _pass_roof(pkg, plan, w, stream, fp32, fp64, l2, hbm_gbs, True)
    out["adjoint"] = e
    del plan

    ext = golden("extensions.json") or {}
    # Eq. (4) phase model: the depleted workload with caller index polynomials
    w = W.eq4_case()
    plan = pkg.Plan(w)
    plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    run = lambda: (plan.propagate(stream), plan.efficiency())  # noqa: E731
    run()
    ms = statistics.median(_event_ms(run, 10, stream))
    eta = plan.efficiency()[0]
    e = {"workload": w.name, "value": w.point_steps / (ms * 1e-3), "unit": UNIT,
         "ms_per_propagation": ms, "us_per_z_step": 1e3 * ms / w.nz, "dtype": "f32",
         "path": "single 128^2 plan: the cluster-resident kernel, Eq. (4) phase table"}
    if "eq4" in ext:
        e["eta_rel_err_vs_oracle"] = _rel(eta, ext["eq4"]["eta"])
    out["eq4"] = e
    del plan

    # three-wave mixing: sum- and difference-frequency generation, 128^2 x 1000
    for key, w in (("sfg", W.sfg_case(n=128, nz=1000)), ("dfg", W.dfg_case(n=128, nz=1000))):
        plan = pkg.Plan3(w)
        plan.set_temperature(w.dT, w.t_lx, w.t_ly)
        run = lambda: (plan.propagate(stream), plan.powers())  # noqa: E731
        run()
        ms = statistics.median(_event_ms(run, 5, stream))
        P = plan.powers()
        pts = w.nx * w.ny * w.nz
        e = {"workload": w.name, "value": pts / (ms * 1e-3), "unit": UNIT,
             "ms_per_propagation": ms, "us_per_z_step": 1e3 * ms / w.nz,
             "path": "single 128^2 plan: the cluster-resident three-wave kernel, map through "
                     "the per-point table",
             "powers_W": list(P), "dtype": "f32",
             "alu_frac_whole_propagation": threewave_flops_per_point_step(w.nx, True) * pts
             / (ms * 1e-3) / (fp32 * 1e12)}
        if key in ext:
            ref = ext[key]["powers"]
            e["powers_err_vs_oracle"] = max(abs(a - b) for a, b in zip(P, ref)) / max(ref)
        out["threewave_" + key] = e
        del plan

    # thermal: 1024^2, nz = 8000, 6 outer iterations with heat solves
    w = W.thermal_loop()
    plan = pkg.Plan(w, thermal=True)
    res = {}

    def loop():
        res["etas"], res["changes"] = pkg.shg_thermal_loop(plan.handle, w.n_outer, 200000, 1e-6,
                                                           stream)
    ms = statistics.median(_event_ms(loop, 1, stream))
    e = {"workload": "thermal_1024x1024_nz8000_x6", "value": w.n_outer * w.point_steps /
         (ms * 1e-3), "unit": UNIT, "ms_per_loop": ms, "etas": res["etas"],
         "changes_K": res["changes"], "dtype": "f32"}
    tp = golden("thermal_pass_1024_nz8000.npz")
    if tp is not None:
        e["first_pass_eta_rel_err_vs_oracle"] = _rel(res["etas"][0], float(tp["eta"]))
    # heat solves alone, each method on the same deposits: a cold start
    # (dT = 0 with the first pass's deposits) and a warm start (from that
    # solution after the second pass)
    hs = {"grid": f"{w.hx}x{w.hy}x{w.hz}", "tol_K": 1e-6}
    # (the SOR takes oven-held faces only; the direct solve also the convective
    # faces of Eq. 10: the end facets in air, h = 10 W/(m^2 K))
    for name, wk, method in (("direct", w, pkg.SHG_HEAT_DIRECT), ("sor", w, pkg.SHG_HEAT_SOR),
                             ("direct_convective_end_facets",
                              W.with_oven(w, "surrounded", h_conv=10.0), pkg.SHG_HEAT_DIRECT)):
        plan2 = pkg.Plan(wk, thermal=True)
        pkg.shg_set_heat_method(plan2.handle, method)
        plan2.propagate(stream)
        plan2.efficiency()
        sw = {}
        cold = _event_ms(lambda: sw.__setitem__("cold", pkg.shg_heat_solve(
            plan2.handle, 200000, 1e-6, stream)), 1, stream)
        plan2.propagate(stream)
        plan2.efficiency()
        warm = _event_ms(lambda: sw.__setitem__("warm", pkg.shg_heat_solve(
            plan2.handle, 200000, 1e-6, stream)), 1, stream)
        hs[name] = {"cold_ms": cold[0], "cold_iterations": sw["cold"][1],
                    "warm_ms": warm[0], "warm_iterations": sw["warm"][1]}
        del plan2
    hs["cold_speedup_direct_over_sor"] = hs["sor"]["cold_ms"] / hs["direct"]["cold_ms"]
    e["heat_solve"] = hs
    e["passes"] = _pass_roof(pkg, plan, w, stream, fp32, fp64, l2, hbm_gbs, True)
    out["thermal"] = e
    del plan
    return out


# --------------------------------------------------------------- our path ----

def run_ours(args, rank, world):
    import paper_2410_04994_gb300 as pkg
    from paper_2410_04994_gb300 import build as pbuild

    if rank == 0:
        pbuild.build()
    if world > 1:
        torch.distributed.barrier()
    pkg.load()
    dev = torch.cuda.current_device()
    groups_arg = tuple((int(a), int(b)) for a, b in
                       (g.split(":") for g in args.groups.split(","))) if args.groups else W.SWEEP_GROUPS
    insts = rank_instances(rank, nz=args.nz, groups=groups_arg)
    npoint_steps = sum(w.nx * w.ny * w.nz for w in insts)
    plans = [pkg.Plan(w) for w in insts]
    maps = [torch.as_tensor(w.dT).to("cuda") for w in insts]
    for p, w, m in zip(plans, insts, maps):
        p.set_temperature(m, w.t_lx, w.t_ly)
    handles = [p.handle for p in plans]
    stream = torch.cuda.current_stream()

    def step():
        return pkg.shg_batch_submit(handles, stream)

    for _ in range(max(args.warmup, 1)):
        etas = step()
    kernels_per_step = 0
    groups = {}
    for w in insts:
        groups.setdefault((w.nx, w.ny, w.nz), 0)
        groups[(w.nx, w.ny, w.nz)] += 1
    for (nx, ny, nz), _ in groups.items():   # two passes per step; recounted below from the
        kernels_per_step += 2 + (nz + 1) + nz + 2   # schedule each group reports

    l2_flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        l2_flush.fill_(k & 0xFF)   # evict L2 between timed steps (not timed)
        ev[k][0].record(stream)
        torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select the timed launches
        etas = step()
        torch.cuda.nvtx.range_pop()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    value, t_total = aggregate_rate(npoint_steps * args.steps, sum(ms) / 1e3, world, "cuda")
    if not all(math.isfinite(e) for e in etas):
        raise RuntimeError("non-finite efficiency")

    # ---- end to end: host maps -> device, tables, propagation, eta -> host.
    # The maps of the sweep share one shape, so they live in one pinned host
    # buffer and cross in one copy per step, into one of two device buffers
    # (views per plan): step k+1's maps are uploaded on a copy stream while
    # step k propagates.  The timed region is the whole loop of K steps, from
    # the first upload to the last step's efficiencies on the host.
    host_all = torch.stack([m.cpu() for m in maps]).pin_memory()
    bufs = [torch.empty(host_all.shape, dtype=host_all.dtype, device="cuda") for _ in range(2)]
    views = [[b[i] for i in range(len(maps))] for b in bufs]
    h2d = host_all.numel() * 4
    d2h = 16 * len(insts)
    copy_stream = torch.cuda.Stream()
    uploaded = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    lx_all, ly_all = [w.t_lx for w in insts], [w.t_ly for w in insts]

    def upload(b, after=None):
        with torch.cuda.stream(copy_stream):
            if after is not None:
                copy_stream.wait_event(after)   # the table build of step k-1 read this buffer
            bufs[b].copy_(host_all, non_blocking=True)
            uploaded[b].record(copy_stream)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload(0)
    for k in range(args.steps):
        b = k & 1
        if k + 1 < args.steps:
            upload(b ^ 1, consumed[b ^ 1] if k >= 1 else None)
        stream.wait_event(uploaded[b])
        pkg.shg_set_temperature_batch(handles, views[b], lx_all, ly_all, stream)
        consumed[b].record(stream)
        step()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = aggregate_rate(npoint_steps * args.steps, e2e_s, world, "cuda")

    result = None
    if rank == 0:
        result = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                      warmup=args.warmup, ms_per_step=1e3 * t_total / args.steps,
                      higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                      data="synthetic",
                      config={"workload": ("sweep_384_mixed_nz2000" if (not args.groups and
                                                                          args.nz == 2000)
                                           else f"sweep_{args.groups or 'default'}_nz{args.nz}"),
                              "instances": len(insts),
                              "grids": " + ".join(f"{c}x{n}^2" for n, c in groups_arg),
                              "nz": args.nz,
                              "temperature_maps": "64x64x128 per instance",
                              "point_steps_per_gpu_step": npoint_steps,
                              "l2": "256 MB buffer written between timed steps; inputs "
                                    "(126 MB fields + 1.6 GB maps/tables) exceed L2",
                              "parallelism": f"instances sharded, {world} rank(s), no "
                                             "data-path collective"},
                      clocks={"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                              "reasons": clk["reasons"]},
                      e2e={"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                           "d2h_bytes_per_step": d2h,
                           "how": "each step: its 384 maps from pinned host memory (one copy, "
                                  "on a copy stream during the previous step's propagation, "
                                  "into one of two device buffers), shg_set_temperature_batch, "
                                  "shg_batch_submit, eta to the host; wall time of all K steps"},
                      gpu_launches=kernels_per_step * args.steps)

    # ---- measured ceilings of this device (timed kernels; no setting changes)
    pk = peaks()
    mpk = pkg.shg_measure_peaks(stream)
    fp32_peak = max(mpk["fp32_tflops"], mpk["fp32_scalar_tflops"])
    mp = dict(mpk, fp32_peak_tflops=fp32_peak)

    # ---- per-kernel launch times (CUDA events on the launching stream)
    pkg.shg_pass_times(handles, nsteps=2, stream=stream)
    runs = [pkg.shg_pass_times(handles, nsteps=10, stream=stream) for _ in range(3)]
    times = [dict(g, row_ms=min(r[i]["row_ms"] for r in runs), col_ms=min(r[i]["col_ms"] for r in runs))
             for i, g in enumerate(runs[0])]
    for g in times:
        npts = g["nx"] * g["ny"] * g["instances"]
        one = g["passes_per_step"] == 1
        g["row_alu_frac"] = ((step_flops_per_point if one else row_flops_per_point)(g["nx"], True)
                             * npts / (g["row_ms"] * 1e-3) / (fp32_peak * 1e12))
        if one:
            g["col_alu_frac"] = (step_flops_per_point(g["ny"], True) * npts / (g["col_ms"] * 1e-3)
                                 / (fp32_peak * 1e12))
        gbs = col_bytes_per_point() * npts / (g["col_ms"] * 1e-3) / 1e9
        g["col_gbs"] = gbs
        g["col_hbm_frac"] = gbs / pk["hbm_gbs"]
        g["col_l2_frac"] = gbs / mpk["l2_read_gbs"]
    # launches per timed step: 2 init + 2 power + the passes of each group
    # (nz + 1 on the one-pass-per-step schedule, 2 nz + 1 otherwise)
    kernels_per_step = sum(4 + (args.nz + 1 if g["passes_per_step"] == 1 else 2 * args.nz + 1)
                           for g in times)
    if rank == 0:
        result["gpu_launches"] = kernels_per_step * args.steps
    best = None
    for g in times:
        npts = g["nx"] * g["ny"] * g["instances"]
        nz = args.nz
        # launches per propagation: one pass per step (even s in the row
        # layout, odd s in the column layout) or a row and a column pass
        launches = ((nz // 2 + 1, (nz + 1) // 2) if g["passes_per_step"] == 1 else (nz + 1, nz))
        for kind, t_ms, n_l in (("row", g["row_ms"], launches[0]), ("col", g["col_ms"], launches[1])):
            share = t_ms * n_l
            if best is None or share > best[0]:
                best = (share, kind, g, t_ms, npts)
    _, kind, g, t_ms, npts = best
    alu_peak = {"peak": fp32_peak, "unit": "TFLOP/s",
                "peak_source": "measured: FP32 FMA throughput kernel (shg_measure_peaks), "
                               "burst, timed alone like the pass",
                "derived_peak_at_sm_max": N_SM * FP32_LANES_PER_SM * 2
                * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12}
    if g["passes_per_step"] == 1:
        n = g["nx"] if kind == "row" else g["ny"]
        per_point = step_flops_per_point(n, True)
        achieved = per_point * npts / (t_ms * 1e-3) / 1e12
        name = (f"k_row_pass<float,{n}> (row-layout step pass: Lx, N, Lx)" if kind == "row"
                else f"k_col_step<{n}> (column-layout step pass: Ly, N, Ly)")
        roof = dict({"bound": "alu", "kernel": name, "achieved": achieved,
                     "frac": achieved / fp32_peak}, **alu_peak,
                    algorithmic_per_point=per_point, points_per_launch=npts, launch_ms=t_ms,
                    traffic=None)
    elif kind == "row":
        flops = row_flops_per_point(g["nx"], True) * npts
        achieved = flops / (t_ms * 1e-3) / 1e12
        roof = dict({"bound": "alu", "kernel": f"k_row_pass<float,{g['nx']}>", "achieved": achieved,
                     "frac": achieved / fp32_peak}, **alu_peak,
                    algorithmic_per_point=row_flops_per_point(g["nx"], True),
                    points_per_launch=npts, launch_ms=t_ms, traffic=None)
    else:
        byts = col_bytes_per_point() * npts
        peak = pk["hbm_gbs"]
        achieved = byts / (t_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"k_col_pass<float,{g['ny']}>", "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_per_point": col_bytes_per_point(), "points_per_launch": npts,
                "launch_ms": t_ms, "traffic": None}
    traffic_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(traffic_file):
        tr = json.load(open(traffic_file)).get(roof["kernel"])
        if tr is not None:
            roof["traffic"] = tr
    if rank == 0:
        result["roofline"] = roof
        result["pass_times_ms"] = times
        result["measured_peaks"] = dict(mp, hbm_gbs=pk["hbm_gbs"],
                                        how="shg_measure_peaks on this GPU during this run; "
                                            "HBM from MEASURED_PEAKS.json")

    # ---- comparisons (rank 0, N = 1): plain GPU forms, oracle, eta check, every config
    if rank == 0 and world == 1 and not args.skip_baselines:
        g256 = [w for w in insts if w.nx == 256]
        fused_256 = [g for g in times if g["nx"] == 256]
        try:
            plain, how = plain_gpu_rate(g256[:1], 50)
            result["plain_fp64_gpu"] = {
                "value": plain, "unit": UNIT,
                "sample": f"one 256^2 instance, 50 z-steps, complex128 torch + torch.fft, "
                          f"unfused; {how}",
                "speedup_of_fused_fp32": value / plain}
        except Exception as e:  # a comparison only: never lose the measured line for it
            result["plain_fp64_gpu"] = {"error": f"{type(e).__name__}: {e}"[:200]}
        try:
            p32, how = plain_gpu_rate(g256, 50, torch.float32)
            ent = {"value": p32, "unit": UNIT,
                   "sample": f"all {len(g256)} 256^2 instances of the sweep batched, 50 z-steps, "
                             f"complex64 torch + torch.fft (cuFFT) with unfused elementwise "
                             f"steps (the paper's design); {how}",
                   "speedup_of_fused_fp32": value / p32}
            if fused_256:
                f = fused_256[0]
                rate = f["nx"] * f["ny"] * f["instances"] / ((f["row_ms"] + f["col_ms"]) * 1e-3)
                ent["fused_same_group"] = rate
                ent["speedup_of_fused_same_group"] = rate / p32
            result["plain_fp32_gpu"] = ent
        except Exception as e:
            result["plain_fp32_gpu"] = {"error": f"{type(e).__name__}: {e}"[:200]}
        sample = sample_instances(insts)
        result["cpu_baseline"] = oracle_baseline(sample, args.ref_zsteps // 2 + 10, 10)
        # eta of the first instance against the FP64 oracle at full length
        cfg_eta = golden("configs_eta.json") or {}
        w0 = insts[0]
        if args.nz == 2000 and not args.groups and w0.name in cfg_eta.get("sweep", {}):
            eta_ref = cfg_eta["sweep"][w0.name]["eta"]
            src_ref = "stored FP64-oracle value (tests/golden/configs_eta.json)"
        else:
            from oracle import ssfm
            eta_ref = float(ssfm.run(w0)[2])
            src_ref = "FP64 oracle run live"
        result["eta_rel_err_vs_oracle"] = {"instance": w0.name, "value": _rel(etas[0], eta_ref),
                                           "oracle": src_ref}
        if not args.skip_configs:
            result["configs"] = time_configs(pkg, stream, mp, pk["hbm_gbs"])
    if rank == 0:
        print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-zsteps", type=int, default=100)
    ap.add_argument("--skip-baselines", action="store_true",
                    help="only the sweep line (no comparisons, no other configs)")
    ap.add_argument("--skip-configs", action="store_true",
                    help="no timing of the other workloads")
    ap.add_argument("--nz", type=int, default=2000,
                    help="z-steps per instance (2000 is the benchmarked workload; smaller "
                         "values are for profiling captures)")
    ap.add_argument("--groups", default="",
                    help="grid:count list, e.g. 256:64 (default: the 384-instance sweep)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank)
        return
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    run_ours(args, rank, world)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
