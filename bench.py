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


# ----------------------------------------------------- plain FP64 GPU form ----

def plain_form(w, dev: str = "cuda", f64=torch.float64):
    """The same split step written plainly in PyTorch: complex fields with
    torch.fft, one instance, unfused elementwise ops (real type f64; complex
    the matching type).  Returns (A_F(0), A_SH(0), step), step(a, s, z)
    advancing one z-step from z."""
    c128 = torch.complex128 if f64 == torch.float64 else torch.complex64
    eps0c = 8.8541878128e-12 * 299792458.0
    nx, ny, dz = w.nx, w.ny, w.L / w.nz
    x = (torch.arange(nx, dtype=f64, device=dev) - nx // 2) * (w.lx / nx)
    y = (torch.arange(ny, dtype=f64, device=dev) - ny // 2) * (w.ly / ny)
    kF = 2 * math.pi * w.n_f / w.lambda_f
    kS = 2 * math.pi * w.n_sh / (w.lambda_f / 2)
    zr = w.w0 ** 2 * kF / 2
    q = complex(1.0, -w.z_focus / zr)
    r2 = (x[None, :] ** 2 + y[:, None] ** 2).to(c128)
    AF = torch.exp(-r2 / (w.w0 ** 2 * q)) / q
    AF = AF * math.sqrt(w.p1 / float(0.5 * eps0c * w.n_f * (AF.abs() ** 2).sum()
                                     * (w.lx / nx) * (w.ly / ny)))
    AS = torch.zeros_like(AF)
    Kx = 2 * math.pi * torch.fft.fftfreq(nx, d=w.lx / nx, dtype=f64, device=dev)
    Ky = 2 * math.pi * torch.fft.fftfreq(ny, d=w.ly / ny, dtype=f64, device=dev)
    K2 = Kx[None, :] ** 2 + Ky[:, None] ** 2
    PF = torch.exp(-1j * K2 * dz / (2 * kF)) * math.exp(-w.alpha_f * dz / 2)
    PS = torch.exp(-1j * K2 * dz / (2 * kS)) * math.exp(-w.alpha_sh * dz / 2)
    dT = torch.as_tensor(w.dT, dtype=f64, device=dev)
    tz, ty, tx = dT.shape
    dZ = w.L / (tz - 1)
    C = torch.cumsum(torch.cat([torch.zeros_like(dT[:1]), 0.5 * dZ * (dT[1:] + dT[:-1])]), 0)

    def cell(coord, lo, n, length):
        u = ((coord - lo) / (length / (n - 1))).clamp(0, n - 1)
        i = torch.floor(u).clamp(max=n - 2)
        return i.long(), u - i

    ix, fx = cell(x, -w.t_lx / 2, tx, w.t_lx)
    iy, fy = cell(y, -w.t_ly / 2, ty, w.t_ly)

    def bil(t2):
        a = t2[iy][:, ix]; b = t2[iy][:, ix + 1]; c = t2[iy + 1][:, ix]; d = t2[iy + 1][:, ix + 1]
        return (1 - fy[:, None]) * ((1 - fx) * a + fx * b) + fy[:, None] * ((1 - fx) * c + fx * d)

    cF, cS = 0.5 * eps0c * w.n_f, 0.5 * eps0c * w.n_sh
    kapF = 2 * math.pi * w.d_eff / (w.n_f * w.lambda_f)
    kapS = 2 * math.pi * w.d_eff / (w.n_sh * w.lambda_f)
    k0F, k0S = 2 * math.pi / w.lambda_f, 4 * math.pi / w.lambda_f

    def coef(z):
        u = min(max(z / dZ, 0.0), tz - 1.0)
        l = min(int(u), tz - 2)
        t = u - l
        d = (1 - t) * bil(dT[l]) + t * bil(dT[l + 1]) + w.t_off
        c = (1 - t) * bil(C[l]) + t * bil(C[l + 1])
        phi = (w.dk0 + w.ddk_dT * w.t_off) * z + w.ddk_dT * c
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


def plain_gpu_rate(w, nsteps: int, real=torch.float64) -> float:
    """plain_form on the GPU (complex128 by default; complex64 is the paper's
    own design: cuFFT plus unfused elementwise steps in FP32).  Returns
    grid-point-steps/s over `nsteps` z-steps."""
    AF, AS, step = plain_form(w, "cuda", real)
    nx, ny, dz = w.nx, w.ny, w.L / w.nz
    for k in range(3):
        AF, AS = step(AF, AS, k * dz)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(nsteps):
        AF, AS = step(AF, AS, (3 + k) * dz)
    torch.cuda.synchronize()
    return nx * ny * nsteps / (time.perf_counter() - t0)


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
                             "cores": torch.get_num_threads(), "sample": desc},
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
    for (nx, ny, nz), _ in groups.items():
        kernels_per_step += 2 + (nz + 1) + nz + 2

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

    # ---- end to end: host maps -> device, tables, propagation, eta -> host
    host_maps = [m.cpu().pin_memory() for m in maps]
    h2d = sum(m.numel() * 4 for m in host_maps)
    d2h = 16 * len(insts)
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(args.steps):
        l2_flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for hm, dm in zip(host_maps, maps):
            dm.copy_(hm, non_blocking=True)
        pkg.shg_set_temperature_batch(handles, maps, [w.t_lx for w in insts],
                                      [w.t_ly for w in insts])
        step()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value, _ = aggregate_rate(npoint_steps, statistics.median(e2e_ms) / 1e3, world, "cuda")

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
                           "d2h_bytes_per_step": d2h},
                      gpu_launches=kernels_per_step * args.steps)

    # ---- per-kernel launch times (CUDA events on the launching stream)
    pk = peaks()
    pkg.shg_pass_times(handles, nsteps=2, stream=stream)
    runs = [pkg.shg_pass_times(handles, nsteps=10, stream=stream) for _ in range(3)]
    times = [dict(g, row_ms=min(r[i]["row_ms"] for r in runs), col_ms=min(r[i]["col_ms"] for r in runs))
             for i, g in enumerate(runs[0])]
    best = None
    for g in times:
        npts = g["nx"] * g["ny"] * g["instances"]
        nz = args.nz
        for kind, t_ms, launches in (("row", g["row_ms"], nz + 1), ("col", g["col_ms"], nz)):
            share = t_ms * launches
            if best is None or share > best[0]:
                best = (share, kind, g, t_ms, npts)
    _, kind, g, t_ms, npts = best
    if kind == "row":
        flops = row_flops_per_point(g["nx"], True) * npts
        peak = N_SM * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        achieved = flops / (t_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": f"k_row_pass<float,{g['nx']}>", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x sm_max_mhz",
                "algorithmic_per_point": row_flops_per_point(g["nx"], True),
                "points_per_launch": npts, "launch_ms": t_ms, "traffic": None}
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

    # ---- comparisons (rank 0, N = 1): plain FP64 GPU form, oracle, eta check
    if rank == 0 and world == 1 and not args.skip_baselines:
        w256 = [w for w in insts if w.nx == 256][0]
        plain = plain_gpu_rate(w256, 50)
        result["plain_fp64_gpu"] = {"value": plain, "unit": UNIT,
                                    "sample": "one 256^2 instance, 50 z-steps, complex128 torch"
                                              " + torch.fft, unfused",
                                    "speedup_of_fused_fp32": value / plain}
        try:
            p32 = plain_gpu_rate(w256, 200, torch.float32)
            result["plain_fp32_gpu"] = {"value": p32, "unit": UNIT,
                                        "sample": "one 256^2 instance, 200 z-steps, complex64 torch"
                                                  " + torch.fft (cuFFT), unfused: the paper's design",
                                        "speedup_of_fused_fp32": value / p32}
        except Exception as e:  # a comparison only: never lose the measured line for it
            result["plain_fp32_gpu"] = {"error": f"{type(e).__name__}: {e}"[:200]}
        sample = sample_instances(insts)
        nref = 3 * args.ref_zsteps  # about 10-15 s of CPU work
        rate, dt = oracle_sample_rate(sample, nref)
        result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": torch.get_num_threads(),
                                  "kind": "oracle",
                                  "sample": f"{nref} z-steps of one instance per grid "
                                            f"size ({dt:.1f} s of CPU work)"}
        # eta against the FP64 oracle on a full-length instance
        from oracle import ssfm
        w0 = insts[0]
        _, _, eta_ref = ssfm.run(w0)
        result["eta_rel_err_vs_oracle"] = {"instance": w0.name,
                                           "value": abs(etas[0] / float(eta_ref) - 1)}
    if rank == 0:
        print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-zsteps", type=int, default=100)
    ap.add_argument("--skip-baselines", action="store_true")
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
