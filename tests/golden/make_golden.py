"""Write the stored expected values of the full-size parity tests.

Every value written here comes from the FP64 CPU oracle (``oracle/``) on the
seeded inputs of ``workloads.py``; nothing is read from the CUDA path.  The
GPU tests load these files and compare the library's results with them.

    python tests/golden/make_golden.py adjoint_fd      # ~30 min on 8 cores
    python tests/golden/make_golden.py thermal_pass    # ~70 min on 8 cores
    python tests/golden/make_golden.py thermal_loop2   # ~15 min on 8 cores
    python tests/golden/make_golden.py configs         # ~5 min on 8 cores
    python tests/golden/make_golden.py extensions      # ~10 min on 8 cores

adjoint_fd (adjoint workload: 256 x 256, nz = 2000, 64 x 64 x 128 map, seed 0)
    eta and central finite differences of eta with respect to the waist w0,
    the focus position z_focus, the oven offset T_off (step 1e-4 |p|, with an
    absolute 1e-4 K for T_off = 0), and along three seeded directions of the
    temperature-map nodes (step 1e-3 K).  The grid and window stay fixed at
    the nominal waist, so the differences measure the discrete map alone.

thermal_pass (thermal workload: 1024 x 1024, nz = 8000, 128 x 128 x 256 heat
grid): the first pass of the self-consistent loop (Fig. 2), i.e. the
propagation with dT = 0 that deposits q_dot (Eq. 8).  Stored: eta, P_F(L),
P_SH(L), the deposited heat per heat-grid layer, and both output fields on a
stride-16 subgrid plus the central 32 x 32 block.

configs: eta, P_F(L) and P_SH(L) of the plain workload (32 x 32, nz = 100),
the depleted workload (128 x 128, nz = 1000, seed-0 map) and the first
instance of each grid of the 384-instance sweep (nz = 2000, seed 1).

extensions: eta, P_F(L) and P_SH(L) of the Eq. (4) workload (W.eq4_case:
128 x 128, nz = 1000, the depleted map), and the powers of the three waves of
sum- and difference-frequency generation (W.sfg_case, W.dfg_case at 128 x 128,
nz = 1000, seeded map).

thermal_loop2 (the thermal workload with nz = 100 and n_outer = 2): both
iterations of the loop, including the SOR solve on the full 128 x 128 x 256
heat grid between them.  Stored per iteration: eta, P_F, P_SH, the change of
dT, the deposited heat per layer; and the final dT on a subgrid, the total
deposit and both output fields of the second pass (subgrid + central block).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import heat, ssfm  # noqa: E402

ADJOINT_FD = os.path.join(HERE, "adjoint_fd_256_nz2000.json")
THERMAL_PASS = os.path.join(HERE, "thermal_pass_1024_nz8000.npz")
THERMAL_LOOP2 = os.path.join(HERE, "thermal_loop2_1024_nz100.npz")
CONFIGS = os.path.join(HERE, "configs_eta.json")
EXTENSIONS = os.path.join(HERE, "extensions.json")

FIELD_STRIDE = 16
CENTRE = 32
DIRECTION_SEED = 11
N_DIRECTIONS = 3


def field_samples(A: torch.Tensor):
    """(stride-16 subgrid, central 32 x 32 block) of a [ny][nx] field."""
    a = A.detach().numpy()
    ny, nx = a.shape
    c0, c1 = ny // 2 - CENTRE // 2, nx // 2 - CENTRE // 2
    return a[::FIELD_STRIDE, ::FIELD_STRIDE].copy(), a[c0:c0 + CENTRE, c1:c1 + CENTRE].copy()


def map_directions(shape):
    rng = np.random.default_rng(DIRECTION_SEED)
    return [rng.normal(size=shape) for _ in range(N_DIRECTIONS)]


def adjoint_fd():
    w = W.adjoint_case()
    dT0 = torch.tensor(w.dT, dtype=torch.float64)

    def eta(**kw):
        t = time.time()
        v = float(ssfm.run(w, **kw)[2])
        print(f"  eta={v:.15e} ({time.time() - t:.0f} s)", flush=True)
        return v

    def central(fun, x, h):
        return (fun(x + h) - fun(x - h)) / (2 * h), h

    out = {"_source": "FP64 CPU oracle, tests/golden/make_golden.py adjoint_fd",
           "workload": "adjoint_case(): 256x256, nz=2000, P1=30 W, xi=2.84, 64x64x128 map seed 0",
           "eta": eta()}
    g, h = central(lambda v: eta(w0=v), w.w0, 1e-4 * abs(w.w0))
    out["d_w0"] = {"value": g, "h": h}
    g, h = central(lambda v: eta(z_focus=v), w.z_focus, 1e-4 * abs(w.z_focus))
    out["d_zf"] = {"value": g, "h": h}
    g, h = central(lambda v: eta(t_off=v), w.t_off, max(1e-4 * abs(w.t_off), 1e-4))
    out["d_toff"] = {"value": g, "h": h}
    dirs = []
    for k, d in enumerate(map_directions(tuple(dT0.shape))):
        dd = torch.tensor(d)
        g, h = central(lambda s: eta(dT=dT0 + s * dd), 0.0, 1e-3)
        dirs.append({"seed": DIRECTION_SEED, "index": k, "value": g, "h": h})
    out["d_map_directions"] = dirs
    json.dump(out, open(ADJOINT_FD, "w"), indent=1)
    print(json.dumps(out, indent=1))


def _layer_sums(Q: torch.Tensor):
    return Q.sum(dim=(1, 2)).numpy()


def thermal_pass():
    w = W.thermal_loop()
    t = time.time()
    hist = heat.thermal_loop(w, 1)
    h = hist[0]
    p = ssfm.params_from_workload(w)
    pf = float(ssfm.power(h["AF"], p.n_f, p.dx, p.dy))
    psh = float(ssfm.power(h["AS"], p.n_sh, p.dx, p.dy))
    fs, fc = field_samples(h["AF"])
    ss, sc = field_samples(h["AS"])
    np.savez_compressed(THERMAL_PASS, eta=h["eta"], p_f=pf, p_sh=psh,
                        q_layers=_layer_sums(h["Q"]), q_total=float(h["Q"].sum()),
                        af_sub=fs, af_centre=fc, ash_sub=ss, ash_centre=sc,
                        stride=FIELD_STRIDE, centre=CENTRE)
    print(f"thermal_pass: eta={h['eta']:.12e} P_F={pf:.12e} P_SH={psh:.12e} "
          f"Q={float(h['Q'].sum()):.6e} ({time.time() - t:.0f} s)")


def thermal_loop2():
    w = W.thermal_loop(nz=100, n_outer=2)
    t = time.time()
    hist = heat.thermal_loop(w, 2, tol=1e-6)
    p = ssfm.params_from_workload(w)
    rec = {}
    for k, h in enumerate(hist):
        rec[f"eta{k}"] = h["eta"]
        rec[f"change{k}"] = h["change"]
        rec[f"sweeps{k}"] = h["sweeps"]
        rec[f"p_f{k}"] = float(ssfm.power(h["AF"], p.n_f, p.dx, p.dy))
        rec[f"p_sh{k}"] = float(ssfm.power(h["AS"], p.n_sh, p.dx, p.dy))
        rec[f"q_layers{k}"] = _layer_sums(h["Q"])
    last = hist[-1]
    dT = last["dT"].numpy()
    fs, fc = field_samples(last["AF"])
    ss, sc = field_samples(last["AS"])
    np.savez_compressed(THERMAL_LOOP2, **rec, dT_sub=dT[::8, ::4, ::4].copy(),
                        dT_max=float(np.abs(dT).max()), q_total=float(last["Q"].sum()),
                        af_sub=fs, af_centre=fc, ash_sub=ss, ash_centre=sc,
                        stride=FIELD_STRIDE, centre=CENTRE)
    print(f"thermal_loop2: " + " ".join(f"{k}={v}" for k, v in rec.items()
                                        if not isinstance(v, np.ndarray))
          + f" ({time.time() - t:.0f} s)")


def _eta_record(w):
    AF, AS, eta = ssfm.run(w)
    p = ssfm.params_from_workload(w)
    return {"eta": float(eta), "p_f": float(ssfm.power(AF, p.n_f, p.dx, p.dy)),
            "p_sh": float(ssfm.power(AS, p.n_sh, p.dx, p.dy))}


def configs():
    out = {"_source": "FP64 CPU oracle, tests/golden/make_golden.py configs",
           "plain": _eta_record(W.plain_focused()),
           "depleted": _eta_record(W.depleted_absorbing()),
           "sweep": {}}
    seen = set()
    for w in W.sweep_instances():
        if w.nx in seen:
            continue
        seen.add(w.nx)
        t = time.time()
        out["sweep"][w.name] = _eta_record(w)
        print(w.name, out["sweep"][w.name], f"{time.time() - t:.0f} s", flush=True)
    json.dump(out, open(CONFIGS, "w"), indent=1)
    print(json.dumps(out, indent=1))


def extensions():
    from oracle import threewave
    out = {"_source": "FP64 CPU oracle, tests/golden/make_golden.py extensions"}
    t = time.time()
    out["eq4"] = _eta_record(W.eq4_case())
    print("eq4", out["eq4"], f"{time.time() - t:.0f} s", flush=True)
    for name, w in (("sfg", W.sfg_case(n=128, nz=1000)), ("dfg", W.dfg_case(n=128, nz=1000))):
        t = time.time()
        _, powers = threewave.run(w)
        out[name] = {"workload": w.name, "powers": [float(p) for p in powers]}
        print(name, out[name], f"{time.time() - t:.0f} s", flush=True)
    json.dump(out, open(EXTENSIONS, "w"), indent=1)


if __name__ == "__main__":
    jobs = {"adjoint_fd": adjoint_fd, "thermal_pass": thermal_pass,
            "thermal_loop2": thermal_loop2, "configs": configs, "extensions": extensions}
    for name in sys.argv[1:] or list(jobs):
        jobs[name]()
