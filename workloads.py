"""Seeded synthetic inputs for the focused-Gaussian-beam SHG workloads.

This module only *describes* inputs: crystal and beam parameters, grid sizes,
the transverse window and the seeded temperature maps.  It holds none of the
split-step arithmetic; the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2410_04994_gb300``) each implement that on their own and both read
their inputs from here.

Workload recipe (paper, Sec. 2 and Sec. 5; all SI units):

* SHG 1064 nm -> 532 nm in a 30 mm QPM crystal, n_F = 2.14, n_SH = 2.18,
  d_eff = 10 pm/V, QPM period chosen so that the cold mismatch dk0 = 0.
* The pump is a TEM00 beam (Eq. 5/6) focused at the crystal centre with
  focusing parameter xi = L / (2 z_R), z_R = w0^2 k_F / 2, so that
  w0 = sqrt(L / (xi k_F)).  xi = 2.84 gives w0 = 28.9 um, the 29 um quoted in
  the paper's Example 1 and Example 2 (Sec. 5.1, 5.2).
* The transverse window is square with side 10 w(0), w(z) the Gaussian beam
  radius w0 sqrt(1 + ((z - f)/z_R)^2) at the crystal entrance.
* Temperature maps (node-centred, spanning the window in x, y and [0, L] in z)
  are 2 K exp(-2 r^2 / w(z)^2) plus i.i.d. N(0, 0.01 K) noise per node, drawn
  from ``numpy.random.default_rng(seed)``.
* Losses of the absorbing workloads: alpha_F = 0.002 /cm, alpha_SH = 0.02 /cm,
  beta_SH = 0.1 cm/GW (= 1e-12 m/W), beta_F = 0; dDk/dT = -0.6 /(m K),
  dn/dT = 1e-5 /K.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

LAMBDA_F = 1.064e-6
N_F = 2.14
N_SH = 2.18
D_EFF = 10e-12
L_CRYSTAL = 0.03
ALPHA_F = 0.2        # 0.002 /cm
ALPHA_SH = 2.0       # 0.02 /cm
BETA_SH = 1e-12      # 0.1 cm/GW
DDK_DT = -0.6
DN_DT = 1e-5
KAPPA_TH = 8.4
CRYSTAL_WX = 2e-3
CRYSTAL_WY = 1e-3


def k_pump(lambda_f: float = LAMBDA_F, n_f: float = N_F) -> float:
    """Pump wavenumber inside the crystal, k_F = 2 pi n_F / lambda_F."""
    return 2.0 * math.pi * n_f / lambda_f


def waist_for_xi(xi: float, L: float = L_CRYSTAL, lambda_f: float = LAMBDA_F,
                 n_f: float = N_F) -> float:
    """Waist w0 that gives focusing parameter xi = L/(2 z_R), z_R = w0^2 k_F/2."""
    return math.sqrt(L / (xi * k_pump(lambda_f, n_f)))


def beam_radius(z: float, w0: float, z_focus: float, lambda_f: float = LAMBDA_F,
                n_f: float = N_F) -> float:
    z_r = w0 * w0 * k_pump(lambda_f, n_f) / 2.0
    return w0 * math.sqrt(1.0 + ((z - z_focus) / z_r) ** 2)


def window_for_beam(w0: float, z_focus: float, lambda_f: float = LAMBDA_F,
                    n_f: float = N_F) -> float:
    """Square window side: 10 times the beam radius at the crystal entrance."""
    return 10.0 * beam_radius(0.0, w0, z_focus, lambda_f, n_f)


@dataclass(frozen=True)
class Qpm:
    """Inputs of the phase-matching model of Eq. (4): oven temperature (deg C),
    grating period at 25 C (m), its thermal-expansion coefficients (the
    paper's MgO:sPPLT values by default) and polynomial coefficients of the
    refractive indices in (T - 25 C), n_j(T) = sum_k c_k (T - 25)^k (the
    paper gives no index data, so these are the caller's)."""
    t_oven: float
    lambda25: float
    a_lambda: float = 2.2e-6
    b_lambda: float = -5.9e-9
    n_f_t: tuple = (0.0,)
    n_sh_t: tuple = (0.0,)


@dataclass
class Workload:
    """One SSFM instance: grid, crystal, beam and an optional temperature map."""
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    # crystal
    L: float = L_CRYSTAL
    lambda_f: float = LAMBDA_F
    n_f: float = N_F
    n_sh: float = N_SH
    d_eff: float = D_EFF
    alpha_f: float = 0.0
    alpha_sh: float = 0.0
    beta_f: float = 0.0
    beta_sh: float = 0.0
    dk0: float = 0.0
    ddk_dT: float = 0.0
    dn_dT: float = 0.0
    kappa_th: float = KAPPA_TH
    wx: float = CRYSTAL_WX
    wy: float = CRYSTAL_WY
    walkoff_f: float = 0.0      # walk-off angles (rad) toward +x
    walkoff_sh: float = 0.0
    # beams
    p1: float = 1.0
    w0: float = 30e-6
    z_focus: float = L_CRYSTAL / 2
    t_off: float = 0.0
    undepleted: bool = False
    # precision of the fast path ("f32" or "f64")
    precision: str = "f32"
    # temperature map [tz][ty][tx] (float32) and its transverse extent
    dT: Optional[np.ndarray] = None
    t_lx: float = 0.0
    t_ly: float = 0.0
    # heat grid (nodes incl. faces) for the self-consistent loop; 0 = none
    hx: int = 0
    hy: int = 0
    hz: int = 0
    n_outer: int = 0
    # heat boundary of each face x-, x+, y-, y+, z-, z+: "D" held at the oven
    # temperature (Eq. 9) or "C" convective (Eq. 10) with coefficient h_conv
    # (W/(m^2 K); one value or six) toward the ambient T_oven + t_inf (K)
    heat_faces: tuple = ("D",) * 6
    h_conv: object = 0.0
    t_inf: float = 0.0
    # phase-matching model of Eq. (4), or None for dk0 + dDk/dT dT
    qpm: Optional[Qpm] = None

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    @property
    def point_steps(self) -> int:
        return self.nx * self.ny * self.nz


def gaussian_dT_map(tx: int, ty: int, tz: int, t_lx: float, t_ly: float, L: float,
                    w0: float, z_focus: float, rng: np.random.Generator,
                    amp: float = 2.0, sigma: float = 0.01) -> np.ndarray:
    """amp * exp(-2 r^2 / w(z)^2) + N(0, sigma) on node-centred points [tz][ty][tx]."""
    X = -t_lx / 2 + np.arange(tx) * (t_lx / (tx - 1))
    Y = -t_ly / 2 + np.arange(ty) * (t_ly / (ty - 1))
    Z = np.arange(tz) * (L / (tz - 1))
    z_r = w0 * w0 * k_pump() / 2.0
    wz = w0 * np.sqrt(1.0 + ((Z - z_focus) / z_r) ** 2)
    r2 = X[None, None, :] ** 2 + Y[None, :, None] ** 2
    base = amp * np.exp(-2.0 * r2 / (wz[:, None, None] ** 2))
    noise = rng.normal(0.0, sigma, size=(tz, ty, tx))
    return (base + noise).astype(np.float32)


def _lossy(w: Workload) -> Workload:
    return w.with_(alpha_f=ALPHA_F, alpha_sh=ALPHA_SH, beta_sh=BETA_SH,
                   ddk_dT=DDK_DT, dn_dT=DN_DT)


def plain_focused(n: int = 32, nz: int = 100, xi: float = 2.84, p1: float = 10.0,
                  undepleted: bool = False, precision: str = "f64") -> Workload:
    """Plain SSFM, single instance: no losses, uniform temperature, dk0 = 0."""
    w0 = waist_for_xi(xi)
    lw = window_for_beam(w0, L_CRYSTAL / 2)
    return Workload(name=f"plain_{n}x{n}_nz{nz}", nx=n, ny=n, nz=nz, lx=lw, ly=lw,
                    p1=p1, w0=w0, z_focus=L_CRYSTAL / 2, undepleted=undepleted,
                    precision=precision)


def depleted_absorbing(n: int = 128, nz: int = 1000, xi: float = 1.0, p1: float = 50.0,
                       seed: int = 0, tgrid=(64, 64, 128)) -> Workload:
    """Depleted pump with alpha, beta and a seeded temperature map (FP32 fields)."""
    w0 = waist_for_xi(xi)
    lw = window_for_beam(w0, L_CRYSTAL / 2)
    rng = np.random.default_rng(seed)
    tx, ty, tz = tgrid
    dT = gaussian_dT_map(tx, ty, tz, lw, lw, L_CRYSTAL, w0, L_CRYSTAL / 2, rng)
    return _lossy(Workload(name=f"depleted_{n}x{n}_nz{nz}", nx=n, ny=n, nz=nz, lx=lw,
                           ly=lw, p1=p1, w0=w0, z_focus=L_CRYSTAL / 2, dT=dT,
                           t_lx=lw, t_ly=lw))


SWEEP_GROUPS = ((64, 128), (128, 192), (256, 64))


def sweep_instances(nz: int = 2000, seed: int = 1, groups=SWEEP_GROUPS,
                    tgrid=(64, 64, 128), with_maps: bool = True) -> List[Workload]:
    """Batched focusing/power/oven sweep on mixed grids.

    Within each size group xi = 0.3 * 20**(i/(n-1)) (log-spaced over [0.3, 6]).
    P1 ~ U[5, 60] W and the oven offset ~ U[-1, 1] K are drawn first from one
    seeded stream over all instances in order, then one temperature map per
    instance from the same stream.
    """
    n_total = sum(c for _, c in groups)
    rng = np.random.default_rng(seed)
    p1s = rng.uniform(5.0, 60.0, size=n_total)
    toffs = rng.uniform(-1.0, 1.0, size=n_total)
    out = []
    idx = 0
    tx, ty, tz = tgrid
    for n, count in groups:
        for i in range(count):
            xi = 0.3 * 20.0 ** (i / (count - 1)) if count > 1 else 1.0
            w0 = waist_for_xi(xi)
            lw = window_for_beam(w0, L_CRYSTAL / 2)
            dT = None
            if with_maps:
                dT = gaussian_dT_map(tx, ty, tz, lw, lw, L_CRYSTAL, w0, L_CRYSTAL / 2, rng)
            out.append(_lossy(Workload(name=f"sweep{idx}_{n}x{n}", nx=n, ny=n, nz=nz,
                                       lx=lw, ly=lw, p1=float(p1s[idx]), w0=w0,
                                       z_focus=L_CRYSTAL / 2, t_off=float(toffs[idx]),
                                       dT=dT, t_lx=lw, t_ly=lw)))
            idx += 1
    return out


def adjoint_case(n: int = 256, nz: int = 2000, xi: float = 2.84, p1: float = 30.0,
                 seed: int = 0, tgrid=(64, 64, 128)) -> Workload:
    """Gradient workload: losses of the absorbing case, seeded map on a coarse grid."""
    w0 = waist_for_xi(xi)
    lw = window_for_beam(w0, L_CRYSTAL / 2)
    rng = np.random.default_rng(seed)
    tx, ty, tz = tgrid
    dT = gaussian_dT_map(tx, ty, tz, lw, lw, L_CRYSTAL, w0, L_CRYSTAL / 2, rng)
    return _lossy(Workload(name=f"adjoint_{n}x{n}_nz{nz}", nx=n, ny=n, nz=nz, lx=lw,
                           ly=lw, p1=p1, w0=w0, z_focus=L_CRYSTAL / 2, dT=dT,
                           t_lx=lw, t_ly=lw))


def thermal_loop(n: int = 1024, nz: int = 8000, xi: float = 2.84, p1: float = 100.0,
                 heat=(128, 128, 256), n_outer: int = 6) -> Workload:
    """Self-consistent thermal loop in a 2 x 1 x 30 mm crystal, Dirichlet oven faces."""
    w0 = waist_for_xi(xi)
    lw = window_for_beam(w0, L_CRYSTAL / 2)
    hx, hy, hz = heat
    return _lossy(Workload(name=f"thermal_{n}x{n}_nz{nz}", nx=n, ny=n, nz=nz, lx=lw,
                           ly=lw, p1=p1, w0=w0, z_focus=L_CRYSTAL / 2, hx=hx, hy=hy,
                           hz=hz, n_outer=n_outer, t_lx=CRYSTAL_WX, t_ly=CRYSTAL_WY))


@dataclass
class ThreeWave:
    """One three-wave mixing instance (sum- or difference-frequency
    generation, omega_3 = omega_1 + omega_2): grid, crystal, the three input
    beams (power 0: no input at that wave) and an optional temperature map."""
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lambda1: float
    lambda2: float
    n1: float
    n2: float
    n3: float
    L: float = L_CRYSTAL
    d_eff: float = D_EFF
    alpha: tuple = (0.0, 0.0, 0.0)
    beta: tuple = (0.0, 0.0, 0.0)
    dk0: float = 0.0
    ddk_dT: float = 0.0
    dn_dT: float = 0.0
    walkoff: tuple = (0.0, 0.0, 0.0)
    p: tuple = (1.0, 1.0, 0.0)
    w0: tuple = (30e-6, 30e-6, 30e-6)
    z_focus: tuple = (L_CRYSTAL / 2,) * 3
    t_off: float = 0.0
    undepleted: bool = False
    precision: str = "f32"
    dT: Optional[np.ndarray] = None
    t_lx: float = 0.0
    t_ly: float = 0.0

    def with_(self, **kw) -> "ThreeWave":
        return replace(self, **kw)


def sfg_case(n: int = 64, nz: int = 200, p=(20.0, 30.0, 0.0), xi: float = 1.5,
             seed: int = 0, tgrid=(16, 16, 32), with_map: bool = True) -> ThreeWave:
    """Sum-frequency generation 1550 nm + 1064 nm -> 631 nm in the 30 mm QPM
    crystal: both inputs focused at the centre with the same confocal
    parameter (xi for the 1550 nm beam), the losses and temperature
    coefficients of the absorbing SHG workloads, a seeded map."""
    l1, l2 = 1.55e-6, LAMBDA_F
    n1, n2, n3 = 2.13, N_F, 2.165
    k1 = 2 * math.pi * n1 / l1
    k2 = 2 * math.pi * n2 / l2
    zr = L_CRYSTAL / (2 * xi)
    w01, w02 = math.sqrt(2 * zr / k1), math.sqrt(2 * zr / k2)
    lw = 10.0 * max(w01, w02) * math.sqrt(1 + xi * xi)
    dT = None
    if with_map:
        rng = np.random.default_rng(seed)
        tx, ty, tz = tgrid
        dT = gaussian_dT_map(tx, ty, tz, lw, lw, L_CRYSTAL, w02, L_CRYSTAL / 2, rng)
    return ThreeWave(name=f"sfg_{n}x{n}_nz{nz}", nx=n, ny=n, nz=nz, lx=lw, ly=lw, lambda1=l1,
                     lambda2=l2, n1=n1, n2=n2, n3=n3, alpha=(0.1, ALPHA_F, 1.0),
                     beta=(0.0, 0.0, BETA_SH), ddk_dT=DDK_DT, dn_dT=DN_DT, p=tuple(p),
                     w0=(w01, w02, w02), dT=dT, t_lx=lw, t_ly=lw)


def dfg_case(n: int = 64, nz: int = 200, **kw) -> ThreeWave:
    """Difference-frequency generation 631 nm - 1064 nm -> 1550 nm: the same
    crystal with the pump at omega_3 and a seed at omega_2; wave 1 grows."""
    w = sfg_case(n=n, nz=nz, p=(0.0, 2.0, 40.0), **kw)
    return w.with_(name=f"dfg_{n}x{n}_nz{nz}")


# Inputs of the Eq. (4) phase model for the measured extension workload:
# synthetic index polynomials in (T - 25 C) (the paper gives no index data)
# and the paper's grating expansion; EQ4_LAMBDA25 is the grating period at
# 25 C that phase-matches these polynomials at 60 C (evaluated once, stated
# here as a number).
EQ4_N_F = (2.14, 2e-6, 3e-9, -1e-11)
EQ4_N_SH = (2.18, 4e-6, -4e-9, 2e-11)
EQ4_LAMBDA25 = 1.3278254691754094e-05


def eq4_case(n: int = 128, nz: int = 1000, t_oven: float = 58.0, t_off: float = 1.5) -> Workload:
    """The depleted workload (seed-0 map) with the Eq. (4) phase model: oven at
    58 C plus a 1.5 K offset, 0.5 K from the constructed phase-matching point."""
    w = depleted_absorbing(n=n, nz=nz)
    q = Qpm(t_oven=t_oven, lambda25=EQ4_LAMBDA25, n_f_t=EQ4_N_F, n_sh_t=EQ4_N_SH)
    return w.with_(qpm=q, t_off=t_off, name=f"eq4_{n}x{n}_nz{nz}")


# Oven arrangements of Sec. 4.2 (the crystal surrounded by the oven, or an
# oven under one face): the faces held at the oven temperature, the rest
# cooled by convection.
OVENS = {
    "all": ("D",) * 6,
    "surrounded": ("D", "D", "D", "D", "C", "C"),   # side faces in the oven, end facets in air
    "bottom": ("C", "C", "D", "C", "C", "C"),       # one oven under the y- face
}


def with_oven(w: Workload, oven: str, h_conv=10.0, t_inf: float = 0.0) -> Workload:
    """The workload with one of the paper's oven arrangements (h_conv and the
    ambient temperature are not given in the paper: free convection in air is
    of order 10 W/(m^2 K))."""
    return w.with_(heat_faces=OVENS[oven], h_conv=h_conv, t_inf=t_inf)


# The five workloads at full size, in the order they are quoted.
def full_size(name: str):
    if name == "plain":
        return plain_focused()
    if name == "depleted":
        return depleted_absorbing()
    if name == "sweep":
        return sweep_instances()
    if name == "adjoint":
        return adjoint_case()
    if name == "thermal":
        return thermal_loop()
    raise KeyError(name)
