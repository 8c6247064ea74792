"""FP64 CPU oracle of the steady heat solve and the self-consistent loop.

TEST INFRASTRUCTURE ONLY (see ``oracle/ssfm.py``).

* Steady heat equation kappa lap T + q_dot = 0 (Eq. 7), discretised with the
  7-point second-order stencil of Eq. (16) on a node grid [hz][hy][hx] that
  includes the faces.  All six faces are Dirichlet T = T_oven (Eq. 9); the
  unknown is dT = T - T_oven, zero on the faces.
* Solved by red-black successive over-relaxation with the optimal factor
  omega = 2 / (1 + sqrt(1 - rho_J^2)) from the Jacobi spectral radius of the
  anisotropic stencil.  Stops when the largest Jacobi correction over the
  interior is below ``tol`` (kelvin), checked after every full sweep.
* Self-consistent loop (Fig. 2): q_dot = 0 -> T -> Dk(T), lens -> SSFM ->
  q_dot -> ... for a fixed number of outer iterations.
"""
from __future__ import annotations

import math

import torch

from . import ssfm

F64 = torch.float64


def spacings(hx: int, hy: int, hz: int, wx: float, wy: float, L: float):
    return wx / (hx - 1), wy / (hy - 1), L / (hz - 1)


def sor_omega(hx, hy, hz, dx, dy, dz) -> float:
    ax, ay, az = 1.0 / dx ** 2, 1.0 / dy ** 2, 1.0 / dz ** 2
    rho = (ax * math.cos(math.pi / (hx - 1)) + ay * math.cos(math.pi / (hy - 1))
           + az * math.cos(math.pi / (hz - 1))) / (ax + ay + az)
    return 2.0 / (1.0 + math.sqrt(1.0 - rho * rho))


def jacobi_target(T: torch.Tensor, q: torch.Tensor, kappa: float, dx, dy, dz) -> torch.Tensor:
    """Value that solves Eq. (16) at every interior node given its neighbours."""
    ax, ay, az = 1.0 / dx ** 2, 1.0 / dy ** 2, 1.0 / dz ** 2
    s = (ax * (T[1:-1, 1:-1, 2:] + T[1:-1, 1:-1, :-2])
         + ay * (T[1:-1, 2:, 1:-1] + T[1:-1, :-2, 1:-1])
         + az * (T[2:, 1:-1, 1:-1] + T[:-2, 1:-1, 1:-1])
         + q[1:-1, 1:-1, 1:-1] / kappa)
    return s / (2.0 * (ax + ay + az))


def max_correction(T, q, kappa, dx, dy, dz) -> float:
    return float((jacobi_target(T, q, kappa, dx, dy, dz) - T[1:-1, 1:-1, 1:-1]).abs().max())


def sor_solve(q: torch.Tensor, kappa: float, wx: float, wy: float, L: float,
              tol: float = 1e-6, max_sweeps: int = 100000, T0=None, omega=None):
    """Red-black SOR for dT with zero faces.  q is [hz][hy][hx] in W/m^3.
    Returns (dT, sweeps, final max correction)."""
    hz, hy, hx = q.shape
    dx, dy, dz = spacings(hx, hy, hz, wx, wy, L)
    w = sor_omega(hx, hy, hz, dx, dy, dz) if omega is None else omega
    T = torch.zeros_like(q, dtype=F64) if T0 is None else T0.clone().to(F64)
    T[0] = 0; T[-1] = 0; T[:, 0] = 0; T[:, -1] = 0; T[:, :, 0] = 0; T[:, :, -1] = 0
    l, j, i = torch.meshgrid(torch.arange(1, hz - 1), torch.arange(1, hy - 1),
                             torch.arange(1, hx - 1), indexing="ij")
    red = ((l + j + i) % 2) == 0
    black = ~red
    sweeps = 0
    corr = max_correction(T, q, kappa, dx, dy, dz)
    while corr >= tol and sweeps < max_sweeps:
        for mask in (red, black):
            tgt = jacobi_target(T, q, kappa, dx, dy, dz)
            inner = T[1:-1, 1:-1, 1:-1]
            inner[mask] = inner[mask] + w * (tgt[mask] - inner[mask])
        sweeps += 1
        corr = max_correction(T, q, kappa, dx, dy, dz)
    return T, sweeps, corr


def thermal_loop(w, n_outer: int, tol: float = 1e-6, max_sweeps: int = 100000,
                 nsteps=None):
    """Fig. 2 loop.  Returns the list of (eta, dT, max|dT_i - dT_{i-1}|, sweeps)."""
    p = ssfm.params_from_workload(w)
    q = torch.zeros((w.hz, w.hy, w.hx), dtype=F64)
    dT_prev = torch.zeros_like(q)
    history = []
    for it in range(n_outer):
        dT, sweeps, _ = sor_solve(q, w.kappa_th, w.wx, w.wy, w.L, tol, max_sweeps,
                                  T0=dT_prev)
        change = float((dT - dT_prev).abs().max())
        dep = ssfm.HeatDeposit(p, w.hx, w.hy, w.hz, w.wx, w.wy)
        temp = ssfm.TemperatureField(p, dT, w.wx, w.wy, w.t_off)
        AF0 = ssfm.initial_pump(p, w.p1, w.w0, w.z_focus)
        AS0 = torch.zeros_like(AF0)
        AF, AS = ssfm.propagate(p, AF0, AS0, temp, dep)
        eta = float(ssfm.power(AS, p.n_sh, p.dx, p.dy) / w.p1)
        q = dep.qdot_nodes()
        history.append(dict(eta=eta, dT=dT, change=change, sweeps=sweeps, AF=AF, AS=AS,
                            Q=dep.Q.clone()))
        dT_prev = dT
    return history
