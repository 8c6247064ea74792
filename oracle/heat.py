"""FP64 CPU oracle of the steady heat solve and the self-consistent loop.

TEST INFRASTRUCTURE ONLY (see ``oracle/ssfm.py``).

* Steady heat equation kappa lap T + q_dot = 0 (Eq. 7), discretised with the
  7-point second-order stencil of Eq. (16) on a node grid [hz][hy][hx] that
  includes the faces.  The unknown is dT = T - T_oven.
* Each of the six faces is either held at the oven temperature, dT = 0
  (Dirichlet, Eq. 9), or cooled by convection, -kappa dT/dn = h (T - T_inf)
  (Eq. 10).  Sec. 3.2 computes the face nodes "using the boundary
  conditions"; here a convective face node is an unknown whose stencil uses
  a ghost node beyond the face, eliminated by the central difference of
  Eq. (10): T_ghost = T_inner - 2 d (h / kappa) (T_face - T_inf), d the
  spacing normal to the face.  A node on a Dirichlet face is fixed even
  where it also lies on a convective face.  Default: all faces Dirichlet.
* Solved by red-black successive over-relaxation with the factor
  omega = 2 / (1 + sqrt(1 - rho_J^2)) from the Jacobi spectral radius of the
  all-Dirichlet stencil (optimal there; any omega in (0, 2) converges).
  Stops when the largest Jacobi correction over the unknown nodes is below
  ``tol`` (kelvin), checked after every full sweep.
* Self-consistent loop (Fig. 2): q_dot = 0 -> T -> Dk(T), lens -> SSFM ->
  q_dot -> ... for a fixed number of outer iterations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import ssfm

F64 = torch.float64

FACES = ("x-", "x+", "y-", "y+", "z-", "z+")


@dataclass(frozen=True)
class HeatBC:
    """Boundary condition of each face of the crystal, in the order of FACES:
    "D" held at T_oven (Eq. 9) or "C" convective (Eq. 10) with that face's
    heat transfer coefficient h (W/(m^2 K); one number for all faces, or six)
    and the ambient temperature T_inf = T_oven + t_inf."""
    faces: tuple = ("D",) * 6
    h: object = 0.0
    t_inf: float = 0.0

    def convective(self, k: int) -> bool:
        return self.faces[k] == "C"

    def h_of(self, k: int) -> float:
        return float(self.h[k]) if isinstance(self.h, (tuple, list)) else float(self.h)


DIRICHLET = HeatBC()


def bc_of(w) -> HeatBC:
    """The heat boundary condition of a workload (all Dirichlet by default)."""
    h = getattr(w, "h_conv", 0.0)
    return HeatBC(tuple(getattr(w, "heat_faces", ("D",) * 6)),
                  tuple(float(v) for v in h) if isinstance(h, (tuple, list)) else float(h),
                  float(getattr(w, "t_inf", 0.0)))


def spacings(hx: int, hy: int, hz: int, wx: float, wy: float, L: float):
    return wx / (hx - 1), wy / (hy - 1), L / (hz - 1)


def sor_omega(hx, hy, hz, dx, dy, dz) -> float:
    ax, ay, az = 1.0 / dx ** 2, 1.0 / dy ** 2, 1.0 / dz ** 2
    rho = (ax * math.cos(math.pi / (hx - 1)) + ay * math.cos(math.pi / (hy - 1))
           + az * math.cos(math.pi / (hz - 1))) / (ax + ay + az)
    return 2.0 / (1.0 + math.sqrt(1.0 - rho * rho))


def _face_terms(shape, dx, dy, dz, kappa, bc: HeatBC):
    """Diagonal and right-hand-side additions of the ghost-node convective
    faces: 2 a_d d (h / kappa) on the diagonal and that times t_inf on the
    right-hand side of every node on a convective face (a_d = 1 / d^2)."""
    hz, hy, hx = shape
    diag = torch.zeros(shape, dtype=F64)
    for k, (axis, d) in enumerate(((2, dx), (2, dx), (1, dy), (1, dy), (0, dz), (0, dz))):
        if not bc.convective(k):
            continue
        layer = [slice(None)] * 3
        layer[axis] = 0 if k % 2 == 0 else shape[axis] - 1
        diag[tuple(layer)] += 2.0 * (1.0 / d ** 2) * d * bc.h_of(k) / kappa
    return diag, diag * bc.t_inf


def unknown_mask(shape, bc: HeatBC) -> torch.Tensor:
    """Nodes whose temperature is solved for: all but those on a Dirichlet face."""
    m = torch.ones(shape, dtype=torch.bool)
    for k, axis in enumerate((2, 2, 1, 1, 0, 0)):
        if not bc.convective(k):
            layer = [slice(None)] * 3
            layer[axis] = 0 if k % 2 == 0 else shape[axis] - 1
            m[tuple(layer)] = False
    return m


def _neighbour_sum(T: torch.Tensor, axis: int) -> torch.Tensor:
    """T[i-1] + T[i+1] along `axis`; at the two end layers the ghost node's
    T_inner part doubles the inner neighbour (2 T[1], 2 T[n-2])."""
    n = T.shape[axis]
    S = torch.zeros_like(T)
    sl = lambda a, b: tuple(slice(a, b) if k == axis else slice(None) for k in range(3))  # noqa: E731
    S[sl(1, n - 1)] = T[sl(2, n)] + T[sl(0, n - 2)]
    S[sl(0, 1)] = 2.0 * T[sl(1, 2)]
    S[sl(n - 1, n)] = 2.0 * T[sl(n - 2, n - 1)]
    return S


def jacobi_target(T: torch.Tensor, q: torch.Tensor, kappa: float, dx, dy, dz,
                  bc: HeatBC = DIRICHLET) -> torch.Tensor:
    """Value that solves the node's equation of Eq. (16) given its neighbours,
    at every node of the grid (meaningful on the unknown nodes only)."""
    ax, ay, az = 1.0 / dx ** 2, 1.0 / dy ** 2, 1.0 / dz ** 2
    s = (ax * _neighbour_sum(T, 2) + ay * _neighbour_sum(T, 1) + az * _neighbour_sum(T, 0)
         + q / kappa)
    diag = 2.0 * (ax + ay + az)
    if any(bc.convective(k) for k in range(6)):
        d_add, r_add = _face_terms(tuple(T.shape), dx, dy, dz, kappa, bc)
        return (s + r_add) / (diag + d_add)
    return s / diag


def max_correction(T, q, kappa, dx, dy, dz, bc: HeatBC = DIRICHLET) -> float:
    m = unknown_mask(tuple(T.shape), bc)
    return float((jacobi_target(T, q, kappa, dx, dy, dz, bc) - T)[m].abs().max())


def sor_solve(q: torch.Tensor, kappa: float, wx: float, wy: float, L: float,
              tol: float = 1e-6, max_sweeps: int = 100000, T0=None, omega=None,
              bc: HeatBC = DIRICHLET):
    """Red-black SOR for dT (zero on Dirichlet faces).  q is [hz][hy][hx] in
    W/m^3.  Returns (dT, sweeps, final max correction)."""
    hz, hy, hx = q.shape
    dx, dy, dz = spacings(hx, hy, hz, wx, wy, L)
    w = sor_omega(hx, hy, hz, dx, dy, dz) if omega is None else omega
    T = torch.zeros_like(q, dtype=F64) if T0 is None else T0.clone().to(F64)
    unknown = unknown_mask(tuple(q.shape), bc)
    T[~unknown] = 0
    l, j, i = torch.meshgrid(torch.arange(hz), torch.arange(hy), torch.arange(hx), indexing="ij")
    red = (((l + j + i) % 2) == 0) & unknown
    black = (((l + j + i) % 2) == 1) & unknown
    sweeps = 0
    corr = max_correction(T, q, kappa, dx, dy, dz, bc)
    while corr >= tol and sweeps < max_sweeps:
        for mask in (red, black):
            tgt = jacobi_target(T, q, kappa, dx, dy, dz, bc)
            T[mask] = T[mask] + w * (tgt[mask] - T[mask])
        sweeps += 1
        corr = max_correction(T, q, kappa, dx, dy, dz, bc)
    return T, sweeps, corr


def thermal_loop(w, n_outer: int, tol: float = 1e-6, max_sweeps: int = 100000,
                 nsteps=None):
    """Fig. 2 loop.  Returns the list of (eta, dT, max|dT_i - dT_{i-1}|, sweeps)."""
    p = ssfm.params_from_workload(w)
    bc = bc_of(w)
    q = torch.zeros((w.hz, w.hy, w.hx), dtype=F64)
    dT_prev = torch.zeros_like(q)
    history = []
    for it in range(n_outer):
        dT, sweeps, _ = sor_solve(q, w.kappa_th, w.wx, w.wy, w.L, tol, max_sweeps,
                                  T0=dT_prev, bc=bc)
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
