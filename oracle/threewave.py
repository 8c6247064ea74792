"""FP64 CPU oracle of three-wave mixing: sum- and difference-frequency generation.

TEST INFRASTRUCTURE ONLY (see ``oracle/ssfm.py``).  The paper solves second
harmonic generation and names other three-wave processes as the natural
extension of its coupled-wave model (Sec. 6).  This module is that extension:
the same discrete map as ``ssfm.py`` (symmetric split step of Eqs. (14)-(15),
one RK4 step per half step, K-space diffraction and absorption of App. A)
with three fields at omega_3 = omega_1 + omega_2.

Coupled-wave equations (the field convention of ``ssfm.py``: E = Re[A e^{i(kz-wt)}],
I = eps0 c n |A|^2 / 2; the SHG equations are the degenerate case):
    dA1/dz = i k1 A3 conj(A2) e^{-i phi} - (1/2) beta1 I1 A1 + i psi1 A1
    dA2/dz = i k2 A3 conj(A1) e^{-i phi} - (1/2) beta2 I2 A2 + i psi2 A2
    dA3/dz = i k3 A1 A2 e^{+i phi}       - (1/2) beta3 I3 A3 + i psi3 A3
with k_j = 2 pi d_eff / (n_j lambda_j) (the SHG reading 2 gives k_SH =
2 pi d / (n_SH lambda_F) = pi d / (n_SH lambda_SH), half of this, because the
degenerate polarisation carries a factor 1/2), so that n_j k_j / omega_j = d/c
for every wave (Manley-Rowe).  phi = (dk0 + g T_off) z + g C(x,y,z) and
psi_j = (2 pi / lambda_j)(dn/dT)(dT + T_off) as in ``ssfm.py``.  Linear step per
wave: exp(-i K^2 dz / (2 k_j)) exp(-alpha_j dz / 2) exp(-i tan(rho_j) Kx dz).

Each wave starts as the focused Gaussian of Eq. (5) with its own power, waist
and focus (power 0: a zero field), normalised to its discrete power.
"Undepleted" drops the coupling terms of waves 1 and 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import torch

from . import fft as dft
from . import ssfm

F64 = torch.float64
C128 = torch.complex128


@dataclass
class Params3:
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    L: float
    lambda1: float
    lambda2: float
    n1: float
    n2: float
    n3: float
    d_eff: float
    alpha: tuple = (0.0, 0.0, 0.0)
    beta: tuple = (0.0, 0.0, 0.0)
    dk0: float = 0.0
    ddk_dT: float = 0.0
    dn_dT: float = 0.0
    walkoff: tuple = (0.0, 0.0, 0.0)
    undepleted: bool = False
    qpm: Optional[object] = None   # TemperatureField reads it; the linearised phase only here

    @property
    def lambda3(self) -> float:
        return 1.0 / (1.0 / self.lambda1 + 1.0 / self.lambda2)

    @property
    def lambdas(self):
        return (self.lambda1, self.lambda2, self.lambda3)

    @property
    def ns(self):
        return (self.n1, self.n2, self.n3)

    @property
    def k(self):
        return tuple(2.0 * math.pi * n / lam for n, lam in zip(self.ns, self.lambdas))

    @property
    def kappa(self):
        return tuple(2.0 * math.pi * self.d_eff / (n * lam) for n, lam in zip(self.ns, self.lambdas))

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    @property
    def dz(self) -> float:
        return self.L / self.nz


def params_from(w) -> Params3:
    return Params3(nx=w.nx, ny=w.ny, nz=w.nz, lx=w.lx, ly=w.ly, L=w.L, lambda1=w.lambda1,
                   lambda2=w.lambda2, n1=w.n1, n2=w.n2, n3=w.n3, d_eff=w.d_eff,
                   alpha=tuple(w.alpha), beta=tuple(w.beta), dk0=w.dk0, ddk_dT=w.ddk_dT,
                   dn_dT=w.dn_dT, walkoff=tuple(w.walkoff), undepleted=bool(w.undepleted))


def gaussian(p: Params3, j: int, power, w0, z_focus) -> torch.Tensor:
    """Eq. (5) at z = 0 for wave j (its own wavenumber), at discrete power `power`."""
    if float(power) == 0.0:
        return torch.zeros((p.ny, p.nx), dtype=C128)
    w0 = ssfm._t(w0)
    z_focus = ssfm._t(z_focus)
    x = ssfm.axis(p.nx, p.lx)
    y = ssfm.axis(p.ny, p.ly)
    z_r = w0 * w0 * p.k[j] / 2.0
    q = torch.complex(torch.ones((), dtype=F64), (0.0 - z_focus) / z_r)
    r2 = (x[None, :] ** 2 + y[:, None] ** 2).to(C128)
    g = torch.exp(-r2 / (w0 * w0 * q)) / q
    return torch.sqrt(ssfm._t(power) / ssfm.power(g, p.ns[j], p.dx, p.dy)) * g


class Nonlinear3:
    def __init__(self, p: Params3, temp: ssfm.TemperatureField):
        self.p = p
        self.temp = temp
        self.c = tuple(0.5 * ssfm.EPS0 * ssfm.C_LIGHT * n for n in p.ns)
        self.k0 = tuple(2.0 * math.pi / lam for lam in p.lambdas)

    def coefficients(self, z: float):
        p = self.p
        d, c = self.temp.at(z)
        t_off = self.temp.t_off
        phi = (p.dk0 + p.ddk_dT * t_off) * z + p.ddk_dT * c
        psi = tuple(k0 * p.dn_dT * (d + t_off) for k0 in self.k0)
        return phi, psi

    def rhs(self, A, coef):
        p = self.p
        phi, psi = coef
        e = torch.exp(1j * phi)
        k1, k2, k3 = p.kappa
        out = []
        for j in range(3):
            I = self.c[j] * (A[j].real ** 2 + A[j].imag ** 2)
            out.append(-0.5 * p.beta[j] * I * A[j] + 1j * psi[j] * A[j])
        if not p.undepleted:
            out[0] = out[0] + 1j * k1 * A[2] * torch.conj(A[1]) * torch.conj(e)
            out[1] = out[1] + 1j * k2 * A[2] * torch.conj(A[0]) * torch.conj(e)
        out[2] = out[2] + 1j * k3 * A[0] * A[1] * e
        return out

    def rk4(self, A, z0: float, h: float):
        c0 = self.coefficients(z0)
        cm = self.coefficients(z0 + 0.5 * h)
        c1 = self.coefficients(z0 + h)
        k1 = self.rhs(A, c0)
        k2 = self.rhs([a + 0.5 * h * k for a, k in zip(A, k1)], cm)
        k3 = self.rhs([a + 0.5 * h * k for a, k in zip(A, k2)], cm)
        k4 = self.rhs([a + h * k for a, k in zip(A, k3)], c1)
        return [a + (h / 6.0) * (q1 + 2 * q2 + 2 * q3 + q4)
                for a, q1, q2, q3, q4 in zip(A, k1, k2, k3, k4)]


class Linear3:
    def __init__(self, p: Params3):
        Kx = ssfm.wavenumbers(p.nx, p.lx)
        Ky = ssfm.wavenumbers(p.ny, p.ly)
        K2 = Kx[None, :] ** 2 + Ky[:, None] ** 2
        dz = p.dz
        self.P = []
        for j in range(3):
            f = torch.exp(-1j * K2 * dz / (2.0 * p.k[j])) * math.exp(-0.5 * p.alpha[j] * dz)
            self.P.append(f * torch.exp(-1j * math.tan(p.walkoff[j]) * Kx[None, :] * dz))

    def __call__(self, A):
        return [dft.ifft2(P * dft.fft2(a)) for P, a in zip(self.P, A)]


def propagate(p: Params3, A, temp: ssfm.TemperatureField, nsteps: Optional[int] = None):
    """Symmetric split step (Eq. 15) for the three fields."""
    nl = Nonlinear3(p, temp)
    lin = Linear3(p)
    dz = p.dz
    h = 0.5 * dz
    for s in range(p.nz if nsteps is None else nsteps):
        z = s * dz
        A = nl.rk4(A, z, h)
        A = lin(A)
        A = nl.rk4(A, z + h, h)
    return A


def initial_fields(p: Params3, w):
    return [gaussian(p, j, w.p[j], w.w0[j], w.z_focus[j]) for j in range(3)]


def run(w, A0=None):
    """(A1, A2, A3) at z = L and their discrete powers (W)."""
    p = params_from(w)
    dT = None if w.dT is None else torch.as_tensor(w.dT)
    temp = ssfm.TemperatureField(p, dT, w.t_lx, w.t_ly, w.t_off)
    A = initial_fields(p, w) if A0 is None else [a.to(C128) for a in A0]
    A = propagate(p, A, temp)
    powers = [float(ssfm.power(a, n, p.dx, p.dy)) for a, n in zip(A, p.ns)]
    return A, powers
