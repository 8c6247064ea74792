"""FP64 CPU oracle of the split-step Fourier SHG propagation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline and reference legs of ``bench.py`` may import this package.  It shares no code
with the CUDA path: plain PyTorch CPU ops in float64 / complex128 and the
oracle's own radix-2 DFT (``oracle/fft.c``, no library FFT), with no blocking,
fusion or reordering.

The discrete map it computes (all SI units):

* Coupled-wave equations, Eqs. (1)-(2), in the operator form of Eq. (11):
  the nonlinear operator N is applied pointwise, the linear operator L
  (diffraction + linear absorption, and the walk-off term of Sec. 6 / App. B
  when its angles are non-zero) in K-space, App. A Eqs. (A.1)-(A.5).
* Symmetric split step, Eqs. (14)-(15): every z-step of length dz is
  N(dz/2) -> L(dz) -> N(dz/2).  Each N(dz/2) is one classical RK4 step of
  size h = dz/2 (Sec. 3.1 names RK4 for the nonlinear part); the first half
  covers [z, z+dz/2], the second [z+dz/2, z+dz].
* Pump at the crystal entrance: Eq. (5) at z = 0 (Eq. (6) when f = L/2),
  normalised so that the discrete power (1/2) eps0 c n_F sum |A_F|^2 dx dy
  equals P1.  The SH starts at zero.
* Efficiency eta = P_SH(L) / P_F(0), Eq. (17), with the discrete powers.

Readings of the paper (where it is silent, garbled or inconsistent):

1. Diffraction sign: the Gaussian beam of Eq. (5) solves
   dA/dz = +(i/2k) lap_perp A, so the K-space factor is
   exp(-i (Kx^2+Ky^2) dz / (2 k_j)) with K = 2 pi q (App. A's sign flipped).
2. SH coupling: kappa_SH = 2 pi d_eff / (n_SH lambda_F), so that
   n_F kappa_F = n_SH kappa_SH (Manley-Rowe) with I = eps0 c n |A|^2 / 2.
3. TPA: -(1/2) beta_j I_j A_j with I_j = eps0 c n_j |A_j|^2 / 2.
4. Phase: e^{-i phi} on the pump equation, e^{+i phi} on the SH equation,
   phi = int_0^z Dk dz' (Eq. 3), taken literally.
5. Linear absorption alpha_j sits in L: exp(-alpha_j dz/2) on the amplitude
   inside the K-space multiply (Eq. 11).
6. Thermal lens: an extra i psi_j A_j term in N, psi_j = (2 pi / lambda_j)
   (dn/dT) dT_eff, the same dn/dT for both waves.
7. Dk(T) is linearised: Dk = dk0 + (dDk/dT) dT_eff, dT_eff = dT + T_off.
   phi = (dk0 + g T_off) z + g C(x,y,z), g = dDk/dT, C the trapezoid
   cumulative integral of dT along z on the temperature-grid nodes,
   trilinearly interpolated (clamped to the edge outside the grid).
8. Undepleted pump (Sec. 5.1): only the coupling term of the pump equation
   is removed; beta_F and psi_F stay.
9. Heat source samples (Eq. 8) are taken at z_s = s dz, s = 0..nz, with
   trapezoid weights in z, and box-summed into the nearest heat node.
10. Dk(T) of Eq. (4) (optional, ``Params.qpm``): with the oven at T_oven the
   local temperature is T = T_oven + T_off + dT, and
   Dk(T) = (4 pi / lambda_F)(n_SH(T) - n_F(T)) - 2 pi / Lambda(T),
   Lambda(T) = Lambda(25 C)(1 + a (T - 25) + b (T - 25)^2), n_j(T) a
   polynomial in (T - 25 C) (the paper gives no index data).  With
   T_ref = T_oven + T_off: phi = Dk(T_ref) z + C'(x,y,z), C' the trapezoid
   cumulative integral of Dk(T_ref + dT) - Dk(T_ref) on the map nodes,
   interpolated like C.  dk0 and dDk/dT are not used then; the lens phase
   (reading 6) keeps dn/dT.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import torch

from . import fft as dft

F64 = torch.float64
C128 = torch.complex128

EPS0 = 8.8541878128e-12   # vacuum permittivity, F/m
C_LIGHT = 299792458.0     # speed of light, m/s


def _t(v) -> torch.Tensor:
    if isinstance(v, torch.Tensor):
        return v.to(F64)
    return torch.tensor(float(v), dtype=F64)


@dataclass
class QPM:
    """Temperature model of the phase mismatch, Eq. (4) with Lambda(T)."""
    t_oven: float               # oven temperature (deg C)
    lambda25: float             # grating period Lambda(25 C) (m)
    a_lambda: float = 2.2e-6    # thermal expansion of the period (1/K), the paper's MgO:sPPLT
    b_lambda: float = -5.9e-9   # (1/K^2)
    n_f_t: tuple = (0.0,)       # n_F(T) = sum_k n_f_t[k] (T - 25)^k
    n_sh_t: tuple = (0.0,)

    def dk(self, lambda_f: float, T):
        u = T - 25.0
        nF = sum(c * u ** k for k, c in enumerate(self.n_f_t))
        nS = sum(c * u ** k for k, c in enumerate(self.n_sh_t))
        lam = self.lambda25 * (1.0 + self.a_lambda * u + self.b_lambda * u * u)
        return 4.0 * math.pi / lambda_f * (nS - nF) - 2.0 * math.pi / lam


@dataclass
class Params:
    """Physical inputs of one instance (crystal, beams, grid)."""
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    L: float
    lambda_f: float
    n_f: float
    n_sh: float
    d_eff: float
    alpha_f: float = 0.0
    alpha_sh: float = 0.0
    beta_f: float = 0.0
    beta_sh: float = 0.0
    dk0: float = 0.0
    ddk_dT: float = 0.0
    dn_dT: float = 0.0
    undepleted: bool = False
    walkoff_f: float = 0.0      # spatial walk-off angles rho_j (rad) toward +x
    walkoff_sh: float = 0.0
    qpm: Optional[QPM] = None   # Eq. (4) phase mismatch instead of dk0 + dDk/dT dT

    @property
    def lambda_sh(self) -> float:
        return self.lambda_f / 2.0

    @property
    def k_f(self) -> float:
        return 2.0 * math.pi * self.n_f / self.lambda_f

    @property
    def k_sh(self) -> float:
        return 2.0 * math.pi * self.n_sh / self.lambda_sh

    @property
    def kappa_f(self) -> float:
        # Eq. (1): 2 pi d_eff / (n_F lambda_F)
        return 2.0 * math.pi * self.d_eff / (self.n_f * self.lambda_f)

    @property
    def kappa_sh(self) -> float:
        # Reading 2: 2 pi d_eff / (n_SH lambda_F)
        return 2.0 * math.pi * self.d_eff / (self.n_sh * self.lambda_f)

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    @property
    def dz(self) -> float:
        return self.L / self.nz


def params_from_workload(w) -> Params:
    return Params(nx=w.nx, ny=w.ny, nz=w.nz, lx=w.lx, ly=w.ly, L=w.L,
                  lambda_f=w.lambda_f, n_f=w.n_f, n_sh=w.n_sh, d_eff=w.d_eff,
                  alpha_f=w.alpha_f, alpha_sh=w.alpha_sh, beta_f=w.beta_f,
                  beta_sh=w.beta_sh, dk0=w.dk0, ddk_dT=w.ddk_dT, dn_dT=w.dn_dT,
                  undepleted=bool(w.undepleted), walkoff_f=getattr(w, "walkoff_f", 0.0),
                  walkoff_sh=getattr(w, "walkoff_sh", 0.0), qpm=_qpm_of(w))


def _qpm_of(w) -> Optional["QPM"]:
    q = getattr(w, "qpm", None)
    if q is None:
        return None
    return QPM(q.t_oven, q.lambda25, q.a_lambda, q.b_lambda, tuple(q.n_f_t), tuple(q.n_sh_t))


# ---------------------------------------------------------------- grid ----

def axis(n: int, length: float) -> torch.Tensor:
    """Sample positions x_m = (m - n/2) dx, dx = length / n."""
    return (torch.arange(n, dtype=F64) - n // 2) * (length / n)


def wavenumbers(n: int, length: float) -> torch.Tensor:
    """Angular spatial frequency of DFT bin b: K_b = 2 pi m_b / length with
    m_b = b for b < n/2 and b - n above (the bin's signed frequency index)."""
    b = torch.arange(n, dtype=F64)
    m = torch.where(b < (n + 1) // 2, b, b - n)
    return 2.0 * math.pi * m / length


def power(A: torch.Tensor, n_j: float, dx: float, dy: float) -> torch.Tensor:
    """P = (1/2) eps0 c n sum |A|^2 dx dy (Sec. 2.2 intensity, summed over the grid)."""
    return 0.5 * EPS0 * C_LIGHT * n_j * (A.real ** 2 + A.imag ** 2).sum() * dx * dy


# ---------------------------------------------------------------- init ----

def initial_pump(p: Params, p1, w0, z_focus) -> torch.Tensor:
    """Eq. (5) at z = 0: A_F0/(1 + i tau0) exp(-r^2 / (w0^2 (1 + i tau0))),
    tau0 = -f/z_R, z_R = w0^2 k_F / 2, scaled to discrete power P1."""
    w0 = _t(w0)
    z_focus = _t(z_focus)
    p1 = _t(p1)
    x = axis(p.nx, p.lx)
    y = axis(p.ny, p.ly)
    z_r = w0 * w0 * p.k_f / 2.0
    tau0 = (0.0 - z_focus) / z_r
    q = torch.complex(torch.ones((), dtype=F64), tau0)
    r2 = (x[None, :] ** 2 + y[:, None] ** 2).to(C128)
    g = torch.exp(-r2 / (w0 * w0 * q)) / q
    a0 = torch.sqrt(p1 / power(g, p.n_f, p.dx, p.dy))
    return a0 * g


# --------------------------------------------------- temperature tables ----

def cumulative_dT(dT: torch.Tensor, L: float) -> torch.Tensor:
    """C[l] = int_0^{Z_l} dT dz' by the trapezoid rule on the z-nodes (Eq. 3)."""
    tz = dT.shape[0]
    dZ = L / (tz - 1)
    rows = [torch.zeros_like(dT[0])]
    for l in range(1, tz):
        rows.append(rows[-1] + 0.5 * dZ * (dT[l - 1] + dT[l]))
    return torch.stack(rows, 0)


def _lin_index(coord: torch.Tensor, origin: float, spacing: float, n: int):
    """Clamped linear-interpolation cell and fraction for node-centred samples."""
    u = ((coord - origin) / spacing).clamp(0.0, float(n - 1))
    i = torch.floor(u).clamp(max=n - 2)
    return i.long(), u - i


class TemperatureField:
    """dT(x,y,z) on a node-centred grid [tz][ty][tx] over
    [-t_lx/2, t_lx/2] x [-t_ly/2, t_ly/2] x [0, L], plus the uniform offset T_off.
    Provides dT and the cumulative C trilinearly interpolated at the field points."""

    def __init__(self, p: Params, dT: Optional[torch.Tensor], t_lx: float, t_ly: float,
                 t_off=0.0):
        if dT is None:
            dT = torch.zeros((2, 2, 2), dtype=F64)
            t_lx = t_lx or p.lx
            t_ly = t_ly or p.ly
        if not isinstance(dT, torch.Tensor):
            dT = torch.as_tensor(dT)
        self.dT = dT.to(F64)
        self.t_off = _t(t_off)
        self.L = p.L
        tz, ty, tx = self.dT.shape
        self.tz = tz
        if p.qpm is None:
            self.C = cumulative_dT(self.dT, p.L)
        else:
            # reading 10: the integrand is Dk(T_ref + dT) - Dk(T_ref) at every node
            t_ref = p.qpm.t_oven + self.t_off
            self.C = cumulative_dT(p.qpm.dk(p.lambda_f, t_ref + self.dT)
                                   - p.qpm.dk(p.lambda_f, t_ref), p.L)
        t_lx = t_lx or p.lx
        t_ly = t_ly or p.ly
        x = axis(p.nx, p.lx)
        y = axis(p.ny, p.ly)
        self.ix, self.fx = _lin_index(x, -t_lx / 2, t_lx / (tx - 1), tx)
        self.iy, self.fy = _lin_index(y, -t_ly / 2, t_ly / (ty - 1), ty)
        self.dZ = p.L / (tz - 1)

    def _bilinear(self, table2d: torch.Tensor) -> torch.Tensor:
        ix, fx, iy, fy = self.ix, self.fx, self.iy, self.fy
        t00 = table2d[iy][:, ix]
        t01 = table2d[iy][:, ix + 1]
        t10 = table2d[iy + 1][:, ix]
        t11 = table2d[iy + 1][:, ix + 1]
        fxr = fx[None, :]
        fyc = fy[:, None]
        return ((1 - fyc) * ((1 - fxr) * t00 + fxr * t01)
                + fyc * ((1 - fxr) * t10 + fxr * t11))

    def at(self, z: float):
        """(dT_interp, C_interp) at every field point of the plane z."""
        u = min(max(z / self.dZ, 0.0), float(self.tz - 1))
        l = min(int(math.floor(u)), self.tz - 2)
        t = u - l
        d = (1 - t) * self._bilinear(self.dT[l]) + t * self._bilinear(self.dT[l + 1])
        c = (1 - t) * self._bilinear(self.C[l]) + t * self._bilinear(self.C[l + 1])
        return d, c


# ----------------------------------------------------- nonlinear step ----

class Nonlinear:
    """Pointwise right-hand side of Eqs. (1)-(2) without diffraction and alpha
    (those live in L), plus the thermal-lens phase (reading 6)."""

    def __init__(self, p: Params, temp: TemperatureField):
        self.p = p
        self.temp = temp
        self.cF = 0.5 * EPS0 * C_LIGHT * p.n_f
        self.cS = 0.5 * EPS0 * C_LIGHT * p.n_sh
        self.k0F = 2.0 * math.pi / p.lambda_f
        self.k0S = 2.0 * math.pi / p.lambda_sh

    def coefficients(self, z: float):
        """phi and psi_F, psi_S at every field point of the plane z."""
        p = self.p
        d, c = self.temp.at(z)
        t_off = self.temp.t_off
        if p.qpm is None:
            g = p.ddk_dT
            phi = (p.dk0 + g * t_off) * z + g * c
        else:
            phi = p.qpm.dk(p.lambda_f, p.qpm.t_oven + t_off) * z + c
        dT_eff = d + t_off
        psiF = self.k0F * p.dn_dT * dT_eff
        psiS = self.k0S * p.dn_dT * dT_eff
        return phi, psiF, psiS

    def rhs(self, AF, AS, coef):
        p = self.p
        phi, psiF, psiS = coef
        e = torch.exp(1j * phi)
        IF = self.cF * (AF.real ** 2 + AF.imag ** 2)
        IS = self.cS * (AS.real ** 2 + AS.imag ** 2)
        fF = -0.5 * p.beta_f * IF * AF + 1j * psiF * AF
        if not p.undepleted:
            fF = fF + 1j * p.kappa_f * AS * torch.conj(AF) * torch.conj(e)
        fS = 1j * p.kappa_sh * AF * AF * e - 0.5 * p.beta_sh * IS * AS + 1j * psiS * AS
        return fF, fS

    def rk4(self, AF, AS, z0: float, h: float):
        """One classical RK4 step of size h from z0 (stages at z0, z0+h/2, z0+h)."""
        c0 = self.coefficients(z0)
        cm = self.coefficients(z0 + 0.5 * h)
        c1 = self.coefficients(z0 + h)
        k1F, k1S = self.rhs(AF, AS, c0)
        k2F, k2S = self.rhs(AF + 0.5 * h * k1F, AS + 0.5 * h * k1S, cm)
        k3F, k3S = self.rhs(AF + 0.5 * h * k2F, AS + 0.5 * h * k2S, cm)
        k4F, k4S = self.rhs(AF + h * k3F, AS + h * k3S, c1)
        AF = AF + (h / 6.0) * (k1F + 2 * k2F + 2 * k3F + k4F)
        AS = AS + (h / 6.0) * (k1S + 2 * k2S + 2 * k3S + k4S)
        return AF, AS


# -------------------------------------------------------- linear step ----

class Linear:
    """exp(L dz) applied in K-space: diffraction (reading 1), exp(-alpha dz/2)
    and the walk-off term.  The walk-off term (Sec. 6, App. B) adds -tan(rho) dA/dx to
    dA/dz, i.e. the factor exp(-i tan(rho) Kx dz): the field drifts toward +x
    by tan(rho) per unit length."""

    def __init__(self, p: Params):
        Kx = wavenumbers(p.nx, p.lx)
        Ky = wavenumbers(p.ny, p.ly)
        K2 = Kx[None, :] ** 2 + Ky[:, None] ** 2
        dz = p.dz
        self.PF = torch.exp(-1j * K2 * dz / (2.0 * p.k_f)) * math.exp(-0.5 * p.alpha_f * dz)
        self.PS = torch.exp(-1j * K2 * dz / (2.0 * p.k_sh)) * math.exp(-0.5 * p.alpha_sh * dz)
        self.PF = self.PF * torch.exp(-1j * math.tan(p.walkoff_f) * Kx[None, :] * dz)
        self.PS = self.PS * torch.exp(-1j * math.tan(p.walkoff_sh) * Kx[None, :] * dz)

    def __call__(self, AF, AS):
        AF = dft.ifft2(self.PF * dft.fft2(AF))
        AS = dft.ifft2(self.PS * dft.fft2(AS))
        return AF, AS


# ------------------------------------------------------ heat deposits ----

class HeatDeposit:
    """Box-sums q_dot dV (Eq. 8) of the field samples into the nearest node of
    a heat grid [hz][hy][hx] spanning [-wx/2, wx/2] x [-wy/2, wy/2] x [0, L]."""

    def __init__(self, p: Params, hx: int, hy: int, hz: int, wx: float, wy: float):
        self.p = p
        self.shape = (hz, hy, hx)
        self.Q = torch.zeros(self.shape, dtype=F64)   # sum of q_dot dV per node, W
        self.hdx = wx / (hx - 1)
        self.hdy = wy / (hy - 1)
        self.hdz = p.L / (hz - 1)
        x = axis(p.nx, p.lx)
        y = axis(p.ny, p.ly)
        self.ix = torch.floor((x + wx / 2) / self.hdx + 0.5).long()
        self.iy = torch.floor((y + wy / 2) / self.hdy + 0.5).long()
        self.okx = (self.ix >= 0) & (self.ix < hx)
        self.oky = (self.iy >= 0) & (self.iy < hy)
        self.cF = 0.5 * EPS0 * C_LIGHT * p.n_f
        self.cS = 0.5 * EPS0 * C_LIGHT * p.n_sh

    def qdot(self, AF, AS):
        p = self.p
        IF = self.cF * (AF.real ** 2 + AF.imag ** 2)
        IS = self.cS * (AS.real ** 2 + AS.imag ** 2)
        return p.alpha_f * IF + p.beta_f * IF ** 2 + p.alpha_sh * IS + p.beta_sh * IS ** 2

    def add(self, AF, AS, z: float, wz: float):
        l = int(math.floor(z / self.hdz + 0.5))
        if l < 0 or l >= self.shape[0]:
            return
        q = self.qdot(AF, AS) * (self.p.dx * self.p.dy * wz)
        mask = self.oky[:, None] & self.okx[None, :]
        jj = self.iy[:, None].expand_as(q)[mask]
        ii = self.ix[None, :].expand_as(q)[mask]
        ll = torch.full_like(jj, l)
        self.Q.index_put_((ll, jj, ii), q[mask].detach(), accumulate=True)

    def qdot_nodes(self) -> torch.Tensor:
        """Node source density q_dot = Q / V, V the volume of the node's cell:
        hdx hdy hdz, halved once for every face the node lies on (a face
        node's cell lies half outside the crystal, and only samples inside
        are binned to it).  Nodes on faces held at T_oven are not solved
        for, so there the factor has no effect."""
        hz, hy, hx = self.shape
        vol = torch.full(self.shape, self.hdx * self.hdy * self.hdz, dtype=F64)
        for axis, n in ((0, hz), (1, hy), (2, hx)):
            for end in (0, n - 1):
                sl = [slice(None)] * 3
                sl[axis] = end
                vol[tuple(sl)] *= 0.5
        return self.Q / vol


# ---------------------------------------------------------- propagate ----

def propagate(p: Params, AF: torch.Tensor, AS: torch.Tensor, temp: TemperatureField,
              deposit: Optional[HeatDeposit] = None, nsteps: Optional[int] = None):
    """March nz symmetric split steps (Eq. 15): N(dz/2) L(dz) N(dz/2)."""
    nl = Nonlinear(p, temp)
    lin = Linear(p)
    dz = p.dz
    h = 0.5 * dz
    nz = p.nz if nsteps is None else nsteps
    for s in range(nz):
        z = s * dz
        if deposit is not None:
            deposit.add(AF, AS, z, dz * (0.5 if s == 0 else 1.0))
        AF, AS = nl.rk4(AF, AS, z, h)
        AF, AS = lin(AF, AS)
        AF, AS = nl.rk4(AF, AS, z + h, h)
    if deposit is not None and nz == p.nz:
        deposit.add(AF, AS, p.L, 0.5 * dz)
    return AF, AS


def run(w, AF0: Optional[torch.Tensor] = None, AS0: Optional[torch.Tensor] = None,
        w0=None, z_focus=None, t_off=None, dT=None, deposit: Optional[HeatDeposit] = None):
    """Initial fields + full propagation for a workload description.
    Returns (AF(L), AS(L), eta).  w0, z_focus, t_off, dT may be tensors that
    require grad (the oracle's gradients are autograd of this map)."""
    p = params_from_workload(w)
    w0 = w.w0 if w0 is None else w0
    z_focus = w.z_focus if z_focus is None else z_focus
    t_off = w.t_off if t_off is None else t_off
    if dT is None and w.dT is not None:
        dT = torch.as_tensor(w.dT)
    temp = TemperatureField(p, dT, w.t_lx, w.t_ly, t_off)
    if AF0 is None:
        AF0 = initial_pump(p, w.p1, w0, z_focus)
    if AS0 is None:
        AS0 = torch.zeros((p.ny, p.nx), dtype=C128)
    AF, AS = propagate(p, AF0.to(C128), AS0.to(C128), temp, deposit)
    eta = power(AS, p.n_sh, p.dx, p.dy) / _t(w.p1)
    return AF, AS, eta
