"""Independent references that pin the oracle: closed forms and brute force.

Nothing here calls the oracle's arithmetic; these are the textbook results the
oracle must reproduce.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad

EPS0 = 8.8541878128e-12
C_LIGHT = 299792458.0


def bk_h(sigma: float, xi: float) -> float:
    """Boyd-Kleinman focusing function without walk-off,
    h(sigma, xi) = (1/4xi) |int_{-xi}^{xi} e^{i sigma t} / (1 + i t) dt|^2,
    by adaptive quadrature of its real and imaginary parts."""
    re = quad(lambda t: (math.cos(sigma * t) + t * math.sin(sigma * t)) / (1 + t * t),
              -xi, xi, limit=400, epsabs=1e-13, epsrel=1e-12)[0]
    im = quad(lambda t: (math.sin(sigma * t) - t * math.cos(sigma * t)) / (1 + t * t),
              -xi, xi, limit=400, epsabs=1e-13, epsrel=1e-12)[0]
    return (re * re + im * im) / (4.0 * xi)


def bk_constant(d_eff, L, n_f, n_sh, lambda_f) -> float:
    """Prefactor of Eq. (17): 16 pi^2 d^2 L / (eps0 c n_F n_SH lambda_F^3)."""
    return 16 * math.pi ** 2 * d_eff ** 2 * L / (EPS0 * C_LIGHT * n_f * n_sh * lambda_f ** 3)


def brute_dft2(a: np.ndarray) -> np.ndarray:
    """O(N^4) 2-D DFT, X[k,l] = sum_{m,n} a[m,n] exp(-2 pi i (k m / M + l n / N))."""
    M, N = a.shape
    out = np.zeros((M, N), dtype=np.complex128)
    for k in range(M):
        for l in range(N):
            s = 0j
            for m in range(M):
                for n in range(N):
                    s += a[m, n] * np.exp(-2j * np.pi * (k * m / M + l * n / N))
            out[k, l] = s
    return out


def gaussian_beam(x, y, z, w0, z_focus, k):
    """Unnormalised Eq. (5) without the carrier: exp(-r^2/(w0^2 (1+i tau)))/(1+i tau)."""
    z_r = w0 * w0 * k / 2.0
    q = 1 + 1j * (z - z_focus) / z_r
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    return np.exp(-r2 / (w0 * w0 * q)) / q


def tpa_plane_wave(I0, alpha, beta, z):
    """dI/dz = -alpha I - beta I^2:  I = I0 e^{-a z} / (1 + b I0 (1 - e^{-a z}) / a)."""
    e = math.exp(-alpha * z)
    return I0 * e / (1 + beta * I0 * (1 - e) / alpha)


def discrete_laplacian_eigen(hx, hy, hz, dx, dy, dz):
    """Eigenvalue of the 7-point Laplacian (Eq. 16) for the lowest sine mode that
    vanishes on all faces: -sum (4/d^2) sin^2(pi d / (2 W))."""
    lam = 0.0
    for n, d in ((hx, dx), (hy, dy), (hz, dz)):
        W = (n - 1) * d
        lam -= 4.0 / d ** 2 * math.sin(math.pi * d / (2 * W)) ** 2
    return lam
