"""The oracle's own discrete Fourier transform (radix-2, FP64, plain C).

TEST INFRASTRUCTURE ONLY (see ``oracle/ssfm.py``).  The linear step of the
split step (App. A, Eqs. (A.3)-(A.5)) transforms the fields to K-space,
multiplies and transforms back.  Its DFT is ``oracle/fft.c``: the textbook
iterative Cooley-Tukey radix-2 algorithm in double precision, compiled here
with gcc (OpenMP over rows when available) and called through ctypes.  No
library FFT is used.

Conventions (those of the DFT's definition):
    fft(x)[k]  = sum_m x[m] exp(-2 pi i k m / n)
    ifft(X)[m] = (1/n) sum_k X[k] exp(+2 pi i k m / n)
fft2 / ifft2 apply them along the last axis, then along the one before.

Both are linear, so their vector-Jacobian products are the adjoint maps:
fft^H = n ifft and ifft^H = fft / n (PyTorch's complex gradients are the
conjugate Wirtinger derivatives, for which a linear map's VJP is its
conjugate transpose).  That lets the oracle's autograd gradients pass
through the transform.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fft.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle_fft.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fft.c into a shared library (gcc; with -fopenmp if it links)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("the oracle's FFT needs a C compiler (gcc)")
    os.makedirs(BUILD, exist_ok=True)
    tmp = f"{LIB}.{os.getpid()}.tmp"
    base = [cc, "-O2", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:3] + ["-fopenmp"] + base[3:], capture_output=True, text=True)
    if r.returncode != 0:   # no OpenMP runtime: the same code, one thread
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed on {SRC}:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_dft_rows.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_long,
                                            ctypes.c_int]
            lib.oracle_dft_rows.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads of the DFT's row loop (n <= 0 only queries); returns the count."""
    return int(_load().oracle_set_threads(int(n)))


def _rows(x: torch.Tensor, sign: int) -> torch.Tensor:
    """Unnormalised DFT (sign -1) or its conjugate sum (sign +1) of every
    row along the last axis; returns a new complex128 tensor."""
    y = x.detach().to(torch.complex128).contiguous().clone()
    n = y.shape[-1]
    if y.numel() == 0:
        return y
    rc = _load().oracle_dft_rows(y.data_ptr(), y.numel() // n, n, sign)
    if rc != 0:
        raise ValueError(f"DFT length {n} is not a power of two")
    return y


class _DFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, inverse: bool):
        ctx.inverse = inverse
        n = x.shape[-1]
        return _rows(x, +1) / n if inverse else _rows(x, -1)

    @staticmethod
    def backward(ctx, g):
        n = g.shape[-1]
        if ctx.inverse:              # (ifft)^H g = fft(g) / n
            return _rows(g, -1) / n, None
        return _rows(g, +1), None    # (fft)^H g = n ifft(g) = unnormalised +1 sum


def fft(x: torch.Tensor) -> torch.Tensor:
    """Forward DFT along the last axis."""
    return _DFT.apply(x, False)


def ifft(x: torch.Tensor) -> torch.Tensor:
    """Inverse DFT (with 1/n) along the last axis."""
    return _DFT.apply(x, True)


def fft2(x: torch.Tensor) -> torch.Tensor:
    """2-D forward DFT over the last two axes ([..., ny, nx])."""
    return fft(fft(x).transpose(-1, -2)).transpose(-1, -2)


def ifft2(x: torch.Tensor) -> torch.Tensor:
    """2-D inverse DFT over the last two axes."""
    return ifft(ifft(x).transpose(-1, -2)).transpose(-1, -2)
