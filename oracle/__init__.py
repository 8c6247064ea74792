"""FP64 CPU oracle of the SHG split-step Fourier path and its heat loop.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product package.
It is plain PyTorch CPU code in float64/complex128, with its own radix-2 DFT
in plain C (``fft.c``), and shares no code with the CUDA path.
"""
from . import fft, ssfm, heat  # noqa: F401
