"""GB300 SpMM library: Y = A X and A^T X for power-law sparse A (paper arXiv
1602.02864, Section 3) behind the C-ABI in include/spmm.h.

The CUDA library is loaded on first use of the binding::

    from paper_1602_02864_gb300 import spmm
    A = spmm.SparseMatrix.from_csr(csr)
    Y = A.apply(X)
"""
from __future__ import annotations

import importlib

__all__ = ["spmm", "build"]


def __getattr__(name):
    if name in ("spmm", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
