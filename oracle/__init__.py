"""FP64 CPU oracle for the SpMM library -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
``oracle.c`` is compiled on its own with gcc and takes plain numpy arrays.

Each function is the plain definition from the paper, summed in double:

* ``spmm``        Y = A X / A^T X (Section 3, Algorithm 1: a nonzero a_ij adds
                  a_ij * X[j, :] to output row i)
* ``spmm_rows``   the forward product for selected output rows
* ``spmm_t_rows`` the transposed product for selected output rows
* ``pagerank``    the Section 4.1 update rule, dangling mass spread uniformly
* ``nmf``         the Section 4.3 multiplicative updates (H first, then W)
* ``lanczos``     top eigenpairs of a symmetric sparse matrix (Section 4.2 uses
                  a Krylov eigensolver; here block Lanczos with full
                  re-orthogonalisation)
* ``svds``        top singular values (Section 5.5.2) by the same Lanczos on
                  A^T A, applied as two products
* ``sym_eigh``    the dense symmetric eigen-decomposition of the projected
                  matrix: Householder tridiagonalisation, Sturm bisection,
                  inverse iteration
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (gcc -O2, OpenMP for the row-parallel
    forward product only)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.oracle_num_threads.restype = i32
            lib.oracle_spmm.argtypes = [i64, i64, P, P, P, i32, P, i32, i64, i32, P, i64, i32, i32]
            lib.oracle_spmm_rows.argtypes = [P, P, P, i32, P, i32, i64, i32, P, i64, P, i32]
            lib.oracle_spmm_t_rows.argtypes = [i64, P, P, P, i32, P, i32, i64, i32, P, i64, P]
            lib.oracle_pagerank.argtypes = [i64, P, P, f64, i32, P, P]
            lib.oracle_nmf.argtypes = [i64, i64, P, P, P, i32, i32, i32, f64, P, P, P]
            lib.oracle_sym_eigh.argtypes = [i32, P, P, P]
            lib.oracle_sym_eigh.restype = i32
            lib.oracle_lanczos.argtypes = [i64, i64, P, P, P, i32, i32, i32, i32, P, i32, P, P]
            lib.oracle_lanczos.restype = i32
            _lib = lib
    return _lib


class using_library:
    """Temporarily route every call through another build of oracle.c (the
    mutation tests use it to check that the pins catch planted mistakes)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("oracle_num_threads", "oracle_spmm", "oracle_spmm_rows", "oracle_spmm_t_rows",
                     "oracle_pagerank", "oracle_nmf", "oracle_sym_eigh", "oracle_lanczos"):
            f, g = getattr(self._saved, name), getattr(lib, name)
            g.argtypes, g.restype = f.argtypes, f.restype
        with _lock:
            _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _vals(values):
    if values is None:
        return None, 0
    v = np.asarray(values)
    if v.dtype == np.float32:
        return np.ascontiguousarray(v), 1
    return np.ascontiguousarray(v, dtype=np.float64), 2


def _dense(X):
    X = np.asarray(X)
    if X.dtype == np.float32:
        X = np.ascontiguousarray(X)
        return X, 1
    return np.ascontiguousarray(X, dtype=np.float64), 2


def _csr(row_ptr, col_idx):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col_idx, dtype=np.int32))


def spmm(n_rows, n_cols, row_ptr, col_idx, values, X, transpose=False, threads=1) -> np.ndarray:
    """Y = A X (n_rows x k) or A^T X (n_cols x k) in float64.  X is float32 or
    float64, shape (n_rows or n_cols, k); values None means pattern-only."""
    rp, ci = _csr(row_ptr, col_idx)
    v, vt = _vals(values)
    Xc, xt = _dense(X)
    k = Xc.shape[1]
    out_rows = n_cols if transpose else n_rows
    Y = np.zeros((out_rows, k), dtype=np.float64)
    _load().oracle_spmm(n_rows, n_cols, _p(rp), _p(ci), _p(v), vt, _p(Xc), xt, Xc.shape[1], k, _p(Y), k,
                        int(bool(transpose)), int(threads))
    return Y


def spmm_rows(row_ptr, col_idx, values, X, rows, threads=1, k=None) -> np.ndarray:
    """Forward product for the listed output rows: returns len(rows) x k.
    With k given, only the first k columns of the (contiguous) X are used,
    without copying it."""
    rp, ci = _csr(row_ptr, col_idx)
    v, vt = _vals(values)
    Xc, xt = _dense(X)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    k = Xc.shape[1] if k is None else int(k)
    if not 1 <= k <= Xc.shape[1]:
        raise ValueError("k out of range")
    Y = np.zeros((len(rows), k), dtype=np.float64)
    _load().oracle_spmm_rows(_p(rp), _p(ci), _p(v), vt, _p(Xc), xt, Xc.shape[1], k, _p(rows), len(rows),
                             _p(Y), int(threads))
    return Y


def spmm_t_rows(n_rows, n_cols, row_ptr, col_idx, values, X, rows) -> np.ndarray:
    """Transposed product for the listed output rows (distinct ids)."""
    rp, ci = _csr(row_ptr, col_idx)
    v, vt = _vals(values)
    Xc, xt = _dense(X)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if len(np.unique(rows)) != len(rows):
        raise ValueError("spmm_t_rows needs distinct row ids")
    slot = np.full(n_cols, -1, dtype=np.int64)
    slot[rows] = np.arange(len(rows), dtype=np.int64)
    k = Xc.shape[1]
    Y = np.zeros((len(rows), k), dtype=np.float64)
    _load().oracle_spmm_t_rows(n_rows, _p(rp), _p(ci), _p(v), vt, _p(Xc), xt, Xc.shape[1], k, _p(slot),
                               len(rows), _p(Y))
    return Y


def pagerank(n, row_ptr, col_idx, damping=0.85, iters=30, x0=None):
    """Returns (x, residuals): x after `iters` iterations from x0 (default 1/N),
    residuals[t] = L1 change of iteration t."""
    rp, ci = _csr(row_ptr, col_idx)
    x = np.full(n, 1.0 / n, dtype=np.float64) if x0 is None else np.array(x0, dtype=np.float64)
    res = np.zeros(iters, dtype=np.float64)
    _load().oracle_pagerank(n, _p(rp), _p(ci), float(damping), int(iters), _p(x), _p(res))
    return x, res


def nmf(n_rows, n_cols, row_ptr, col_idx, values, W0, Ht0, steps, eps=1e-12):
    """Returns (W, Ht, objective[steps+1]) after `steps` H-then-W updates."""
    rp, ci = _csr(row_ptr, col_idx)
    v, vt = _vals(values)
    W = np.array(W0, dtype=np.float64, order="C")
    Ht = np.array(Ht0, dtype=np.float64, order="C")
    k = W.shape[1]
    if k > 64:
        raise ValueError("k <= 64")
    obj = np.zeros(steps + 1, dtype=np.float64)
    _load().oracle_nmf(n_rows, n_cols, _p(rp), _p(ci), _p(v), vt, k, int(steps), float(eps), _p(W), _p(Ht),
                       _p(obj))
    return W, Ht, obj


def sym_eigh(M):
    """All eigenpairs of a dense symmetric matrix: (evals ascending, V with
    unit eigenvector columns), by Householder tridiagonalisation, Sturm
    bisection and inverse iteration (oracle_sym_eigh)."""
    M = np.array(M, dtype=np.float64, order="C")
    m = M.shape[0]
    ev = np.zeros(m, dtype=np.float64)
    V = np.zeros((m, m), dtype=np.float64)
    if _load().oracle_sym_eigh(m, _p(M), _p(ev), _p(V)) != 0:
        raise MemoryError("oracle_sym_eigh: allocation failed")
    return ev, V


def lanczos(n, row_ptr, col_idx, values, Q0, nev, m_max):
    """Top-nev eigenpairs (descending) of the symmetric n x n CSR matrix S:
    (evals, vectors n x nev, basis size)."""
    rp, ci = _csr(row_ptr, col_idx)
    v, vt = _vals(values)
    Q0 = np.ascontiguousarray(Q0, dtype=np.float64)
    b = Q0.shape[1]
    ev = np.zeros(nev, dtype=np.float64)
    V = np.zeros((n, nev), dtype=np.float64)
    m = _load().oracle_lanczos(n, n, _p(rp), _p(ci), _p(v), vt, 0, b, int(m_max), _p(Q0), nev, _p(ev), _p(V))
    if m < 0:
        raise MemoryError("oracle_lanczos: allocation failed")
    return ev, V, m


def svds(n_rows, n_cols, row_ptr, col_idx, values, Q0, nsv, m_max):
    """Top-nsv singular values (descending) of the n_rows x n_cols CSR matrix
    A, from block Lanczos on A^T A applied as A q then A^T (A q): (singular
    values, right singular vectors n_cols x nsv, basis size)."""
    rp, ci = _csr(row_ptr, col_idx)
    v, vt = _vals(values)
    Q0 = np.ascontiguousarray(Q0, dtype=np.float64)
    b = Q0.shape[1]
    ev = np.zeros(nsv, dtype=np.float64)
    V = np.zeros((n_cols, nsv), dtype=np.float64)
    m = _load().oracle_lanczos(n_rows, n_cols, _p(rp), _p(ci), _p(v), vt, 1, b, int(m_max), _p(Q0), nsv, _p(ev),
                               _p(V))
    if m < 0:
        raise MemoryError("oracle_lanczos: allocation failed")
    return np.sqrt(np.maximum(ev, 0.0)), V, m
