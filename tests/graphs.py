"""Small hand-made graphs for tests (CSR from explicit edge lists)."""
import numpy as np

import synth


def csr_from_edges(n_rows, n_cols, src, dst, values=None):
    """CSR with rows sorted, duplicates merged (values of duplicates summed)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if len(src) == 0:
        return synth.CSR(n_rows, n_cols, np.zeros(n_rows + 1, np.int64), np.zeros(0, np.int32),
                         None if values is None else np.zeros(0, np.float32))
    key = src * n_cols + dst
    order = np.argsort(key, kind="stable")
    key = key[order]
    uk, first = np.unique(key, return_index=True)
    rows = uk // n_cols
    cols = (uk % n_cols).astype(np.int32)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    vals = None
    if values is not None:
        v = np.asarray(values, dtype=np.float64)[order]
        vals = np.add.reduceat(v, first).astype(np.float32)
    return synth.CSR(n_rows, n_cols, row_ptr, cols, vals)


def cycle(n):
    i = np.arange(n)
    return csr_from_edges(n, n, i, (i + 1) % n)


def complete(n, loops=False):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    m = np.ones((n, n), bool) if loops else ~np.eye(n, dtype=bool)
    return csr_from_edges(n, n, i[m], j[m])


def star(n):
    """vertex 0 -> every other vertex"""
    return csr_from_edges(n, n, np.zeros(n - 1, np.int64), np.arange(1, n))


def path(n):
    i = np.arange(n - 1)
    return csr_from_edges(n, n, i, i + 1)


def dense_of(A, dtype=np.float64):
    D = np.zeros((A.n_rows, A.n_cols), dtype=dtype)
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    v = np.ones(A.nnz) if A.values is None else A.values.astype(np.float64)
    np.add.at(D, (rows, A.col_idx.astype(np.int64)), v)
    return D


def random_csr(n_rows, n_cols, density, seed, weighted=True, empty_rows=0.2):
    rng = np.random.default_rng(seed)
    m = max(1, int(n_rows * n_cols * density))
    src = rng.integers(0, n_rows, m)
    dst = rng.integers(0, n_cols, m)
    keep_rows = rng.random(n_rows) >= empty_rows
    sel = keep_rows[src]
    src, dst = src[sel], dst[sel]
    vals = rng.random(len(src)).astype(np.float32) if weighted else None
    return csr_from_edges(n_rows, n_cols, src, dst, vals)
