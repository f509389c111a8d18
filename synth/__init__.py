"""Seeded synthetic inputs (graphs, edge values, dense matrices).

This module serves both the CUDA library and the CPU oracle with identical
inputs and holds none of the SpMM arithmetic.  The C source ``synth.c`` is
compiled with gcc on first use (or by ``__graft_entry__.build()``).

Graph recipes (paper Section 5 "graph datasets"; R-MAT quadrant probabilities
a/b/c/d = 0.57/0.19/0.19/0.05):

* ``rmat_csr(scale, n_edges)``: R-MAT edges, duplicates merged, self-loops kept.
* ``chunglu_csr(g)``: graph ``g`` of a batch of Chung-Lu power-law graphs
  (exponent 2.1, size log-uniform in [1e3, 2e5], average degree U[8, 32]).
* ``sbm_csr(n, clusters, avg_deg, p_in, permuted)``: stochastic block model,
  clustered ids or a seeded random relabelling (Section 5.1's ordering study).
* ``rmat_permuted_csr(scale)``: R-MAT with randomly relabelled vertices.
* ``sym_rmat_csr(scale)``: symmetrised R-MAT (8*N directed edges, union with the
  transpose), lognormal(0,1) pair weights, normalised D^-1/2 A D^-1/2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile libsynth.so in place (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_CU_SRC = os.path.join(_HERE, "rmat_cuda.cu")
_CU_LIB_PATH = os.path.join(_HERE, "libsynth_cuda.so")
_cu_lib = None


def build_cuda(force: bool = False) -> str:
    """Compile libsynth_cuda.so (the GPU R-MAT generator) in place with nvcc."""
    if force or not os.path.exists(_CU_LIB_PATH) or os.path.getmtime(_CU_LIB_PATH) < os.path.getmtime(_CU_SRC):
        import shutil
        nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _CU_LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                               "-Xcompiler", "-fPIC", "-o", tmp, _CU_SRC])
        os.replace(tmp, _CU_LIB_PATH)
    return _CU_LIB_PATH


def _load_cuda():
    global _cu_lib
    with _lock:
        if _cu_lib is None:
            build_cuda()
            lib = ctypes.CDLL(_CU_LIB_PATH)
            P, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.synth_rmat_block_count.argtypes = [i32, i64, f64, f64, f64, u64, i32, P, P]
            lib.synth_rmat_block_fill.argtypes = [i32, i64, f64, f64, f64, u64, i32, P, P, P, P, P]
            lib.synth_host_alloc.argtypes = [u64]
            lib.synth_host_alloc.restype = P
            lib.synth_host_free.argtypes = [P]
            _cu_lib = lib
    return _cu_lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.synth_philox4x32_10.argtypes = [P, P, P]
            lib.synth_rmat_edges.argtypes = [i32, i64, f64, f64, f64, u64, P, P]
            lib.synth_edges_to_csr.argtypes = [i64, i64, i64, P, P, i32, P, P]
            lib.synth_edges_to_csr.restype = i64
            lib.synth_uniform01_f32.argtypes = [u64, u64, i64, P]
            lib.synth_dense_f32.argtypes = [u64, u64, i64, i64, i32, i64, i32, P]
            lib.synth_dense_rows_f32.argtypes = [u64, u64, P, i64, i32, i32, P]
            lib.synth_sample_rows.argtypes = [u64, i64, i64, P]
            lib.synth_chunglu_size.argtypes = [u64, i64, f64, f64, f64, f64, P]
            lib.synth_chunglu_size.restype = i64
            lib.synth_chunglu_edges.argtypes = [u64, i64, i64, i64, f64, P, P]
            lib.synth_chunglu_edges.restype = i32
            lib.synth_sym_lognormal.argtypes = [u64, i64, P, P, i32, P]
            lib.synth_permutation.argtypes = [u64, i64, P]
            lib.synth_relabel_edges.argtypes = [i64, P, P, P]
            lib.synth_sbm_edges.argtypes = [u64, i64, i64, i64, f64, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().synth_philox4x32_10(_p(c), _p(k), _p(out))
    return out


class CSR:
    """A host CSR matrix: int64 row pointers, int32 column indices, optional
    float32 values (None = pattern-only, every stored entry is 1)."""

    def __init__(self, n_rows, n_cols, row_ptr, col_idx, values=None):
        self.n_rows = int(n_rows)
        self.n_cols = int(n_cols)
        self.row_ptr = row_ptr
        self.col_idx = col_idx
        self.values = values

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def rmat_edges(scale: int, n_edges: int, seed: int = 0, abc=RMAT_ABC):
    src = np.empty(n_edges, dtype=np.uint32)
    dst = np.empty(n_edges, dtype=np.uint32)
    a, b, c = abc
    _load().synth_rmat_edges(scale, n_edges, a, b, c, seed, _p(src), _p(dst))
    return src, dst


def edges_to_csr(n_rows: int, n_cols: int, src, dst, symmetrize: bool = False) -> CSR:
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    m = len(src) * (2 if symmetrize else 1)
    row_ptr = np.empty(n_rows + 1, dtype=np.int64)
    col_idx = np.empty(max(m, 1), dtype=np.int32)
    nnz = _load().synth_edges_to_csr(n_rows, n_cols, len(src), _p(src), _p(dst), int(symmetrize),
                                     _p(row_ptr), _p(col_idx))
    if nnz < 0:
        raise MemoryError("synth_edges_to_csr: allocation failed")
    return CSR(n_rows, n_cols, row_ptr, col_idx[:nnz].copy())


def uniform01(n: int, seed: int = 0, seed2: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float32)
    _load().synth_uniform01_f32(seed, seed2, n, _p(out))
    return out


def host_empty(n: int, dtype) -> np.ndarray:
    """An uninitialised host array in anonymous memory advised for transparent
    huge pages (fewer, larger pages: pinned copies of it run at the full link
    rate).  The mapping lives as long as the array."""
    import mmap
    dtype = np.dtype(dtype)
    m = mmap.mmap(-1, max(int(n) * dtype.itemsize, 1), flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    try:
        m.madvise(mmap.MADV_HUGEPAGE)
    except (AttributeError, OSError, ValueError):
        pass
    return np.frombuffer(m, dtype=dtype, count=int(n))


def host_empty_pinned(n: int, dtype) -> np.ndarray:
    """An uninitialised page-locked host array (cudaHostAlloc), freed when the
    array and every view of it are gone."""
    import weakref
    lib = _load_cuda()
    dtype = np.dtype(dtype)
    nbytes = max(int(n) * dtype.itemsize, 1)
    ptr = lib.synth_host_alloc(nbytes)
    if not ptr:
        raise MemoryError(f"cudaHostAlloc of {nbytes} bytes failed")
    raw = (ctypes.c_uint8 * nbytes).from_address(ptr)
    weakref.finalize(raw, lib.synth_host_free, ptr)
    return np.frombuffer(raw, dtype=dtype, count=int(n))


def rmat_csr_cuda(scale: int, n_edges: int | None = None, seed: int = 0, block_bits: int = 10,
                  abc=RMAT_ABC, pinned: bool = False) -> CSR:
    """rmat_csr (pattern) built on the GPU: the same draws, so the same graph,
    for edge lists too large to sort on the host.  The edges are bucketed by
    row block on the device (8 bytes per edge), each block is sorted and
    deduplicated there, and the CSR is assembled in host memory (int64 row
    pointers, int32 columns) -- page-locked memory if pinned (for streaming
    the matrix to the GPU), else anonymous memory advised for huge pages."""
    import torch
    lib = _load_cuda()
    n = 1 << scale
    m = 16 * n if n_edges is None else int(n_edges)
    a, b, c = abc
    t0, t1, t2 = a, a + b, a + b + c
    bb = min(block_bits, scale)
    nb = 1 << bb
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    hist = torch.zeros(nb, dtype=torch.int64, device=dev)
    if lib.synth_rmat_block_count(scale, m, t0, t1, t2, seed, bb, hist.data_ptr(), stream) != 0:
        raise RuntimeError("synth_rmat_block_count failed")
    base = torch.zeros(nb + 1, dtype=torch.int64, device=dev)
    base[1:] = torch.cumsum(hist, 0)
    keys = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
    cursor = torch.zeros(nb, dtype=torch.int64, device=dev)
    overflow = torch.zeros(1, dtype=torch.int64, device=dev)
    if lib.synth_rmat_block_fill(scale, m, t0, t1, t2, seed, bb, base.data_ptr(), cursor.data_ptr(),
                                 keys.data_ptr(), overflow.data_ptr(), stream) != 0:
        raise RuntimeError("synth_rmat_block_fill failed")
    if int(overflow.item()) != 0 or not torch.equal(cursor, hist):
        raise RuntimeError("R-MAT block fill does not match the block counts")
    base_h = base.cpu().numpy()
    rpb = n >> bb
    alloc = host_empty_pinned if pinned else host_empty
    row_ptr = alloc(n + 1, np.int64)
    row_ptr[:] = 0
    col = alloc(max(m, 1), np.int32)
    col_t = torch.from_numpy(col)
    nnz = 0
    mask = n - 1
    for blk in range(nb):
        lo, hi = int(base_h[blk]), int(base_h[blk + 1])
        if hi == lo:
            continue
        u = torch.unique_consecutive(torch.sort(keys[lo:hi])[0])
        rows = (u >> scale) - blk * rpb
        row_ptr[blk * rpb + 1:(blk + 1) * rpb + 1] = torch.bincount(rows, minlength=rpb).cpu().numpy()
        col_t[nnz:nnz + u.numel()].copy_((u & mask).to(torch.int32))
        nnz += u.numel()
        del u, rows
    del keys
    np.cumsum(row_ptr, out=row_ptr)
    return CSR(n, n, row_ptr, col[:nnz])


def rmat_csr(scale: int, n_edges: int | None = None, seed: int = 0, weighted: bool = False,
             abc=RMAT_ABC) -> CSR:
    """R-MAT graph with 2^scale vertices and n_edges (default 16 * 2^scale)
    directed edges; duplicates merged, self-loops kept.  If weighted, values are
    U[0,1) float32 drawn per CSR position after the merge."""
    n = 1 << scale
    if n_edges is None:
        n_edges = 16 * n
    src, dst = rmat_edges(scale, n_edges, seed, abc)
    A = edges_to_csr(n, n, src, dst)
    del src, dst
    if weighted:
        A.values = uniform01(A.nnz, seed=seed, seed2=0x7661)
    return A


def sym_rmat_csr(scale: int, seed: int = 0, normalise: bool = True) -> CSR:
    """Symmetrised R-MAT: 8*N directed edges, union with the transpose (a
    self-loop is stored once), lognormal(0,1) weight per unordered pair, then
    D^-1/2 A D^-1/2 with D the weighted degree (zero rows stay zero)."""
    n = 1 << scale
    src, dst = rmat_edges(scale, 8 * n, seed)
    A = edges_to_csr(n, n, src, dst, symmetrize=True)
    del src, dst
    val = np.empty(A.nnz, dtype=np.float32)
    _load().synth_sym_lognormal(seed, n, _p(A.row_ptr), _p(A.col_idx), int(normalise), _p(val))
    A.values = val
    return A


def chunglu_size(g: int, seed: int = 0, nmin=1e3, nmax=2e5, dmin=8.0, dmax=32.0):
    d = np.zeros(1, dtype=np.float64)
    n = _load().synth_chunglu_size(seed, g, nmin, nmax, dmin, dmax, _p(d))
    return int(n), float(d[0])


def chunglu_csr(g: int, seed: int = 0, gamma: float = 2.1, nmin=1e3, nmax=2e5, dmin=8.0,
                dmax=32.0, n: int | None = None, avg_deg: float | None = None) -> CSR:
    """Graph g of a seeded batch of directed Chung-Lu power-law graphs."""
    n0, d0 = chunglu_size(g, seed, nmin, nmax, dmin, dmax)
    n = n0 if n is None else n
    avg_deg = d0 if avg_deg is None else avg_deg
    m = int(round(n * avg_deg))
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    if _load().synth_chunglu_edges(seed, g, n, m, gamma, _p(src), _p(dst)) != 0:
        raise MemoryError("synth_chunglu_edges: allocation failed")
    return edges_to_csr(n, n, src, dst)


def dense(n_rows: int, k: int, seed: int = 0, mode: str = "uniform", row0: int = 0,
          ld: int | None = None, seed2: int = 0) -> np.ndarray:
    """Dense float32 matrix; element (i, j) depends only on (seed, seed2, i, j).
    mode: 'uniform' U[-1,1), 'int' integers 0..7, 'unit' U[0,1)."""
    ld = k if ld is None else ld
    m = {"uniform": 0, "int": 1, "unit": 2}[mode]
    out = np.zeros((n_rows, ld), dtype=np.float32)
    _load().synth_dense_f32(seed, seed2, row0, n_rows, k, ld, m, _p(out))
    return out


def dense_rows(rows, k: int, seed: int = 0, mode: str = "uniform", seed2: int = 0) -> np.ndarray:
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    m = {"uniform": 0, "int": 1, "unit": 2}[mode]
    out = np.empty((len(rows), k), dtype=np.float32)
    _load().synth_dense_rows_f32(seed, seed2, _p(rows), len(rows), k, m, _p(out))
    return out


def sample_rows(n_rows: int, n: int, seed: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _load().synth_sample_rows(seed, n_rows, n, _p(out))
    return out


def permutation(n: int, seed: int = 0) -> np.ndarray:
    """A seeded uniform random permutation of 0..n-1 (uint32)."""
    out = np.empty(n, dtype=np.uint32)
    _load().synth_permutation(seed, n, _p(out))
    return out


def relabel_edges(src, dst, perm) -> None:
    """Map both endpoints of an edge list through perm, in place."""
    assert src.dtype == np.uint32 and dst.dtype == np.uint32 and perm.dtype == np.uint32
    _load().synth_relabel_edges(len(src), _p(src), _p(dst), _p(np.ascontiguousarray(perm)))


def sbm_edges(n: int, n_clusters: int, m: int, p_in: float, seed: int = 0):
    """Stochastic block model edge list: equal clusters of consecutive ids,
    uniform sources, destination inside the source's cluster with probability
    p_in, else uniform outside it."""
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    _load().synth_sbm_edges(seed, n, n_clusters, m, p_in, _p(src), _p(dst))
    return src, dst


def sbm_csr(n: int, n_clusters: int, avg_deg: float, p_in: float, seed: int = 0, permuted: bool = False) -> CSR:
    """SBM graph in CSR (duplicates merged); clustered ids, or ids relabelled
    by a seeded uniform permutation (the unclustered order)."""
    src, dst = sbm_edges(n, n_clusters, int(round(n * avg_deg)), p_in, seed)
    if permuted:
        relabel_edges(src, dst, permutation(n, seed=seed + 1))
    A = edges_to_csr(n, n, src, dst)
    del src, dst
    return A


def rmat_permuted_csr(scale: int, n_edges: int | None = None, seed: int = 0) -> CSR:
    """R-MAT graph with its vertex ids relabelled by a seeded uniform permutation
    (hubs no longer sit at low ids)."""
    n = 1 << scale
    src, dst = rmat_edges(scale, 16 * n if n_edges is None else n_edges, seed)
    relabel_edges(src, dst, permutation(n, seed=seed + 1))
    A = edges_to_csr(n, n, src, dst)
    del src, dst
    return A


def largest_component(A: CSR) -> CSR:
    """The largest connected component of a symmetric graph, vertices kept in
    their original relative order, values carried along (no renormalisation)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    n = A.n_rows
    M = csr_matrix((np.ones(A.nnz, dtype=np.int8), A.col_idx, A.row_ptr), shape=(n, n))
    ncomp, lab = connected_components(M, directed=False)
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    new_id = np.full(n, -1, dtype=np.int64)
    new_id[keep] = np.arange(len(keep))
    deg = np.diff(A.row_ptr)
    rows = np.repeat(np.arange(n), deg)
    sel = (new_id[rows] >= 0) & (new_id[A.col_idx] >= 0)
    r, c = new_id[rows[sel]], new_id[A.col_idx[sel]]
    row_ptr = np.zeros(len(keep) + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    vals = None if A.values is None else A.values[sel].copy()
    return CSR(len(keep), len(keep), row_ptr, c.astype(np.int32), vals)


def sym_rmat_lcc(scale: int, seed: int = 0) -> CSR:
    """Largest connected component of the symmetrised R-MAT graph with
    lognormal pair weights, normalised D^-1/2 A D^-1/2 on the component."""
    A = sym_rmat_csr(scale, seed=seed, normalise=False)
    L = largest_component(A)
    # renormalise on the component (its degrees are unchanged: no edge leaves it)
    deg = np.zeros(L.n_rows)
    rows = np.repeat(np.arange(L.n_rows), np.diff(L.row_ptr))
    np.add.at(deg, rows, L.values.astype(np.float64))
    inv = 1.0 / np.sqrt(deg)
    L.values = (L.values.astype(np.float64) * inv[rows] * inv[L.col_idx]).astype(np.float32)
    return L
