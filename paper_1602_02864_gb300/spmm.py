"""ctypes binding of libspmm.so (include/spmm.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.  Importing
this module fails loudly if the compiled library is missing -- there is no CPU
fallback.

Functions keep the C names (``spmm_create_csr``, ``spmm_apply``, ...);
``SparseMatrix`` is a small convenience wrapper around a handle that accepts
numpy arrays for A and torch CUDA tensors for X and Y.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspmm.so")

SPMM_F32, SPMM_BF16, SPMM_F16, SPMM_F64 = 0, 1, 2, 3
SPMM_OK = 0
SPMM_ERR_ARG, SPMM_ERR_CUDA, SPMM_ERR_OOM, SPMM_ERR_FORMAT, SPMM_ERR_TIMEOUT, SPMM_ERR_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6)
SPMM_ERR_IO = -7
SPMM_WANT_TRANSPOSE = 0x1
SPMM_HOST_STREAMING = 0x2
SPMM_REORDER = 0x4
SPMM_FILE_DIRECT = 0x8
SPMM_RELABEL = 0x10

_STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_FORMAT", -5: "ERR_TIMEOUT",
           -6: "ERR_UNSUPPORTED", -7: "ERR_IO"}


class SpmmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class spmm_opts(ctypes.Structure):
    _fields_ = [("task_nnz", ctypes.c_int32), ("task_rows", ctypes.c_int32), ("long_row", ctypes.c_int32),
                ("short_max", ctypes.c_int32), ("x_l2_policy", ctypes.c_int32), ("stream_slot_kib", ctypes.c_int32),
                ("debug_fail_block", ctypes.c_int32), ("compensated", ctypes.c_int32),
                ("short_runs", ctypes.c_int32), ("hot_cols", ctypes.c_int32)]


class spmm_tile_desc(ctypes.Structure):
    _fields_ = [("tile_row", ctypes.c_int64), ("tile_col", ctypes.c_int64), ("n_scsr_words", ctypes.c_int64),
                ("n_coo", ctypes.c_int64), ("data", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class spmm_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_rows", "n_cols", "nnz", "n_tasks", "n_split_rows", "n_segments",
                                              "n_tasks_t", "n_split_rows_t", "n_segments_t", "device_bytes")] + [
        ("value_dtype", ctypes.c_int32), ("has_transpose", ctypes.c_int32), ("n_graphs", ctypes.c_int32),
        ("relabelled", ctypes.c_int32), ("walk_eff", ctypes.c_double * 4), ("walk_eff_t", ctypes.c_double * 4),
        ("n_hot", ctypes.c_int64), ("n_hot_t", ctypes.c_int64)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(the library has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_i32, _i64, _u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32

_lib.spmm_create_csr.argtypes = [ctypes.POINTER(_P), _i64, _i64, _i64, _P, _P, _P, ctypes.c_int, _u32,
                                 ctypes.POINTER(spmm_opts), _P]
_lib.spmm_create_csr.restype = ctypes.c_int
_lib.spmm_apply.argtypes = [_P, _P, _i64, _i32, ctypes.c_int, _P, _i64, ctypes.c_int, _i32, _P]
_lib.spmm_apply.restype = ctypes.c_int
_lib.spmm_get_info.argtypes = [_P, ctypes.POINTER(spmm_info)]
_lib.spmm_get_info.restype = ctypes.c_int
_lib.spmm_destroy.argtypes = [_P]
_lib.spmm_destroy.restype = ctypes.c_int
_lib.spmm_sync_status.argtypes = [_P, _P]
_lib.spmm_sync_status.restype = ctypes.c_int
_lib.spmm_debug_wait_timeout.argtypes = [ctypes.c_uint64, _P]
_lib.spmm_debug_wait_timeout.restype = ctypes.c_int
_lib.spmm_plan_tasks.argtypes = [_i64, _P, ctypes.POINTER(spmm_opts), _P, ctypes.POINTER(_i64),
                                 ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
_lib.spmm_plan_tasks.restype = ctypes.c_int
_lib.spmm_plan_walk_eff.argtypes = [_i64, _P, ctypes.POINTER(spmm_opts), ctypes.POINTER(ctypes.c_double)]
_lib.spmm_plan_walk_eff.restype = ctypes.c_int
_lib.spmm_plan_runs.argtypes = [_i64, _P, ctypes.POINTER(spmm_opts), _i32, _P, ctypes.POINTER(_i32)]
_lib.spmm_plan_runs.restype = ctypes.c_int
_lib.spmm_apply_csr_static.argtypes = [_i64, _i64, _i64, _P, _P, _P, ctypes.c_int, _P, _i64, _i64, _P, _i64,
                                       _i32, ctypes.c_int, _P, _i64, _P]
_lib.spmm_apply_csr_static.restype = ctypes.c_int
_lib.spmm_apply_batched.argtypes = [_i32, _P, _P, _P, _P, ctypes.c_int, _i32, _P]
_lib.spmm_apply_batched.restype = ctypes.c_int
_lib.spmm_eigs_filtered.argtypes = [_P, _i32, _i32, _i32, ctypes.c_double, _i32, ctypes.c_double, ctypes.c_int, _P,
                                    _P, _P, _P, _P, _P]
_lib.spmm_eigs_filtered.restype = ctypes.c_int
_lib.spmm_static_status.argtypes = [_P]
_lib.spmm_static_status.restype = ctypes.c_int
_lib.spmm_pagerank.argtypes = [_P, ctypes.c_double, _i32, _P, _P, _P, _P]
_lib.spmm_pagerank.restype = ctypes.c_int
_lib.spmm_create_batched.argtypes = [ctypes.POINTER(_P), _i32, _P, _P, _P, _P, _P, ctypes.c_int, _u32,
                                     ctypes.POINTER(spmm_opts), _P]
_lib.spmm_create_batched.restype = ctypes.c_int
_lib.spmm_nmf.argtypes = [_P, _i32, _i32, _P, _P, ctypes.c_int, ctypes.c_double, _P, _P]
_lib.spmm_nmf.restype = ctypes.c_int
_lib.spmm_eigs.argtypes = [_P, _i32, _i32, _i32, _i32, ctypes.c_double, ctypes.c_int, _P, _P, _P, _P, _P, _P]
_lib.spmm_eigs.restype = ctypes.c_int
_lib.spmm_replan.argtypes = [_P, ctypes.POINTER(spmm_opts), _i32, _P]
_lib.spmm_replan.restype = ctypes.c_int
_lib.spmm_autotune.argtypes = [_P, _i32, ctypes.c_int, _i32, _P, _i32, _i32, ctypes.POINTER(_i32), _P, _P]
_lib.spmm_autotune.restype = ctypes.c_int
_lib.spmm_create_tiles.argtypes = [ctypes.POINTER(_P), _i64, _i64, _i32, _i64, ctypes.POINTER(spmm_tile_desc),
                                   ctypes.c_int, _u32, ctypes.POINTER(spmm_opts), _P]
_lib.spmm_create_tiles.restype = ctypes.c_int
_lib.spmm_svds.argtypes = [_P, _i32, _i32, _i32, _i32, ctypes.c_double, ctypes.c_int, _P, _P, _P, _P, _P, _P]
_lib.spmm_svds.restype = ctypes.c_int
_lib.spmm_vpart_cols.argtypes = [_i64, _i64, _i32, ctypes.c_int, _i64, _P]
_lib.spmm_vpart_cols.restype = ctypes.c_int
_lib.spmm_apply_host.argtypes = [_P, _P, _i64, _i32, ctypes.c_int, _P, _i64, _i32, _i32, _i64, _P, _P]
_lib.spmm_apply_host.restype = ctypes.c_int
_lib.spmm_apply_host_parts.argtypes = [_P, _P, _P, _P, _i32, ctypes.c_int, _i32, _P]
_lib.spmm_apply_host_parts.restype = ctypes.c_int
_lib.spmm_write_csr_file.argtypes = [ctypes.c_char_p, _i64, _i64, _i64, _P, _P, _P, ctypes.c_int]
_lib.spmm_write_csr_file.restype = ctypes.c_int
_lib.spmm_create_file.argtypes = [ctypes.POINTER(_P), ctypes.c_char_p, ctypes.c_uint32, _P, _P]
_lib.spmm_create_file.restype = ctypes.c_int
_lib.spmm_apply_relabelled.argtypes = [_P, _P, _i64, _i32, ctypes.c_int, _P, _i64, ctypes.c_int, _i32, _P]
_lib.spmm_apply_relabelled.restype = ctypes.c_int
_lib.spmm_relabel_rows.argtypes = [_P, _P, _i64, _i32, ctypes.c_int, _P, _i64, _i32, _P]
_lib.spmm_relabel_rows.restype = ctypes.c_int
_lib.spmm_get_relabel.argtypes = [_P, _P]
_lib.spmm_get_relabel.restype = ctypes.c_int
_lib.spmm_relabel_order.argtypes = [_i64, _P, _P, _P]
_lib.spmm_relabel_order.restype = ctypes.c_int
_lib.spmm_last_error.argtypes = []
_lib.spmm_last_error.restype = ctypes.c_char_p


def lib() -> ctypes.CDLL:
    return _lib


def spmm_last_error() -> str:
    return _lib.spmm_last_error().decode()


def _check(rc: int):
    if rc != SPMM_OK:
        raise SpmmError(rc, spmm_last_error())


def _ptr(a) -> _P:
    if a is None:
        return _P(0)
    if isinstance(a, np.ndarray):
        return _P(a.ctypes.data)
    return _P(a.data_ptr())   # torch tensor


def _torch_dtype_code(t) -> int:
    import torch
    return {torch.float32: SPMM_F32, torch.bfloat16: SPMM_BF16, torch.float16: SPMM_F16,
            torch.float64: SPMM_F64}[t.dtype]


def _np_dtype_code(a) -> int:
    if a.dtype == np.float32:
        return SPMM_F32
    if a.dtype == np.float16:
        return SPMM_F16
    raise TypeError("host values must be float32 or float16 numpy arrays (bf16: pass a torch CPU tensor)")


def _stream_handle(stream) -> _P:
    if stream is None:
        import torch
        return _P(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _P(stream)
    return _P(stream.cuda_stream)


def spmm_create_csr(n_rows, n_cols, row_ptr, col_idx, values=None, flags=0, opts: spmm_opts | None = None,
                    stream=None) -> _P:
    """Returns a handle (c_void_p).  row_ptr/col_idx/values are host arrays."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    vtype = SPMM_F32
    vptr = _P(0)
    vkeep = None
    if values is not None:
        try:
            import torch
            if isinstance(values, torch.Tensor):
                vkeep = values.contiguous().cpu()
                vtype = _torch_dtype_code(vkeep)
                vptr = _P(vkeep.data_ptr())
        except ImportError:  # pragma: no cover
            pass
        if vkeep is None:
            vkeep = np.ascontiguousarray(values)
            vtype = _np_dtype_code(vkeep)
            vptr = _P(vkeep.ctypes.data)
    h = _P(0)
    _check(_lib.spmm_create_csr(ctypes.byref(h), int(n_rows), int(n_cols), int(rp[-1]) if len(rp) else 0,
                                _ptr(rp), _ptr(ci), vptr, vtype, int(flags),
                                ctypes.byref(opts) if opts is not None else None, _stream_handle(stream)))
    return h


def spmm_apply(h, X, ldx, k, xtype, Y, ldy, transpose=0, stream=None):
    _check(_lib.spmm_apply(h, _ptr(X), int(ldx), int(k), int(xtype), _ptr(Y), int(ldy), SPMM_F32,
                           int(transpose), _stream_handle(stream)))


def spmm_apply_relabelled(h, X, ldx, k, xtype, Y, ldy, transpose=0, stream=None):
    """spmm_apply with X and Y in the handle's vertex order (SPMM_RELABEL)."""
    _check(_lib.spmm_apply_relabelled(h, _ptr(X), int(ldx), int(k), int(xtype), _ptr(Y), int(ldy), SPMM_F32,
                                      int(transpose), _stream_handle(stream)))


def spmm_relabel_rows(h, src, dst, to_handle_order, stream=None):
    """dst = src's rows in the handle's order (to_handle_order) or back in
    the input order; src, dst 2-D CUDA tensors of one dtype, unit column
    stride."""
    if src.dim() != 2 or dst.dim() != 2 or src.stride(1) != 1 or dst.stride(1) != 1:
        raise ValueError("src and dst must be 2-D with unit column stride")
    if src.dtype != dst.dtype or src.shape != dst.shape:
        raise ValueError("src and dst must have one dtype and shape")
    _check(_lib.spmm_relabel_rows(h, _ptr(src), int(src.stride(0)), int(src.shape[1]), _torch_dtype_code(src),
                                  _ptr(dst), int(dst.stride(0)), int(bool(to_handle_order)), _stream_handle(stream)))


def spmm_get_relabel(h, n) -> np.ndarray:
    """old_of_new of the handle (the identity without SPMM_RELABEL)."""
    out = np.empty(int(n), dtype=np.int32)
    _check(_lib.spmm_get_relabel(h, _P(out.ctypes.data)))
    return out


def spmm_relabel_order(n, row_ptr, col_idx) -> np.ndarray:
    """Host-only: the vertex order SPMM_RELABEL gives an n x n CSR matrix
    (old_of_new: decreasing row + column entry count, ties by vertex)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    out = np.empty(int(n), dtype=np.int32)
    _check(_lib.spmm_relabel_order(int(n), _P(rp.ctypes.data), _P(ci.ctypes.data) if ci.size else None,
                                   _P(out.ctypes.data)))
    return out


def spmm_apply_batched(handles, Xs, Ys, transpose=False, stream=None):
    """Y_i = A_i X_i (or A_i^T X_i) for lists of handles, contiguous CUDA
    tensors X_i (one dtype) and float32 CUDA tensors Y_i (see spmm.h)."""
    n = len(handles)
    if len(Xs) != n or len(Ys) != n or n == 0:
        raise ValueError("need as many X and Y tensors as handles (at least one)")
    xtype = _torch_dtype_code(Xs[0])
    for X, Y in zip(Xs, Ys):
        if _torch_dtype_code(X) != xtype or not X.is_contiguous() or not Y.is_contiguous() \
                or X.shape[1] != Y.shape[1]:
            raise ValueError("X tensors of one dtype, X and Y contiguous with equal columns")
    hs = (_P * n)(*[h.value if isinstance(h, _P) else h for h in handles])
    xs = (_P * n)(*[X.data_ptr() for X in Xs])
    ys = (_P * n)(*[Y.data_ptr() for Y in Ys])
    ks = (_i32 * n)(*[int(X.shape[1]) for X in Xs])
    _check(_lib.spmm_apply_batched(n, hs, xs, ys, ks, xtype, int(bool(transpose)), _stream_handle(stream)))


def spmm_sync_status(h, stream=None):
    """Raise SpmmError(SPMM_ERR_TIMEOUT) if a device-side wait ran out."""
    _check(_lib.spmm_sync_status(h, _stream_handle(stream)))


def spmm_debug_wait_timeout(wait_ns: int, stream=None) -> int:
    """Run the never-completing bounded wait; returns the status code."""
    return _lib.spmm_debug_wait_timeout(int(wait_ns), _stream_handle(stream))


def spmm_plan_tasks(row_ptr, opts: spmm_opts | None = None):
    """Host-only plan of a row-pointer array: returns (tasks int32 [n+1, 4],
    n_split_rows, n_segments)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    n_rows = len(rp) - 1
    nt, ns, nseg = _i64(0), _i64(0), _i64(0)
    o = ctypes.byref(opts) if opts is not None else None
    _check(_lib.spmm_plan_tasks(n_rows, _ptr(rp), o, None, ctypes.byref(nt), ctypes.byref(ns), ctypes.byref(nseg)))
    tasks = np.zeros((nt.value + 1, 4), dtype=np.int32)
    _check(_lib.spmm_plan_tasks(n_rows, _ptr(rp), o, _ptr(tasks), ctypes.byref(nt), ctypes.byref(ns),
                                ctypes.byref(nseg)))
    return tasks, ns.value, nseg.value


def spmm_plan_runs(row_ptr, max_runs=4, opts: spmm_opts | None = None) -> np.ndarray:
    """Host-only runs of whole tasks of the plan (the host-buffer calls use
    4): int64 [n_runs, 6] rows {t0, t1, r0, r1, s0, s1}."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = np.zeros((max(int(max_runs), 1), 6), dtype=np.int64)
    n = ctypes.c_int32(0)
    o = ctypes.byref(opts) if opts is not None else None
    _check(_lib.spmm_plan_runs(len(rp) - 1, _ptr(rp), o, int(max_runs), _ptr(out), ctypes.byref(n)))
    return out[:n.value]


def spmm_plan_walk_eff(row_ptr, opts: spmm_opts | None = None) -> list[float]:
    """Host-only row-walk efficiency of the plan for 2, 4, 8, 16 lane groups."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = (ctypes.c_double * 4)()
    o = ctypes.byref(opts) if opts is not None else None
    _check(_lib.spmm_plan_walk_eff(len(rp) - 1, _ptr(rp), o, out))
    return list(out)


def spmm_apply_csr_static(n_rows, n_cols, nnz, row_ptr, col_idx, values, vtype, tasks, n_tasks, n_segments, X,
                          ldx, k, xtype, Y, ldy, stream=None):
    """Allocation-free Y = A X on caller-owned device buffers (see spmm.h)."""
    _check(_lib.spmm_apply_csr_static(int(n_rows), int(n_cols), int(nnz), _ptr(row_ptr), _ptr(col_idx),
                                      _ptr(values), int(vtype), _ptr(tasks), int(n_tasks), int(n_segments), _ptr(X),
                                      int(ldx), int(k), int(xtype), _ptr(Y), int(ldy), _stream_handle(stream)))


def spmm_static_status(stream=None):
    """Raise SpmmError if the last spmm_apply_csr_static call on this device
    timed out or named partial-sum slots beyond the static scratch."""
    _check(_lib.spmm_static_status(_stream_handle(stream)))


def spmm_pagerank(h, damping, iters, x, x0=None, stream=None) -> np.ndarray:
    """PageRank into the float32 CUDA tensor x; returns the FP64 residuals."""
    res = np.zeros(max(int(iters), 1), dtype=np.float64)
    _check(_lib.spmm_pagerank(h, float(damping), int(iters), _ptr(x), _ptr(x0), _P(res.ctypes.data),
                              _stream_handle(stream)))
    return res[:int(iters)]


def spmm_create_batched(graphs, flags=0, opts: spmm_opts | None = None, stream=None, weighted=True) -> _P:
    """One block-diagonal handle for a list of host CSR graphs (objects with
    n_rows, n_cols, row_ptr, col_idx, values)."""
    n = len(graphs)
    nr = np.array([g.n_rows for g in graphs], dtype=np.int64)
    nc = np.array([g.n_cols for g in graphs], dtype=np.int64)
    rps = [np.ascontiguousarray(g.row_ptr, dtype=np.int64) for g in graphs]
    cis = [np.ascontiguousarray(g.col_idx, dtype=np.int32) for g in graphs]
    rp_arr = (_P * n)(*[_P(a.ctypes.data) for a in rps])
    ci_arr = (_P * n)(*[_P(a.ctypes.data) for a in cis])
    use_vals = weighted and all(g.values is not None for g in graphs)
    vals = [np.ascontiguousarray(g.values, dtype=np.float32) for g in graphs] if use_vals else None
    v_arr = (_P * n)(*[_P(a.ctypes.data) for a in vals]) if use_vals else None
    h = _P(0)
    _check(_lib.spmm_create_batched(ctypes.byref(h), n, _ptr(nr), _ptr(nc), rp_arr, ci_arr, v_arr, SPMM_F32,
                                    int(flags), ctypes.byref(opts) if opts is not None else None,
                                    _stream_handle(stream)))
    return h


def spmm_nmf(h, k, steps, W, Ht, ftype=SPMM_F32, eps=1e-12, n_graphs=1, stream=None) -> np.ndarray:
    """NMF in place on float32 CUDA tensors W, Ht; returns objective
    [n_graphs, steps+1] (FP64)."""
    obj = np.zeros((n_graphs, int(steps) + 1), dtype=np.float64)
    _check(_lib.spmm_nmf(h, int(k), int(steps), _ptr(W), _ptr(Ht), int(ftype), float(eps), _P(obj.ctypes.data),
                         _stream_handle(stream)))
    return obj


def spmm_eigs(h, nev, V0, block=16, max_basis=64, max_restarts=100, tol=1e-6, xtype=SPMM_F32, evecs=None,
              stream=None):
    """Top-nev eigenpairs; V0 is a float64 CUDA tensor (n x block).  Returns
    (evals, residuals, restarts)."""
    ev = np.zeros(nev, dtype=np.float64)
    rs = np.zeros(nev, dtype=np.float64)
    nr = ctypes.c_int32(0)
    _check(_lib.spmm_eigs(h, int(nev), int(block), int(max_basis), int(max_restarts), float(tol), int(xtype),
                          _ptr(V0), _P(ev.ctypes.data), _ptr(evecs), _P(rs.ctypes.data), ctypes.byref(nr),
                          _stream_handle(stream)))
    return ev, rs, nr.value


def spmm_eigs_filtered(h, nev, V0, degree=20, lower=-1.0, max_iters=100, tol=1e-6, xtype=SPMM_F32, evecs=None,
                       stream=None):
    """Top-nev eigenpairs by Chebyshev-filtered subspace iteration; V0 is a
    float64 CUDA tensor (n x block).  Returns (evals, residuals, iterations)."""
    ev = np.zeros(nev, dtype=np.float64)
    rs = np.zeros(nev, dtype=np.float64)
    ni = ctypes.c_int32(0)
    _check(_lib.spmm_eigs_filtered(h, int(nev), int(V0.shape[1]), int(degree), float(lower), int(max_iters),
                                   float(tol), int(xtype), _ptr(V0), _P(ev.ctypes.data), _ptr(evecs),
                                   _P(rs.ctypes.data), ctypes.byref(ni), _stream_handle(stream)))
    return ev, rs, ni.value


def spmm_replan(h, opts: spmm_opts | None = None, transpose=0, stream=None):
    _check(_lib.spmm_replan(h, ctypes.byref(opts) if opts is not None else None, int(transpose),
                            _stream_handle(stream)))


BUILTIN_GRID = [dict(task_nnz=tn, short_max=sm, long_row=512, x_l2_policy=pol)
                for tn in (128, 256, 512) for sm in (7, 15, 31, 63) for pol in (1, 2) if sm < tn]


def spmm_autotune(h, k, xtype=SPMM_F32, transpose=0, candidates=None, reps=3, stream=None):
    """Returns (best index, times_ms, candidate list as dicts); the handle is
    left on the best plan."""
    if candidates is None:
        cands, arr, n = BUILTIN_GRID, None, len(BUILTIN_GRID)
    else:
        cands = list(candidates)
        n = len(cands)
        arr = (spmm_opts * n)(*[spmm_opts(**c) for c in cands])
    times = np.zeros(n, dtype=np.float64)
    best = _i32(-1)
    _check(_lib.spmm_autotune(h, int(k), int(xtype), int(transpose), arr, n if arr is not None else 0, int(reps),
                              ctypes.byref(best), _P(times.ctypes.data), _stream_handle(stream)))
    return best.value, times, cands


def spmm_create_tiles(n_rows, n_cols, tile, tiles, flags=0, opts: spmm_opts | None = None, stream=None) -> _P:
    """tiles: list of (tile_row, tile_col, scsr_words uint16, coo_pairs uint16 [n,2], values float32 or None)."""
    keep = []
    arr = (spmm_tile_desc * max(len(tiles), 1))()
    for i, (tr, tc, scsr, coo, vals) in enumerate(tiles):
        data = np.ascontiguousarray(np.concatenate([np.asarray(scsr, np.uint16), np.asarray(coo, np.uint16).ravel()]))
        v = None if vals is None else np.ascontiguousarray(vals, dtype=np.float32)
        keep += [data, v]
        arr[i] = spmm_tile_desc(tr, tc, len(scsr), len(coo), data.ctypes.data, None if v is None else v.ctypes.data)
    h = _P(0)
    _check(_lib.spmm_create_tiles(ctypes.byref(h), int(n_rows), int(n_cols), int(tile), len(tiles), arr, SPMM_F32,
                                  int(flags), ctypes.byref(opts) if opts is not None else None,
                                  _stream_handle(stream)))
    return h


def spmm_write_csr_file(path, A, values=None) -> None:
    """Write host CSR ``A`` (synth.CSR-like; values float32/bf16-as-uint16/float16
    or None) to ``path`` in the library's file layout (host only)."""
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    vals = A.values if values is None else values
    vt, vp = SPMM_F32, None
    if vals is not None:
        vals = np.ascontiguousarray(vals)
        vt = {np.dtype(np.float32): SPMM_F32, np.dtype(np.float16): SPMM_F16,
              np.dtype(np.uint16): SPMM_BF16}[vals.dtype]
        vp = _P(vals.ctypes.data)
    _check(_lib.spmm_write_csr_file(os.fsencode(path), int(A.n_rows), int(A.n_cols), int(rp[-1]),
                                    _P(rp.ctypes.data), _P(ci.ctypes.data), vp, vt))


def spmm_create_file(path, direct=False, opts=None, stream=None):
    h = _P(0)
    _check(_lib.spmm_create_file(ctypes.byref(h), os.fsencode(path), SPMM_FILE_DIRECT if direct else 0,
                                 ctypes.byref(opts) if opts is not None else None, _stream_handle(stream)))
    return h


def spmm_vpart_cols(n_in, n_out, p, xtype, budget_bytes) -> int:
    """Column-group width for vertical partitions under a device budget (host only)."""
    c = ctypes.c_int32(0)
    _check(_lib.spmm_vpart_cols(int(n_in), int(n_out), int(p), int(xtype), int(budget_bytes), ctypes.byref(c)))
    return c.value


def spmm_apply_host(h, X, Y, transpose=False, group_cols=0, budget_bytes=0, stream=None) -> int:
    """Y = A X (or A^T X) for host numpy (or pinned CPU torch) matrices, in
    vertical partitions; returns the number of column groups."""
    xt, ldx, p, xp = _host_matrix(X)
    yt, ldy, py, yp = _host_matrix(Y)
    if yt != SPMM_F32 or py != p:
        raise ValueError("Y must be float32 with the same number of columns as X")
    g = ctypes.c_int32(0)
    _check(_lib.spmm_apply_host(h, xp, ldx, p, xt, yp, ldy, int(bool(transpose)), int(group_cols),
                                int(budget_bytes), ctypes.byref(g), _stream_handle(stream)))
    return g.value


def spmm_apply_host_parts(h, X_parts, Y_parts, transpose=False, stream=None):
    """Y = A X for a dense matrix stored as contiguous row-major vertical
    partitions (lists of host matrices, part i of X and Y with equal columns)."""
    if len(X_parts) != len(Y_parts) or not X_parts:
        raise ValueError("need as many Y parts as X parts (at least one)")
    xs, ys, cols, xtype = [], [], [], None
    for Xp, Yp in zip(X_parts, Y_parts):
        xt, ldx, w, xp = _host_matrix(Xp)
        yt, ldy, wy, yp = _host_matrix(Yp)
        if ldx != w or ldy != wy or yt != SPMM_F32 or wy != w or (xtype is not None and xt != xtype):
            raise ValueError("parts must be contiguous, Y float32, same columns, one X dtype")
        xtype = xt
        xs.append(xp.value)
        ys.append(yp.value)
        cols.append(w)
    n = len(cols)
    xa, ya, ca = (ctypes.c_void_p * n)(*xs), (ctypes.c_void_p * n)(*ys), (ctypes.c_int32 * n)(*cols)
    _check(_lib.spmm_apply_host_parts(h, xa, ya, ca, n, xtype, int(bool(transpose)), _stream_handle(stream)))


def _host_matrix(M):
    """(dtype code, leading dimension, columns, pointer) of a row-major host
    matrix: a 2-D numpy array or CPU torch tensor with unit column stride."""
    if isinstance(M, np.ndarray):
        if M.ndim != 2 or M.strides[1] != M.itemsize or M.strides[0] % M.itemsize:
            raise ValueError("host matrix must be 2-D with unit column stride")
        code = {np.dtype(np.float32): SPMM_F32, np.dtype(np.float16): SPMM_F16}.get(M.dtype)
        if code is None:
            raise ValueError(f"unsupported host dtype {M.dtype}")
        return code, M.strides[0] // M.itemsize, M.shape[1], _P(M.ctypes.data)
    import torch
    if M.device.type != "cpu" or M.dim() != 2 or M.stride(1) != 1:
        raise ValueError("host tensor must be a 2-D CPU tensor with unit column stride")
    code = {torch.float32: SPMM_F32, torch.bfloat16: SPMM_BF16, torch.float16: SPMM_F16}.get(M.dtype)
    if code is None:
        raise ValueError(f"unsupported host dtype {M.dtype}")
    return code, M.stride(0), M.shape[1], _P(M.data_ptr())


def spmm_svds(h, nsv, V0, block=16, max_basis=64, max_restarts=100, tol=1e-6, xtype=SPMM_F32, right_vecs=None,
              stream=None):
    """Top-nsv singular values of A (via A^T A): (svals, residuals, restarts)."""
    sv = np.zeros(nsv, dtype=np.float64)
    rs = np.zeros(nsv, dtype=np.float64)
    nr = ctypes.c_int32(0)
    _check(_lib.spmm_svds(h, int(nsv), int(block), int(max_basis), int(max_restarts), float(tol), int(xtype),
                          _ptr(V0), _P(sv.ctypes.data), _ptr(right_vecs), _P(rs.ctypes.data), ctypes.byref(nr),
                          _stream_handle(stream)))
    return sv, rs, nr.value


def spmm_get_info(h) -> dict:
    info = spmm_info()
    _check(_lib.spmm_get_info(h, ctypes.byref(info)))
    out = {name: getattr(info, name) for name, _ in info._fields_}
    out["walk_eff"] = list(info.walk_eff)
    out["walk_eff_t"] = list(info.walk_eff_t)
    return out


def spmm_destroy(h):
    _check(_lib.spmm_destroy(h))


class SparseMatrix:
    """A sparse matrix resident in HBM: ``SparseMatrix(A_csr).apply(X)``."""

    def __init__(self, n_rows, n_cols, row_ptr, col_idx, values=None, transpose=False,
                 opts: spmm_opts | None = None, stream=None, streaming=False, reorder=False, relabel=False):
        self.n_rows, self.n_cols = int(n_rows), int(n_cols)
        flags = ((SPMM_WANT_TRANSPOSE if transpose else 0) | (SPMM_HOST_STREAMING if streaming else 0)
                 | (SPMM_REORDER if reorder else 0) | (SPMM_RELABEL if relabel else 0))
        if streaming:
            # the library borrows these host arrays until close(): keep them alive
            self._borrowed = (np.ascontiguousarray(row_ptr, dtype=np.int64),
                              np.ascontiguousarray(col_idx, dtype=np.int32),
                              None if values is None else np.ascontiguousarray(values))
            row_ptr, col_idx, values = self._borrowed
        self.handle = spmm_create_csr(n_rows, n_cols, row_ptr, col_idx, values, flags, opts, stream)

    @classmethod
    def from_tiles(cls, n_rows, n_cols, tile, tiles, transpose=False, opts: spmm_opts | None = None, stream=None):
        """Handle from SCSR + COO tiles (see spmm_create_tiles)."""
        self = cls.__new__(cls)
        self.n_rows, self.n_cols = int(n_rows), int(n_cols)
        self.handle = spmm_create_tiles(n_rows, n_cols, tile, tiles, SPMM_WANT_TRANSPOSE if transpose else 0, opts,
                                        stream)
        return self

    @classmethod
    def from_file(cls, path, n_rows, n_cols, direct=False, opts: spmm_opts | None = None, stream=None):
        """Handle whose matrix stays in a file written by spmm_write_csr_file."""
        self = cls.__new__(cls)
        self.n_rows, self.n_cols = int(n_rows), int(n_cols)
        self.handle = spmm_create_file(path, direct, opts, stream)
        return self

    @classmethod
    def batched(cls, graphs, transpose=False, weighted=True, opts: spmm_opts | None = None, stream=None,
                reorder=False, relabel=False):
        """Block-diagonal handle over a list of graphs (one launch per apply)."""
        self = cls.__new__(cls)
        self.n_rows = int(sum(g.n_rows for g in graphs))
        self.n_cols = int(sum(g.n_cols for g in graphs))
        flags = ((SPMM_WANT_TRANSPOSE if transpose else 0) | (SPMM_REORDER if reorder else 0)
                 | (SPMM_RELABEL if relabel else 0))
        self.handle = spmm_create_batched(graphs, flags, opts, stream, weighted)
        return self

    def apply_host(self, X, Y, transpose=False, group_cols=0, budget_bytes=0, stream=None) -> int:
        """Y = A X with host X, Y (vertical partitions); returns the group count."""
        return spmm_apply_host(self.handle, X, Y, transpose, group_cols, budget_bytes, stream)

    def apply_host_parts(self, X_parts, Y_parts, transpose=False, stream=None) -> None:
        """Y = A X for contiguous row-major vertical partitions (host)."""
        spmm_apply_host_parts(self.handle, X_parts, Y_parts, transpose, stream)

    def svds(self, nsv, V0, **kw):
        """Top-nsv singular values (needs transpose=True): (svals, residuals, restarts)."""
        return spmm_svds(self.handle, nsv, V0, **kw)

    def eigs(self, nev, V0, **kw):
        """Top-nev eigenpairs of a symmetric matrix: (evals, residuals, restarts)."""
        return spmm_eigs(self.handle, nev, V0, **kw)

    def eigs_filtered(self, nev, V0, **kw):
        """Top-nev eigenpairs by Chebyshev-filtered subspace iteration:
        (evals, residuals, iterations)."""
        return spmm_eigs_filtered(self.handle, nev, V0, **kw)

    def nmf(self, k, steps, W, Ht, ftype=SPMM_F32, eps=1e-12, stream=None):
        """NMF in place on W (rows x k) and Ht (cols x k); returns objective."""
        return spmm_nmf(self.handle, k, steps, W, Ht, ftype, eps, self.info()["n_graphs"], stream)

    @classmethod
    def from_csr(cls, A, transpose=False, values=None, **kw):
        vals = A.values if values is None else values
        return cls(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vals, transpose=transpose, **kw)

    def apply(self, X, transpose=False, Y=None, stream=None):
        """Y = A X (or A^T X).  X: 2-D CUDA tensor (float32/bfloat16/float16)
        with unit column stride; returns / fills a float32 CUDA tensor."""
        import torch
        if X.dim() != 2 or X.stride(1) != 1:
            raise ValueError("X must be 2-D with unit column stride")
        k = X.shape[1]
        out_rows = self.n_cols if transpose else self.n_rows
        if Y is None:
            Y = torch.empty((out_rows, k), dtype=torch.float32, device=X.device)
        if Y.dim() != 2 or Y.stride(1) != 1 or Y.dtype != torch.float32:
            raise ValueError("Y must be a 2-D float32 tensor with unit column stride")
        spmm_apply(self.handle, X, X.stride(0), k, _torch_dtype_code(X), Y, Y.stride(0), int(transpose), stream)
        return Y

    def apply_relabelled(self, X, transpose=False, Y=None, stream=None):
        """apply() with X and Y in the handle's vertex order (SPMM_RELABEL)."""
        import torch
        if X.dim() != 2 or X.stride(1) != 1:
            raise ValueError("X must be 2-D with unit column stride")
        k = X.shape[1]
        out_rows = self.n_cols if transpose else self.n_rows
        if Y is None:
            Y = torch.empty((out_rows, k), dtype=torch.float32, device=X.device)
        if Y.dim() != 2 or Y.stride(1) != 1 or Y.dtype != torch.float32:
            raise ValueError("Y must be a 2-D float32 tensor with unit column stride")
        spmm_apply_relabelled(self.handle, X, X.stride(0), k, _torch_dtype_code(X), Y, Y.stride(0), int(transpose),
                              stream)
        return Y

    def to_handle_order(self, M, out=None, stream=None):
        """M's rows (input vertex order) in the handle's order."""
        import torch
        out = torch.empty_like(M) if out is None else out
        spmm_relabel_rows(self.handle, M, out, True, stream)
        return out

    def to_input_order(self, M, out=None, stream=None):
        """M's rows (handle's vertex order) back in the input order."""
        import torch
        out = torch.empty_like(M) if out is None else out
        spmm_relabel_rows(self.handle, M, out, False, stream)
        return out

    def vertex_order(self) -> np.ndarray:
        """old_of_new: the input vertex that is each vertex of the handle."""
        return spmm_get_relabel(self.handle, self.n_rows)

    def info(self) -> dict:
        return spmm_get_info(self.handle)

    def sync_status(self, stream=None):
        spmm_sync_status(self.handle, stream)

    def pagerank(self, damping=0.85, iters=30, x0=None, x=None, stream=None):
        """Returns (x, residuals) -- x a float32 CUDA tensor of the ranks."""
        import torch
        if x is None:
            x = torch.empty(self.n_rows, dtype=torch.float32, device="cuda")
        res = spmm_pagerank(self.handle, damping, iters, x, x0, stream)
        return x, res

    def close(self):
        if self.handle is not None and self.handle.value:
            spmm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
