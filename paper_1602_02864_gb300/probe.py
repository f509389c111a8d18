"""ctypes binding of libspmm_probe.so (paper_1602_02864_gb300/diag/spmm_probe.h):
the gather-rate diagnostics the benchmark reports beside the SpMM.  They
are not part of the library's interface."""
from __future__ import annotations

import ctypes
import os

from . import spmm as _sp

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libspmm_probe.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)
_P, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lib.spmm_probe_gather.argtypes = [_i64, _i32, _dp, _dp, _P]
_lib.spmm_probe_gather.restype = ctypes.c_int
_lib.spmm_probe_gather_cols.argtypes = [_P, _i32, _i32, _dp, _dp, _P]
_lib.spmm_probe_gather_cols.restype = ctypes.c_int


def spmm_probe_gather(table_bytes, row_bytes, stream=None):
    """(rows/s, bytes/s) of uniformly random row gathers from a table."""
    r, b = ctypes.c_double(0), ctypes.c_double(0)
    _sp._check(_lib.spmm_probe_gather(int(table_bytes), int(row_bytes), ctypes.byref(r), ctypes.byref(b),
                                      _sp._stream_handle(stream)))
    return r.value, b.value


def spmm_probe_gather_cols(h, transpose, row_bytes, stream=None):
    """(rows/s, bytes/s) of gathering one table row per stored entry of the
    handle's column-index stream."""
    r, b = ctypes.c_double(0), ctypes.c_double(0)
    _sp._check(_lib.spmm_probe_gather_cols(h, int(bool(transpose)), int(row_bytes), ctypes.byref(r),
                                           ctypes.byref(b), _sp._stream_handle(stream)))
    return r.value, b.value
