"""The allocation-free entry point, spmm_apply_csr_static, for callers that
cannot call cudaMalloc (they own every device buffer, so they cannot create a
handle).  It must give the same result as spmm_apply on a handle, call after
call, with its scratch in the library's static device array.  This file sorts
last so a run that stops at the first failure has run everything else."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import abs_product, assert_close_rel

pytestmark = pytest.mark.gpu


def _device_inputs(A, torch):
    """Caller-owned device copies, padded past their ends as the entry point
    requires (its aligned bulk copies may read up to 32 bytes beyond)."""
    rp = torch.zeros(len(A.row_ptr) + 2, dtype=torch.int64, device="cuda")
    rp[:len(A.row_ptr)] = torch.from_numpy(A.row_ptr)
    ci = torch.zeros(A.nnz + 8, dtype=torch.int32, device="cuda")
    ci[:A.nnz] = torch.from_numpy(A.col_idx)
    va = torch.zeros(A.nnz + 8, dtype=torch.float32, device="cuda")
    va[:A.nnz] = torch.from_numpy(A.values)
    return rp, ci, va


def test_static_scratch_entry_matches_apply_twice():
    import torch
    from paper_1602_02864_gb300 import spmm as sp

    A = synth.rmat_csr(14, seed=5, weighted=True)
    tasks, n_split, n_seg = sp.spmm_plan_tasks(A.row_ptr)
    assert n_split > 0 and 0 < n_seg <= 16384          # hub rows use the static scratch
    rp, ci, va = _device_inputs(A, torch)
    tk = torch.from_numpy(tasks).cuda()
    h = sp.SparseMatrix.from_csr(A)
    try:
        for k, seed in ((8, 1), (33, 2)):                # two calls in a row, different shapes
            X = torch.from_numpy(synth.dense(A.n_cols, k, seed=seed)).cuda()
            Yref = h.apply(X)
            Y = torch.full((A.n_rows, k), float("nan"), device="cuda")
            sp.spmm_apply_csr_static(A.n_rows, A.n_cols, A.nnz, rp, ci, va, sp.SPMM_F32, tk, len(tasks) - 1, n_seg,
                                     X, X.stride(0), k, sp.SPMM_F32, Y, Y.stride(0))
            torch.cuda.synchronize()
            Xh = X.cpu().numpy().astype(np.float64)
            scale = abs_product(A, Xh)
            assert_close_rel(Y.cpu().numpy(), Yref.cpu().numpy().astype(np.float64), scale, 1e-5,
                             f"static vs handle k={k}")
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xh)
            assert_close_rel(Y.cpu().numpy(), ref, scale, 1e-5, f"static vs oracle k={k}")
    finally:
        h.close()


def test_static_scratch_entry_rejects_oversized_plan():
    import torch
    from paper_1602_02864_gb300 import spmm as sp

    A = synth.rmat_csr(16, seed=1)
    o = sp.spmm_opts(task_nnz=32, long_row=32, short_max=8)
    tasks, _, n_seg = sp.spmm_plan_tasks(A.row_ptr, o)
    assert n_seg > 16384
    X = torch.zeros((A.n_cols, 4), device="cuda")
    Y = torch.zeros((A.n_rows, 4), device="cuda")
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_apply_csr_static(A.n_rows, A.n_cols, A.nnz, None, None, None, sp.SPMM_F32, None, len(tasks) - 1,
                                 n_seg, X, 4, 4, sp.SPMM_F32, Y, 4)
    assert e.value.status == sp.SPMM_ERR_ARG and "16384" in str(e.value)
