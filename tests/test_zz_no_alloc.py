"""The allocation-free entry point, spmm_apply_csr_static, for callers that
cannot call cudaMalloc (they own every device buffer, so they cannot create a
handle).  It must give the same result as spmm_apply on a handle, call after
call, with its scratch in the library's static device array, for every lane
geometry the handle path uses (one lane per row at k = 1 and 2, two lanes
for 16-byte rows, lane groups, two column chunks), for 16-bit X and values,
and bit for bit on a pattern matrix with small-integer X.  This file sorts
last so a run that stops at the first failure has run everything else."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import abs_product, assert_close_rel, rounded_host

pytestmark = pytest.mark.gpu


def _device_inputs(A, torch, vdtype=None):
    """Caller-owned device copies, padded past their ends as the entry point
    requires (its aligned bulk copies may read up to 32 bytes beyond)."""
    rp = torch.zeros(len(A.row_ptr) + 2, dtype=torch.int64, device="cuda")
    rp[:len(A.row_ptr)] = torch.from_numpy(A.row_ptr)
    ci = torch.zeros(A.nnz + 8, dtype=torch.int32, device="cuda")
    ci[:A.nnz] = torch.from_numpy(A.col_idx)
    va = None
    if A.values is not None:
        va = torch.zeros(A.nnz + 16, dtype=vdtype or torch.float32, device="cuda")
        va[:A.nnz] = torch.from_numpy(A.values).to(va.dtype)
    return rp, ci, va


def _static(sp, A, rp, ci, va, vtype, tk, n_seg, X, k, xtype, Y):
    sp.spmm_apply_csr_static(A.n_rows, A.n_cols, A.nnz, rp, ci, va, vtype, tk, tk.shape[0] - 1, n_seg,
                             X, X.stride(0), k, xtype, Y, Y.stride(0))


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
        # two calls in a row per shape; k = 4 puts a 16-byte row on two lanes,
        # k = 1 and 2 on one lane, k = 33 on two column chunks
        for k, seed in ((8, 1), (33, 2), (1, 3), (4, 4), (2, 5)):
            X = torch.from_numpy(synth.dense(A.n_cols, k, seed=seed)).cuda()
            Yref = h.apply(X)
            Xh = X.cpu().numpy().astype(np.float64)
            scale = abs_product(A, Xh)
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xh)
            for call in range(2):
                Y = torch.full((A.n_rows, k), float("nan"), device="cuda")
                _static(sp, A, rp, ci, va, sp.SPMM_F32, tk, n_seg, X, k, sp.SPMM_F32, Y)
                sp.spmm_static_status()
                assert_close_rel(Y.cpu().numpy(), Yref.cpu().numpy().astype(np.float64), scale, 1e-5,
                                 f"static vs handle k={k} call {call}")
                assert_close_rel(Y.cpu().numpy(), ref, scale, 1e-5, f"static vs oracle k={k} call {call}")
    finally:
        h.close()


@pytest.mark.parametrize("xname,k", [("bf16", 8), ("bf16", 1), ("f16", 2), ("f16", 16), ("bf16", 64)])
def test_static_scratch_entry_16bit_x(xname, k):
    """16-bit X (one lane per row at k = 1, 2; two lanes of 8 bytes for a
    16-byte row at k = 8) with float32 values, against the FP64 oracle on the
    rounded X at the 16-bit tolerance, and against the handle."""
    import torch
    from paper_1602_02864_gb300 import spmm as sp

    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[xname]
    code = {"bf16": sp.SPMM_BF16, "f16": sp.SPMM_F16}[xname]
    A = synth.rmat_csr(13, seed=6, weighted=True)
    tasks, _, n_seg = sp.spmm_plan_tasks(A.row_ptr)
    rp, ci, va = _device_inputs(A, torch)
    tk = torch.from_numpy(tasks).cuda()
    X = torch.from_numpy(synth.dense(A.n_cols, k, seed=11)).cuda().to(tdt)
    Xr = rounded_host(X)
    scale = abs_product(A, Xr)
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xr)
    h = sp.SparseMatrix.from_csr(A)
    try:
        Yref = h.apply(X).cpu().numpy().astype(np.float64)
    finally:
        h.close()
    for call in range(2):
        Y = torch.full((A.n_rows, k), float("nan"), device="cuda")
        _static(sp, A, rp, ci, va, sp.SPMM_F32, tk, n_seg, X, k, code, Y)
        sp.spmm_static_status()
        assert_close_rel(Y.cpu().numpy(), ref, scale, 2e-3, f"{xname} k={k} vs oracle call {call}")
        assert_close_rel(Y.cpu().numpy(), Yref, scale, 2e-3, f"{xname} k={k} vs handle call {call}")


def test_static_scratch_entry_16bit_values():
    """BF16 values with BF16 X (the staged 2-byte value path)."""
    import torch
    from paper_1602_02864_gb300 import spmm as sp

    A = synth.rmat_csr(13, seed=8, weighted=True)
    A.values = torch.from_numpy(A.values).to(torch.bfloat16).float().numpy()   # exactly representable
    tasks, _, n_seg = sp.spmm_plan_tasks(A.row_ptr)
    rp, ci, va = _device_inputs(A, torch, vdtype=torch.bfloat16)
    tk = torch.from_numpy(tasks).cuda()
    for k in (4, 8):
        X = torch.from_numpy(synth.dense(A.n_cols, k, seed=12)).cuda().to(torch.bfloat16)
        Xr = rounded_host(X)
        scale = abs_product(A, Xr)
        ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xr)
        for call in range(2):
            Y = torch.full((A.n_rows, k), float("nan"), device="cuda")
            _static(sp, A, rp, ci, va, sp.SPMM_BF16, tk, n_seg, X, k, sp.SPMM_BF16, Y)
            sp.spmm_static_status()
            assert_close_rel(Y.cpu().numpy(), ref, scale, 2e-3, f"bf16 values k={k} call {call}")


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16, 64])
def test_static_scratch_entry_pattern_integer_exact(k):
    """Pattern-only A with X in {0..7}: every partial sum is an integer below
    2^24, so the result is the oracle's bit for bit, whatever the order."""
    import torch
    from paper_1602_02864_gb300 import spmm as sp

    A = synth.rmat_csr(14, seed=9)
    A.values = None
    assert 7 * int(np.diff(A.row_ptr).max()) < 2 ** 24
    tasks, n_split, n_seg = sp.spmm_plan_tasks(A.row_ptr)
    assert n_split > 0
    rp, ci, _ = _device_inputs(A, torch)
    tk = torch.from_numpy(tasks).cuda()
    Xi = synth.dense(A.n_cols, k, seed=13, mode="int")
    X = torch.from_numpy(Xi).cuda()
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, Xi.astype(np.float64))
    for call in range(2):
        Y = torch.full((A.n_rows, k), float("nan"), device="cuda")
        _static(sp, A, rp, ci, None, sp.SPMM_F32, tk, n_seg, X, k, sp.SPMM_F32, Y)
        sp.spmm_static_status()
        got = Y.cpu().numpy().astype(np.float64)
        assert np.array_equal(got, ref), f"k={k} call {call}: {np.abs(got - ref).max()}"


def test_static_scratch_entry_fails_closed_on_foreign_slots():
    """A task list whose segment slots lie beyond the static array (here: a
    valid plan with every slot shifted past the end) writes nothing outside
    the array; the kernels flag it and spmm_static_status reports it.  The
    next well-formed call clears the flag."""
    import torch
    from paper_1602_02864_gb300 import spmm as sp

    A = synth.rmat_csr(14, seed=5, weighted=True)
    tasks, _, n_seg = sp.spmm_plan_tasks(A.row_ptr)
    assert n_seg > 0
    bad = tasks.copy()
    seg = bad[:-1, 1] < 0
    bad[:-1, 1][seg] -= 16384                           # slot s -> s + 16384
    rp, ci, va = _device_inputs(A, torch)
    X = torch.from_numpy(synth.dense(A.n_cols, 8, seed=1)).cuda()
    Y = torch.zeros((A.n_rows, 8), device="cuda")
    _static(sp, A, rp, ci, va, sp.SPMM_F32, torch.from_numpy(bad).cuda(), n_seg, X, 8, sp.SPMM_F32, Y)
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_static_status()
    assert e.value.status == sp.SPMM_ERR_FORMAT
    # rows that are not split are still complete
    Xh = X.cpu().numpy().astype(np.float64)
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xh)
    split_rows = np.unique(tasks[:-1, 0][tasks[:-1, 1] < 0])
    keep = np.setdiff1d(np.arange(A.n_rows), split_rows)
    assert_close_rel(Y.cpu().numpy()[keep], ref[keep], abs_product(A, Xh)[keep], 1e-5, "unsplit rows")
    _static(sp, A, rp, ci, va, sp.SPMM_F32, torch.from_numpy(tasks).cuda(), n_seg, X, 8, sp.SPMM_F32, Y)
    sp.spmm_static_status()


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
