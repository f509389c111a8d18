"""Y = A X with X and Y in host memory, in vertical partitions (Section 3.3),
against the FP64 oracle and against per-group device applies."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_close_rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


@pytest.fixture(scope="module")
def rmat14():
    return synth.rmat_csr(14, seed=5, weighted=True)


@pytest.fixture(scope="module")
def handles(sp, rmat14):
    A = rmat14
    hp = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)
    hw = sp.SparseMatrix.from_csr(A, transpose=True)
    yield hp, hw
    hp.close()
    hw.close()


@pytest.mark.parametrize("p,g", [(40, 16), (7, 3), (64, 64), (1, 1), (65, 0), (130, 64)])
@pytest.mark.parametrize("transpose", [False, True])
def test_integer_exact(sp, rmat14, handles, p, g, transpose):
    A = rmat14
    hp, _ = handles
    X = synth.dense(A.n_cols, p, seed=p, mode="int")
    Y = np.full((A.n_rows, p), np.nan, dtype=np.float32)
    n = hp.apply_host(X, Y, transpose=transpose, group_cols=g)
    assert n == -(-p // (g if g else min(p, 64)))
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X, transpose=transpose)
    assert np.array_equal(Y.astype(np.float64), ref)


def test_strided_host_and_equals_group_applies(sp, rmat14, handles):
    """Strided host views (ldx, ldy > p) and a weighted matrix: the result is
    bit-identical to device applies of the same column groups, and within the
    FP32 tolerance of the oracle."""
    import torch
    A = rmat14
    _, hw = handles
    p, g = 21, 8
    Xw = synth.dense(A.n_cols, 29, seed=3)
    X = Xw[:, 3:3 + p]
    Yw = np.zeros((A.n_rows, 33), dtype=np.float32)
    Y = Yw[:, 5:5 + p]
    assert hw.apply_host(X, Y, group_cols=g) == 3
    assert np.all(Yw[:, :5] == 0) and np.all(Yw[:, 5 + p:] == 0)
    for c0 in range(0, p, g):
        w = min(g, p - c0)
        Yd = hw.apply(to_dev(np.ascontiguousarray(X[:, c0:c0 + w])))
        assert torch.equal(Yd.cpu(), torch.from_numpy(np.ascontiguousarray(Y[:, c0:c0 + w])))
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X)
    scale = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, np.abs(X))
    assert_close_rel(Y, ref, scale, 1e-5)


@pytest.mark.parametrize("pinned", [False, True])
def test_bf16_torch_host(sp, rmat14, handles, pinned):
    import torch
    A = rmat14
    hp, _ = handles
    p = 24
    Xt = torch.from_numpy(synth.dense(A.n_rows, p, seed=9, mode="int")).to(torch.bfloat16)
    Yt = torch.empty((A.n_cols, p), dtype=torch.float32)
    if pinned:
        Xt, Yt = Xt.pin_memory(), Yt.pin_memory()
    assert hp.apply_host(Xt, Yt, transpose=True, group_cols=10) == 3
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, Xt.float().numpy(), transpose=True)
    assert np.array_equal(Yt.numpy().astype(np.float64), ref)


def test_budget_picks_groups(sp, rmat14, handles):
    A = rmat14
    hp, _ = handles
    p = 10
    per_col = 2 * (A.n_cols * 4 + A.n_rows * 4)
    X = synth.dense(A.n_cols, p, seed=1, mode="int")
    Y = np.zeros((A.n_rows, p), dtype=np.float32)
    assert hp.apply_host(X, Y, budget_bytes=3 * per_col + 5) == 4          # groups of 3: 3+3+3+1
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X)
    assert np.array_equal(Y.astype(np.float64), ref)
    with pytest.raises(sp.SpmmError, match="ERR_OOM"):
        hp.apply_host(X, Y, budget_bytes=per_col - 1)
    with pytest.raises(sp.SpmmError, match="ERR_ARG"):
        hp.apply_host(X, Y, group_cols=65)


def test_streaming_handle(sp, rmat14):
    """X, Y and A all in host memory: A streams through its slots once per group."""
    A = rmat14
    o = sp.spmm_opts(stream_slot_kib=64)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, streaming=True, opts=o)
    p = 12
    X = synth.dense(A.n_cols, p, seed=2)
    Y = np.zeros((A.n_rows, p), dtype=np.float32)
    assert h.apply_host(X, Y, group_cols=5) == 3
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X)
    scale = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, np.abs(X))
    assert_close_rel(Y, ref, scale, 1e-5)
    h.sync_status()
    h.close()


@pytest.mark.parametrize("transpose", [False, True])
def test_contiguous_parts(sp, rmat14, handles, transpose):
    """Section 3.3's layout: each vertical partition its own contiguous
    row-major array (widths 5, 16, 3, 64, 1)."""
    A = rmat14
    hp, _ = handles
    n_in, n_out = (A.n_rows, A.n_cols) if transpose else (A.n_cols, A.n_rows)
    widths = [5, 16, 3, 64, 1]
    X = synth.dense(n_in, sum(widths), seed=4, mode="int")
    cuts = np.cumsum([0] + widths)
    Xp = [np.ascontiguousarray(X[:, a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
    Yp = [np.full((n_out, w), np.nan, dtype=np.float32) for w in widths]
    hp.apply_host_parts(Xp, Yp, transpose=transpose)
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X, transpose=transpose)
    assert np.array_equal(np.concatenate(Yp, axis=1).astype(np.float64), ref)


def test_contiguous_parts_bf16_pinned(sp, rmat14, handles):
    import torch
    A = rmat14
    _, hw = handles
    widths = [8, 8, 4]
    X = torch.from_numpy(synth.dense(A.n_cols, sum(widths), seed=8)).to(torch.bfloat16)
    Xp = [X[:, a:a + w].contiguous().pin_memory() for a, w in zip([0, 8, 16], widths)]
    Yp = [torch.empty((A.n_rows, w), dtype=torch.float32).pin_memory() for w in widths]
    hw.apply_host_parts(Xp, Yp)
    Xf = X.float().numpy()
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xf)
    scale = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, np.abs(Xf))
    assert_close_rel(torch.cat(Yp, dim=1).numpy(), ref, scale, 1e-5)


def test_parts_errors(sp, rmat14, handles):
    A = rmat14
    hp, _ = handles
    X = np.zeros((A.n_cols, 65), dtype=np.float32)
    Y = np.zeros((A.n_rows, 65), dtype=np.float32)
    with pytest.raises(sp.SpmmError, match="ERR_ARG"):
        hp.apply_host_parts([X], [Y])                      # a part wider than 64 columns
    with pytest.raises(ValueError):
        hp.apply_host_parts([X[:, :4].copy()], [])         # unequal part lists


@pytest.mark.parametrize("transpose", [False, True])
def test_parts_by_runs_with_split_rows(sp, transpose):
    """The host-buffer calls multiply in runs of whole tasks and copy each
    run's rows out while the next run multiplies: with many split hub rows
    (short tasks, low split threshold) and hot columns at k = 1, every part
    equals the device product bit for bit and the oracle exactly."""
    import torch
    A = synth.rmat_csr(13, seed=21)
    o = sp.spmm_opts(task_nnz=32, long_row=64, short_max=15, hot_cols=512)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, opts=o)
    try:
        info = h.info()
        assert info["n_split_rows"] > 50 and info["n_hot"] > 0
        widths = [1, 8, 33]
        X = synth.dense(A.n_rows, sum(widths), seed=6, mode="int")
        cuts = np.cumsum([0] + widths)
        Xp = [np.ascontiguousarray(X[:, a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
        Yp = [np.full((A.n_rows, w), np.nan, dtype=np.float32) for w in widths]
        h.apply_host_parts(Xp, Yp, transpose=transpose)
        for x, y in zip(Xp, Yp):
            assert torch.equal(h.apply(to_dev(x), transpose=transpose).cpu(), torch.from_numpy(y))
        ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X, transpose=transpose)
        assert np.array_equal(np.concatenate(Yp, axis=1).astype(np.float64), ref)
        h.sync_status()
    finally:
        h.close()


@pytest.mark.parametrize("n,edges", [(3, [(0, 1), (2, 0)]), (40, []), (1, [(0, 0)])])
def test_parts_tiny_and_empty(sp, n, edges):
    """Fewer tasks than runs, and no stored entries at all."""
    rp = np.zeros(n + 1, dtype=np.int64)
    for r, _ in edges:
        rp[r + 1:] += 1
    ci = np.array([c for _, c in sorted(edges)], dtype=np.int32)
    h = sp.SparseMatrix(n, n, rp, ci, None, transpose=True)
    try:
        X = synth.dense(n, 5, seed=1, mode="int")
        Y = np.full((n, 5), np.nan, dtype=np.float32)
        h.apply_host_parts([X], [Y])
        ref = oracle.spmm(n, n, rp, ci, None, X)
        assert np.array_equal(Y.astype(np.float64), ref)
    finally:
        h.close()
