"""SPMM_REORDER: columns relabelled by decreasing degree inside the handle.
Rows and the entry order within each row are unchanged, so every result must
be bit-identical to a handle without the flag (and so carries the same parity
against the oracle)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


@pytest.fixture(scope="module")
def rmat15():
    return synth.rmat_csr(15, seed=3, weighted=True)


@pytest.fixture(scope="module")
def pair(sp, rmat15):
    A = rmat15
    h0 = sp.SparseMatrix.from_csr(A, transpose=True)
    h1 = sp.SparseMatrix.from_csr(A, transpose=True, reorder=True)
    yield h0, h1
    h0.close()
    h1.close()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16, 33, 64])
@pytest.mark.parametrize("transpose", [False, True])
def test_bit_identical_f32(sp, rmat15, pair, k, transpose):
    import torch
    h0, h1 = pair
    n_in = rmat15.n_rows if transpose else rmat15.n_cols
    X = to_dev(synth.dense(n_in, k, seed=k))
    assert torch.equal(h0.apply(X, transpose=transpose), h1.apply(X, transpose=transpose))


@pytest.mark.parametrize("k", [1, 4, 8, 24])
def test_bit_identical_bf16_and_strided(sp, rmat15, pair, k):
    """A strided, misaligned X is copied into the relabelled order as a
    contiguous aligned array, so the reordered handle equals the plain handle
    on X.contiguous() bit for bit, and the plain handle on the strided X within
    the FP32 tolerance (its vector width follows X's alignment)."""
    import torch
    from tests.gpu_util import assert_close_rel
    A = rmat15
    h0, h1 = pair
    Xw = to_dev(synth.dense(A.n_cols, k + 3, seed=2), torch.bfloat16)
    X = Xw[:, 1:1 + k]                       # unaligned start, ldx = k + 3
    Y1 = h1.apply(X)
    assert torch.equal(h0.apply(X.contiguous()), Y1)
    Xh = X.float().cpu().numpy()
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xh)
    scale = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, np.abs(Xh))
    assert_close_rel(Y1.cpu().numpy(), ref, scale, 1e-5)
    assert_close_rel(h0.apply(X).cpu().numpy(), ref, scale, 1e-5)
    Xf = to_dev(synth.dense(A.n_cols, k + 5, seed=4))[:, 2:2 + k]
    assert torch.equal(h0.apply(Xf.contiguous()), h1.apply(Xf))


def test_matches_oracle(sp, rmat15, pair):
    A = rmat15
    _, h1 = pair
    X = synth.dense(A.n_cols, 5, seed=9, mode="int")
    Ap = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, reorder=True)
    Y = Ap.apply(to_dev(X)).cpu().numpy().astype(np.float64)
    assert np.array_equal(Y, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X))
    Ap.close()


def test_pagerank_and_host_apply_identical(sp, rmat15):
    import torch
    A = rmat15
    h0 = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)
    h1 = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, reorder=True)
    x0, r0 = h0.pagerank(0.85, 20)
    x1, r1 = h1.pagerank(0.85, 20)
    assert torch.equal(x0, x1) and np.array_equal(r0, r1)
    X = synth.dense(A.n_cols, 12, seed=1)
    Y0 = np.zeros((A.n_rows, 12), np.float32)
    Y1 = np.zeros((A.n_rows, 12), np.float32)
    h0.apply_host(X, Y0, group_cols=5)
    h1.apply_host(X, Y1, group_cols=5)
    assert np.array_equal(Y0, Y1)
    info0, info1 = h0.info(), h1.info()
    assert info1["device_bytes"] > info0["device_bytes"]       # the relabelled-index tables and X buffer
    h0.close()
    h1.close()


def test_nmf_identical(sp):
    import torch
    graphs = [synth.chunglu_csr(g, seed=1, nmin=500, nmax=3000) for g in range(3)]
    res = []
    for reorder in (False, True):
        h = sp.SparseMatrix.batched(graphs, transpose=True, weighted=False, reorder=reorder)
        nr = sum(g.n_rows for g in graphs)
        W = torch.from_numpy(synth.dense(nr, 8, seed=1, mode="unit")).cuda()
        Ht = torch.from_numpy(synth.dense(nr, 8, seed=2, mode="unit")).cuda()
        obj = h.nmf(8, 5, W, Ht)
        res.append((W.cpu(), Ht.cpu(), obj))
        h.close()
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2], res[1][2])


def test_streaming_rejects_reorder(sp, rmat15):
    A = rmat15
    with pytest.raises(sp.SpmmError, match="ERR_UNSUPPORTED"):
        sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, streaming=True, reorder=True)
