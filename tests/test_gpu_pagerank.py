"""GPU PageRank (Section 4.1) against the FP64 oracle and closed forms."""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


def handle(sp, A):
    return sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)


@pytest.mark.parametrize("scale", [12, 16])
def test_pagerank_matches_oracle(sp, scale):
    A = synth.rmat_csr(scale, seed=scale)
    h = handle(sp, A)
    x, res = h.pagerank(0.85, 30)
    xr, resr = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 30)
    xg = x.cpu().numpy().astype(np.float64)
    # float32 ranks after 30 contractions: elementwise relative 1e-5
    assert np.all(np.abs(xg - xr) <= 1e-5 * xr + 1e-12), np.max(np.abs(xg - xr) / xr)
    assert abs(xg.sum() - 1.0) < 1e-5 and xg.min() >= 0
    # the L1 change is taken between float32 rank vectors: once it falls to the
    # float32 noise floor (a few ulps of ranks summing to 1, ~2^-24 each per unit
    # of mass) it is compared in absolute terms
    np.testing.assert_allclose(res, resr, rtol=1e-3, atol=4 * 2.0 ** -24)
    x2, res2 = h.pagerank(0.85, 30)
    assert np.array_equal(x2.cpu().numpy(), x.cpu().numpy()) and np.array_equal(res2, res)
    h.sync_status()
    h.close()


def test_pagerank_start_vector_and_zero_iters(sp):
    import torch
    A = synth.rmat_csr(11, seed=3)
    h = handle(sp, A)
    x0 = np.random.default_rng(0).random(A.n_rows).astype(np.float32)
    x0 /= x0.sum()
    x, res = h.pagerank(0.85, 0, x0=torch.from_numpy(x0).cuda())
    assert np.array_equal(x.cpu().numpy(), x0) and len(res) == 0
    x, res = h.pagerank(0.85, 7, x0=torch.from_numpy(x0).cuda())
    xr, resr = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 7, x0=x0.astype(np.float64))
    assert np.all(np.abs(x.cpu().numpy() - xr) <= 1e-5 * xr + 1e-12)
    h.close()


def test_pagerank_closed_forms(sp):
    for A in (graphs.cycle(1000), graphs.complete(50)):
        h = handle(sp, A)
        x, res = h.pagerank(0.85, 30)
        np.testing.assert_allclose(x.cpu().numpy(), 1.0 / A.n_rows, rtol=2e-7)
        h.close()
    A = graphs.csr_from_edges(2, 2, [0], [1])           # 0 -> 1, vertex 1 dangling
    h = handle(sp, A)
    x, _ = h.pagerank(0.85, 200)
    np.testing.assert_allclose(x.cpu().numpy(), [1 / 2.85, 1.85 / 2.85], rtol=1e-6)
    h.close()


def test_pagerank_argument_errors(sp):
    A = graphs.cycle(10)
    h = sp.SparseMatrix(10, 10, A.row_ptr, A.col_idx, None)          # no transpose
    with pytest.raises(sp.SpmmError):
        h.pagerank()
    h.close()
    W = graphs.random_csr(20, 20, 0.2, 1)
    h = sp.SparseMatrix.from_csr(W, transpose=True)                  # weighted
    with pytest.raises(sp.SpmmError):
        h.pagerank()
    h.close()


@pytest.mark.parametrize("opts", [None, (32, 64, 64, 31), (512, 64, 512, 1)])
def test_compensated_plan_gives_the_same_ranks(sp, opts):
    """A compensated plan changes only how hub-row segments are summed, so its
    ranks agree with the plain plan's within 1e-6 and with the oracle within
    1e-5; plans with many split rows (small long_row) or one row per task are
    included."""
    A = synth.rmat_csr(14, seed=4)
    o = None if opts is None else sp.spmm_opts(task_nnz=opts[0], task_rows=opts[1], long_row=opts[2],
                                                 short_max=opts[3])
    hf = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, opts=o)
    oc = sp.spmm_opts(compensated=1) if o is None else sp.spmm_opts(task_nnz=opts[0], task_rows=opts[1],
                                                                     long_row=opts[2], short_max=opts[3],
                                                                     compensated=1)
    hc = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, opts=oc)
    xf, rf = hf.pagerank(0.85, 25)
    xc, rc = hc.pagerank(0.85, 25)
    xf, xc = xf.cpu().numpy().astype(np.float64), xc.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(xf - xc) <= 1e-6 * xc + 1e-12)
    np.testing.assert_allclose(rf, rc, rtol=1e-3, atol=4 * 2.0 ** -24)
    xr, _ = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 25)
    assert np.all(np.abs(xf - xr) <= 1e-5 * xr + 1e-12)
    hf.close()
    hc.close()


def test_pagerank_cached_graph_follows_its_inputs(sp):
    """The handle keeps the captured iterations: a repeated call relaunches
    them, and another output vector, damping, iteration count, start vector
    or plan (spmm_replan) still gives the oracle's ranks."""
    import torch
    A = synth.rmat_csr(13, seed=21)
    h = handle(sp, A)
    try:
        xa = torch.empty(A.n_rows, device="cuda")
        xb = torch.empty(A.n_rows, device="cuda")
        x0 = torch.from_numpy(synth.dense(A.n_rows, 1, seed=4, mode="unit")[:, 0]).cuda()
        x0 /= x0.sum()
        cases = [(xa, 0.85, 30, None), (xa, 0.85, 30, None), (xb, 0.85, 30, None), (xa, 0.5, 30, None),
                 (xa, 0.85, 7, None), (xa, 0.85, 30, x0), (xa, 0.85, 1, None), (xa, 0.85, 0, None),
                 ("replan", None, None, None), (xa, 0.85, 30, None)]
        for x, d, it, start in cases:
            if isinstance(x, str):
                sp.spmm_replan(h.handle, sp.spmm_opts(task_nnz=128, short_max=15), 1)
                continue
            _, res = h.pagerank(d, it, x=x, x0=start)
            s0 = None if start is None else start.double().cpu().numpy()
            xr, resr = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, d, it, x0=s0)
            xg = x.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(xg - xr) <= 1e-5 * xr + 1e-12), (d, it)
            assert len(res) == it
            if it:
                np.testing.assert_allclose(res, resr, rtol=1e-3, atol=4 * 2.0 ** -24)
        h.sync_status()
    finally:
        h.close()
