"""Compensated summation for long rows and split hub rows (option
`compensated`): brute-force check on an adversarial hub row against the exact
FP64 sum, and parity on an R-MAT graph."""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs
from tests.gpu_util import abs_product, assert_close_rel

pytestmark = pytest.mark.gpu


def test_adversarial_hub_row():
    import torch
    from paper_1602_02864_gb300 import spmm as sp
    d = 1_000_000
    A = graphs.csr_from_edges(2, d, np.zeros(d, np.int64), np.arange(d))          # one hub row, one empty row
    j = np.arange(d)
    x = np.where(j % 3 == 0, 1e8, np.where(j % 3 == 1, 1.0, -1e8)).astype(np.float32)
    X = np.stack([x, np.roll(x, 1), 0.5 * x, np.ones(d, np.float32)], axis=1).astype(np.float32)
    exact = oracle.spmm(2, d, A.row_ptr, A.col_idx, None, X)[0]
    out = {}
    for comp in (0, 1):
        h = sp.SparseMatrix(2, d, A.row_ptr, A.col_idx, None, opts=sp.spmm_opts(compensated=comp))
        assert h.info()["n_split_rows"] == 1
        out[comp] = h.apply(torch.from_numpy(X).cuda()).cpu().numpy()[0].astype(np.float64)
        h.close()
    err_c = np.abs(out[1] - exact)
    err_p = np.abs(out[0] - exact)
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    assert np.all(err_c <= 2 * ulp), (err_c, ulp)            # within two float32 ulps of the exact sum
    assert err_p.max() > 100 * max(err_c.max(), 1.0)         # plain float32 sums lose the small terms


def test_compensated_parity_rmat():
    import torch
    from paper_1602_02864_gb300 import spmm as sp
    A = synth.rmat_csr(15, seed=3, weighted=True)
    h = sp.SparseMatrix.from_csr(A, transpose=True, opts=sp.spmm_opts(compensated=1))
    for k in (1, 8, 33):
        for tr in (False, True):
            X = synth.dense(A.n_rows, k, seed=k)
            Y = h.apply(torch.from_numpy(X).cuda(), transpose=tr).cpu().numpy()
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X, transpose=tr)
            assert_close_rel(Y, ref, abs_product(A, X.astype(np.float64), tr), 1e-5, f"comp k={k}")
    Xi = synth.dense(A.n_rows, 8, seed=1, mode="int")
    hp = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, opts=sp.spmm_opts(compensated=1))
    Yi = hp.apply(torch.from_numpy(Xi).cuda()).cpu().numpy().astype(np.float64)
    assert np.array_equal(Yi, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, Xi))
    h.close()
    hp.close()
