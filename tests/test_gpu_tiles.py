"""Handles imported from SCSR + COO tiles compute the same product as the CSR
they encode (FP64 oracle on the original CSR)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import abs_product, assert_close_rel
from tests.tiles_encode import encode

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile", [256, 4096, 32768])
def test_tiles_import_matches_oracle(tile):
    import torch
    from paper_1602_02864_gb300 import spmm as sp
    A = synth.rmat_csr(14, seed=8, weighted=True)
    h = sp.SparseMatrix.from_tiles(A.n_rows, A.n_cols, tile, encode(A, tile), transpose=True)
    assert h.info()["nnz"] == A.nnz
    for tr in (False, True):
        X = synth.dense(A.n_rows, 8, seed=3)
        Y = h.apply(torch.from_numpy(X).cuda(), transpose=tr).cpu().numpy()
        ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X, transpose=tr)
        assert_close_rel(Y, ref, abs_product(A, X.astype(np.float64), tr), 1e-5, f"tiles t={tile}")
    h.close()
    P = synth.rmat_csr(13, seed=2)
    hp = sp.SparseMatrix.from_tiles(P.n_rows, P.n_cols, 512, encode(P, 512))
    Xi = synth.dense(P.n_cols, 5, seed=4, mode="int")
    Y = hp.apply(torch.from_numpy(Xi).cuda()).cpu().numpy().astype(np.float64)
    assert np.array_equal(Y, oracle.spmm(P.n_rows, P.n_cols, P.row_ptr, P.col_idx, None, Xi))
    hp.close()
