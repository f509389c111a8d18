"""Streaming mode (matrix in pinned host memory, streamed per call through two
staging slots) against the resident mode and the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import abs_product, assert_close_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


@pytest.mark.parametrize("slot_kib", [16, 256])
def test_streaming_matches_resident_and_oracle(sp, slot_kib):
    import torch
    A = synth.rmat_csr(15, seed=4, weighted=True)
    o = sp.spmm_opts(stream_slot_kib=slot_kib)
    hs = sp.SparseMatrix.from_csr(A, opts=o, streaming=True)
    hr = sp.SparseMatrix.from_csr(A, opts=o)
    hp = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, opts=o, streaming=True)
    for k in (1, 8, 33):
        X = torch.from_numpy(synth.dense(A.n_cols, k, seed=k)).cuda()
        Ys = hs.apply(X)
        Yr = hr.apply(X)
        assert torch.equal(Ys, Yr)                     # same plan, same kernel, same order
        ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X.cpu().numpy())
        assert_close_rel(Ys.cpu().numpy(), ref, abs_product(A, X.cpu().numpy().astype(np.float64)), 1e-5, "stream")
        Xi = synth.dense(A.n_cols, k, seed=k, mode="int")
        Yi = hp.apply(torch.from_numpy(Xi).cuda()).cpu().numpy().astype(np.float64)
        assert np.array_equal(Yi, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, Xi))
    hs.sync_status()
    for h in (hs, hr, hp):
        h.close()


def test_streaming_injected_copy_failure_drains(sp):
    import torch
    A = synth.rmat_csr(13, seed=2)
    bad = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, streaming=True,
                          opts=sp.spmm_opts(stream_slot_kib=16, debug_fail_block=3))
    X = torch.from_numpy(synth.dense(A.n_cols, 4, seed=1, mode="int")).cuda()
    with pytest.raises(sp.SpmmError) as e:
        bad.apply(X)
    assert e.value.status == sp.SPMM_ERR_CUDA and "injected" in str(e.value)
    bad.close()
    good = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, streaming=True,
                           opts=sp.spmm_opts(stream_slot_kib=16))
    Y = good.apply(X).cpu().numpy().astype(np.float64)
    assert np.array_equal(Y, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X.cpu().numpy()))
    good.close()


def test_streaming_rejects_transpose(sp):
    A = synth.rmat_csr(10, seed=1)
    with pytest.raises(sp.SpmmError) as e:
        sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, streaming=True)
    assert e.value.status == sp.SPMM_ERR_UNSUPPORTED
