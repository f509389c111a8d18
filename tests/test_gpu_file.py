"""A matrix kept in a file (spmm_create_file): read from storage on every
apply, streamed through the HBM slots, identical to the resident handle."""
import os

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
def rmat14():
    return synth.rmat_csr(14, seed=6, weighted=True)


def small_slots(sp):
    return sp.spmm_opts(stream_slot_kib=64)      # ~16 K entries per block: many blocks


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("direct", [False, True])
def test_equals_resident(sp, rmat14, tmp_path, weighted, direct):
    import torch
    A = rmat14
    path = str(tmp_path / "a.spmm")
    vals = A.values if weighted else None
    sp.spmm_write_csr_file(path, synth.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vals))
    try:
        hf = sp.SparseMatrix.from_file(path, A.n_rows, A.n_cols, direct=direct, opts=small_slots(sp))
    except sp.SpmmError as e:
        if direct and "ERR_UNSUPPORTED" in str(e):
            pytest.skip("this file system refuses O_DIRECT")
        raise
    hr = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vals, opts=small_slots(sp))
    for k in (1, 4, 8, 33):
        X = to_dev(synth.dense(A.n_cols, k, seed=k))
        Yf = hf.apply(X)
        assert torch.equal(Yf, hr.apply(X))
    hf.sync_status()
    X = synth.dense(A.n_cols, 3, seed=1, mode="int")
    Yi = hf.apply(to_dev(X)).cpu().numpy().astype(np.float64)
    if not weighted:
        assert np.array_equal(Yi, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X))
    hf.close()
    hr.close()


def test_bf16_values(sp, rmat14, tmp_path):
    import torch
    A = rmat14
    vb = torch.from_numpy(A.values).to(torch.bfloat16)
    path = str(tmp_path / "b.spmm")
    sp.spmm_write_csr_file(path, synth.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx,
                                           vb.view(torch.int16).numpy().view(np.uint16)))
    hf = sp.SparseMatrix.from_file(path, A.n_rows, A.n_cols, opts=small_slots(sp))
    hr = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vb, opts=small_slots(sp))
    X = to_dev(synth.dense(A.n_cols, 8, seed=3), torch.bfloat16)
    Yf = hf.apply(X)
    assert torch.equal(Yf, hr.apply(X))
    Xh = X.float().cpu().numpy()
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vb.float().numpy(), Xh)
    scale = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, np.abs(vb.float().numpy()), np.abs(Xh))
    assert np.all(np.abs(Yf.cpu().numpy() - ref) <= 1e-5 * scale + 1e-30)
    hf.close()
    hr.close()


def test_changed_file_is_caught_on_the_host(sp, rmat14, tmp_path):
    """A column index made out of range after create is found by the host
    readers before the block reaches the GPU; a truncated file is an I/O
    error.  The device stays usable afterwards."""
    import torch
    A = rmat14
    path = str(tmp_path / "c.spmm")
    sp.spmm_write_csr_file(path, synth.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx))
    hf = sp.SparseMatrix.from_file(path, A.n_rows, A.n_cols, opts=small_slots(sp))
    X = to_dev(synth.dense(A.n_cols, 4, seed=2))
    Y0 = hf.apply(X).clone()
    raw = np.fromfile(path, dtype=np.uint8)
    off_ci = int(np.frombuffer(raw[48:56].tobytes(), np.int64)[0])
    with open(path, "r+b") as f:
        f.seek(off_ci + 4 * (A.nnz // 2))
        f.write(np.int32(A.n_cols + 5).tobytes())
    with pytest.raises(sp.SpmmError, match="ERR_FORMAT"):
        hf.apply(X)
    with open(path, "r+b") as f:
        f.truncate(off_ci + 4 * (A.nnz // 3))
    with pytest.raises(sp.SpmmError, match="ERR_IO"):
        hf.apply(X)
    hf.close()
    hr = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, opts=small_slots(sp))
    assert torch.equal(hr.apply(X), Y0)
    hr.close()


def test_open_errors(sp, tmp_path):
    with pytest.raises(sp.SpmmError, match="ERR_IO"):
        sp.SparseMatrix.from_file(str(tmp_path / "missing.spmm"), 1, 1)
    p = tmp_path / "junk.spmm"
    p.write_bytes(b"not a matrix" * 100)
    with pytest.raises(sp.SpmmError, match="ERR_FORMAT"):
        sp.SparseMatrix.from_file(str(p), 1, 1)
