"""The CSR file layout (host only, no GPU): spmm_write_csr_file's output
read back with numpy, and its validation."""
import numpy as np
import pytest

import synth
from tests import graphs

ALIGN = 4096


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


def read_back(path):
    raw = np.fromfile(path, dtype=np.uint8)
    assert raw[:8].tobytes() == b"SPMMCSR1"
    n_rows, n_cols, nnz = np.frombuffer(raw[8:32].tobytes(), dtype=np.int64)
    vtype, zero = np.frombuffer(raw[32:40].tobytes(), dtype=np.int32)
    off_rp, off_ci, off_val = np.frombuffer(raw[40:64].tobytes(), dtype=np.int64)
    assert zero == 0 and len(raw) % ALIGN == 0
    for off in (off_rp, off_ci) + ((off_val,) if vtype >= 0 else ()):
        assert off % ALIGN == 0
    rp = np.frombuffer(raw[off_rp:off_rp + 8 * (n_rows + 1)].tobytes(), dtype=np.int64)
    ci = np.frombuffer(raw[off_ci:off_ci + 4 * nnz].tobytes(), dtype=np.int32)
    vals = None
    if vtype >= 0:
        vb = 4 if vtype == 0 else 2
        vals = raw[off_val:off_val + vb * nnz].tobytes()
    return int(n_rows), int(n_cols), int(nnz), int(vtype), rp, ci, vals


@pytest.mark.parametrize("weighted", [False, True])
def test_roundtrip(sp, tmp_path, weighted):
    A = synth.rmat_csr(10, seed=1, weighted=weighted)
    path = tmp_path / "a.spmm"
    sp.spmm_write_csr_file(str(path), A)
    n_rows, n_cols, nnz, vtype, rp, ci, vals = read_back(path)
    assert (n_rows, n_cols, nnz) == (A.n_rows, A.n_cols, A.nnz)
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(ci, A.col_idx)
    if weighted:
        assert vtype == 0 and vals == A.values.tobytes()
    else:
        assert vtype == -1 and vals is None


def test_empty_and_rectangular(sp, tmp_path):
    E = graphs.csr_from_edges(5, 3, [], [])
    sp.spmm_write_csr_file(str(tmp_path / "e.spmm"), E)
    assert read_back(tmp_path / "e.spmm")[:3] == (5, 3, 0)
    R = graphs.csr_from_edges(3, 7, [0, 2, 2], [6, 0, 5], [1, 2, 3])
    R.values = R.values.astype(np.float16)
    sp.spmm_write_csr_file(str(tmp_path / "r.spmm"), R)
    n_rows, n_cols, nnz, vtype, rp, ci, vals = read_back(tmp_path / "r.spmm")
    assert (n_rows, n_cols, nnz, vtype) == (3, 7, 3, sp.SPMM_F16)
    assert np.frombuffer(vals, np.float16).tolist() == [1, 2, 3]


def test_validation(sp, tmp_path):
    A = synth.rmat_csr(8, seed=2)
    bad = synth.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx.copy())
    bad.col_idx[7] = A.n_cols
    with pytest.raises(sp.SpmmError, match="ERR_FORMAT"):
        sp.spmm_write_csr_file(str(tmp_path / "b.spmm"), bad)
    rp = A.row_ptr.copy()
    rp[3], rp[4] = rp[4], rp[3] - 1
    with pytest.raises(sp.SpmmError, match="ERR_FORMAT"):
        sp.spmm_write_csr_file(str(tmp_path / "b.spmm"), synth.CSR(A.n_rows, A.n_cols, rp, A.col_idx))
    with pytest.raises(sp.SpmmError, match="ERR_IO"):
        sp.spmm_write_csr_file(str(tmp_path / "no_such_dir" / "x.spmm"), A)
    assert not (tmp_path / "b.spmm").exists()
