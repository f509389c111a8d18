"""Tile format (Section 3.2): storage formulas and host-side validation of the
importer (no GPU work happens before a tile set is accepted)."""
import numpy as np
import pytest

import synth
from tests.tiles_encode import encode, storage_bytes


def test_scsr_storage_formula_and_dcsc_ratio():
    A = synth.rmat_csr(13, seed=3)
    t = 1024
    tiles = encode(A, t)
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    cols = A.col_idx
    nnr = nnc = 0
    for tr in range(A.n_rows // t):
        for tc in range(A.n_cols // t):
            m = (rows // t == tr) & (cols // t == tc)
            nnr += len(np.unique(rows[m]))
            nnc += len(np.unique(cols[m]))
    for c in (0, 4):
        assert storage_bytes(tiles, c) == 2 * nnr + (2 + c) * A.nnz          # S_SCSR = 2 nnr + (2 + c) nnz
    s_scsr = 2 * nnr + 2 * A.nnz
    s_dcsc = (2 + 2 + 4) * nnc + 2 * A.nnz
    assert 0.4 <= s_scsr / s_dcsc < 1.0                                     # binary matrix, nnr ~ nnc


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import build
    build.build()
    from paper_1602_02864_gb300 import spmm
    return spmm


def test_importer_rejects_bad_tiles_before_gpu_work(sp):
    ok = (0, 0, np.array([0x8000 | 1, 3, 4], np.uint16), np.zeros((0, 2), np.uint16), None)
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_create_tiles(10, 10, 40000, [ok], stream=0)                 # tile > 32768
    assert e.value.status == sp.SPMM_ERR_ARG
    cases = [
        (0, 0, np.array([3, 0x8000 | 1, 2], np.uint16), np.zeros((0, 2), np.uint16), None),   # column first
        (0, 0, np.array([0x8000 | 1, 0x8000 | 2, 5], np.uint16), np.zeros((0, 2), np.uint16), None),  # empty row
        (0, 0, np.array([0x8000 | 9, 1], np.uint16), np.zeros((0, 2), np.uint16), None),      # row >= tile
        (0, 0, np.array([], np.uint16), np.array([[1, 0x8001]], np.uint16), None),            # top bit in COO
        (3, 0, np.array([0x8000, 1], np.uint16), np.zeros((0, 2), np.uint16), None),          # tile outside
    ]
    for bad in cases:
        with pytest.raises(sp.SpmmError) as e:
            sp.spmm_create_tiles(20, 20, 8, [ok, bad] if bad[0] != 3 else [bad], stream=0)
        assert e.value.status == sp.SPMM_ERR_FORMAT, bad
