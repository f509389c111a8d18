"""SPMM_RELABEL's vertex order, host side (no GPU): spmm_relabel_order
against its definition (decreasing row + column entry count, ties in vertex
order), and the create-time checks that reject the flag before any device
work."""
import ctypes

import numpy as np
import pytest

import synth
from tests import graphs


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import build
    build.build()
    from paper_1602_02864_gb300 import spmm
    return spmm


def reference_order(n, row_ptr, col_idx):
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64)) + np.bincount(np.asarray(col_idx, dtype=np.int64), minlength=n)
    return np.lexsort((np.arange(n), -deg)).astype(np.int32)


@pytest.mark.parametrize("scale,seed", [(8, 0), (10, 3), (12, 5)])
def test_order_matches_definition_rmat(sp, scale, seed):
    A = synth.rmat_csr(scale, seed=seed)
    got = sp.spmm_relabel_order(A.n_rows, A.row_ptr, A.col_idx)
    np.testing.assert_array_equal(got, reference_order(A.n_rows, A.row_ptr, A.col_idx))


def test_order_special_cases(sp):
    # star: the hub first, then the leaves in vertex order (all degree 2: one
    # out-entry and one in-entry each)
    n = 9
    i = np.arange(1, n)
    S = graphs.csr_from_edges(n, n, np.r_[np.zeros(n - 1, int), i], np.r_[i, np.zeros(n - 1, int)])
    np.testing.assert_array_equal(sp.spmm_relabel_order(n, S.row_ptr, S.col_idx), np.arange(n, dtype=np.int32))
    # isolated vertices last, in vertex order; a self-loop counts twice
    rp = np.array([0, 0, 1, 1, 3, 3], dtype=np.int64)
    ci = np.array([3, 3, 1], dtype=np.int32)       # 1 -> 3, 3 -> 3 (loop), 3 -> 1
    got = sp.spmm_relabel_order(5, rp, ci)
    np.testing.assert_array_equal(got, reference_order(5, rp, ci))
    assert list(got[:2]) == [3, 1] and list(got[2:]) == [0, 2, 4]
    # repeated entries count once per stored entry
    rp = np.array([0, 3, 3, 4], dtype=np.int64)
    ci = np.array([2, 2, 2, 1], dtype=np.int32)
    np.testing.assert_array_equal(sp.spmm_relabel_order(3, rp, ci), reference_order(3, rp, ci))
    # the empty matrix keeps the vertex order
    np.testing.assert_array_equal(sp.spmm_relabel_order(4, np.zeros(5, np.int64), np.zeros(0, np.int32)),
                                  np.arange(4, dtype=np.int32))


def test_order_is_a_permutation_with_decreasing_degree(sp):
    A = synth.chunglu_csr(3, seed=0)
    n = A.n_rows
    o = sp.spmm_relabel_order(n, A.row_ptr, A.col_idx)
    assert sorted(o.tolist()) == list(range(n))
    deg = np.diff(A.row_ptr) + np.bincount(A.col_idx, minlength=n)
    d = deg[o]
    assert np.all(np.diff(d) <= 0)
    ties = np.diff(d) == 0
    assert np.all(np.diff(o)[ties] > 0)


def test_order_rejects_bad_input(sp):
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_relabel_order(3, np.array([0, 2, 1, 3]), np.array([0, 1, 2]))
    assert e.value.status == sp.SPMM_ERR_FORMAT
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_relabel_order(3, np.array([0, 1, 2, 3]), np.array([0, 3, 2]))
    assert e.value.status == sp.SPMM_ERR_FORMAT


def test_create_rejects_relabel_combinations_on_host(sp):
    lib = sp.lib()
    h = ctypes.c_void_p(0)
    rp = np.array([0, 1, 2, 3], dtype=np.int64)
    ci = np.array([0, 1, 1], dtype=np.int32)

    def create(n_rows, n_cols, flags):
        return lib.spmm_create_csr(ctypes.byref(h), n_rows, n_cols, 3, ctypes.c_void_p(rp.ctypes.data),
                                   ctypes.c_void_p(ci.ctypes.data), None, 0, flags, None, None)
    assert create(3, 4, sp.SPMM_RELABEL) == sp.SPMM_ERR_ARG                       # not square
    assert create(3, 3, sp.SPMM_RELABEL | sp.SPMM_REORDER) == sp.SPMM_ERR_ARG
    assert create(3, 3, sp.SPMM_RELABEL | sp.SPMM_HOST_STREAMING) == sp.SPMM_ERR_UNSUPPORTED
    assert not h.value
