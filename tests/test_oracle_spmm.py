"""Pins for the oracle's SpMM against things other than itself: dense matmul,
closed forms of special graphs, degree identities, sampled-row consistency."""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_vs_dense_matmul(seed, weighted, k):
    A = graphs.random_csr(97, 131, 0.05, seed, weighted=weighted)
    D = graphs.dense_of(A)
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (131, k))
    Y = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X)
    np.testing.assert_allclose(Y, D @ X, rtol=1e-13, atol=1e-13)
    Xt = rng.uniform(-1, 1, (97, k))
    Yt = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xt, transpose=True)
    np.testing.assert_allclose(Yt, D.T @ Xt, rtol=1e-13, atol=1e-13)


def test_rmat_vs_dense_float32_input():
    A = synth.rmat_csr(8, 3000, seed=4, weighted=True)
    X = synth.dense(256, 5, seed=1)          # float32 input, widened exactly
    D = graphs.dense_of(A)
    Y = oracle.spmm(256, 256, A.row_ptr, A.col_idx, A.values, X)
    np.testing.assert_allclose(Y, D @ X.astype(np.float64), rtol=1e-13, atol=1e-13)


def test_ones_give_degrees():
    A = synth.rmat_csr(10, seed=7)
    n = A.n_rows
    one = np.ones((n, 1))
    out_deg = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, one)[:, 0]
    in_deg = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, one, transpose=True)[:, 0]
    assert np.array_equal(out_deg, np.diff(A.row_ptr).astype(np.float64))
    assert np.array_equal(in_deg, np.bincount(A.col_idx, minlength=n).astype(np.float64))


def test_cycle_shifts_rows():
    n = 37
    A = graphs.cycle(n)
    X = np.arange(n * 3, dtype=np.float64).reshape(n, 3)
    Y = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, X)
    assert np.array_equal(Y, np.roll(X, -1, axis=0))
    Yt = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, X, transpose=True)
    assert np.array_equal(Yt, np.roll(X, 1, axis=0))


def test_complete_graph_column_sums():
    n = 23
    A = graphs.complete(n)
    X = np.random.default_rng(0).integers(-5, 6, (n, 4)).astype(np.float64)
    Y = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, X)
    assert np.array_equal(Y, X.sum(0)[None, :] - X)


def test_star_and_empty_rows():
    n = 50
    A = graphs.star(n)
    X = np.random.default_rng(1).uniform(-1, 1, (n, 2))
    Y = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, X)
    np.testing.assert_allclose(Y[0], X[1:].sum(0), rtol=1e-14)
    assert np.all(Y[1:] == 0)
    Yt = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, X, transpose=True)
    assert np.all(Yt[0] == 0) and np.array_equal(Yt[1:], np.repeat(X[:1], n - 1, 0))


def test_degenerate_sizes():
    E = graphs.csr_from_edges(5, 4, [], [])
    Y = oracle.spmm(5, 4, E.row_ptr, E.col_idx, None, np.ones((4, 3)))
    assert Y.shape == (5, 3) and np.all(Y == 0)
    one = graphs.csr_from_edges(1, 1, [0], [0], [2.5])
    assert oracle.spmm(1, 1, one.row_ptr, one.col_idx, one.values, np.array([[4.0]]))[0, 0] == 10.0


def test_sampled_rows_and_threads_agree():
    A = synth.rmat_csr(11, seed=9, weighted=True)
    n = A.n_rows
    X = synth.dense(n, 8, seed=2)
    Y1 = oracle.spmm(n, n, A.row_ptr, A.col_idx, A.values, X, threads=1)
    Y4 = oracle.spmm(n, n, A.row_ptr, A.col_idx, A.values, X, threads=4)
    assert np.array_equal(Y1, Y4)
    rows = synth.sample_rows(n, 300, seed=1)
    assert np.array_equal(oracle.spmm_rows(A.row_ptr, A.col_idx, A.values, X, rows, threads=3), Y1[rows])
    Yt = oracle.spmm(n, n, A.row_ptr, A.col_idx, A.values, X, transpose=True)
    ur = np.unique(rows)
    assert np.array_equal(oracle.spmm_t_rows(n, n, A.row_ptr, A.col_idx, A.values, X, ur), Yt[ur])
