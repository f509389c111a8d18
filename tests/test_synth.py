"""Pins for the seeded input generators (no SpMM arithmetic lives there)."""
import numpy as np
import pytest

import synth


def test_philox_known_answers():
    # Known-answer vectors published with the Philox4x32-10 definition.
    assert synth.philox4x32_10([0, 0, 0, 0], [0, 0]).tolist() == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert synth.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2).tolist() == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert synth.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]).tolist() == [
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_rmat_quadrant_frequencies():
    # Each level picks quadrant a/b/c/d = .57/.19/.19/.05, so a row bit is 0
    # with probability a+b = .76 and a column bit with a+c = .76, and both are
    # 0 with probability a = .57 (paper, Section 5 footnote on R-MAT).
    scale, m = 12, 400_000
    src, dst = synth.rmat_edges(scale, m, seed=3)
    assert src.max() < (1 << scale) and dst.max() < (1 << scale)
    sd = np.sqrt(0.76 * 0.24 / m)
    for lvl in range(scale):
        bit = scale - 1 - lvl
        r0 = ((src >> bit) & 1) == 0
        c0 = ((dst >> bit) & 1) == 0
        assert abs(r0.mean() - 0.76) < 6 * sd
        assert abs(c0.mean() - 0.76) < 6 * sd
        assert abs((r0 & c0).mean() - 0.57) < 6 * np.sqrt(0.57 * 0.43 / m)


def test_edges_to_csr_matches_numpy_unique():
    src, dst = synth.rmat_edges(10, 30_000, seed=1)
    A = synth.edges_to_csr(1024, 1024, src, dst)
    keys = np.unique(src.astype(np.int64) * 1024 + dst)
    assert A.nnz == len(keys)
    rows = np.repeat(np.arange(1024), np.diff(A.row_ptr))
    assert np.array_equal(rows * 1024 + A.col_idx, keys)
    assert np.all(np.diff(A.row_ptr) >= 0) and A.row_ptr[0] == 0


def test_symmetrize_and_weights():
    A = synth.sym_rmat_csr(9, seed=2, normalise=False)
    n = 1 << 9
    D = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    D[rows, A.col_idx] = A.values
    assert np.array_equal(D, D.T)
    assert np.all(A.values > 0)
    S = synth.sym_rmat_csr(9, seed=2, normalise=True)
    deg = D.sum(1)
    inv = np.where(deg > 0, 1.0 / np.sqrt(np.where(deg > 0, deg, 1)), 0.0)
    Sd = np.zeros((n, n))
    Sd[rows, S.col_idx] = S.values
    np.testing.assert_allclose(Sd, (inv[:, None] * D * inv[None, :]).astype(np.float32), rtol=2e-7, atol=0)


def test_dense_is_elementwise_function():
    X8 = synth.dense(100, 8, seed=5)
    X3 = synth.dense(100, 3, seed=5)
    assert np.array_equal(X8[:, :3], X3)
    rows = np.array([7, 99, 0, 7])
    assert np.array_equal(synth.dense_rows(rows, 8, seed=5), X8[rows])
    Xo = synth.dense(50, 8, seed=5, row0=50)
    assert np.array_equal(Xo, X8[50:])
    assert X8.min() >= -1 and X8.max() < 1
    Xi = synth.dense(1000, 8, mode="int")
    assert set(np.unique(Xi)) <= set(range(8)) and len(np.unique(Xi)) == 8


def test_chunglu_batch_sizes():
    ns = [synth.chunglu_size(g)[0] for g in range(64)]
    assert min(ns) >= 1000 and max(ns) <= 200_000
    A = synth.chunglu_csr(3)
    n, d = synth.chunglu_size(3)
    assert A.n_rows == n
    assert 0.5 * d * n < A.nnz <= d * n + 1
    deg = A.degrees()
    assert deg.max() > 20 * deg.mean()       # heavy tail


# ---- vertex relabelling and the stochastic block model (ordering study)

def test_permutation_is_uniform_bijection():
    for n in (1, 2, 10, 1000):
        p = synth.permutation(n, seed=4)
        assert np.array_equal(np.sort(p), np.arange(n))
    assert np.array_equal(synth.permutation(50, seed=1), synth.permutation(50, seed=1))
    assert not np.array_equal(synth.permutation(50, seed=1), synth.permutation(50, seed=2))
    # all 3! orders equally likely (an off-by-one in Fisher-Yates skews this)
    counts = {}
    trials = 6000
    for s in range(trials):
        key = tuple(synth.permutation(3, seed=s))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 6
    exp = trials / 6
    sd = np.sqrt(trials * (1 / 6) * (5 / 6))
    assert all(abs(c - exp) < 5 * sd for c in counts.values()), counts


@pytest.mark.parametrize("n,C,p_in", [(1 << 14, 16, 0.9), (10007, 7, 0.5), (5000, 1, 1.0), (4096, 64, 0.0)])
def test_sbm_inside_fraction_and_clusters(n, C, p_in):
    m = 200_000
    src, dst = synth.sbm_edges(n, C, m, p_in, seed=3)
    assert src.max() < n and dst.max() < n
    cs = src.astype(np.int64) * C // n
    cd = dst.astype(np.int64) * C // n
    inside = (cs == cd).mean()
    if C == 1:
        assert inside == 1.0
    else:
        sd = np.sqrt(p_in * (1 - p_in) / m)
        assert abs(inside - p_in) <= 5 * sd + 1e-12, (inside, p_in)
    # sources uniform over the vertices: cluster shares match cluster sizes
    sizes = np.bincount(np.arange(n) * C // n, minlength=C)
    share = np.bincount(cs, minlength=C) / m
    assert np.all(np.abs(share - sizes / n) < 5 * np.sqrt(sizes / n / m) + 1e-12)


def test_relabelling_preserves_degrees():
    A = synth.sbm_csr(1 << 13, 8, 12, 0.8, seed=2)
    B = synth.sbm_csr(1 << 13, 8, 12, 0.8, seed=2, permuted=True)
    assert A.nnz == B.nnz
    assert np.array_equal(np.sort(np.diff(A.row_ptr)), np.sort(np.diff(B.row_ptr)))
    assert np.array_equal(np.sort(np.bincount(A.col_idx, minlength=A.n_cols)),
                          np.sort(np.bincount(B.col_idx, minlength=B.n_cols)))
    R = synth.rmat_csr(12, seed=5)
    P = synth.rmat_permuted_csr(12, seed=5)
    assert R.nnz == P.nnz
    assert np.array_equal(np.sort(np.diff(R.row_ptr)), np.sort(np.diff(P.row_ptr)))
    # the permutation moves the hubs away from the low ids
    assert np.diff(R.row_ptr)[:16].sum() > 4 * np.diff(P.row_ptr)[:16].sum()
