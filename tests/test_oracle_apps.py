"""Pins for the oracle's PageRank, NMF and eigensolver: closed forms,
invariants and independent dense formulations (numpy), never the oracle
itself."""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs


# ------------------------------------------------------------------ PageRank
def google_dense_iterate(A, d, iters):
    """Dense Google-matrix power iteration: x <- G x with
    G = d * (P + dangling/N) + (1-d)/N, P[u, v] = 1/L(v) for an edge v -> u."""
    n = A.n_rows
    D = graphs.dense_of(A)
    out = D.sum(1)
    P = np.zeros((n, n))
    nz = out > 0
    P[:, nz] = (D[nz] / out[nz, None]).T
    P[:, ~nz] = 1.0 / n
    G = d * P + (1 - d) / n
    x = np.full(n, 1.0 / n)
    for _ in range(iters):
        x = G @ x
    return x


def test_pagerank_vs_dense_google_matrix():
    A = synth.rmat_csr(8, 2000, seed=3)
    x, res = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 30)
    np.testing.assert_allclose(x, google_dense_iterate(A, 0.85, 30), rtol=1e-12, atol=1e-15)
    assert abs(x.sum() - 1) < 1e-12 and np.all(x > 0)
    assert res.shape == (30,) and np.all(res >= 0)


def test_pagerank_residuals_are_l1_changes():
    """residuals[t] = sum_u |x_{t+1}(u) - x_t(u)|, against the dense Google
    iteration's own iterates."""
    A = synth.rmat_csr(7, 900, seed=6)
    _, res = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 12)
    prev = np.full(A.n_rows, 1.0 / A.n_rows)
    for t in range(12):
        cur = google_dense_iterate(A, 0.85, t + 1)
        np.testing.assert_allclose(res[t], np.abs(cur - prev).sum(), rtol=1e-9, atol=1e-16)
        prev = cur
    assert res[0] > 1e-3                       # a skewed graph moves away from 1/N


def test_pagerank_uniform_on_regular_graphs():
    for A in (graphs.cycle(19), graphs.complete(11)):
        x, res = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 30)
        np.testing.assert_allclose(x, 1.0 / A.n_rows, rtol=1e-14)
        assert res.max() < 1e-15


def test_pagerank_two_node_closed_form():
    # 0 -> 1, vertex 1 dangling: stationary x0 = 1/(2+d), x1 = (1+d)/(2+d)
    A = graphs.csr_from_edges(2, 2, [0], [1])
    d = 0.85
    x, _ = oracle.pagerank(2, A.row_ptr, A.col_idx, d, 400)
    np.testing.assert_allclose(x, [1 / (2 + d), (1 + d) / (2 + d)], rtol=1e-14)


def test_pagerank_sums_to_one_every_iteration():
    A = synth.rmat_csr(10, seed=1)
    x = None
    for t in range(5):
        x, _ = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 1, x0=x)
        assert abs(x.sum() - 1) < 1e-12 and x.min() >= 0


# ----------------------------------------------------------------------- NMF
def nmf_dense(D, W, H, steps, eps):
    W, H = W.copy(), H.copy()
    obj = [np.linalg.norm(D - W @ H) ** 2]
    for _ in range(steps):
        H = H * (W.T @ D) / (W.T @ W @ H + eps)
        W = W * (D @ H.T) / (W @ H @ H.T + eps)
        obj.append(np.linalg.norm(D - W @ H) ** 2)
    return W, H, np.array(obj)


@pytest.mark.parametrize("weighted", [False, True])
def test_nmf_vs_dense_updates(weighted):
    A = graphs.random_csr(40, 30, 0.15, seed=5, weighted=weighted)
    D = graphs.dense_of(A)
    k = 4
    W0 = synth.dense(40, k, seed=1, mode="unit").astype(np.float64) + 0.01
    Ht0 = synth.dense(30, k, seed=2, mode="unit").astype(np.float64) + 0.01
    W, Ht, obj = oracle.nmf(40, 30, A.row_ptr, A.col_idx, A.values, W0, Ht0, 12)
    Wd, Hd, objd = nmf_dense(D, W0, Ht0.T, 12, 1e-12)
    np.testing.assert_allclose(W, Wd, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(Ht, Hd.T, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(obj, objd, rtol=1e-9, atol=1e-9)


def test_nmf_objective_non_increasing():
    A = synth.rmat_csr(9, seed=2)
    k = 8
    W0 = synth.dense(A.n_rows, k, seed=3, mode="unit") + 0.01
    Ht0 = synth.dense(A.n_cols, k, seed=4, mode="unit") + 0.01
    W, Ht, obj = oracle.nmf(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, W0, Ht0, 20)
    assert np.all(np.diff(obj) <= 1e-9 * obj[:-1])
    assert W.min() >= 0 and Ht.min() >= 0


# ---------------------------------------------------------------- eigensolver
def test_sym_eigh_vs_numpy_eigh():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((17, 17))
    M = M + M.T
    ev, V = oracle.sym_eigh(M)
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(M), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(M @ V, V * ev[None, :], atol=1e-11)
    np.testing.assert_allclose(V.T @ V, np.eye(17), atol=1e-12)


def test_sym_eigh_repeated_and_clustered_eigenvalues():
    """A multiple eigenvalue and a tight cluster: the vectors of each must
    still be orthonormal eigenvectors (inverse iteration re-orthogonalises
    within clusters)."""
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((24, 24)))
    lam = np.r_[np.full(5, 0.75), 0.5 + 1e-9 * np.arange(4), np.linspace(-1, 0.4, 15)]
    M = (Q * lam[None, :]) @ Q.T
    M = 0.5 * (M + M.T)
    ev, V = oracle.sym_eigh(M)
    np.testing.assert_allclose(ev, np.sort(lam), atol=1e-13)
    np.testing.assert_allclose(M @ V, V * ev[None, :], atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(24), atol=1e-10)


def test_sym_eigh_tridiagonal_and_diagonal_inputs():
    # already tridiagonal (Householder leaves it), and diagonal with zeros off it
    m = 30
    d = np.linspace(-2, 3, m)
    T = np.diag(d) + np.diag(np.full(m - 1, 0.3), 1) + np.diag(np.full(m - 1, 0.3), -1)
    ev, V = oracle.sym_eigh(T)
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(T), atol=1e-13)
    np.testing.assert_allclose(T @ V, V * ev[None, :], atol=1e-12)
    D = np.diag(np.r_[3.0, -1.0, 2.0, 2.0, 0.0])
    ev, V = oracle.sym_eigh(D)
    np.testing.assert_allclose(ev, [-1.0, 0.0, 2.0, 2.0, 3.0], atol=1e-15)
    np.testing.assert_allclose(np.abs(V.T @ V), np.eye(5), atol=1e-12)


def test_svds_vs_numpy_svd():
    """Singular values through Lanczos on A^T A (two products per step)."""
    A = synth.rmat_csr(8, seed=4, weighted=True)
    D = graphs.dense_of(A)
    Q0 = synth.dense(A.n_cols, 6, seed=2).astype(np.float64)
    sv, V, m = oracle.svds(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Q0, 5, A.n_cols)
    ref = np.linalg.svd(D, compute_uv=False)[:5]
    np.testing.assert_allclose(sv, ref, rtol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(D @ V, axis=0), sv, rtol=1e-9)      # ||A v|| = s
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-9)


def test_svds_rectangular_closed_form():
    """A 3 x 5 matrix with orthogonal rows of norms 3, 2, 1: singular values
    3, 2, 1 whatever the column count."""
    rows = [[0, 1], [2], [3, 4]]
    vals = [[3 / np.sqrt(2), 3 / np.sqrt(2)], [2.0], [0.6, 0.8]]
    rp = np.r_[0, np.cumsum([len(r) for r in rows])].astype(np.int64)
    ci = np.concatenate(rows).astype(np.int32)
    va = np.concatenate(vals).astype(np.float64)
    Q0 = synth.dense(5, 3, seed=1).astype(np.float64)
    sv, _, _ = oracle.svds(3, 5, rp, ci, va, Q0, 3, 5)
    np.testing.assert_allclose(sv, [3.0, 2.0, 1.0], atol=1e-12)


def _normalised(A):
    D = graphs.dense_of(A)
    deg = D.sum(1)
    inv = np.where(deg > 0, 1 / np.sqrt(np.where(deg > 0, deg, 1)), 0)
    S = inv[:, None] * D * inv[None, :]
    Sc = graphs.csr_from_edges(A.n_rows, A.n_cols, *np.nonzero(S), S[np.nonzero(S)])
    return S, Sc


def test_lanczos_cycle_closed_form():
    # normalised adjacency of the undirected cycle C_n is A/2: eigenvalues cos(2 pi j / n)
    n = 40
    i = np.arange(n)
    A = graphs.csr_from_edges(n, n, np.r_[i, (i + 1) % n], np.r_[(i + 1) % n, i])
    S, Sc = _normalised(A)
    Q0 = synth.dense(n, 4, seed=1).astype(np.float64)
    ev, V, m = oracle.lanczos(n, Sc.row_ptr, Sc.col_idx, Sc.values.astype(np.float64), Q0, 5, 40)
    expect = np.sort(np.cos(2 * np.pi * np.arange(n) / n))[::-1][:5]
    np.testing.assert_allclose(ev, expect, atol=1e-10)
    np.testing.assert_allclose(S @ V, V * ev[None, :], atol=1e-9)


def test_lanczos_complete_graph():
    n = 12
    A = graphs.complete(n)
    S, Sc = _normalised(A)
    Q0 = synth.dense(n, 3, seed=2).astype(np.float64)
    ev, _, _ = oracle.lanczos(n, Sc.row_ptr, Sc.col_idx, Sc.values.astype(np.float64), Q0, 3, 12)
    np.testing.assert_allclose(ev, [1.0, -1.0 / (n - 1), -1.0 / (n - 1)], atol=1e-12)


def test_lanczos_vs_dense_eigh_on_rmat():
    A = synth.sym_rmat_csr(8, seed=3, normalise=True)
    n = A.n_rows
    S = graphs.dense_of(A)
    Q0 = synth.dense(n, 8, seed=5).astype(np.float64)
    ev, V, m = oracle.lanczos(n, A.row_ptr, A.col_idx, A.values, Q0, 6, n)
    np.testing.assert_allclose(ev, np.sort(np.linalg.eigvalsh(S))[::-1][:6], atol=1e-9)


def test_lanczos_vs_dense_eigh_on_normalised_lcc():
    # the eigensolver's benchmark matrix family: normalised symmetric R-MAT,
    # largest connected component, top eigenvalue 1 (simple)
    S = synth.sym_rmat_lcc(9, seed=2)
    D = graphs.dense_of(S)
    assert np.allclose(D, D.T)
    ref = np.sort(np.linalg.eigvalsh(D))[::-1][:8]
    Q0 = synth.dense(S.n_rows, 8, seed=3).astype(np.float64)
    ev, V, m = oracle.lanczos(S.n_rows, S.row_ptr, S.col_idx, S.values, Q0, 8, 200)
    np.testing.assert_allclose(ev, ref, atol=1e-9)
    assert abs(ev[0] - 1.0) < 1e-9 and ev[1] < 1 - 1e-6
