"""GPU block eigensolver (Section 4.2) against closed forms and the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


@pytest.fixture(scope="module")
def lcc12():
    return synth.sym_rmat_lcc(12, seed=1)


def start_block(n, b, seed=0):
    import torch
    return torch.from_numpy(synth.dense(n, b, seed=seed).astype(np.float64)).cuda()


def test_cycle_closed_form(sp):
    n = 200
    i = np.arange(n)
    C = graphs.csr_from_edges(n, n, np.r_[i, (i + 1) % n], np.r_[(i + 1) % n, i], np.full(2 * n, 0.5))
    h = sp.SparseMatrix.from_csr(C)
    ev, res, _ = h.eigs(8, start_block(n, 8), block=8, max_basis=32, max_restarts=400, tol=1e-6)
    expect = np.sort(np.cos(2 * np.pi * np.arange(n) / n))[::-1][:8]
    np.testing.assert_allclose(ev, expect, atol=2e-6)
    assert np.all(res <= 1e-6)
    h.close()


@pytest.mark.parametrize("xdtype,tol,atol", [("f32", 1e-6, 2e-6), ("bf16", 5e-3, 2e-3)])
def test_rmat_lcc_matches_oracle(sp, lcc12, xdtype, tol, atol):
    import torch
    S = lcc12
    n = S.n_rows
    h = sp.SparseMatrix.from_csr(S)
    evecs = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    xt = sp.SPMM_F32 if xdtype == "f32" else sp.SPMM_BF16
    ev, res, nrest = h.eigs(8, start_block(n, 16), block=16, max_basis=64, max_restarts=300, tol=tol, xtype=xt,
                            evecs=evecs)
    Q0 = synth.dense(n, 8, seed=9).astype(np.float64)
    evr, _, _ = oracle.lanczos(n, S.row_ptr, S.col_idx, S.values, Q0, 8, 400)
    np.testing.assert_allclose(ev, evr, atol=atol)
    assert np.all(res <= tol), res
    U = evecs.cpu().numpy()
    SU = oracle.spmm(n, n, S.row_ptr, S.col_idx, S.values, U)
    true_res = np.linalg.norm(SU - U * ev[None, :], axis=0)
    assert np.all(true_res <= 20 * tol), true_res
    np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-8 if xdtype == "f32" else 1e-6)
    h.close()


def test_eigs_argument_errors(sp):
    n = 100
    C = graphs.cycle(n)
    h = sp.SparseMatrix(n, n, C.row_ptr, C.col_idx, None)
    with pytest.raises(sp.SpmmError):                       # nev + 2*block > max_basis
        h.eigs(8, start_block(n, 16), block=16, max_basis=32)
    with pytest.raises(sp.SpmmError):                       # basis larger than n
        h.eigs(4, start_block(n, 8), block=8, max_basis=200)
    h.close()


def test_svds_matches_dense_svd(sp):
    """Top singular values of a directed R-MAT graph (via A^T A) against
    numpy's dense SVD."""
    import torch
    A = synth.rmat_csr(11, seed=4, weighted=True)
    D = graphs.dense_of(A)
    ref = np.linalg.svd(D, compute_uv=False)[:6]
    h = sp.SparseMatrix.from_csr(A, transpose=True)
    V = torch.zeros((A.n_cols, 6), dtype=torch.float64, device="cuda")
    sv, res, _ = h.svds(6, start_block(A.n_cols, 16), block=16, max_basis=64, max_restarts=300, tol=1e-5,
                        right_vecs=V)
    np.testing.assert_allclose(sv, ref, rtol=1e-6)
    v = V.cpu().numpy()
    np.testing.assert_allclose(np.linalg.norm(D @ v, axis=0), sv, rtol=1e-5)     # ||A v|| = s
    h.close()


def test_svds_matches_oracle(sp):
    """Top singular values of a weighted directed R-MAT graph (Section 5.5.2's
    SVD of a directed graph) against the FP64 oracle's Lanczos on A^T A, and
    the right singular vectors' ||A v|| = s through the oracle's product."""
    import torch
    A = synth.rmat_csr(12, seed=6, weighted=True)
    Q0 = synth.dense(A.n_cols, 8, seed=3).astype(np.float64)
    ref, _, _ = oracle.svds(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Q0, 6, 400)
    h = sp.SparseMatrix.from_csr(A, transpose=True)
    try:
        V = torch.zeros((A.n_cols, 6), dtype=torch.float64, device="cuda")
        sv, res, _ = h.svds(6, start_block(A.n_cols, 16), block=16, max_basis=64, max_restarts=400, tol=1e-6,
                            right_vecs=V)
        np.testing.assert_allclose(sv, ref, rtol=1e-6)
        v = V.cpu().numpy()
        Av = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, v)
        np.testing.assert_allclose(np.linalg.norm(Av, axis=0), sv, rtol=1e-5)
    finally:
        h.close()


def test_filtered_cycle_closed_form(sp):
    n = 200
    i = np.arange(n)
    C = graphs.csr_from_edges(n, n, np.r_[i, (i + 1) % n], np.r_[(i + 1) % n, i], np.full(2 * n, 0.5))
    h = sp.SparseMatrix.from_csr(C)
    try:
        ev, res, it = h.eigs_filtered(8, start_block(n, 16), degree=10, lower=-1.0, max_iters=400, tol=1e-6)
        expect = np.sort(np.cos(2 * np.pi * np.arange(n) / n))[::-1][:8]
        np.testing.assert_allclose(ev, expect, atol=2e-6)
        assert np.all(res <= 1e-6), res
    finally:
        h.close()


@pytest.mark.parametrize("xdtype,tol,atol", [("f32", 1e-6, 2e-6), ("bf16", 5e-3, 2e-3)])
def test_filtered_rmat_lcc_matches_oracle(sp, lcc12, xdtype, tol, atol):
    """Chebyshev-filtered subspace iteration on the normalised R-MAT LCC:
    eigenvalues against the FP64 oracle's Lanczos, true residuals through the
    oracle's product, orthonormal vectors."""
    import torch
    S = lcc12
    n = S.n_rows
    h = sp.SparseMatrix.from_csr(S)
    try:
        evecs = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
        xt = sp.SPMM_F32 if xdtype == "f32" else sp.SPMM_BF16
        ev, res, it = h.eigs_filtered(8, start_block(n, 16), degree=16, lower=-1.0, max_iters=300, tol=tol,
                                      xtype=xt, evecs=evecs)
        Q0 = synth.dense(n, 8, seed=9).astype(np.float64)
        evr, _, _ = oracle.lanczos(n, S.row_ptr, S.col_idx, S.values, Q0, 8, 400)
        np.testing.assert_allclose(ev, evr, atol=atol)
        assert np.all(res <= tol), res
        U = evecs.cpu().numpy()
        SU = oracle.spmm(n, n, S.row_ptr, S.col_idx, S.values, U)
        true_res = np.linalg.norm(SU - U * ev[None, :], axis=0)
        assert np.all(true_res <= 20 * tol), true_res
        np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-8 if xdtype == "f32" else 1e-6)
    finally:
        h.close()


def test_filtered_argument_errors(sp):
    n = 100
    C = graphs.cycle(n)
    h = sp.SparseMatrix(n, n, C.row_ptr, C.col_idx, None)
    try:
        with pytest.raises(sp.SpmmError):                   # block must exceed nev
            h.eigs_filtered(8, start_block(n, 8), degree=4)
        with pytest.raises(sp.SpmmError):                   # degree 0
            h.eigs_filtered(4, start_block(n, 8), degree=0)
        with pytest.raises(sp.SpmmError):                   # the lower bound lies above the block's Ritz values
            h.eigs_filtered(4, start_block(n, 8), degree=4, lower=5.0, tol=1e-12)
    finally:
        h.close()


def test_filtered_scale18_vs_stored_oracle(sp):
    """Section 4.2's eigenproblem at the size the precision configuration
    reports its errors on (normalised symmetrised R-MAT LCC, scale 18): the
    FP32 filtered solve against the FP64 oracle's stored eigenvalues."""
    import json
    import os
    import torch
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "eigs_symrmat_lcc18_top8.json")) as f:
        rec = json.load(f)
    S = synth.sym_rmat_lcc(18, seed=0)
    assert (S.n_rows, S.nnz) == (rec["graph"]["n"], rec["graph"]["nnz"])
    h = sp.SparseMatrix.from_csr(S)
    try:
        ev, res, it = h.eigs_filtered(8, start_block(S.n_rows, 16, seed=1), degree=20, lower=-1.0, max_iters=300,
                                      tol=1e-6)
        assert np.all(res <= 1e-6), res
        np.testing.assert_allclose(ev, rec["evals"], rtol=0, atol=2e-7)
    finally:
        h.close()


@pytest.mark.parametrize("values,block,nev", [((1.0,), 4, 4), ((1.0, 0.5, 0.0), 2, 2)])
def test_krylov_on_invariant_subspace(sp, values, block, nev):
    """A diagonal S with few distinct eigenvalues: the block Krylov space is
    invariant after a few expansions.  Whatever the device-side expansions do
    beyond it (a CholQR2 breakdown that ends the basis, or rounding noise
    orthonormalised into new directions), the Ritz values are the exact top
    eigenvalue (1, of multiplicity >= nev) at the first Rayleigh-Ritz step,
    with residuals at the rounding level of the FP32 products (~1e-8)."""
    n = 60
    d = np.array([values[i % len(values)] for i in range(n)])
    C = graphs.csr_from_edges(n, n, np.arange(n), np.arange(n), d)
    h = sp.SparseMatrix.from_csr(C)
    try:
        ev, res, nrest = h.eigs(nev, start_block(n, block, seed=3), block=block, max_basis=4 * block + nev,
                                max_restarts=5, tol=1e-6)
        np.testing.assert_allclose(ev, np.ones(nev), atol=1e-7)
        assert np.all(res <= 1e-6) and nrest == 0, (res, nrest)
    finally:
        h.close()
