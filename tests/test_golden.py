"""The stored oracle reference under tests/golden, pinned on the CPU: it
describes the graph the generator makes today, it obeys the closed forms of a
normalised adjacency matrix, and an independent eigensolver (ARPACK through
scipy) finds the same eigenvalues."""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def eigs18():
    with open(os.path.join(GOLDEN, "eigs_symrmat_lcc18_top8.json")) as f:
        rec = json.load(f)
    S = synth.sym_rmat_lcc(rec["graph"]["scale"], seed=rec["graph"]["seed"])
    return rec, S


def test_eigs_reference_describes_the_generated_graph(eigs18):
    import hashlib
    rec, S = eigs18
    assert (S.n_rows, S.nnz) == (rec["graph"]["n"], rec["graph"]["nnz"])
    h = hashlib.sha256()
    for a in (np.ascontiguousarray(S.row_ptr, dtype=np.int64), np.ascontiguousarray(S.col_idx, dtype=np.int32),
              np.ascontiguousarray(S.values, dtype=np.float32)):
        h.update(a.tobytes())
    assert h.hexdigest() == rec["graph"]["csr_sha256"]


def test_eigs_reference_closed_forms(eigs18):
    """S = D^-1/2 A D^-1/2 of a connected graph: every eigenvalue lies in
    [-1, 1] and the largest is 1 (eigenvector D^1/2 1), up to the FP32
    rounding of the stored values."""
    rec, _ = eigs18
    ev = np.asarray(rec["evals"])
    assert len(ev) == 8 and np.all(np.diff(ev) <= 0)
    assert np.all(np.abs(ev) <= 1.0 + 1e-12)
    assert abs(ev[0] - 1.0) < 1e-9
    assert max(rec["residuals"]) < 1e-6


def test_eigs_reference_vs_arpack(eigs18):
    sp = pytest.importorskip("scipy.sparse")
    sla = pytest.importorskip("scipy.sparse.linalg")
    rec, S = eigs18
    M = sp.csr_matrix((np.asarray(S.values, dtype=np.float64), S.col_idx, S.row_ptr), shape=(S.n_rows, S.n_cols))
    w = np.sort(sla.eigsh(M, k=8, which="LA", tol=1e-12, return_eigenvectors=False, v0=np.ones(S.n_rows)))[::-1]
    np.testing.assert_allclose(np.asarray(rec["evals"]), w, rtol=0, atol=1e-8)
