"""SPMM_RELABEL: the handle stores P A P^T with the vertices numbered by
decreasing degree.  Every call that takes vectors in the input order must
give the oracle's result in the input order (integer-exact for pattern A and
integer X; within the FP32 tolerance otherwise); the relabelled-order entry
point must agree with the permuted input-order one; the applications must
match the oracle as on a plain handle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import abs_product, assert_close_rel, rounded_host, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


@pytest.fixture(scope="module")
def rmat14():
    return synth.rmat_csr(14, seed=2)


@pytest.fixture(scope="module")
def rmat14w():
    return synth.rmat_csr(14, seed=4, weighted=True)


@pytest.fixture(scope="module")
def hp(sp, rmat14):
    h = sp.SparseMatrix.from_csr(rmat14, transpose=True, relabel=True)
    yield h
    h.close()


@pytest.fixture(scope="module")
def hw(sp, rmat14w):
    h = sp.SparseMatrix.from_csr(rmat14w, transpose=True, relabel=True)
    yield h
    h.close()


def test_info_and_order(sp, rmat14, hp):
    A = rmat14
    assert hp.info()["relabelled"] == 1
    o = hp.vertex_order()
    np.testing.assert_array_equal(o, sp.spmm_relabel_order(A.n_rows, A.row_ptr, A.col_idx))
    h0 = sp.SparseMatrix.from_csr(A)
    try:
        assert h0.info()["relabelled"] == 0
        np.testing.assert_array_equal(h0.vertex_order(), np.arange(A.n_rows, dtype=np.int32))
    finally:
        h0.close()


@pytest.mark.parametrize("k", [1, 2, 3, 8, 33, 64])
@pytest.mark.parametrize("transpose", [False, True])
def test_integer_exact(sp, rmat14, hp, k, transpose):
    A = rmat14
    X = synth.dense(A.n_rows, k, seed=k, mode="int")
    Y = hp.apply(to_dev(X), transpose=transpose).cpu().numpy().astype(np.float64)
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X, transpose=transpose)
    assert np.array_equal(Y, ref)


@pytest.mark.parametrize("k", [1, 4, 16, 64])
@pytest.mark.parametrize("transpose", [False, True])
def test_weighted_f32(sp, rmat14w, hw, k, transpose):
    A = rmat14w
    X = synth.dense(A.n_rows, k, seed=10 + k)
    Y = hw.apply(to_dev(X), transpose=transpose).cpu().numpy()
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X, transpose=transpose)
    assert_close_rel(Y, ref, abs_product(A, X.astype(np.float64), transpose), 1e-5, "relabel f32")


@pytest.mark.parametrize("k", [2, 8])
def test_bf16_x_and_strided(sp, rmat14w, hw, k):
    import torch
    A = rmat14w
    Xw = to_dev(synth.dense(A.n_rows, k + 3, seed=k), torch.bfloat16)
    X = Xw[:, 1:1 + k]                            # unaligned, ldx = k + 3
    Yw = torch.full((A.n_rows, k + 2), -7.0, device="cuda")
    Y = hw.apply(X, Y=Yw[:, :k])
    Xh = rounded_host(X)
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xh)
    assert_close_rel(Y.cpu().numpy(), ref, abs_product(A, Xh), 1e-5, "relabel bf16")
    assert torch.all(Yw[:, k:] == -7.0)           # columns past k untouched


def test_relabelled_order_entry_points(sp, rmat14w, hw):
    """apply_relabelled on rows moved into the handle's order, moved back, is
    apply() bit for bit; the moves are the permutation old_of_new."""
    import torch
    A = rmat14w
    o = hw.vertex_order()
    for k, dt in ((1, torch.float32), (8, torch.float32), (16, torch.bfloat16)):
        X = to_dev(synth.dense(A.n_rows, k, seed=20 + k), dt)
        Xr = hw.to_handle_order(X)
        assert torch.equal(Xr.cpu(), X.cpu()[torch.from_numpy(o.astype(np.int64))])
        assert torch.equal(hw.to_input_order(Xr), X)
        for tr in (False, True):
            Yr = hw.apply_relabelled(Xr, transpose=tr)
            assert torch.equal(hw.to_input_order(Yr), hw.apply(X, transpose=tr))
    V = to_dev(synth.dense(A.n_rows, 3, seed=1).astype(np.float64))      # F64 rows move too
    assert torch.equal(hw.to_input_order(hw.to_handle_order(V)), V)


def test_pagerank_matches_oracle(sp, rmat14, hp):
    A = rmat14
    x, res = hp.pagerank(0.85, 30)
    xr, resr = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 30)
    xg = x.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(xg - xr) <= 1e-5 * xr + 1e-12), np.max(np.abs(xg - xr) / xr)
    np.testing.assert_allclose(res, resr, rtol=1e-3, atol=4 * 2.0 ** -24)
    x2, res2 = hp.pagerank(0.85, 30)                       # the cached graph
    assert np.array_equal(x2.cpu().numpy(), x.cpu().numpy()) and np.array_equal(res2, res)
    x0 = synth.dense(A.n_rows, 1, seed=3, mode="unit")[:, 0]
    x0 = (x0 / x0.sum()).astype(np.float32)
    x3, _ = hp.pagerank(0.85, 7, x0=to_dev(x0))
    xr3, _ = oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, 7, x0=x0.astype(np.float64))
    assert np.all(np.abs(x3.cpu().numpy() - xr3) <= 1e-5 * xr3 + 1e-12)


def test_eigensolvers_match_oracle(sp):
    import torch
    S = synth.sym_rmat_lcc(12, seed=1)
    n = S.n_rows
    h = sp.SparseMatrix.from_csr(S, relabel=True)
    try:
        Q0 = synth.dense(n, 8, seed=9).astype(np.float64)
        evr, _, _ = oracle.lanczos(n, S.row_ptr, S.col_idx, S.values, Q0, 8, 400)
        V0 = to_dev(synth.dense(n, 16, seed=1).astype(np.float64))
        for solve in ("ks", "filtered"):
            U = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
            if solve == "ks":
                ev, res, _ = h.eigs(8, V0, block=16, max_basis=64, max_restarts=300, tol=1e-6, evecs=U)
            else:
                ev, res, _ = h.eigs_filtered(8, V0, degree=16, lower=-1.0, max_iters=300, tol=1e-6, evecs=U)
            np.testing.assert_allclose(ev, evr, atol=2e-6)
            u = U.cpu().numpy()
            SU = oracle.spmm(n, n, S.row_ptr, S.col_idx, S.values, u)     # vectors in the input order
            assert np.all(np.linalg.norm(SU - u * ev[None, :], axis=0) <= 2e-5), solve
            np.testing.assert_allclose(u.T @ u, np.eye(8), atol=1e-8)
    finally:
        h.close()


def test_svds_matches_oracle(sp):
    import torch
    A = synth.rmat_csr(12, seed=6, weighted=True)
    Q0 = synth.dense(A.n_cols, 8, seed=3).astype(np.float64)
    ref, _, _ = oracle.svds(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Q0, 6, 400)
    h = sp.SparseMatrix.from_csr(A, transpose=True, relabel=True)
    try:
        V = torch.zeros((A.n_cols, 6), dtype=torch.float64, device="cuda")
        sv, _, _ = h.svds(6, to_dev(synth.dense(A.n_cols, 16, seed=0).astype(np.float64)), block=16, max_basis=64,
                          max_restarts=400, tol=1e-6, right_vecs=V)
        np.testing.assert_allclose(sv, ref, rtol=1e-6)
        v = V.cpu().numpy()
        Av = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, v)
        np.testing.assert_allclose(np.linalg.norm(Av, axis=0), sv, rtol=1e-5)
    finally:
        h.close()


def test_nmf_matches_oracle(sp):
    import torch
    A = synth.rmat_csr(11, seed=7, weighted=True)
    k, steps = 8, 30
    W0 = synth.dense(A.n_rows, k, seed=1, mode="unit") + np.float32(0.01)
    H0 = synth.dense(A.n_cols, k, seed=2, mode="unit") + np.float32(0.01)
    h = sp.SparseMatrix.from_csr(A, transpose=True, relabel=True)
    try:
        W, Ht = to_dev(W0.copy()), to_dev(H0.copy())
        obj = h.nmf(k, steps, W, Ht)[0]
        Wr, Hr, objr = oracle.nmf(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, W0, H0, steps)
        np.testing.assert_allclose(obj, objr, rtol=1e-4)
        np.testing.assert_allclose(W.cpu().numpy(), Wr, rtol=1e-2, atol=1e-4 * np.abs(Wr).max())
        np.testing.assert_allclose(Ht.cpu().numpy(), Hr, rtol=1e-2, atol=1e-4 * np.abs(Hr).max())
        assert np.all(np.diff(obj) <= 1e-6 * obj[:-1])
    finally:
        h.close()


def test_unsupported_combinations(sp, rmat14, hp):
    import torch
    A = rmat14
    X = to_dev(synth.dense(A.n_rows, 4, seed=0))
    Y = torch.empty((A.n_rows, 4), device="cuda")
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_apply_batched([hp.handle], [X], [Y])
    assert e.value.status == sp.SPMM_ERR_UNSUPPORTED
    with pytest.raises(sp.SpmmError) as e:
        hp.apply_host(synth.dense(A.n_rows, 4, seed=0), np.empty((A.n_rows, 4), np.float32))
    assert e.value.status == sp.SPMM_ERR_UNSUPPORTED
    with pytest.raises(sp.SpmmError) as e:
        sp.SparseMatrix.batched([A, A], relabel=True)
    assert e.value.status == sp.SPMM_ERR_UNSUPPORTED


@pytest.mark.parametrize("case", ["one_vertex_empty", "empty_5", "loops_and_isolated", "ragged_small"])
def test_degenerate_matrices(sp, case):
    """Tiny and degenerate square matrices through every entry point that
    takes vectors: results in the input order equal the oracle's exactly."""
    import torch
    from tests import graphs
    if case == "one_vertex_empty":
        n, rp, ci = 1, np.array([0, 0]), np.zeros(0, np.int32)
    elif case == "empty_5":
        n, rp, ci = 5, np.zeros(6, np.int64), np.zeros(0, np.int32)
    elif case == "loops_and_isolated":
        n, rp, ci = 6, np.array([0, 1, 1, 3, 3, 4, 4]), np.array([0, 2, 5, 4], np.int32)
    else:
        A = synth.rmat_csr(7, seed=11)
        n, rp, ci = A.n_rows, A.row_ptr, A.col_idx
    rp = np.asarray(rp, np.int64)
    h = sp.SparseMatrix(n, n, rp, ci, None, transpose=True, relabel=True)
    try:
        np.testing.assert_array_equal(h.vertex_order(), sp.spmm_relabel_order(n, rp, ci))
        for k in (1, 3, 64):
            X = synth.dense(n, k, seed=k, mode="int")
            for tr in (False, True):
                Y = h.apply(to_dev(X), transpose=tr).cpu().numpy().astype(np.float64)
                assert np.array_equal(Y, oracle.spmm(n, n, rp, ci, None, X, transpose=tr)), (case, k, tr)
                Yr = h.to_input_order(h.apply_relabelled(h.to_handle_order(to_dev(X)), transpose=tr))
                assert np.array_equal(Yr.cpu().numpy().astype(np.float64), Y)
        if rp[-1] > 0:
            x, _ = h.pagerank(0.85, 5)
            xr, _ = oracle.pagerank(n, rp, ci, 0.85, 5)
            assert np.all(np.abs(x.cpu().numpy() - xr) <= 1e-5 * xr + 1e-12)
    finally:
        h.close()


@pytest.mark.parametrize("vdtype", ["bfloat16", "float16"])
@pytest.mark.parametrize("k", [1, 8, 64])
def test_16bit_values(sp, rmat14w, vdtype, k):
    """Stored 16-bit values move with their entries: X of the same type,
    both orientations, against the oracle on the rounded inputs."""
    import torch
    A = rmat14w
    vt = torch.from_numpy(A.values).to(getattr(torch, vdtype))
    vr = vt.float().numpy().astype(np.float64)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vt, transpose=True, relabel=True)
    try:
        Xd = to_dev(synth.dense(A.n_cols, k, seed=4 + k), getattr(torch, vdtype))
        Xr = rounded_host(Xd)
        for tr in (False, True):
            Y = h.apply(Xd, transpose=tr).cpu().numpy()
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vr, Xr, transpose=tr)
            scale = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, np.abs(vr), np.abs(Xr), transpose=tr)
            assert_close_rel(Y, ref, scale, 2e-3, f"relabel {vdtype} values k={k} t={tr}")
    finally:
        h.close()


@pytest.mark.parametrize("k", [1, 16])
def test_compensated_plan(sp, rmat14w, k):
    """Compensated sums for long rows and hub segments on the relabelled
    matrix: the same parity, and the hub rows' partials still add up."""
    A = rmat14w
    o = sp.spmm_opts(compensated=1, long_row=64, task_nnz=64, short_max=15)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, transpose=True, relabel=True, opts=o)
    try:
        assert h.info()["n_split_rows"] > 0
        X = synth.dense(A.n_rows, k, seed=30 + k)
        for tr in (False, True):
            Y = h.apply(to_dev(X), transpose=tr).cpu().numpy()
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X, transpose=tr)
            assert_close_rel(Y, ref, abs_product(A, X.astype(np.float64), tr), 1e-5, f"compensated k={k} t={tr}")
    finally:
        h.close()


def test_relabelled_entry_strided_and_misaligned(sp, rmat14w, hw):
    """spmm_apply_relabelled with X and Y as column windows of wider arrays
    (leading dimension > k, X starting off a 16-byte boundary): the same
    sums as on contiguous copies, within the FP32 tolerance."""
    import torch
    A = rmat14w
    k = 5
    Xw = to_dev(synth.dense(A.n_rows, k + 3, seed=8))
    X = Xw[:, 1:1 + k]
    Xr = torch.empty((A.n_rows, k + 3), device="cuda")[:, 2:2 + k]
    sp.spmm_relabel_rows(hw.handle, X, Xr, True)
    Yw = torch.full((A.n_rows, k + 4), 5.0, device="cuda")
    hw.apply_relabelled(Xr, Y=Yw[:, :k])
    Y = hw.to_input_order(Yw[:, :k].contiguous())
    Xh = X.cpu().numpy().astype(np.float64)
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xh)
    assert_close_rel(Y.cpu().numpy(), ref, abs_product(A, Xh), 1e-5, "strided relabelled")
    assert torch.all(Yw[:, k:] == 5.0)
