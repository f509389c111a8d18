"""spmm_apply_batched: several handles, each with its own k, in one launch per
kernel instantiation (Section 3.4's single task queue).  Every entry must
match the FP64 oracle (and its own spmm_apply) at the float32 tolerance,
exactly in integer mode, in both orientations, across the launch chunks of
128 entries; misuse is rejected on the host."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import abs_product, assert_close_rel, rounded_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


def _graphs():
    gs = [synth.rmat_csr(12, seed=1, weighted=True), synth.rmat_csr(13, seed=2, weighted=True),
          synth.rmat_csr(11, seed=3, weighted=True)]
    for g in range(5):
        A = synth.chunglu_csr(g)
        A.values = synth.uniform01(A.nnz, seed=g, seed2=7)
        gs.append(A)
    return gs


@pytest.mark.parametrize("transpose", [False, True])
def test_mixed_k_matches_oracle_and_apply(sp, transpose):
    import torch
    gs = _graphs()
    ks = [1, 8, 33, 4, 16, 2, 64, 3]
    hs = [sp.SparseMatrix.from_csr(A, transpose=True) for A in gs]
    try:
        Xs, Ys, refs = [], [], []
        for i, (A, k) in enumerate(zip(gs, ks)):
            n_in, n_out = (A.n_rows, A.n_cols) if transpose else (A.n_cols, A.n_rows)
            Xh = synth.dense(n_in, k, seed=10 + i)
            Xs.append(torch.from_numpy(Xh).cuda())
            Ys.append(torch.full((n_out, k), float("nan"), device="cuda"))
            refs.append(Xh.astype(np.float64))
        sp.spmm_apply_batched([h.handle for h in hs], Xs, Ys, transpose=transpose)
        for i, (A, h) in enumerate(zip(gs, hs)):
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, refs[i], transpose=transpose)
            scale = abs_product(A, refs[i], transpose)
            assert_close_rel(Ys[i].cpu().numpy(), ref, scale, 1e-5, f"entry {i} k={ks[i]}")
            own = h.apply(Xs[i], transpose=transpose).cpu().numpy().astype(np.float64)
            assert_close_rel(Ys[i].cpu().numpy(), own, scale, 1e-5, f"entry {i} vs spmm_apply")
    finally:
        for h in hs:
            h.close()


def test_integer_exact_many_entries_two_launch_chunks(sp):
    """150 pattern graphs (two chunks of at most 128 entries), k cycling over
    1, 8, 33: exactly the oracle's result for every entry."""
    import torch
    gs = [synth.chunglu_csr(g, nmax=2e4) for g in range(150)]
    ks = [(1, 8, 33)[i % 3] for i in range(150)]
    hs = [sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None) for A in gs]
    try:
        Xs = [synth.dense(A.n_cols, k, seed=i, mode="int") for i, (A, k) in enumerate(zip(gs, ks))]
        Xd = [torch.from_numpy(X).cuda() for X in Xs]
        Ys = [torch.empty((A.n_rows, k), device="cuda") for A, k in zip(gs, ks)]
        for rep in range(2):                         # twice: the shared counter is reset per launch
            sp.spmm_apply_batched([h.handle for h in hs], Xd, Ys)
            for i, A in enumerate(gs):
                ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, Xs[i].astype(np.float64))
                assert np.array_equal(Ys[i].cpu().numpy().astype(np.float64), ref), (rep, i)
    finally:
        for h in hs:
            h.close()


def test_16bit_x_and_compensated_entries(sp):
    import torch
    gs = _graphs()[:4]
    o = sp.spmm_opts(compensated=1, task_nnz=128, long_row=128)
    hs = [sp.SparseMatrix.from_csr(A, opts=o if i % 2 else None) for i, A in enumerate(gs)]
    try:
        ks = [1, 8, 16, 2]
        Xs = [torch.from_numpy(synth.dense(A.n_cols, k, seed=i)).cuda().to(torch.bfloat16)
              for i, (A, k) in enumerate(zip(gs, ks))]
        Ys = [torch.empty((A.n_rows, k), device="cuda") for A, k in zip(gs, ks)]
        sp.spmm_apply_batched([h.handle for h in hs], Xs, Ys)
        for i, A in enumerate(gs):
            Xr = rounded_host(Xs[i])
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xr)
            assert_close_rel(Ys[i].cpu().numpy(), ref, abs_product(A, Xr), 2e-3, f"bf16 entry {i}")
    finally:
        for h in hs:
            h.close()


def test_batched_misuse_is_rejected(sp):
    import torch
    A = synth.rmat_csr(10, seed=1)
    h = sp.SparseMatrix.from_csr(A)
    hr = sp.SparseMatrix.from_csr(A, reorder=True)
    hs_ = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, streaming=True)
    X = torch.zeros((A.n_cols, 4), device="cuda")
    Y = torch.zeros((A.n_rows, 4), device="cuda")
    Y2 = torch.zeros((A.n_rows, 4), device="cuda")
    try:
        with pytest.raises(sp.SpmmError) as e:
            sp.spmm_apply_batched([h.handle, h.handle], [X, X], [Y, Y2])       # same handle twice
        assert e.value.status == sp.SPMM_ERR_ARG
        for bad in (hr, hs_):
            with pytest.raises(sp.SpmmError) as e:
                sp.spmm_apply_batched([h.handle, bad.handle], [X, X], [Y, Y2])
            assert e.value.status == sp.SPMM_ERR_UNSUPPORTED
        with pytest.raises(sp.SpmmError) as e:                                 # no transposed copy
            sp.spmm_apply_batched([h.handle], [X], [Y], transpose=True)
        assert e.value.status == sp.SPMM_ERR_ARG
    finally:
        h.close()
        hr.close()
        hs_.close()
