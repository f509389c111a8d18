"""Hot columns (spmm_opts.hot_cols): a second copy of each orientation's
column indices names the most-referenced columns by rank, and calls whose X
rows take at most 4 bytes gather those rows from a copy in shared memory.
Only the address a row is read from changes, so a handle with hot columns
must give the same float32 result as one without, bit for bit, in both
orientations, for every k and X type (wider rows simply do not use the hot
copy); and the integer mode must match the FP64 oracle exactly."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import abs_product, assert_close_rel, rounded_host

pytestmark = pytest.mark.gpu


def _handles(A, H, transpose=True, values=None):
    from paper_1602_02864_gb300 import spmm as sp
    vals = A.values if values is None else values
    plain = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vals, transpose=transpose,
                            opts=sp.spmm_opts(hot_cols=-1))
    hot = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vals, transpose=transpose,
                          opts=sp.spmm_opts(hot_cols=H))
    return plain, hot


def _expected_hot(counts, H):
    return int(min(H, int((counts >= 2).sum())))


@pytest.mark.parametrize("H,weighted", [(1, True), (100, True), (1000, True), (1 << 20, True), (8192, False),
                                        (1 << 20, False)])
def test_hot_handle_equals_plain_handle(H, weighted):
    import torch
    A = synth.rmat_csr(14, seed=3, weighted=weighted)
    plain, hot = _handles(A, H)
    try:
        info = hot.info()
        indeg = np.bincount(A.col_idx, minlength=A.n_cols)
        outdeg = np.diff(A.row_ptr)
        for got, cnt in ((info["n_hot"], indeg), (info["n_hot_t"], outdeg)):
            if H <= 1000 or (not weighted and H <= 8192):   # room for them: exactly the columns asked for
                assert got == _expected_hot(cnt, H)
            else:               # capped by the room in shared memory beside the staging buffers
                assert 0 < got <= _expected_hot(cnt, H)
        assert plain.info()["n_hot"] == 0 and plain.info()["n_hot_t"] == 0
        for k in (1, 2, 4, 8, 16, 33, 64):
            X = torch.from_numpy(synth.dense(A.n_cols, k, seed=k)).cuda()
            for tr in (False, True):
                Yp = plain.apply(X, transpose=tr)
                Yh = hot.apply(X, transpose=tr)
                assert torch.equal(Yp, Yh), f"H={H} k={k} transpose={tr}"
    finally:
        plain.close()
        hot.close()


def test_hot_default_is_automatic_by_size():
    from paper_1602_02864_gb300 import spmm as sp
    small = synth.rmat_csr(12, seed=1)
    big = synth.rmat_csr(17, seed=1)          # > 2^20 stored entries
    assert small.nnz < 1 << 20 <= big.nnz
    hs = sp.SparseMatrix.from_csr(small, transpose=True)
    hb = sp.SparseMatrix.from_csr(big, transpose=True)
    try:
        assert hs.info()["n_hot"] == 0 and hs.info()["n_hot_t"] == 0
        assert hb.info()["n_hot"] == 8192 and hb.info()["n_hot_t"] == 8192
    finally:
        hs.close()
        hb.close()


def test_hot_compensated_and_repeated_calls():
    import torch
    from paper_1602_02864_gb300 import spmm as sp
    A = synth.rmat_csr(13, seed=4, weighted=True)
    o = dict(compensated=1, task_nnz=128, long_row=128)
    plain = sp.SparseMatrix.from_csr(A, transpose=True, opts=sp.spmm_opts(hot_cols=-1, **o))
    hot = sp.SparseMatrix.from_csr(A, transpose=True, opts=sp.spmm_opts(hot_cols=2000, **o))
    try:
        for k in (1, 4):
            for rep in range(3):            # the hot copy is refreshed from each call's X
                X = torch.from_numpy(synth.dense(A.n_cols, k, seed=10 * k + rep)).cuda()
                for tr in (False, True):
                    assert torch.equal(plain.apply(X, transpose=tr), hot.apply(X, transpose=tr)), (k, rep, tr)
    finally:
        plain.close()
        hot.close()


@pytest.mark.parametrize("xname", ["bf16", "f16"])
def test_hot_16bit_x_and_values(xname):
    import torch
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[xname]
    A = synth.rmat_csr(13, seed=5, weighted=True)
    v16 = torch.from_numpy(A.values).to(tdt)
    for vals in (None, v16):
        plain, hot = _handles(A, 1000, values=vals)
        try:
            for k in (1, 2, 3, 8, 16):
                X = torch.from_numpy(synth.dense(A.n_cols, k, seed=k + 2)).cuda().to(tdt)
                for tr in (False, True):
                    assert torch.equal(plain.apply(X, transpose=tr), hot.apply(X, transpose=tr)), (xname, k, tr)
        finally:
            plain.close()
            hot.close()


def test_hot_integer_exact_vs_oracle_and_strided_x():
    """Pattern A, X in {0..7}, X a column slice of a wider array (ldx > k):
    exact against the FP64 oracle in both orientations."""
    import torch
    from paper_1602_02864_gb300 import spmm as sp
    A = synth.rmat_csr(15, seed=6)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True,
                        opts=sp.spmm_opts(hot_cols=5000))
    try:
        Xw = synth.dense(A.n_cols, 24, seed=9, mode="int")
        Xd = torch.from_numpy(Xw).cuda()
        for k in (1, 2, 3, 8, 16):
            Xs = Xd[:, 4:4 + k]                   # ldx = 24, offset 4 elements
            for tr in (False, True):
                got = h.apply(Xs, transpose=tr).cpu().numpy().astype(np.float64)
                ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None,
                                  np.ascontiguousarray(Xw[:, 4:4 + k]).astype(np.float64), transpose=tr)
                assert np.array_equal(got, ref), (k, tr)
    finally:
        h.close()


def test_hot_pagerank_and_batched_match_plain():
    import torch
    from paper_1602_02864_gb300 import spmm as sp
    A = synth.rmat_csr(14, seed=7)
    plain = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True,
                            opts=sp.spmm_opts(hot_cols=-1))
    hot = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True,
                          opts=sp.spmm_opts(hot_cols=3000))
    try:
        xp, rp = plain.pagerank(0.85, 30)
        xh, rh = hot.pagerank(0.85, 30)
        assert torch.equal(xp, xh) and np.array_equal(rp, rh)
    finally:
        plain.close()
        hot.close()
    graphs = [synth.chunglu_csr(g) for g in range(6)]
    bp = sp.SparseMatrix.batched(graphs, transpose=True, weighted=False, opts=sp.spmm_opts(hot_cols=-1))
    bh = sp.SparseMatrix.batched(graphs, transpose=True, weighted=False, opts=sp.spmm_opts(hot_cols=2000))
    try:
        n = sum(g.n_cols for g in graphs)
        X = torch.from_numpy(synth.dense(n, 8, seed=1)).cuda()
        for tr in (False, True):
            assert torch.equal(bp.apply(X, transpose=tr), bh.apply(X, transpose=tr))
    finally:
        bp.close()
        bh.close()


def test_hot_weighted_vs_oracle_bf16():
    import torch
    from paper_1602_02864_gb300 import spmm as sp
    A = synth.rmat_csr(14, seed=8, weighted=True)
    h = sp.SparseMatrix.from_csr(A, transpose=True, opts=sp.spmm_opts(hot_cols=8192))
    try:
        for k in (1, 8, 64):
            X = torch.from_numpy(synth.dense(A.n_cols, k, seed=3)).cuda().to(torch.bfloat16)
            Xr = rounded_host(X)
            for tr in (False, True):
                ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xr, transpose=tr)
                assert_close_rel(h.apply(X, transpose=tr).cpu().numpy(), ref, abs_product(A, Xr, tr), 2e-3,
                                 f"bf16 k={k} tr={tr}")
    finally:
        h.close()
