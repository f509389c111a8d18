"""GPU parity: the CUDA SpMM (through the C-ABI) against the FP64 oracle.

Tolerances: bit-exact for a pattern matrix with integer X in 0..7 (every
partial sum is an integer below 2^24, so every summation order is exact);
otherwise |Y - Y*| <= 1e-5 * (|A||X|) for float32 inputs and 2e-3 for 16-bit
inputs, Y* being the oracle on the already-rounded inputs.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import graphs
from tests.gpu_util import abs_product, assert_close_rel, rounded_host, to_dev

pytestmark = pytest.mark.gpu

KS = [1, 2, 3, 4, 5, 7, 8, 13, 16, 31, 32, 33, 64]


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


@pytest.fixture(scope="module")
def rmat16():
    return synth.rmat_csr(16, seed=0, weighted=True)


@pytest.fixture(scope="module")
def rmat16_handles(sp, rmat16):
    A = rmat16
    hw = sp.SparseMatrix.from_csr(A, transpose=True)
    hp = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)
    yield hw, hp
    hw.close()
    hp.close()


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("transpose", [False, True])
def test_bit_exact_pattern_integer_x(sp, rmat16, rmat16_handles, k, transpose):
    import torch
    A = rmat16
    _, hp = rmat16_handles
    n_in = A.n_rows if transpose else A.n_cols
    assert 7 * max(A.degrees().max(), np.bincount(A.col_idx).max()) < 2 ** 24
    X = synth.dense(n_in, k, seed=11, mode="int")
    Y = hp.apply(to_dev(X), transpose=transpose)
    torch.cuda.synchronize()
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X, transpose=transpose)
    assert np.array_equal(Y.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("transpose", [False, True])
def test_f32_weighted(sp, rmat16, rmat16_handles, k, transpose):
    A = rmat16
    hw, _ = rmat16_handles
    n_in = A.n_rows if transpose else A.n_cols
    X = synth.dense(n_in, k, seed=0)
    Y = hw.apply(to_dev(X), transpose=transpose).cpu().numpy()
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, X, transpose=transpose)
    assert_close_rel(Y, ref, abs_product(A, X.astype(np.float64), transpose), 1e-5, f"k={k} t={transpose}")


@pytest.mark.parametrize("xdtype", ["bfloat16", "float16"])
@pytest.mark.parametrize("k", [1, 2, 4, 8, 16, 24, 64])
@pytest.mark.parametrize("transpose", [False, True])
def test_16bit_x(sp, rmat16, rmat16_handles, xdtype, k, transpose):
    import torch
    A = rmat16
    hw, _ = rmat16_handles
    n_in = A.n_rows if transpose else A.n_cols
    Xd = to_dev(synth.dense(n_in, k, seed=3), getattr(torch, xdtype))
    Y = hw.apply(Xd, transpose=transpose).cpu().numpy()
    Xr = rounded_host(Xd)
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xr, transpose=transpose)
    assert_close_rel(Y, ref, abs_product(A, Xr, transpose), 2e-3, f"{xdtype} k={k}")


@pytest.fixture(scope="module")
def rmat16_16bit_handles(sp, rmat16):
    """Handles of the weighted scale-16 graph with bf16 and f16 stored values."""
    import torch
    out = {}
    for vdtype in ("bfloat16", "float16"):
        vt = torch.from_numpy(rmat16.values).to(getattr(torch, vdtype))
        out[vdtype] = (sp.SparseMatrix(rmat16.n_rows, rmat16.n_cols, rmat16.row_ptr, rmat16.col_idx, vt,
                                       transpose=True), vt.float().numpy().astype(np.float64))
    yield out
    for h, _ in out.values():
        h.close()


@pytest.mark.parametrize("vdtype", ["bfloat16", "float16"])
@pytest.mark.parametrize("k", [1, 2, 8, 16, 64])
def test_16bit_values(sp, rmat16, rmat16_16bit_handles, vdtype, k):
    """Stored 16-bit values with X of the same type: every lane geometry (one
    lane per row at k = 1, 2; two lanes at k = 8; lane groups at 16; two
    column chunks of 16-bit lanes at 64), both orientations."""
    import torch
    A = rmat16
    h, vr = rmat16_16bit_handles[vdtype]
    Xd = to_dev(synth.dense(A.n_cols, k, seed=4 + k), getattr(torch, vdtype))
    Xr = rounded_host(Xd)
    for tr in (False, True):
        Y = h.apply(Xd, transpose=tr).cpu().numpy()
        ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vr, Xr, transpose=tr)
        scale = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, np.abs(vr), np.abs(Xr), transpose=tr)
        assert_close_rel(Y, ref, scale, 2e-3, f"{vdtype} values k={k} t={tr}")


@pytest.mark.parametrize("graph", ["sbm16_clustered", "sbm16_unclustered", "sbm1024_p90_clustered",
                                   "rmat_permuted"])
@pytest.mark.parametrize("k", [1, 4, 8, 32])
def test_ordering_study_graphs_integer_exact(sp, graph, k):
    """The ordering study's inputs (Section 5.1: SBM graphs with clustered or
    randomly relabelled ids, R-MAT with relabelled ids) through the CUDA
    path, pattern A with integer X, exactly the oracle's result."""
    import torch
    n = 1 << 15
    A = {"sbm16_clustered": lambda: synth.sbm_csr(n, 16, 16, 0.5, seed=1),
         "sbm16_unclustered": lambda: synth.sbm_csr(n, 16, 16, 0.5, seed=1, permuted=True),
         "sbm1024_p90_clustered": lambda: synth.sbm_csr(n, 1024, 16, 0.9, seed=2),
         "rmat_permuted": lambda: synth.rmat_permuted_csr(15, seed=3)}[graph]()
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)
    try:
        X = synth.dense(n, k, seed=k, mode="int")
        for tr in (False, True):
            got = h.apply(torch.from_numpy(X).cuda(), transpose=tr).cpu().numpy().astype(np.float64)
            ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X.astype(np.float64), transpose=tr)
            assert np.array_equal(got, ref), (graph, k, tr)
    finally:
        h.close()


def test_deterministic_repeat(sp, rmat16, rmat16_handles):
    import torch
    hw, _ = rmat16_handles
    Xd = to_dev(synth.dense(rmat16.n_cols, 16, seed=5))
    Y1 = hw.apply(Xd).clone()
    Y2 = hw.apply(Xd)
    assert torch.equal(Y1, Y2)
    T1 = hw.apply(Xd, transpose=True).clone()
    T2 = hw.apply(Xd, transpose=True)
    assert torch.equal(T1, T2)


@pytest.mark.parametrize("opts", [(32, 1, 32, 1), (32, 64, 64, 31), (64, 8, 128, 8), (512, 64, 512, 200),
                                  (100, 3, 100, 50), (256, 64, 512, 1), (256, 64, 512, 255)])
def test_plan_shapes_agree(sp, opts):
    """Different task sizes, short-row limits and split thresholds (many
    splits, one row per task, maximal tasks, every row long, no row long)
    all give the oracle's answer exactly in integer mode."""
    A = synth.rmat_csr(14, seed=2)
    o = sp.spmm_opts(task_nnz=opts[0], task_rows=opts[1], long_row=opts[2], short_max=opts[3])
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, opts=o)
    info = h.info()
    assert info["n_split_rows"] > 0
    for k in (1, 2, 4, 8, 33):
        X = synth.dense(A.n_cols, k, seed=k, mode="int")
        for tr in (False, True):
            Y = h.apply(to_dev(X), transpose=tr).cpu().numpy().astype(np.float64)
            assert np.array_equal(Y, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X, transpose=tr))
    h.sync_status()
    h.close()


@pytest.mark.parametrize("kind", ["uniform", "geometric", "bimodal", "sparse"])
@pytest.mark.parametrize("task_nnz", [32, 100, 512])
@pytest.mark.parametrize("short_runs", [0, 1, 2])
def test_merge_rows_cross_lane_pieces(sp, kind, task_nnz, short_runs):
    """One lane per X row (k = 2 in FP32, k = 2 and 4 in BF16) cuts each
    short-row run into 32 equal pieces of nonzeros, and rows on several lanes
    of at most 4 elements (k = 4, 16, 32, 64 in FP32; 8, 16, 32 in BF16 and
    FP16) cut it into one piece per lane group; rows that start before a
    piece, span several pieces or have no nonzeros must all come out right.
    Degree mixes: uniform 0..63, geometric, mostly 0..2 with 10% of 30..63,
    and 0/1.  short_runs 1 and 2 force whole rows or pieces per lane group
    where the automatic choice (0) would take the other."""
    import torch
    rng = np.random.default_rng({"uniform": 1, "geometric": 2, "bimodal": 3, "sparse": 4}[kind])
    n = 3000
    deg = {"uniform": lambda: rng.integers(0, 64, n),
           "geometric": lambda: rng.geometric(0.2, n) - 1,
           "bimodal": lambda: np.where(rng.random(n) < 0.1, rng.integers(30, 64, n), rng.integers(0, 3, n)),
           "sparse": lambda: rng.integers(0, 2, n)}[kind]()
    deg = np.minimum(deg, 63)
    src = np.repeat(np.arange(n), deg)
    dst = np.concatenate([rng.choice(n, d, replace=False) for d in deg]) if deg.sum() else np.zeros(0, int)
    A = graphs.csr_from_edges(n, n, src, dst, rng.random(len(src)).astype(np.float32))
    o = sp.spmm_opts(task_nnz=task_nnz, task_rows=64, long_row=512, short_max=63, short_runs=short_runs)
    hp = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, opts=o)
    hw = sp.SparseMatrix.from_csr(A, transpose=True, opts=o)
    for tr in (False, True):
        X = synth.dense(n, 2, seed=5, mode="int")
        Y = hp.apply(to_dev(X), transpose=tr).cpu().numpy().astype(np.float64)
        assert np.array_equal(Y, oracle.spmm(n, n, A.row_ptr, A.col_idx, None, X, transpose=tr))
        for k in (2, 4):
            Xb = torch.from_numpy(synth.dense(n, k, seed=6, mode="int")).to(torch.bfloat16).cuda()
            Yb = hp.apply(Xb, transpose=tr).cpu().numpy().astype(np.float64)
            ref = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, Xb.float().cpu().numpy(), transpose=tr)
            assert np.array_equal(Yb, ref)
        for k in (4, 16, 32, 64):
            X = synth.dense(n, k, seed=8 + k, mode="int")
            Y = hp.apply(to_dev(X), transpose=tr).cpu().numpy().astype(np.float64)
            assert np.array_equal(Y, oracle.spmm(n, n, A.row_ptr, A.col_idx, None, X, transpose=tr)), k
        for dt in (torch.bfloat16, torch.float16):
            for k in (8, 16, 32):
                Xb = torch.from_numpy(synth.dense(n, k, seed=k, mode="int")).to(dt).cuda()
                Yb = hp.apply(Xb, transpose=tr).cpu().numpy().astype(np.float64)
                ref = oracle.spmm(n, n, A.row_ptr, A.col_idx, None, Xb.float().cpu().numpy(), transpose=tr)
                assert np.array_equal(Yb, ref), (dt, k)
        for k in (2, 16):
            Xf = synth.dense(n, k, seed=7)
            Yw = hw.apply(to_dev(Xf), transpose=tr).cpu().numpy()
            ref = oracle.spmm(n, n, A.row_ptr, A.col_idx, A.values, Xf, transpose=tr)
            scale = oracle.spmm(n, n, A.row_ptr, A.col_idx, A.values, np.abs(Xf), transpose=tr)
            assert_close_rel(Yw, ref, scale, 1e-5)
    hp.sync_status()
    hp.close()
    hw.close()


def test_edge_cases(sp):
    import torch
    cases = {
        "empty": graphs.csr_from_edges(7, 5, [], []),
        "single": graphs.csr_from_edges(1, 1, [0], [0], [2.5]),
        "hub_all_columns": graphs.csr_from_edges(3, 5000, np.zeros(5000, np.int64), np.arange(5000),
                                                 np.linspace(0, 1, 5000)),
        "all_degree_one": graphs.csr_from_edges(3000, 3000, np.arange(3000), (np.arange(3000) * 7) % 3000,
                                                np.ones(3000)),
        "rect_wide": graphs.random_csr(50, 4000, 0.01, 1),
        "rect_tall": graphs.random_csr(4000, 30, 0.05, 2, empty_rows=0.6),
        "cycle": graphs.cycle(1000),
        "complete": graphs.complete(70),
        "star": graphs.star(3000),
    }
    for name, A in cases.items():
        h = sp.SparseMatrix.from_csr(A, transpose=True)
        for k in (1, 3, 8, 64):
            for tr in (False, True):
                n_in = A.n_rows if tr else A.n_cols
                X = synth.dense(n_in, k, seed=1, mode="int")
                Y = h.apply(to_dev(X), transpose=tr)
                torch.cuda.synchronize()
                v = None if A.values is None else A.values
                ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, v, X, transpose=tr)
                if A.values is None:
                    assert np.array_equal(Y.cpu().numpy().astype(np.float64), ref), name
                else:
                    assert_close_rel(Y.cpu().numpy(), ref, abs_product(A, X.astype(np.float64), tr), 1e-5, name)
        h.close()


def test_strided_and_misaligned(sp, rmat16, rmat16_handles):
    """ld > k and an X that starts one element off a 16-byte boundary (forces
    narrower vectors); only the first k columns of Y are written."""
    import torch
    A = rmat16
    hw, _ = rmat16_handles
    k, ld = 8, 13
    Xfull = synth.dense(A.n_cols, ld + 1, seed=6)
    Xd = to_dev(Xfull)[:, 1:1 + k]                 # ld = ld+1, offset 4 bytes
    assert Xd.stride(0) == ld + 1
    Y = torch.full((A.n_rows, 11), 7.0, device="cuda")
    hw.apply(Xd, Y=Y[:, :k])
    ref = oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.values, Xfull[:, 1:1 + k])
    Yh = Y.cpu().numpy()
    assert_close_rel(Yh[:, :k], ref, abs_product(A, np.abs(Xfull[:, 1:1 + k]).astype(np.float64)), 1e-5, "strided")
    assert np.all(Yh[:, k:] == 7.0)


def test_error_codes(sp):
    import torch
    A = graphs.cycle(10)
    with pytest.raises(sp.SpmmError) as e:
        sp.SparseMatrix(10, 10, np.array([0, 1, 0] + [10] * 8), A.col_idx)
    assert e.value.status == sp.SPMM_ERR_FORMAT
    bad = A.col_idx.copy()
    bad[3] = 10
    with pytest.raises(sp.SpmmError) as e:
        sp.SparseMatrix(10, 10, A.row_ptr, bad)
    assert e.value.status == sp.SPMM_ERR_FORMAT
    h = sp.SparseMatrix.from_csr(A)
    X = torch.zeros((10, 4), device="cuda")
    Y = torch.zeros((10, 4), device="cuda")
    for args in [(X, 10, 0), (X, 2, 4), (X, 65, 65)]:
        with pytest.raises(sp.SpmmError) as e:
            sp.spmm_apply(h.handle, args[0], args[1], args[2], sp.SPMM_F32, Y, 4)
        assert e.value.status == sp.SPMM_ERR_ARG
    with pytest.raises(sp.SpmmError) as e:          # no transposed copy was built
        sp.spmm_apply(h.handle, X, 4, 4, sp.SPMM_F32, Y, 4, transpose=1)
    assert e.value.status == sp.SPMM_ERR_ARG
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_apply(h.handle, X, 4, 4, sp.SPMM_F64, Y, 4)
    assert e.value.status == sp.SPMM_ERR_ARG
    h.close()


def test_bounded_wait_times_out_and_context_survives(sp, rmat16, rmat16_handles):
    """A staging wait that can never complete runs out after its bound and is
    reported as SPMM_ERR_TIMEOUT; the context stays usable afterwards."""
    import torch
    assert sp.spmm_debug_wait_timeout(2_000_000) == sp.SPMM_ERR_TIMEOUT
    hw, hp = rmat16_handles
    hp.sync_status()                     # no timeout recorded on a real handle
    X = synth.dense(rmat16.n_cols, 8, seed=2, mode="int")
    Y = hp.apply(to_dev(X)).cpu().numpy().astype(np.float64)
    hp.sync_status()
    ref = oracle.spmm(rmat16.n_rows, rmat16.n_cols, rmat16.row_ptr, rmat16.col_idx, None, X)
    assert np.array_equal(Y, ref)


def test_info_walk_eff_matches_host_plan(sp):
    """The handle's row-walk efficiency (which the automatic short_runs
    choice reads) is the host plan's, for both orientations and after a
    replan."""
    A = synth.rmat_csr(14, seed=4)
    o = sp.spmm_opts(task_nnz=256, short_max=31)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True, opts=o)
    rpt = np.concatenate([[0], np.cumsum(np.bincount(A.col_idx, minlength=A.n_cols))]).astype(np.int64)
    info = h.info()
    assert info["walk_eff"] == sp.spmm_plan_walk_eff(A.row_ptr, o)
    assert info["walk_eff_t"] == sp.spmm_plan_walk_eff(rpt, o)
    o2 = sp.spmm_opts(task_nnz=512, short_max=63)
    sp.spmm_replan(h.handle, o2, 0)
    assert h.info()["walk_eff"] == sp.spmm_plan_walk_eff(A.row_ptr, o2)
    h.close()
