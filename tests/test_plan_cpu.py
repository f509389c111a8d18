"""Host-side checks of the warp-task plan (no GPU): the task kernel's staging
windows and shared-memory indexing are only in bounds if these hold."""
import numpy as np
import pytest

import synth
from tests import graphs

MAX_TASK_NNZ, MAX_TASK_ROWS = 512, 64
COL_BUF_INTS, VAL_BUF_BYTES, RP_BUF_LONGS = MAX_TASK_NNZ + 8, (MAX_TASK_NNZ + 8) * 4, MAX_TASK_ROWS + 4


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import build
    build.build()
    from paper_1602_02864_gb300 import spmm
    return spmm


def check_plan(sp, A, opts=None):
    rp = A.row_ptr
    n, nnz = A.n_rows, A.nnz
    tasks, n_split, n_seg = sp.spmm_plan_tasks(rp, opts)
    e0 = (tasks[:, 2].astype(np.int64) & 0xFFFFFFFF) | (tasks[:, 3].astype(np.int64) << 32)
    assert e0[-1] == nnz and tasks[-1, 0] == n          # sentinel
    cnt = np.diff(e0)
    assert np.all(cnt >= 0) and np.all(cnt <= MAX_TASK_NNZ)
    covered = np.zeros(n, dtype=np.int64)
    slots = []
    for t in range(len(tasks) - 1):
        r0, x = int(tasks[t, 0]), int(tasks[t, 1])
        if x > 0:
            assert x <= MAX_TASK_ROWS and e0[t] == rp[r0] and e0[t + 1] == rp[r0 + x]
            covered[r0:r0 + x] += 1
            # row-pointer window: 16-byte aligned start, inside the 2-entry padding
            rs, re = r0 & ~1, (r0 + x + 2) & ~1
            assert re - rs <= RP_BUF_LONGS and re <= n + 3
            assert (r0 & 1) + x < RP_BUF_LONGS
        elif x == 0:
            assert e0[t] == rp[r0] and e0[t + 1] == rp[r0 + 1]
            covered[r0] += 1
        else:
            slots.append(-x - 1)
            assert rp[r0] <= e0[t] < e0[t + 1] <= rp[r0 + 1]
            if e0[t + 1] == rp[r0 + 1]:
                covered[r0] += 1                            # last segment of the row
        cs, ce = e0[t] & ~3, (e0[t + 1] + 3) & ~3
        assert ce - cs <= COL_BUF_INTS and ce <= nnz + 8
        for vb in (4, 2):                                   # value windows, f32 and 16-bit
            epb = 16 // vb
            vs, ve = e0[t] & ~(epb - 1), (e0[t + 1] + epb - 1) & ~(epb - 1)
            assert (ve - vs) * vb <= VAL_BUF_BYTES and ve <= nnz + 8
    assert np.all(covered == 1)
    assert sorted(slots) == list(range(n_seg))
    return tasks, n_split, n_seg


@pytest.mark.parametrize("opts", [None, (32, 1, 32, 1), (512, 64, 512, 511), (100, 3, 100, 50), (256, 64, 512, 1)])
def test_plan_invariants_rmat(sp, opts):
    A = synth.rmat_csr(15, seed=1)
    o = None if opts is None else sp.spmm_opts(task_nnz=opts[0], task_rows=opts[1], long_row=opts[2],
                                                short_max=opts[3])
    tasks, n_split, n_seg = check_plan(sp, A, o)
    assert n_split > 0 and n_seg > n_split


def test_plan_invariants_special(sp):
    for A in (graphs.csr_from_edges(9, 4, [], []), graphs.star(5000), graphs.cycle(300),
              graphs.csr_from_edges(1, 100000, np.zeros(100000, np.int64), np.arange(100000)),
              graphs.random_csr(3000, 3000, 0.01, 3, empty_rows=0.7)):
        check_plan(sp, A)


def test_plan_classes(sp):
    """Degree bins: empty and short rows are packed, long rows get a task of
    their own, hub rows are split into segments of at most task_nnz."""
    deg = np.array([0, 1, 2, 40, 0, 3, 600, 5, 1500], dtype=np.int64)
    rp = np.concatenate([[0], np.cumsum(deg)])
    tasks, n_split, n_seg = sp.spmm_plan_tasks(rp, sp.spmm_opts(task_nnz=256, short_max=31, long_row=512))
    kinds = [(int(t[0]), int(t[1])) for t in tasks[:-1]]
    assert kinds[0] == (0, 3)                        # rows 0-2 packed
    assert kinds[1] == (3, 0)                        # degree 40 > 31: long
    assert kinds[2] == (4, 2)                        # rows 4-5 packed
    assert [k[0] for k in kinds[3:6]] == [6, 6, 6] and all(k[1] < 0 for k in kinds[3:6])   # 600 -> 3 segments
    assert kinds[6] == (7, 1)
    assert len(kinds) == 7 + 6 and n_split == 2 and n_seg == 9      # 1500 -> 6 segments


def test_plan_rejects_bad_row_ptr(sp):
    with pytest.raises(sp.SpmmError) as e:
        sp.spmm_plan_tasks(np.array([0, 3, 2], dtype=np.int64))
    assert e.value.status == sp.SPMM_ERR_FORMAT


def test_plan_invariants_random_degrees(sp):
    """Property test over random degree sequences and plan options: the plan
    covers every row once, keeps every staging window in bounds, and splits a
    hub row into segments of equal length except the last (the allocation-free
    entry point finds a row's first segment from that)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    degree = st.one_of(st.integers(0, 3), st.integers(0, 70), st.integers(0, 5000))

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(deg=st.lists(degree, min_size=1, max_size=300),
               task_nnz=st.integers(32, 512), task_rows=st.integers(1, 64),
               long_row=st.integers(1, 512), short_max=st.integers(1, 511))
    def prop(deg, task_nnz, task_rows, long_row, short_max):
        n = len(deg)
        rp = np.zeros(n + 1, dtype=np.int64)
        rp[1:] = np.cumsum(deg)
        A = synth.CSR(n, max(1, n), rp, np.zeros(int(rp[-1]), dtype=np.int32))
        o = sp.spmm_opts(task_nnz=task_nnz, task_rows=task_rows, long_row=long_row, short_max=short_max)
        tasks, n_split, n_seg = check_plan(sp, A, o)
        e0 = (tasks[:, 2].astype(np.int64) & 0xFFFFFFFF) | (tasks[:, 3].astype(np.int64) << 32)
        seg_rows = {}
        for t in range(len(tasks) - 1):
            if tasks[t, 1] < 0:
                seg_rows.setdefault(int(tasks[t, 0]), []).append(int(e0[t + 1] - e0[t]))
        assert len(seg_rows) == n_split
        for lens in seg_rows.values():
            assert len(lens) >= 2 and len(set(lens[:-1])) == 1 and lens[-1] <= lens[0]

    prop()


def walk_eff_by_definition(sp, rp, opts=None):
    """Row-walk efficiency written out from its definition in spmm.h over the
    plan's short-row tasks: per round of G consecutive rows of a task, the
    batches of 4 nonzeros summed, over G x the longest (at least 1)."""
    tasks, _, _ = sp.spmm_plan_tasks(rp, opts)
    deg = np.diff(rp)
    out = []
    for G in (2, 4, 8, 16):
        done = taken = 0
        for t in range(len(tasks) - 1):
            r0, x = int(tasks[t, 0]), int(tasks[t, 1])
            if x < 1:
                continue
            for j in range(0, x, G):
                b = [(int(deg[r0 + q]) + 3) // 4 for q in range(j, min(j + G, x))]
                done += sum(b)
                taken += G * max(1, max(b))
        out.append(done / taken if taken else 1.0)
    return out


def test_walk_eff_closed_forms(sp):
    # one row of 4 nonzeros and three empty rows: one batch done per round
    # of G groups (two rounds at G = 2)
    assert sp.spmm_plan_walk_eff(np.array([0, 4, 4, 4, 4])) == [0.25, 0.25, 0.125, 0.0625]
    # 64 rows of 8 nonzeros: every round is full
    assert sp.spmm_plan_walk_eff(np.arange(65, dtype=np.int64) * 8) == [1.0, 1.0, 1.0, 1.0]
    # only long rows (no short-row runs): 1 by definition
    assert sp.spmm_plan_walk_eff(np.array([0, 100, 300], dtype=np.int64)) == [1.0, 1.0, 1.0, 1.0]
    # rows of 1 and 5 nonzeros alternating: batches 1, 2; at G = 2 each
    # round does 3 of 4; wider rounds hold both lengths too
    rp = np.concatenate([[0], np.cumsum(np.tile([1, 5], 32))]).astype(np.int64)
    assert sp.spmm_plan_walk_eff(rp) == [0.75, 0.75, 0.75, 0.75]
    # empty matrix
    assert sp.spmm_plan_walk_eff(np.zeros(1, dtype=np.int64)) == [1.0, 1.0, 1.0, 1.0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_walk_eff_matches_definition(sp, seed):
    rng = np.random.default_rng(seed)
    n = 5000
    deg = np.where(rng.random(n) < 0.3, 0, rng.geometric(0.08, n))
    hubs = rng.random(n) < 0.01
    deg[hubs] = rng.integers(64, 2000, int(hubs.sum()))
    rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    for o in (None, sp.spmm_opts(task_nnz=128, short_max=31, task_rows=40)):
        np.testing.assert_allclose(sp.spmm_plan_walk_eff(rp, o), walk_eff_by_definition(sp, rp, o), rtol=1e-12)


def test_walk_eff_orders_graph_families(sp):
    """The automatic short_runs rule reads this statistic: on R-MAT most
    rounds wait on one long row (efficiency well below 0.5 for 8 and 16
    groups), on a Chung-Lu batch and an SBM graph rows are closer in length
    (above 0.5)."""
    rm = sp.spmm_plan_walk_eff(synth.rmat_csr(16, seed=0).row_ptr)
    assert rm == sorted(rm, reverse=True) and rm[3] < 0.35 and rm[2] < 0.45
    for A in (synth.sbm_csr(1 << 16, 16, 16.0, 0.5, seed=0), synth.chunglu_csr(3, seed=0)):
        e = sp.spmm_plan_walk_eff(A.row_ptr)
        assert e == sorted(e, reverse=True) and min(e) > 0.5, e


def test_walk_eff_rejects_bad_row_ptr(sp):
    with pytest.raises(sp.SpmmError):
        sp.spmm_plan_walk_eff(np.array([1, 2, 3], dtype=np.int64))
    with pytest.raises(sp.SpmmError):
        sp.spmm_plan_walk_eff(np.array([0, 5, 3], dtype=np.int64))


def check_runs(sp, rp, max_runs, opts=None):
    """The runs of whole tasks the host-buffer calls multiply one at a time:
    they tile the task list, the rows and the split rows in order, never cut
    between two segments of one split row, and each run but the last ends at
    the first task boundary past its share of the stored entries."""
    tasks, n_split, _ = sp.spmm_plan_tasks(rp, opts)
    runs = sp.spmm_plan_runs(rp, max_runs, opts)
    nt, n = len(tasks) - 1, len(rp) - 1
    if nt == 0:
        assert len(runs) == 0
        return runs
    e0 = (tasks[:, 2].astype(np.int64) & 0xFFFFFFFF) | (tasks[:, 3].astype(np.int64) << 32)
    split_rows = np.array(sorted({int(t[0]) for t in tasks[:-1] if t[1] < 0}), dtype=np.int64)
    assert split_rows.size == n_split
    assert 1 <= len(runs) <= max_runs
    assert runs[0, 0] == 0 and runs[0, 2] == 0 and runs[0, 4] == 0
    assert runs[-1, 1] == nt and runs[-1, 3] == n and runs[-1, 5] == n_split
    total = int(rp[-1])
    for j, (t0, t1, r0, r1, s0, s1) in enumerate(runs):
        assert t0 < t1
        if j + 1 < len(runs):
            assert (t1, r1, s1) == tuple(runs[j + 1, [0, 2, 4]])
        assert r0 == tasks[t0, 0] and r1 == tasks[t1, 0]          # rows of the run's tasks
        assert t0 == 0 or tasks[t0, 0] != tasks[t0 - 1, 0]        # a split row is never cut
        # the split rows of the run are exactly those among its rows
        assert list(split_rows[s0:s1]) == [r for r in split_rows if r0 <= r < r1]
        if j + 1 < len(runs):
            goal = total * (j + 1) // max_runs
            assert e0[t1] >= goal
            # no earlier boundary past the goal that starts a new row
            for u in range(t0 + 1, t1):
                assert e0[u] < goal or tasks[u, 0] == tasks[u - 1, 0]
    return runs


@pytest.mark.parametrize("max_runs", [1, 2, 4, 7])
def test_runs_invariants_rmat(sp, max_runs):
    A = synth.rmat_csr(12, seed=3)
    runs = check_runs(sp, A.row_ptr, max_runs)
    assert len(runs) == max_runs
    o = sp.spmm_opts(task_nnz=32, long_row=64, short_max=15)    # many split rows
    check_runs(sp, A.row_ptr, max_runs, o)


def test_runs_small_and_special(sp):
    assert len(check_runs(sp, np.zeros(1, dtype=np.int64), 4)) == 0          # no rows
    assert len(check_runs(sp, np.zeros(41, dtype=np.int64), 4)) == 1         # 40 empty rows, one task
    # one hub row split into many segments followed by short rows: the hub's
    # segments stay together although they hold most of the entries
    rp = np.concatenate([[0, 5000], 5000 + np.arange(1, 200)]).astype(np.int64)
    runs = check_runs(sp, rp, 4)
    assert runs[0, 2] == 0 and runs[0, 3] >= 1
    for opts in (None, sp.spmm_opts(task_nnz=64, long_row=64, short_max=3)):
        for seed in range(4):
            rng = np.random.default_rng(seed)
            deg = rng.zipf(1.8, size=500).clip(0, 3000)
            check_runs(sp, np.concatenate([[0], np.cumsum(deg)]).astype(np.int64), 4, opts)


def test_runs_reject_bad_input(sp):
    with pytest.raises(sp.SpmmError, match="ERR_FORMAT"):
        sp.spmm_plan_runs(np.array([0, 3, 2], dtype=np.int64))
    with pytest.raises(sp.SpmmError, match="ERR_ARG"):
        sp.spmm_plan_runs(np.array([0, 1], dtype=np.int64), 0)
