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
