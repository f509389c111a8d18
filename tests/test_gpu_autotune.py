"""Autotuner: candidate plans are timed, the handle ends on the fastest, the
result stays exact, and the JSON cache re-plans without searching."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_stays_exact(tmp_path):
    import torch
    from paper_1602_02864_gb300 import autotune, spmm as sp
    A = synth.rmat_csr(14, seed=6)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)
    cands = [dict(task_nnz=64, short_max=7, long_row=128), dict(task_nnz=256, short_max=31, long_row=512),
             dict(task_nnz=512, short_max=63, long_row=512, x_l2_policy=1)]
    best, times, _ = sp.spmm_autotune(h.handle, 8, sp.SPMM_F32, 0, cands, reps=2)
    assert 0 <= best < 3 and np.all(times > 0) and times[best] == times.min()
    tasks, _, _ = sp.spmm_plan_tasks(A.row_ptr, sp.spmm_opts(**cands[best]))
    assert h.info()["n_tasks"] == len(tasks) - 1
    X = synth.dense(A.n_cols, 8, seed=2, mode="int")
    Y = h.apply(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    assert np.array_equal(Y, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X))
    # built-in grid on the transposed plan
    best_t, times_t, grid = sp.spmm_autotune(h.handle, 1, sp.SPMM_F32, 1, None, reps=1)
    assert len(times_t) == len(grid) == 24 and np.all(times_t > 0)
    Yt = h.apply(torch.from_numpy(X[:, :1].copy()).cuda(), transpose=True).cpu().numpy().astype(np.float64)
    assert np.array_equal(Yt, oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, X[:, :1], transpose=True))
    # cache round trip
    path = str(tmp_path / "tune.json")
    c1 = autotune.tune(h, 8, cache_path=path, candidates=cands, reps=1)
    c2 = autotune.tune(h, 8, cache_path=path, candidates=cands, reps=1)
    assert not c1["cached"] and c2["cached"]
    assert {n: c2[n] for n in cands[0]} == {n: c1[n] for n in cands[0]}
    h.sync_status()
    h.close()


def test_tune_batched_leaves_every_handle_on_one_plan_and_exact():
    """The batch-level tuner times the batched call for each candidate, leaves
    every handle on the fastest, and the batched results stay exact."""
    import torch
    from paper_1602_02864_gb300 import autotune, spmm as sp
    graphs = [synth.chunglu_csr(g, seed=0, nmin=1000, nmax=20000) for g in range(6)]
    hs = [sp.SparseMatrix(g.n_rows, g.n_cols, g.row_ptr, g.col_idx, None) for g in graphs]
    try:
        ks = [1, 8, 16, 8, 33, 4]
        Xh = [synth.dense(g.n_cols, k, seed=i, mode="int") for i, (g, k) in enumerate(zip(graphs, ks))]
        Xs = [torch.from_numpy(x).cuda() for x in Xh]
        Ys = [torch.empty((g.n_rows, k), device="cuda") for g, k in zip(graphs, ks)]
        cands = [dict(task_nnz=128, short_max=15, long_row=512), dict(task_nnz=512, short_max=63, long_row=512),
                 dict(task_nnz=256, short_max=31, long_row=256, x_l2_policy=1)]
        r = autotune.tune_batched(hs, Xs, Ys, candidates=cands, reps=2)
        assert len(r["candidate_ms"]) == 3 and r["ms"] == min(r["candidate_ms"])
        chosen = {n: r[n] for n in cands[0]}
        assert chosen in [{n: c[n] for n in cands[0]} for c in cands]
        for g, h in zip(graphs, hs):
            tasks, _, _ = sp.spmm_plan_tasks(g.row_ptr, sp.spmm_opts(**chosen))
            assert h.info()["n_tasks"] == len(tasks) - 1
        sp.spmm_apply_batched([h.handle for h in hs], Xs, Ys)
        for g, x, y in zip(graphs, Xh, Ys):
            ref = oracle.spmm(g.n_rows, g.n_cols, g.row_ptr, g.col_idx, None, x)
            assert np.array_equal(y.cpu().numpy().astype(np.float64), ref)
    finally:
        for h in hs:
            h.close()
