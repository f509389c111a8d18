"""Concurrent host threads: separate handles applied from several threads at
once (ctypes releases the GIL during each call), each on its own stream,
including the first calls of kernel instantiations, must give the results of
the same calls made one at a time."""
import threading

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_concurrent_handles_match_serial():
    import torch
    from paper_1602_02864_gb300 import spmm
    graphs = [synth.rmat_csr(12 + (i % 3), seed=i, weighted=bool(i % 2)) for i in range(6)]
    ks = [3, 5, 7, 11, 13, 24]                  # instantiations the other tests may not have used yet
    handles = [spmm.SparseMatrix.from_csr(A, transpose=True) for A in graphs]
    Xs = [torch.from_numpy(synth.dense(A.n_cols, k, seed=7)).cuda() for A, k in zip(graphs, ks)]
    out = [None] * len(graphs)
    errors = []

    def work(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(10):
                    Y = handles[i].apply(Xs[i], stream=s)
                    Yt = handles[i].apply(Y, transpose=True, stream=s)      # square graphs
                s.synchronize()
                out[i] = (Y.cpu(), Yt.cpu())
        except Exception as e:                     # reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(graphs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i in range(len(graphs)):
        Y = handles[i].apply(Xs[i])
        assert torch.equal(Y.cpu(), out[i][0])
        assert torch.equal(handles[i].apply(Y, transpose=True).cpu(), out[i][1])
        handles[i].sync_status()
        handles[i].close()


def test_orientations_of_one_handle_overlap():
    """On one handle, A X products (a host-buffer sweep and device applies)
    from one thread and PageRank's A^T products from another run at once and
    give the results of the same calls made one at a time."""
    import torch
    from paper_1602_02864_gb300 import spmm
    A = synth.rmat_csr(15, seed=11)
    h = spmm.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)
    ks = (1, 8, 33)
    Xp = [torch.from_numpy(synth.dense(A.n_cols, k, seed=k)).pin_memory() for k in ks]
    Yp = [torch.empty((A.n_rows, k), dtype=torch.float32).pin_memory() for k in ks]
    Xd = torch.from_numpy(synth.dense(A.n_cols, 4, seed=4)).cuda()
    x = torch.empty(A.n_rows, dtype=torch.float32, device="cuda")
    try:
        # one at a time: these calls also grow the host-call buffers and
        # capture the PageRank graph, which must not overlap anything
        h.apply_host_parts(Xp, Yp)
        Y_ref = [y.clone() for y in Yp]
        Yd_ref = h.apply(Xd).cpu()
        _, res_ref = h.pagerank(0.85, 12, x=x)
        x_ref = x.cpu()
        torch.cuda.synchronize()
        errors = []

        def ranks():
            try:
                s = torch.cuda.Stream()
                for _ in range(4):
                    _, res = h.pagerank(0.85, 12, x=x, stream=s)
                    assert np.array_equal(res, res_ref)
                s.synchronize()
            except Exception as e:                 # reported below
                errors.append(e)

        for _ in range(3):
            for y in Yp:
                y.fill_(float("nan"))
            t = threading.Thread(target=ranks)
            t.start()
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                h.apply_host_parts(Xp, Yp, stream=s)
                Yd = h.apply(Xd, stream=s)
            s.synchronize()
            t.join()
            assert not errors, errors
            for y, r in zip(Yp, Y_ref):
                assert torch.equal(y, r)
            assert torch.equal(Yd.cpu(), Yd_ref)
            assert torch.equal(x.cpu(), x_ref)
        h.sync_status()
    finally:
        h.close()
