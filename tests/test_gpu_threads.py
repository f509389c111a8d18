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
