"""The GPU R-MAT generator (for graphs too large to sort on the host) makes
the same draws as the CPU one, so both must give the same CSR bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scale,n_edges,block_bits,seed", [(8, None, 0, 0), (12, 50_001, 3, 1), (16, None, 10, 0),
                                                           (16, 2_000_003, 12, 7), (1, 9, 1, 2)])
def test_gpu_rmat_equals_cpu(scale, n_edges, block_bits, seed):
    A = synth.rmat_csr(scale, n_edges, seed=seed)
    B = synth.rmat_csr_cuda(scale, n_edges, seed=seed, block_bits=block_bits, pinned=scale == 12)
    assert A.n_rows == B.n_rows and A.nnz == B.nnz
    assert np.array_equal(A.row_ptr, B.row_ptr)
    assert np.array_equal(A.col_idx, B.col_idx)
