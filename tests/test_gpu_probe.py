"""Gather-rate diagnostics: argument checks and sane magnitudes."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    """The library binding with the diagnostics' two calls beside it."""
    import types
    from paper_1602_02864_gb300 import probe, spmm
    ns = types.SimpleNamespace(**{n: getattr(spmm, n) for n in dir(spmm) if not n.startswith("__")})
    ns.spmm_probe_gather = probe.spmm_probe_gather
    ns.spmm_probe_gather_cols = probe.spmm_probe_gather_cols
    return ns


def test_uniform_probe(sp):
    r_l2, b_l2 = sp.spmm_probe_gather(16 << 20, 16)
    assert r_l2 > 1e9 and abs(b_l2 - 16 * r_l2) < 1e-6 * b_l2
    with pytest.raises(sp.SpmmError):
        sp.spmm_probe_gather(16 << 20, 12)           # not a power of two
    with pytest.raises(sp.SpmmError):
        sp.spmm_probe_gather(1024, 16)               # table too small


def test_matrix_stream_probe(sp):
    A = synth.rmat_csr(14, seed=2)
    h = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, transpose=True)
    for t in (0, 1):
        for rb in (4, 12, 32, 256):
            r, b = sp.spmm_probe_gather_cols(h.handle, t, rb)
            assert r > 1e8 and abs(b - (rb + 4) * r) < 1e-6 * b
    with pytest.raises(sp.SpmmError):
        sp.spmm_probe_gather_cols(h.handle, 0, 6)
    h.close()
    hs = sp.SparseMatrix(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, None, streaming=True)
    with pytest.raises(sp.SpmmError):
        sp.spmm_probe_gather_cols(hs.handle, 0, 4)
    hs.close()
