"""Vertical partitions: the column-group width rule (host only, no GPU).

Section 3.6: with M' bytes for the dense matrices, a p-column input is
processed in ceil(p / cols) passes over the sparse matrix, so cols should be
as large as the memory allows.  Each column of a group costs two X buffers
and two Y buffers on the device."""
import pytest


@pytest.fixture(scope="module")
def sp():
    from paper_1602_02864_gb300 import spmm
    return spmm


def per_col(n_in, n_out, xbytes):
    return 2 * (n_in * xbytes + n_out * 4)


@pytest.mark.parametrize("n_in,n_out,p,xt,xb", [(1 << 20, 1 << 20, 32, "SPMM_F32", 4),
                                                (1000, 3000, 7, "SPMM_BF16", 2),
                                                (5, 0, 100, "SPMM_F16", 2)])
def test_widest_group_that_fits(sp, n_in, n_out, p, xt, xb):
    xtype = getattr(sp, xt)
    c = per_col(n_in, n_out, xb)
    for cols in (1, 2, 3, 5, 16, 64):
        want = min(cols, p, 64)
        assert sp.spmm_vpart_cols(n_in, n_out, p, xtype, cols * c) == want        # exact fit
        assert sp.spmm_vpart_cols(n_in, n_out, p, xtype, cols * c + c - 1) == want  # just below the next
    assert sp.spmm_vpart_cols(n_in, n_out, p, xtype, 10 ** 15) == min(p, 64)


def test_passes_decrease_with_memory(sp):
    n, p = 1 << 22, 32
    passes = []
    for cols in (1, 2, 4, 8, 16, 32):
        g = sp.spmm_vpart_cols(n, n, p, sp.SPMM_F32, cols * per_col(n, n, 4))
        passes.append(-(-p // g))
    assert passes == [32, 16, 8, 4, 2, 1]


def test_errors(sp):
    with pytest.raises(sp.SpmmError, match="ERR_OOM"):
        sp.spmm_vpart_cols(1 << 20, 1 << 20, 8, sp.SPMM_F32, per_col(1 << 20, 1 << 20, 4) - 1)
    for bad in [(-1, 5, 4, 0, 10 ** 9), (5, 5, 0, 0, 10 ** 9), (5, 5, 4, 0, -1), (5, 5, 4, 7, 10 ** 9)]:
        with pytest.raises(sp.SpmmError, match="ERR_ARG"):
            sp.spmm_vpart_cols(*bad)
