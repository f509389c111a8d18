"""Helpers for the GPU parity tests: run the CUDA path through the C-ABI and
compare with the FP64 oracle on the same seeded inputs."""
import numpy as np

import oracle


def to_dev(X, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(X))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rounded_host(Xd):
    """The exact values a device tensor holds, as float64 (bf16/f16 widen exactly)."""
    import torch
    return Xd.float().cpu().numpy().astype(np.float64)


def abs_product(A, Xh, transpose=False):
    """(|A| |X|): the scale of the float32 summation error for each output."""
    vals = None if A.values is None else np.abs(A.values.astype(np.float64))
    return oracle.spmm(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vals, np.abs(Xh), transpose=transpose)


def assert_close_rel(Y, Yref, scale, rtol, what=""):
    """|Y - Yref| <= rtol * (|A||X|) + 1e-30 elementwise."""
    Y = np.asarray(Y, dtype=np.float64)
    err = np.abs(Y - Yref)
    bound = rtol * scale + 1e-30
    bad = err > bound
    if bad.any():
        i = np.argwhere(bad)[0]
        ratio = (err / np.maximum(scale, 1e-300)).max()
        raise AssertionError(f"{what}: {bad.sum()} entries exceed rtol={rtol}; first at {tuple(i)}: "
                             f"got {Y[tuple(i)]!r} want {Yref[tuple(i)]!r} scale {scale[tuple(i)]!r}; "
                             f"max err/scale {ratio:.3e}")
