"""bench.py helpers that run without a GPU: the source digest that keys the
stored traffic record ignores comments and layout but not code."""
import bench


def test_code_tokens_drops_comments_keeps_literals():
    src = 'int a = 1; // note\n/* block\n comment */ char* s = "x // y /* z */"; char q = \'"\';\n\n  float b;'
    assert bench.code_tokens(src) == 'int a = 1; char* s = "x // y /* z */"; char q = \'"\'; float b;'
    assert bench.code_tokens('a = "esc \\" // still string"; // gone') == 'a = "esc \\" // still string";'


def test_comment_edits_keep_the_digest_code_edits_change_it():
    base = "__global__ void k(float* y) {\n    y[0] = 1.f;   // one\n}\n"
    reworded = "// a kernel\n__global__ void k(float* y) {\n    y[0] = 1.f;   /* the value one */\n}\n"
    changed = "__global__ void k(float* y) {\n    y[0] = 2.f;\n}\n"
    assert bench.code_tokens(base) == bench.code_tokens(reworded)
    assert bench.code_tokens(base) != bench.code_tokens(changed)


def test_vertical_parts_cover_every_column_once():
    ks = [1, 2, 4, 8, 16, 32, 64]
    for P in (1, 3, 16, 32, 64, 100):
        parts = bench.vertical_parts(ks, P)
        w = min(64, max(1, P))
        assert all(1 <= c1 - c0 <= w for _, c0, c1 in parts)
        for k in ks:
            mine = [(c0, c1) for kk, c0, c1 in parts if kk == k]
            assert mine[0][0] == 0 and mine[-1][1] == k                      # whole X_k, in order
            assert all(a[1] == b[0] for a, b in zip(mine, mine[1:]))
            assert len(mine) == -(-k // w)                                     # one pass over A each
        assert sum(c1 - c0 for _, c0, c1 in parts) == sum(ks)                 # the bytes the step moves
    assert len(bench.vertical_parts(ks, 16)) == 11


def test_host_cpu_names_the_machine_and_cores():
    import os
    import platform
    s = bench.host_cpu()
    assert s.startswith(platform.machine()) and s.endswith(f"{os.cpu_count()} logical cores")


def test_algorithmic_bytes_of_the_scale24_sweep():
    """A once, X once, Y once: nnz * (4 + value bytes) + 8 (N + 1) + N k (x + 4).
    At R-MAT scale 24 with 2^28 stored entries this is 1.342 GB at k = 1 and
    9.798 GB at k = 64 (FP32 X, pattern)."""
    nnz, n = 1 << 28, 1 << 24
    assert bench.alg_bytes(nnz, n, n, 1, 4) == 4 * nnz + 8 * (n + 1) + 8 * n
    assert round(bench.alg_bytes(nnz, n, n, 1, 4) / 1e9, 3) == 1.342
    assert round(bench.alg_bytes(nnz, n, n, 64, 4) / 1e9, 3) == 9.798
    # a weighted matrix adds its values; BF16 X halves the X side only
    assert bench.alg_bytes(nnz, n, n, 8, 4, 4) - bench.alg_bytes(nnz, n, n, 8, 4) == 4 * nnz
    assert bench.alg_bytes(nnz, n, n, 8, 4) - bench.alg_bytes(nnz, n, n, 8, 2) == 2 * 8 * n
    # one PageRank iteration: the k = 1 A^T product plus the update's five vectors
    assert bench.pagerank_iter_bytes(nnz, n) == bench.alg_bytes(nnz, n, n, 1, 4) + 20 * n
