"""Plant plausible mistakes in a copy of oracle.c (on the CPU) and check that
the pins fail on each one.  A pin that cannot tell a mutant from the real
oracle would not be pinning anything."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_apps as apps
from tests import test_oracle_spmm as sp

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    # forward product reads the output row's own X row (wrong index)
    "fwd_wrong_index": ("* xget(X, xtype, (int64_t)col_idx[p] * ldx + j);\n                Y[i * ldy + j] = s;",
                        "* xget(X, xtype, (int64_t)i * ldx + j);\n                Y[i * ldy + j] = s;",
                        [lambda: sp.test_vs_dense_matmul(0, True, 3)]),
    # forward product drops the edge value
    "fwd_drop_value": ("s += vget(val, vtype, p) * xget(X, xtype, (int64_t)col_idx[p] * ldx + j);",
                       "s += xget(X, xtype, (int64_t)col_idx[p] * ldx + j);",
                       [lambda: sp.test_vs_dense_matmul(1, True, 1)]),
    # transposed product uses the transposed operand's row
    "t_transposed_operand": ("Y[c * ldy + j] += a * xget(X, xtype, i * ldx + j);",
                             "Y[c * ldy + j] += a * xget(X, xtype, c * ldx + j);",
                             [sp.test_cycle_shifts_rows]),
    # PageRank forgets the dangling mass
    "pr_no_dangling": ("d * dangling / (double)n;", "0.0 * dangling;",
                       [apps.test_pagerank_two_node_closed_form, apps.test_pagerank_vs_dense_google_matrix]),
    # PageRank forgets to divide by the out-degree
    "pr_no_outdegree": ("double share = x[v] / (double)L;", "double share = x[v];",
                        [apps.test_pagerank_vs_dense_google_matrix]),
    # NMF objective with the cross term's factor 2 dropped
    "nmf_objective_cross": ("return a2 - 2.0 * cross + quad;", "return a2 - cross + quad;",
                            [lambda: apps.test_nmf_vs_dense_updates(False)]),
    # NMF W update with an off-by-one numerator column
    "nmf_w_numerator": ("W[i * k + r] *= AH[i * k + r] / (den[r] + eps);",
                        "W[i * k + r] *= AH[i * k + (r + 1) % k] / (den[r] + eps);",
                        [lambda: apps.test_nmf_vs_dense_updates(True)]),
    # Householder update of the trailing block with a dropped rank-one term
    "house_dropped_term": ("M[i * m + j] += -2.0 * v[i] * p[j] - 2.0 * p[i] * v[j] + 4.0 * vp * v[i] * v[j];",
                           "M[i * m + j] += -2.0 * v[i] * p[j] - 2.0 * p[i] * v[j];",
                           [apps.test_sym_eigh_vs_numpy_eigh]),
    # Sturm count off by one comparison (counts eigenvalues at or above x)
    "sturm_sign": ("if (q < 0.0) ++cnt;", "if (q > 0.0) ++cnt;", [apps.test_sym_eigh_vs_numpy_eigh]),
    # no re-orthogonalisation inside clusters
    "inverse_iteration_no_reorth": ("for (int32_t q = c0; q < r; ++q) {", "for (int32_t q = r; q < r; ++q) {",
                                    [apps.test_sym_eigh_repeated_and_clustered_eigenvalues]),
    # the A^T A operator applies A twice instead of A then A^T
    "svd_operator": ("w[col_idx[p]] += vget(val, vtype, p) * t[i];", "w[i] += vget(val, vtype, p) * t[col_idx[p]];",
                     [apps.test_svds_vs_numpy_svd]),
    # the sampled-rows product reads the output row's own X row
    "rows_wrong_index": ("acc += vget(val, vtype, p) * xget(X, xtype, (int64_t)col_idx[p] * ldx + j);",
                         "acc += vget(val, vtype, p) * xget(X, xtype, (int64_t)i * ldx + j);",
                         [sp.test_sampled_rows_and_threads_agree]),
    # the sampled transposed product gathers instead of scattering
    "t_rows_transposed_operand": ("Y[s * k + j] += a * xget(X, xtype, i * ldx + j);",
                                  "Y[s * k + j] += a * xget(X, xtype, (int64_t)col_idx[p] * ldx + j);",
                                  [sp.test_sampled_rows_and_threads_agree]),
    # PageRank's teleport term not divided by N
    "pr_teleport_not_divided": ("double base = (1.0 - d) / (double)n + d * dangling / (double)n;",
                                "double base = (1.0 - d) + d * dangling / (double)n;",
                                [apps.test_pagerank_two_node_closed_form, apps.test_pagerank_sums_to_one_every_iteration]),
    # NMF H update with an off-by-one numerator column
    "nmf_h_numerator": ("Ht[c * k + r] *= AtW[c * k + r] / (den[r] + eps);",
                        "Ht[c * k + r] *= AtW[c * k + (r + 1) % k] / (den[r] + eps);",
                        [lambda: apps.test_nmf_vs_dense_updates(True)]),
    # the forward product skips each row's first stored entry
    "fwd_skips_first_entry": ("for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)\n                    s += vget(",
                              "for (int64_t p = row_ptr[i] + 1; p < row_ptr[i + 1]; ++p)\n                    s += vget(",
                              [lambda: sp.test_vs_dense_matmul(0, True, 3), sp.test_ones_give_degrees]),
    # PageRank's residual adds signed changes (they cancel: both vectors sum to 1)
    "pr_residual_signed": ("r += fabs(nx[u] - x[u]);", "r += nx[u] - x[u];",
                           [apps.test_pagerank_residuals_are_l1_changes]),
    # PageRank spreads the rank of the vertices that have out-links instead of the dangling ones
    "pr_dangling_inverted": ("if (row_ptr[v + 1] == row_ptr[v]) dangling += x[v];",
                             "if (row_ptr[v + 1] != row_ptr[v]) dangling += x[v];",
                             [apps.test_pagerank_two_node_closed_form, apps.test_pagerank_vs_dense_google_matrix]),
    # NMF objective without ||A||_F^2
    "nmf_objective_no_a2": ("a2 += a * a;", "a2 += 0.0 * a;", [lambda: apps.test_nmf_vs_dense_updates(True)]),
    # block Lanczos always expands the first block instead of the newest one
    "lanczos_expands_first_block": ("Q + (size_t)(lo + c) * n,", "Q + (size_t)c * n,",
                                    [apps.test_lanczos_vs_dense_eigh_on_rmat, apps.test_lanczos_cycle_closed_form]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new, pins = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mpath = tmp_path / "oracle_mut.c"
    mpath.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-o", str(lib), str(mpath), "-lm"])
    with oracle.using_library(str(lib)):
        for pin in pins:
            with pytest.raises(AssertionError):
                pin()
