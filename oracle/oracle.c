/*
 * oracle.c -- plain, slow, FP64 CPU reference for the paper's sparse-matrix
 * dense-matrix multiplication (SpMM) and the applications built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls
 * this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * Every function is the plain definition, in the paper's order, accumulated
 * in double precision:
 *   oracle_spmm        Y = A X and Y = A^T X                (Section 3, Algorithm 1:
 *                      each nonzero a_ij adds a_ij * X[j,:] to output row i)
 *   oracle_spmm_rows   the same for a list of output rows
 *   oracle_pagerank    PR(u) = (1-d)/N + d * sum_{v in B(u)} PR(v)/L(v)
 *                      (Section 4.1), dangling mass spread uniformly
 *   oracle_nmf         H <- H o (W^T A) / (W^T W H),  W <- W o (A H^T) / (W H H^T)
 *                      (Section 4.3, multiplicative updates, H first)
 *   oracle_lanczos     top eigenpairs of a symmetric sparse matrix (Section 4.2
 *                      needs eigenpairs; block Lanczos with full
 *                      re-orthogonalisation, cyclic Jacobi on the projection)
 * Types: vtype 0 = pattern (every stored entry is 1), 1 = float32, 2 = float64.
 *        xtype 1 = float32, 2 = float64.  Inputs are read in their own type and
 *        widened to double exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline double vget(const void* v, int32_t vtype, int64_t p) {
    if (vtype == 0 || v == NULL) return 1.0;
    if (vtype == 1) return (double)((const float*)v)[p];
    return ((const double*)v)[p];
}

static inline double xget(const void* x, int32_t xtype, int64_t idx) {
    if (xtype == 1) return (double)((const float*)x)[idx];
    return ((const double*)x)[idx];
}

int32_t oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Y[i, j] = sum_{p in row i} a_p * X[col_p, j]        (transpose == 0)
 * Y[c, j] = sum over stored (i, c): a_p * X[i, j]      (transpose != 0)
 * Y is n_rows x k (forward) or n_cols x k (transpose), leading dimension ldy.
 * The forward product runs rows in parallel when nthreads > 1 (rows are
 * independent; each row is still summed in CSR order).  The transpose is
 * summed serially, rows in order. */
void oracle_spmm(int64_t n_rows, int64_t n_cols, const int64_t* row_ptr, const int32_t* col_idx,
                 const void* val, int32_t vtype, const void* X, int32_t xtype, int64_t ldx,
                 int32_t k, double* Y, int64_t ldy, int32_t transpose, int32_t nthreads) {
    if (!transpose) {
#ifdef _OPENMP
        if (nthreads < 1) nthreads = 1;
        #pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
#endif
        for (int64_t i = 0; i < n_rows; ++i) {
            for (int32_t j = 0; j < k; ++j) {
                double s = 0.0;
                for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                    s += vget(val, vtype, p) * xget(X, xtype, (int64_t)col_idx[p] * ldx + j);
                Y[i * ldy + j] = s;
            }
        }
    } else {
        for (int64_t c = 0; c < n_cols; ++c)
            for (int32_t j = 0; j < k; ++j) Y[c * ldy + j] = 0.0;
        for (int64_t i = 0; i < n_rows; ++i)
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                double a = vget(val, vtype, p);
                int64_t c = col_idx[p];
                for (int32_t j = 0; j < k; ++j) Y[c * ldy + j] += a * xget(X, xtype, i * ldx + j);
            }
    }
}

/* Forward product for the listed output rows only: Y is n_sample x k. */
void oracle_spmm_rows(const int64_t* row_ptr, const int32_t* col_idx, const void* val,
                      int32_t vtype, const void* X, int32_t xtype, int64_t ldx, int32_t k,
                      const int64_t* rows, int64_t n_sample, double* Y, int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
    #pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n_sample; ++s) {
        int64_t i = rows[s];
        for (int32_t j = 0; j < k; ++j) {
            double acc = 0.0;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                acc += vget(val, vtype, p) * xget(X, xtype, (int64_t)col_idx[p] * ldx + j);
            Y[s * k + j] = acc;
        }
    }
}

/* Transposed product for the listed output rows (columns of A) only.
 * slot[c] = index into Y for sampled column c, or -1.  Scans every stored
 * entry once, rows in order. */
void oracle_spmm_t_rows(int64_t n_rows, const int64_t* row_ptr, const int32_t* col_idx,
                        const void* val, int32_t vtype, const void* X, int32_t xtype, int64_t ldx,
                        int32_t k, const int64_t* slot, int64_t n_sample, double* Y) {
    for (int64_t s = 0; s < n_sample * k; ++s) Y[s] = 0.0;
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t s = slot[col_idx[p]];
            if (s < 0) continue;
            double a = vget(val, vtype, p);
            for (int32_t j = 0; j < k; ++j) Y[s * k + j] += a * xget(X, xtype, i * ldx + j);
        }
}

/* PageRank power iteration on the pattern of A (row v lists the out-links of
 * v, so B(u) = {v : A[v, u] stored} and L(v) = number of entries in row v).
 * x holds the start vector on entry and the result on exit.  Each iteration:
 *   x'[u] = (1-d)/N + d * (sum_{L(v)=0} x[v]) / N + d * sum_{v in B(u)} x[v] / L(v)
 * residuals[t] = sum_u |x'[u] - x[u]|. */
void oracle_pagerank(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, double d,
                     int32_t iters, double* x, double* residuals) {
    double* nx = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
    for (int32_t t = 0; t < iters; ++t) {
        double dangling = 0.0;
        for (int64_t v = 0; v < n; ++v)
            if (row_ptr[v + 1] == row_ptr[v]) dangling += x[v];
        double base = (1.0 - d) / (double)n + d * dangling / (double)n;
        for (int64_t u = 0; u < n; ++u) nx[u] = base;
        for (int64_t v = 0; v < n; ++v) {
            int64_t L = row_ptr[v + 1] - row_ptr[v];
            if (L == 0) continue;
            double share = x[v] / (double)L;
            for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) nx[col_idx[p]] += d * share;
        }
        double r = 0.0;
        for (int64_t u = 0; u < n; ++u) { r += fabs(nx[u] - x[u]); x[u] = nx[u]; }
        if (residuals) residuals[t] = r;
    }
    free(nx);
}

/* ||A - W H||_F^2 = ||A||_F^2 - 2 tr(W^T (A H^T)) + tr((W^T W)(H H^T)),
 * H stored transposed (Ht is n_cols x k). */
static double nmf_objective(int64_t n_rows, int64_t n_cols, const int64_t* row_ptr,
                            const int32_t* col_idx, const void* val, int32_t vtype, int32_t k,
                            const double* W, const double* Ht) {
    double a2 = 0.0, cross = 0.0, quad = 0.0;
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            double a = vget(val, vtype, p);
            a2 += a * a;
            double wh = 0.0;
            for (int32_t r = 0; r < k; ++r) wh += W[i * k + r] * Ht[(int64_t)col_idx[p] * k + r];
            cross += a * wh;
        }
    double* WtW = (double*)calloc((size_t)k * k, sizeof(double));
    double* HHt = (double*)calloc((size_t)k * k, sizeof(double));
    for (int64_t i = 0; i < n_rows; ++i)
        for (int32_t r = 0; r < k; ++r)
            for (int32_t s = 0; s < k; ++s) WtW[r * k + s] += W[i * k + r] * W[i * k + s];
    for (int64_t c = 0; c < n_cols; ++c)
        for (int32_t r = 0; r < k; ++r)
            for (int32_t s = 0; s < k; ++s) HHt[r * k + s] += Ht[c * k + r] * Ht[c * k + s];
    for (int32_t r = 0; r < k; ++r)
        for (int32_t s = 0; s < k; ++s) quad += WtW[r * k + s] * HHt[s * k + r];
    free(WtW);
    free(HHt);
    return a2 - 2.0 * cross + quad;
}

/* Lee-Seung multiplicative updates, H first then W, for `steps` steps:
 *   Ht <- Ht o (A^T W) / (Ht (W^T W) + eps)
 *   W  <- W  o (A Ht)  / (W (Ht^T Ht) + eps)
 * objective[t] = ||A - W H||_F^2 before step t, objective[steps] after the last. */
void oracle_nmf(int64_t n_rows, int64_t n_cols, const int64_t* row_ptr, const int32_t* col_idx,
                const void* val, int32_t vtype, int32_t k, int32_t steps, double eps, double* W,
                double* Ht, double* objective) {
    double* G = (double*)malloc(sizeof(double) * (size_t)k * k);
    double* AtW = (double*)malloc(sizeof(double) * (size_t)(n_cols ? n_cols : 1) * k);
    double* AH = (double*)malloc(sizeof(double) * (size_t)(n_rows ? n_rows : 1) * k);
    if (objective)
        objective[0] = nmf_objective(n_rows, n_cols, row_ptr, col_idx, val, vtype, k, W, Ht);
    for (int32_t t = 0; t < steps; ++t) {
        /* H update */
        memset(G, 0, sizeof(double) * (size_t)k * k);
        for (int64_t i = 0; i < n_rows; ++i)
            for (int32_t r = 0; r < k; ++r)
                for (int32_t s = 0; s < k; ++s) G[r * k + s] += W[i * k + r] * W[i * k + s];
        oracle_spmm(n_rows, n_cols, row_ptr, col_idx, val, vtype, W, 2, k, k, AtW, k, 1, 1);
        for (int64_t c = 0; c < n_cols; ++c) {
            double den[64];
            for (int32_t r = 0; r < k; ++r) {
                double s = 0.0;
                for (int32_t q = 0; q < k; ++q) s += Ht[c * k + q] * G[q * k + r];
                den[r] = s;
            }
            for (int32_t r = 0; r < k; ++r) Ht[c * k + r] *= AtW[c * k + r] / (den[r] + eps);
        }
        /* W update */
        memset(G, 0, sizeof(double) * (size_t)k * k);
        for (int64_t c = 0; c < n_cols; ++c)
            for (int32_t r = 0; r < k; ++r)
                for (int32_t s = 0; s < k; ++s) G[r * k + s] += Ht[c * k + r] * Ht[c * k + s];
        oracle_spmm(n_rows, n_cols, row_ptr, col_idx, val, vtype, Ht, 2, k, k, AH, k, 0, 1);
        for (int64_t i = 0; i < n_rows; ++i) {
            double den[64];
            for (int32_t r = 0; r < k; ++r) {
                double s = 0.0;
                for (int32_t q = 0; q < k; ++q) s += W[i * k + q] * G[q * k + r];
                den[r] = s;
            }
            for (int32_t r = 0; r < k; ++r) W[i * k + r] *= AH[i * k + r] / (den[r] + eps);
        }
        if (objective)
            objective[t + 1] = nmf_objective(n_rows, n_cols, row_ptr, col_idx, val, vtype, k, W, Ht);
    }
    free(G);
    free(AtW);
    free(AH);
}

/* ------------------------------------------------------------ eigensolver -- */
/* Cyclic Jacobi eigen-decomposition of a dense symmetric m x m matrix M
 * (row-major, destroyed).  On return evals[i] are the eigenvalues and column i
 * of V (row-major m x m) the matching unit eigenvector.  Rotations annihilate
 * one off-diagonal pair at a time until the off-diagonal mass is negligible. */
void oracle_jacobi_eigh(int32_t m, double* M, double* evals, double* V) {
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    for (int32_t sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int32_t i = 0; i < m; ++i)
            for (int32_t j = 0; j < m; ++j) {
                tot += M[i * m + j] * M[i * m + j];
                if (i != j) off += M[i * m + j] * M[i * m + j];
            }
        if (off <= 1e-30 * (tot > 0 ? tot : 1.0) || off == 0.0) break;
        for (int32_t p = 0; p < m; ++p)
            for (int32_t q = p + 1; q < m; ++q) {
                double apq = M[p * m + q];
                if (apq == 0.0) continue;
                double app = M[p * m + p], aqq = M[q * m + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int32_t r = 0; r < m; ++r) {   /* M <- M J (columns p, q) */
                    double mrp = M[r * m + p], mrq = M[r * m + q];
                    M[r * m + p] = c * mrp - s * mrq;
                    M[r * m + q] = s * mrp + c * mrq;
                }
                for (int32_t r = 0; r < m; ++r) {   /* M <- J^T M (rows p, q) */
                    double mpr = M[p * m + r], mqr = M[q * m + r];
                    M[p * m + r] = c * mpr - s * mqr;
                    M[q * m + r] = s * mpr + c * mqr;
                }
                for (int32_t r = 0; r < m; ++r) {   /* V <- V J */
                    double vrp = V[r * m + p], vrq = V[r * m + q];
                    V[r * m + p] = c * vrp - s * vrq;
                    V[r * m + q] = s * vrp + c * vrq;
                }
            }
    }
    for (int32_t i = 0; i < m; ++i) evals[i] = M[i * m + i];
}

/* Block Lanczos with full re-orthogonalisation on a symmetric CSR matrix S
 * (n x n).  Q0 (n x b, row-major) is the start block.  Builds an orthonormal
 * Krylov basis of up to m_max columns (m_max a multiple of b), projects
 * T = Q^T S Q, diagonalises T by Jacobi, and returns the nev largest Ritz
 * values (descending) and their Ritz vectors (n x nev row-major).
 * Returns the basis size used, or -1 on allocation failure. */
int32_t oracle_lanczos(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const void* val,
                       int32_t vtype, int32_t b, int32_t m_max, const double* Q0, int32_t nev,
                       double* evals, double* evecs) {
    double* Q = (double*)calloc((size_t)n * m_max, sizeof(double));   /* column-major n x m */
    double* W = (double*)malloc(sizeof(double) * (size_t)n * b);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n * b);
    if (!Q || !W || !tmp) { free(Q); free(W); free(tmp); return -1; }
    int32_t m = 0;
    /* orthonormalise a block of candidate columns against Q[:, :m] (twice)
     * and against each other by modified Gram-Schmidt; drop dependent ones */
    #define ORTH_APPEND(BLK, NB)                                                        \
        for (int32_t cc = 0; cc < (NB) && m < m_max; ++cc) {                            \
            double* v = (BLK) + (size_t)cc * n;                                         \
            double nrm0 = 0.0;                                                          \
            for (int64_t i = 0; i < n; ++i) nrm0 += v[i] * v[i];                        \
            nrm0 = sqrt(nrm0);                                                          \
            for (int pass = 0; pass < 2; ++pass)                                        \
                for (int32_t j = 0; j < m; ++j) {                                       \
                    double* qj = Q + (size_t)j * n;                                     \
                    double dot = 0.0;                                                   \
                    for (int64_t i = 0; i < n; ++i) dot += qj[i] * v[i];                \
                    for (int64_t i = 0; i < n; ++i) v[i] -= dot * qj[i];                \
                }                                                                       \
            double nrm = 0.0;                                                           \
            for (int64_t i = 0; i < n; ++i) nrm += v[i] * v[i];                         \
            nrm = sqrt(nrm);                                                            \
            if (nrm <= 1e-10 * (nrm0 > 0 ? nrm0 : 1.0)) continue;                      \
            double* qm = Q + (size_t)m * n;                                             \
            for (int64_t i = 0; i < n; ++i) qm[i] = v[i] / nrm;                         \
            ++m;                                                                        \
        }
    for (int32_t c = 0; c < b; ++c)
        for (int64_t i = 0; i < n; ++i) W[(size_t)c * n + i] = Q0[i * b + c];
    ORTH_APPEND(W, b);
    int32_t done = 0;
    while (m < m_max && m > done) {
        int32_t lo = done, hi = m;    /* expand the newest block */
        int32_t nb = hi - lo;
        for (int32_t c = 0; c < nb; ++c) {
            const double* q = Q + (size_t)(lo + c) * n;
            double* w = W + (size_t)c * n;
            for (int64_t i = 0; i < n; ++i) {
                double s = 0.0;
                for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                    s += vget(val, vtype, p) * q[col_idx[p]];
                w[i] = s;
            }
        }
        done = hi;
        ORTH_APPEND(W, nb);
    }
    #undef ORTH_APPEND
    /* T = Q^T S Q */
    double* T = (double*)calloc((size_t)m * m, sizeof(double));
    double* V = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* ev = (double*)malloc(sizeof(double) * (size_t)m);
    double* Sq = (double*)malloc(sizeof(double) * (size_t)n);
    for (int32_t j = 0; j < m; ++j) {
        const double* q = Q + (size_t)j * n;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += vget(val, vtype, p) * q[col_idx[p]];
            Sq[i] = s;
        }
        for (int32_t r = 0; r < m; ++r) {
            const double* qr = Q + (size_t)r * n;
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += qr[i] * Sq[i];
            T[r * m + j] = s;
        }
    }
    for (int32_t r = 0; r < m; ++r)       /* symmetrise rounding */
        for (int32_t j = r + 1; j < m; ++j) {
            double a = 0.5 * (T[r * m + j] + T[j * m + r]);
            T[r * m + j] = a; T[j * m + r] = a;
        }
    oracle_jacobi_eigh(m, T, ev, V);
    /* pick the nev largest */
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    for (int32_t i = 0; i < m; ++i) order[i] = i;
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = i + 1; j < m; ++j)
            if (ev[order[j]] > ev[order[i]]) { int32_t t = order[i]; order[i] = order[j]; order[j] = t; }
    for (int32_t e = 0; e < nev && e < m; ++e) {
        int32_t c = order[e];
        evals[e] = ev[c];
        if (evecs)
            for (int64_t i = 0; i < n; ++i) {
                double s = 0.0;
                for (int32_t j = 0; j < m; ++j) s += Q[(size_t)j * n + i] * V[j * m + c];
                evecs[i * nev + e] = s;
            }
    }
    free(order); free(T); free(V); free(ev); free(Sq);
    free(Q); free(W); free(tmp);
    return m;
}
