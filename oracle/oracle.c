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
 *   oracle_spmm_t_rows A^T X for a list of output rows (columns of A)
 *   oracle_pagerank    PR(u) = (1-d)/N + d * sum_{v in B(u)} PR(v)/L(v)
 *                      (Section 4.1), dangling mass spread uniformly
 *   oracle_nmf         H <- H o (W^T A) / (W^T W H),  W <- W o (A H^T) / (W H H^T)
 *                      (Section 4.3, multiplicative updates, H first)
 *   oracle_lanczos     top eigenpairs of a symmetric sparse matrix, or of A^T A
 *                      for singular values (Sections 4.2, 5.5.2: block Lanczos
 *                      with full re-orthogonalisation; the projection is
 *                      diagonalised by oracle_sym_eigh: Householder
 *                      tridiagonalisation, Sturm bisection, inverse iteration)
 *   oracle_sym_eigh    all eigenpairs of a small dense symmetric matrix (the
 *                      Rayleigh-Ritz step of Section 4.2's eigensolver)
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
/* Dense symmetric eigenproblem, three textbook steps (any numerical linear
 * algebra text; e.g. Golub & Van Loan, Matrix Computations, ch. 8):
 *   1. Householder reduction M = H T H^T, T symmetric tridiagonal;
 *   2. each eigenvalue of T by bisection on its Sturm count (the number of
 *      negative pivots of the LDL^T factorisation of T - x I is the number of
 *      eigenvalues below x);
 *   3. each eigenvector of T by inverse iteration with T - lambda I factored
 *      by Gaussian elimination with partial pivoting, vectors of nearby
 *      eigenvalues re-orthogonalised, then mapped back by H. */

/* Householder tridiagonalisation of the symmetric m x m row-major M
 * (destroyed).  On return d (m) and e (m-1) hold T's diagonal and
 * sub-diagonal, and H (row-major m x m, orthogonal) satisfies M = H T H^T. */
static void house_tridiag(int32_t m, double* M, double* H, double* d, double* e) {
    double* v = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* p = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j) H[i * m + j] = (i == j) ? 1.0 : 0.0;
    for (int32_t k = 0; k + 2 < m; ++k) {
        /* reflect x = M[k+1.., k] onto alpha * e1 with P = I - 2 v v^T */
        double xn = 0.0;
        for (int32_t i = k + 1; i < m; ++i) xn += M[i * m + k] * M[i * m + k];
        xn = sqrt(xn);
        if (xn == 0.0) continue;
        const double x0 = M[(k + 1) * m + k];
        const double alpha = x0 > 0 ? -xn : xn;
        double vn = 0.0;
        for (int32_t i = k + 1; i < m; ++i) {
            v[i] = M[i * m + k] - (i == k + 1 ? alpha : 0.0);
            vn += v[i] * v[i];
        }
        vn = sqrt(vn);
        if (vn == 0.0) continue;
        for (int32_t i = k + 1; i < m; ++i) v[i] /= vn;
        /* trailing block B <- P B P = B - 2 v p^T - 2 p v^T + 4 (v^T p) v v^T, p = B v */
        double vp = 0.0;
        for (int32_t i = k + 1; i < m; ++i) {
            double acc = 0.0;
            for (int32_t j = k + 1; j < m; ++j) acc += M[i * m + j] * v[j];
            p[i] = acc;
        }
        for (int32_t i = k + 1; i < m; ++i) vp += v[i] * p[i];
        for (int32_t i = k + 1; i < m; ++i)
            for (int32_t j = k + 1; j < m; ++j)
                M[i * m + j] += -2.0 * v[i] * p[j] - 2.0 * p[i] * v[j] + 4.0 * vp * v[i] * v[j];
        /* column and row k: P x = alpha e1 */
        for (int32_t i = k + 1; i < m; ++i) {
            M[i * m + k] = (i == k + 1) ? alpha : 0.0;
            M[k * m + i] = M[i * m + k];
        }
        /* H <- H P on columns k+1.. */
        for (int32_t r = 0; r < m; ++r) {
            double hv = 0.0;
            for (int32_t j = k + 1; j < m; ++j) hv += H[r * m + j] * v[j];
            for (int32_t j = k + 1; j < m; ++j) H[r * m + j] -= 2.0 * hv * v[j];
        }
    }
    for (int32_t i = 0; i < m; ++i) d[i] = M[i * m + i];
    for (int32_t i = 0; i + 1 < m; ++i) e[i] = M[(i + 1) * m + i];
    free(v);
    free(p);
}

/* Number of eigenvalues of tridiag(d, e) below x (Sturm count). */
static int32_t sturm_below(int32_t m, const double* d, const double* e, double x, double tiny) {
    int32_t cnt = 0;
    double q = 1.0;
    for (int32_t i = 0; i < m; ++i) {
        const double ee = i > 0 ? e[i - 1] : 0.0;
        q = d[i] - x - (i > 0 ? ee * ee / q : 0.0);
        if (q == 0.0) q = -tiny;       /* a zero pivot: x is an eigenvalue of the leading block */
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

/* Solve (T - lam I) y = b in place (b -> y), T = tridiag(d, e), by Gaussian
 * elimination with partial pivoting; a zero pivot is replaced by `tiny`. */
static void tridiag_solve(int32_t m, const double* d, const double* e, double lam, double tiny, double* b,
                          double* work) {
    /* row i of the working matrix: diagonal a[i], first and second
     * super-diagonals c1[i], c2[i]; sub-diagonal entries are eliminated */
    double* a = work;
    double* c1 = work + m;
    double* c2 = work + 2 * m;
    double* l = work + 3 * m;          /* multipliers */
    int32_t* swapped = (int32_t*)(work + 4 * m);
    for (int32_t i = 0; i < m; ++i) {
        a[i] = d[i] - lam;
        c1[i] = i + 1 < m ? e[i] : 0.0;
        c2[i] = 0.0;
    }
    for (int32_t i = 0; i + 1 < m; ++i) {
        /* rows i and i+1; the sub-diagonal entry of row i+1 is e[i] */
        const double sub = e[i];
        swapped[i] = fabs(sub) > fabs(a[i]);
        if (swapped[i]) {
            /* exchange rows i and i+1 (row i+1: sub, a[i+1], c1[i+1]) */
            const double na = sub, nc1 = a[i + 1], nc2 = c1[i + 1];
            const double oa = a[i], oc1 = c1[i], oc2 = c2[i];
            a[i] = na; c1[i] = nc1; c2[i] = nc2;
            const double tb = b[i]; b[i] = b[i + 1]; b[i + 1] = tb;
            l[i] = oa / na;
            a[i + 1] = oc1 - l[i] * c1[i];
            c1[i + 1] = oc2 - l[i] * c2[i];
        } else {
            if (a[i] == 0.0) a[i] = tiny;
            l[i] = sub / a[i];
            a[i + 1] -= l[i] * c1[i];
            c1[i + 1] -= l[i] * c2[i];
        }
        c2[i + 1] = 0.0;
        b[i + 1] -= l[i] * b[i];
    }
    if (m > 0 && a[m - 1] == 0.0) a[m - 1] = tiny;
    for (int32_t i = m - 1; i >= 0; --i) {        /* back substitution */
        double s = b[i];
        if (i + 1 < m) s -= c1[i] * b[i + 1];
        if (i + 2 < m) s -= c2[i] * b[i + 2];
        b[i] = s / a[i];
    }
}

/* All eigenpairs of the symmetric m x m row-major M (destroyed): evals
 * ascending, V row-major m x m with column i the unit eigenvector of
 * evals[i].  Returns 0, or -1 on allocation failure. */
int32_t oracle_sym_eigh(int32_t m, double* M, double* evals, double* V) {
    if (m <= 0) return 0;
    double* H = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* d = (double*)malloc(sizeof(double) * (size_t)m);
    double* e = (double*)malloc(sizeof(double) * (size_t)m);
    double* Y = (double*)malloc(sizeof(double) * (size_t)m * m);    /* column j at Y + j*m */
    double* work = (double*)malloc(sizeof(double) * (size_t)m * 5 + sizeof(int32_t) * (size_t)m);
    if (!H || !d || !e || !Y || !work) { free(H); free(d); free(e); free(Y); free(work); return -1; }
    house_tridiag(m, M, H, d, e);
    /* Gershgorin bounds of T */
    double lo = d[0], hi = d[0], nrm = 0.0;
    for (int32_t i = 0; i < m; ++i) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
        if (d[i] - r < lo) lo = d[i] - r;
        if (d[i] + r > hi) hi = d[i] + r;
        if (fabs(d[i]) + r > nrm) nrm = fabs(d[i]) + r;
    }
    if (nrm == 0.0) nrm = 1.0;
    const double eps = 2.220446049250313e-16, tiny = eps * nrm;
    lo -= 2 * tiny;
    hi += 2 * tiny;
    /* eigenvalue r (ascending) = the x where the Sturm count passes r */
    for (int32_t r = 0; r < m; ++r) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 2 * eps * (fabs(a) + fabs(b)) + tiny * 1e-3; ++it) {
            const double mid = 0.5 * (a + b);
            if (sturm_below(m, d, e, mid, tiny * 1e-3) > r) b = mid;
            else a = mid;
        }
        evals[r] = 0.5 * (a + b);
    }
    /* inverse iteration; a cluster = eigenvalues within 1e-3 * ||T|| of the previous one */
    uint64_t seed = 0x9e3779b97f4a7c15ull;
    int32_t c0 = 0;
    for (int32_t r = 0; r < m; ++r) {
        if (r > 0 && evals[r] - evals[r - 1] > 1e-3 * nrm) c0 = r;
        double* y = Y + (size_t)r * m;
        for (int32_t i = 0; i < m; ++i) {   /* a fixed pseudo-random start (xorshift) */
            seed ^= seed << 13; seed ^= seed >> 7; seed ^= seed << 17;
            y[i] = (double)(seed >> 11) / 9007199254740992.0 - 0.5;
        }
        for (int it = 0; it < 4; ++it) {
            tridiag_solve(m, d, e, evals[r], tiny, y, work);
            for (int32_t q = c0; q < r; ++q) {    /* orthogonal to the cluster's earlier vectors */
                const double* z = Y + (size_t)q * m;
                double dot = 0.0;
                for (int32_t i = 0; i < m; ++i) dot += z[i] * y[i];
                for (int32_t i = 0; i < m; ++i) y[i] -= dot * z[i];
            }
            double n2 = 0.0;
            for (int32_t i = 0; i < m; ++i) n2 += y[i] * y[i];
            n2 = sqrt(n2);
            for (int32_t i = 0; i < m; ++i) y[i] /= n2;
        }
    }
    /* eigenvectors of M: V[:, r] = H y_r */
    for (int32_t i = 0; i < m; ++i)
        for (int32_t r = 0; r < m; ++r) {
            double s = 0.0;
            for (int32_t j = 0; j < m; ++j) s += H[i * m + j] * Y[(size_t)r * m + j];
            V[i * m + r] = s;
        }
    free(H); free(d); free(e); free(Y); free(work);
    return 0;
}

/* Block Lanczos with full re-orthogonalisation.  op = 0: on the symmetric
 * CSR matrix S (n_rows x n_rows); op = 1: on A^T A for the n_rows x n_cols
 * CSR matrix A, applied as A q then A^T (A q) (its eigenvalues are the
 * squared singular values of A; Section 5.5.2's SVD).  Q0 (n x b,
 * row-major; n = n_rows for op 0, n_cols for op 1) is the start block.
 * Builds an orthonormal Krylov basis of up to m_max columns, projects
 * T = Q^T Op Q, diagonalises T with oracle_sym_eigh, and returns the nev
 * largest Ritz values (descending) and their Ritz vectors (n x nev
 * row-major).  Returns the basis size used, or -1 on allocation failure. */
/* w = Op q for the operator of oracle_lanczos (t: n_rows scratch for op 1) */
static void lanczos_op(int32_t op, int64_t n_rows, int64_t n_cols, const int64_t* row_ptr, const int32_t* col_idx,
                       const void* val, int32_t vtype, const double* q, double* w, double* t) {
    if (op == 0) {
        for (int64_t i = 0; i < n_rows; ++i) {
            double s = 0.0;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += vget(val, vtype, p) * q[col_idx[p]];
            w[i] = s;
        }
        return;
    }
    for (int64_t i = 0; i < n_rows; ++i) {              /* t = A q */
        double s = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += vget(val, vtype, p) * q[col_idx[p]];
        t[i] = s;
    }
    for (int64_t c = 0; c < n_cols; ++c) w[c] = 0.0;     /* w = A^T t, rows in order */
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) w[col_idx[p]] += vget(val, vtype, p) * t[i];
}

int32_t oracle_lanczos(int64_t n_rows, int64_t n_cols, const int64_t* row_ptr, const int32_t* col_idx,
                       const void* val, int32_t vtype, int32_t op, int32_t b, int32_t m_max, const double* Q0,
                       int32_t nev, double* evals, double* evecs) {
    const int64_t n = op ? n_cols : n_rows;
    double* Q = (double*)calloc((size_t)n * m_max, sizeof(double));   /* column-major n x m */
    double* W = (double*)malloc(sizeof(double) * (size_t)n * b);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(n_rows > n ? n_rows : n));
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
        for (int32_t c = 0; c < nb; ++c)
            lanczos_op(op, n_rows, n_cols, row_ptr, col_idx, val, vtype, Q + (size_t)(lo + c) * n,
                       W + (size_t)c * n, tmp);
        done = hi;
        ORTH_APPEND(W, nb);
    }
    #undef ORTH_APPEND
    /* T = Q^T Op Q */
    double* T = (double*)calloc((size_t)m * m, sizeof(double));
    double* V = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* ev = (double*)malloc(sizeof(double) * (size_t)m);
    double* Sq = (double*)malloc(sizeof(double) * (size_t)n);
    for (int32_t j = 0; j < m; ++j) {
        lanczos_op(op, n_rows, n_cols, row_ptr, col_idx, val, vtype, Q + (size_t)j * n, Sq, tmp);
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
    if (oracle_sym_eigh(m, T, ev, V) != 0) m = -1;
    /* the nev largest: eigenvalues come ascending */
    for (int32_t e = 0; m > 0 && e < nev && e < m; ++e) {
        const int32_t c = m - 1 - e;
        evals[e] = ev[c];
        if (evecs)
            for (int64_t i = 0; i < n; ++i) {
                double s = 0.0;
                for (int32_t j = 0; j < m; ++j) s += Q[(size_t)j * n + i] * V[j * m + c];
                evecs[i * nev + e] = s;
            }
    }
    free(T); free(V); free(ev); free(Sq);
    free(Q); free(W); free(tmp);
    return m;
}
