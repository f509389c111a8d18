/*
 * synth.c -- seeded synthetic inputs for the SpMM library, its tests and its
 * benchmark.  This module holds none of the sparse-times-dense arithmetic: it
 * only draws graphs, edge values and dense matrices, so that the CUDA path and
 * the CPU oracle can be fed identical inputs.
 *
 * Randomness: Philox4x32-10, written from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11).  Every draw is a pure function of (seed, index, sub-index, domain),
 * so any element can be regenerated on its own and the result does not depend
 * on the thread count.
 *
 * Graphs:
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with the paper's quadrant
 *     probabilities a/b/c/d = 0.57/0.19/0.19/0.05 (Section 5, graph datasets):
 *     every level draws one quadrant, no noise, no vertex permutation.
 *   - Chung-Lu power-law graphs (expected degree proportional to
 *     (i+1)^(-1/(gamma-1))), destinations relabelled by a seeded permutation.
 *   - stochastic block model graphs (Section 5.1's ordering experiment):
 *     equal clusters of consecutive ids, sources uniform, a destination in
 *     the source's cluster with probability p_in, else uniform outside it;
 *     any graph can be relabelled by a seeded uniform permutation.
 *   - the symmetrised union A + A^T with one lognormal(0,1) weight per
 *     unordered pair and symmetric degree normalisation D^-1/2 A D^-1/2.
 * Edge lists become CSR by a stable LSD radix sort on (row, col) keys and a
 * merge of duplicate keys.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Philox -- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Domain tags keep the draws made for different purposes apart. */
enum {
    DOM_EDGE = 0x45444745u,  /* R-MAT quadrant choices            */
    DOM_VAL  = 0x56414c53u,  /* edge values                        */
    DOM_X    = 0x584d4154u,  /* dense matrices                     */
    DOM_CL   = 0x43484c55u,  /* Chung-Lu endpoint draws            */
    DOM_PERM = 0x5045524du,  /* permutations                       */
    DOM_LOGN = 0x4c4f474eu,  /* lognormal pair weights             */
    DOM_SIZE = 0x53495a45u,  /* per-graph size / degree draws      */
    DOM_SAMP = 0x53414d50u,  /* sampled row ids                    */
    DOM_VPRM = 0x5650524du,  /* vertex relabelling permutations    */
    DOM_SBM  = 0x53424d45u   /* stochastic block model edges       */
};

static inline void draw4(uint64_t seed, uint64_t seed2, uint64_t idx, uint32_t sub,
                         uint32_t dom, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), sub, dom};
    uint32_t key[2] = {(uint32_t)seed ^ (uint32_t)(seed2 * 0x9E3779B9u),
                       (uint32_t)(seed >> 32) ^ (uint32_t)(seed2 >> 32) ^ (uint32_t)(seed2 * 0x85EBCA6Bu)};
    synth_philox4x32_10(ctr, key, out);
}

/* one 53-bit uniform in [0,1) from two words */
static inline double u53(uint32_t hi, uint32_t lo) {
    return (double)(((uint64_t)(hi >> 5) << 26) | (lo >> 6)) * (1.0 / 9007199254740992.0);
}

/* ----------------------------------------------------------------- R-MAT -- */
/* Edge e draws one 32-bit word per level; word w of call j serves level 4j+w.
 * Quadrant 0 = (row bit 0, col bit 0) with probability a, 1 = (0,1) with b,
 * 2 = (1,0) with c, 3 = (1,1) with d = 1-a-b-c.  Level 0 sets the most
 * significant bit. */
void synth_rmat_edges(int32_t scale, int64_t n_edges, double a, double b, double c,
                      uint64_t seed, uint32_t* src, uint32_t* dst) {
    const double t0 = a, t1 = a + b, t2 = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_edges; ++e) {
        uint32_t r = 0, col = 0, w[4];
        for (int32_t l = 0; l < scale; ++l) {
            if ((l & 3) == 0) draw4(seed, 0, (uint64_t)e, (uint32_t)(l >> 2), DOM_EDGE, w);
            double u = (double)w[l & 3] * (1.0 / 4294967296.0);
            int q = (u < t0) ? 0 : (u < t1) ? 1 : (u < t2) ? 2 : 3;
            r |= (uint32_t)(q >> 1) << (scale - 1 - l);
            col |= (uint32_t)(q & 1) << (scale - 1 - l);
        }
        src[e] = r;
        dst[e] = col;
    }
}

/* ----------------------------------------------------- edge list -> CSR -- */
static int bits_for(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

/* Stable LSD radix sort of 64-bit keys on 16-bit digits, OpenMP parallel.
 * On return the sorted keys are in a[]. */
static void radix_sort_u64(uint64_t* a, uint64_t* tmp, int64_t n, int key_bits) {
    int maxt = 1;
#ifdef _OPENMP
    maxt = omp_get_max_threads();
#endif
    int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * 65536 * (size_t)maxt);
    uint64_t* in = a;
    uint64_t* out = tmp;
    for (int shift = 0; shift < key_bits; shift += 16) {
        #pragma omp parallel num_threads(maxt)
        {
            int t = 0, nt = 1;
#ifdef _OPENMP
            t = omp_get_thread_num();
            nt = omp_get_num_threads();
#endif
            int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* h = hist + (size_t)t * 65536;
            memset(h, 0, sizeof(int64_t) * 65536);
            for (int64_t i = lo; i < hi; ++i) h[(in[i] >> shift) & 0xffff]++;
            #pragma omp barrier
            #pragma omp single
            {
                int64_t sum = 0;
                for (int d = 0; d < 65536; ++d)
                    for (int tt = 0; tt < nt; ++tt) {
                        int64_t cnt = hist[(size_t)tt * 65536 + d];
                        hist[(size_t)tt * 65536 + d] = sum;
                        sum += cnt;
                    }
            }
            for (int64_t i = lo; i < hi; ++i) out[h[(in[i] >> shift) & 0xffff]++] = in[i];
        }
        uint64_t* s = in; in = out; out = s;
    }
    if (in != a) memcpy(a, in, sizeof(uint64_t) * (size_t)n);
    free(hist);
}

/* Sort (src, dst) pairs by (src, dst), merge duplicates, and write CSR.
 * row_ptr has n_rows+1 entries; col_idx must hold n_edges entries.
 * If symmetrize != 0 the reversed pair is added for every edge first.
 * Returns nnz, or -1 on allocation failure. */
int64_t synth_edges_to_csr(int64_t n_rows, int64_t n_cols, int64_t n_edges,
                           const uint32_t* src, const uint32_t* dst, int32_t symmetrize,
                           int64_t* row_ptr, int32_t* col_idx) {
    int cb = bits_for(n_cols > n_rows ? n_cols : n_rows);
    int rb = cb;
    int64_t m = symmetrize ? 2 * n_edges : n_edges;
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
    if (!keys || !tmp) { free(keys); free(tmp); return -1; }
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_edges; ++e) {
        keys[e] = ((uint64_t)src[e] << cb) | dst[e];
        if (symmetrize) keys[n_edges + e] = ((uint64_t)dst[e] << cb) | src[e];
    }
    radix_sort_u64(keys, tmp, m, rb + cb);
    free(tmp);
    const uint64_t cmask = ((uint64_t)1 << cb) - 1;
    for (int64_t i = 0; i <= n_rows; ++i) row_ptr[i] = 0;
    int64_t nnz = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (e > 0 && keys[e] == keys[e - 1]) continue;
        uint64_t r = keys[e] >> cb;
        col_idx[nnz++] = (int32_t)(keys[e] & cmask);
        row_ptr[r + 1]++;
    }
    for (int64_t i = 0; i < n_rows; ++i) row_ptr[i + 1] += row_ptr[i];
    free(keys);
    return nnz;
}

/* ------------------------------------------------------ values, matrices -- */
/* val[p] = U[0,1) with 24 random bits (exact in float32), drawn per CSR
 * position p after duplicates are merged. */
void synth_uniform01_f32(uint64_t seed, uint64_t seed2, int64_t n, float* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < (n + 3) / 4; ++q) {
        uint32_t w[4];
        draw4(seed, seed2, (uint64_t)q, 0, DOM_VAL, w);
        for (int j = 0; j < 4; ++j) {
            int64_t p = 4 * q + j;
            if (p < n) out[p] = (float)(w[j] >> 8) * (1.0f / 16777216.0f);
        }
    }
}

/* Dense matrix element (i, j) is a function of (seed, seed2, i, j) only, so the
 * first k columns do not depend on how many columns are drawn.
 *   mode 0: U[-1,1) on a 2^-23 grid (exact in float32)
 *   mode 1: integers 0..7
 *   mode 2: U[0,1) on a 2^-24 grid (non-negative factors) */
static inline float x_elem(uint64_t seed, uint64_t seed2, int64_t i, int32_t j, int32_t mode) {
    uint32_t w[4];
    draw4(seed, seed2, (uint64_t)i, (uint32_t)(j >> 2), DOM_X, w);
    uint32_t r = w[j & 3];
    if (mode == 1) return (float)(r >> 29);
    if (mode == 2) return (float)(r >> 8) * (1.0f / 16777216.0f);
    return (float)(int32_t)(r >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

void synth_dense_f32(uint64_t seed, uint64_t seed2, int64_t row0, int64_t n_rows, int32_t k,
                     int64_t ld, int32_t mode, float* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_rows; ++i)
        for (int32_t j = 0; j < k; ++j) out[i * ld + j] = x_elem(seed, seed2, row0 + i, j, mode);
}

void synth_dense_rows_f32(uint64_t seed, uint64_t seed2, const int64_t* rows, int64_t n, int32_t k,
                          int32_t mode, float* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < k; ++j) out[i * k + j] = x_elem(seed, seed2, rows[i], j, mode);
}

/* n distinct-ish sampled row ids in [0, n_rows) (with replacement). */
void synth_sample_rows(uint64_t seed, int64_t n_rows, int64_t n, int64_t* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t w[4];
        draw4(seed, 0, (uint64_t)i, 0, DOM_SAMP, w);
        out[i] = (int64_t)(u53(w[0], w[1]) * (double)n_rows);
        if (out[i] >= n_rows) out[i] = n_rows - 1;
    }
}

/* -------------------------------------------------------------- Chung-Lu -- */
/* Graph g of a batch: n = round(exp(U[ln nmin, ln nmax])), average degree
 * U[dmin, dmax].  Returns n and writes the average degree. */
int64_t synth_chunglu_size(uint64_t seed, int64_t g, double nmin, double nmax, double dmin,
                           double dmax, double* avg_deg) {
    uint32_t w[4];
    draw4(seed, (uint64_t)g, 0, 0, DOM_SIZE, w);
    double u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
    double ln = log(nmin) + u1 * (log(nmax) - log(nmin));
    int64_t n = (int64_t)llround(exp(ln));
    if (n < 1) n = 1;
    *avg_deg = dmin + u2 * (dmax - dmin);
    return n;
}

/* Draw m directed edges for graph g: the source is drawn with probability
 * proportional to w_i = (i+1)^(-1/(gamma-1)), the destination with the same
 * weights relabelled by a seeded permutation pi (so A^T differs from A).
 * Returns 0, or -1 on allocation failure. */
int32_t synth_chunglu_edges(uint64_t seed, int64_t g, int64_t n, int64_t m, double gamma,
                            uint32_t* src, uint32_t* dst) {
    double* cum = (double*)malloc(sizeof(double) * (size_t)n);
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    if (!cum || !perm) { free(cum); free(perm); return -1; }
    double s = 0.0, ex = -1.0 / (gamma - 1.0);
    for (int64_t i = 0; i < n; ++i) { s += pow((double)(i + 1), ex); cum[i] = s; }
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {   /* Fisher-Yates */
        uint32_t w[4];
        draw4(seed, (uint64_t)g, (uint64_t)i, 0, DOM_PERM, w);
        int64_t j = (int64_t)(u53(w[0], w[1]) * (double)(i + 1));
        if (j > i) j = i;
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t w[4];
        draw4(seed, (uint64_t)g, (uint64_t)e, 0, DOM_CL, w);
        double t1 = u53(w[0], w[1]) * s, t2 = u53(w[2], w[3]) * s;
        int64_t lo = 0, hi = n - 1;                 /* first i with cum[i] > t1 */
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (cum[mid] > t1) hi = mid; else lo = mid + 1; }
        src[e] = (uint32_t)lo;
        lo = 0; hi = n - 1;
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (cum[mid] > t2) hi = mid; else lo = mid + 1; }
        dst[e] = perm[lo];
    }
    free(cum);
    free(perm);
    return 0;
}

/* ----------------------------------------- symmetric weights, normalising -- */
/* For a symmetric pattern (CSR of A + A^T), give pair {i,j} the weight
 * exp(z), z ~ N(0,1) by Box-Muller from the pair's own counter, so
 * w(i,j) == w(j,i) exactly.  Then, if normalise != 0, scale by
 * 1/sqrt(D_i D_j) where D is the weighted degree (rows with D = 0 stay 0).
 * Values are rounded to float32 once, at the end. */
void synth_sym_lognormal(uint64_t seed, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                         int32_t normalise, float* val) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(row_ptr[n] ? row_ptr[n] : 1));
    double* deg = (double*)calloc((size_t)n, sizeof(double));
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t j = col_idx[p];
            uint64_t lo = (uint64_t)(i < j ? i : j), hi = (uint64_t)(i < j ? j : i);
            uint32_t r[4];
            draw4(seed, hi, lo, 0, DOM_LOGN, r);
            double u1 = 1.0 - u53(r[0], r[1]);          /* (0, 1] */
            double u2 = u53(r[2], r[3]);
            double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
            w[p] = exp(z);
            d += w[p];
        }
        deg[i] = d;
    }
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            double v = w[p];
            if (normalise) {
                double dd = deg[i] * deg[col_idx[p]];
                v = dd > 0.0 ? v / sqrt(dd) : 0.0;
            }
            val[p] = (float)v;
        }
    free(w);
    free(deg);
}

/* ------------------------------------------------- vertex relabelling -- */
/* A uniform random permutation of 0..n-1 (Fisher-Yates; position i draws its
 * partner from 53-bit uniforms of its own counter). */
void synth_permutation(uint64_t seed, int64_t n, uint32_t* perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint32_t w[4];
        draw4(seed, 0, (uint64_t)i, 0, DOM_VPRM, w);
        int64_t j = (int64_t)(u53(w[0], w[1]) * (double)(i + 1));
        if (j > i) j = i;
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* Map both endpoints of m edges through perm, in place. */
void synth_relabel_edges(int64_t m, uint32_t* src, uint32_t* dst, const uint32_t* perm) {
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        src[e] = perm[src[e]];
        dst[e] = perm[dst[e]];
    }
}

/* ------------------------------------------------ stochastic block model -- */
/* n vertices in n_clusters equal clusters of consecutive ids (cluster of v is
 * v * n_clusters / n); edge e: source uniform over all vertices; with
 * probability p_in the destination is uniform over the source's cluster,
 * otherwise uniform over the vertices outside it.  Self-loops can occur
 * inside a cluster. */
void synth_sbm_edges(uint64_t seed, int64_t n, int64_t n_clusters, int64_t m, double p_in, uint32_t* src,
                     uint32_t* dst) {
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint32_t w[4], v[4];
        draw4(seed, 0, (uint64_t)e, 0, DOM_SBM, w);
        draw4(seed, 0, (uint64_t)e, 1, DOM_SBM, v);
        int64_t s = (int64_t)(u53(w[0], w[1]) * (double)n);
        if (s >= n) s = n - 1;
        const int64_t c = s * n_clusters / n;
        /* cluster c holds the ids v with v * n_clusters / n == c */
        const int64_t c0 = (c * n + n_clusters - 1) / n_clusters;
        const int64_t c1 = ((c + 1) * n + n_clusters - 1) / n_clusters;
        const double u = u53(w[2], w[3]);
        int64_t d;
        if (u < p_in) {
            d = c0 + (int64_t)(u53(v[0], v[1]) * (double)(c1 - c0));
            if (d >= c1) d = c1 - 1;
        } else {
            const int64_t outside = n - (c1 - c0);
            int64_t t = (int64_t)(u53(v[0], v[1]) * (double)outside);
            if (t >= outside) t = outside - 1;
            d = t < c0 ? t : t + (c1 - c0);
        }
        src[e] = (uint32_t)s;
        dst[e] = (uint32_t)d;
    }
}
