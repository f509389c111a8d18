/*
 * spmm.h -- C-ABI of the GB300 sparse-matrix x dense-matrix library.
 *
 * The library computes Y = A X and Y = A^T X for a sparse n_rows x n_cols
 * matrix A (the adjacency matrix of a power-law graph, optionally weighted)
 * and a dense, row-major X with k = 1..64 columns: the operation of the
 * paper's Section 3 and Algorithm 1 (every nonzero a_ij of a sparse row adds
 * a_ij times row j of the input dense matrix to output row i; the dense
 * matrices are kept row-major, Section 3.3).
 *
 * Conventions for every entry point:
 *   - Status: every call returns an spmm_status (0 = success, < 0 = error).
 *     No exception or abort crosses this boundary.  On error the message is
 *     available from spmm_last_error() (per calling thread) and any handle
 *     passed in is left unchanged.
 *   - Streams: work is enqueued on the given CUDA stream (cudaStream_t passed
 *     as void*, NULL = the legacy default stream).  spmm_apply on a resident
 *     handle does not synchronise the host and allocates nothing (the two
 *     exceptions are stated at spmm_apply).
 *   - Concurrency: calls on one handle must not overlap (from several host
 *     threads, or on several streams at once), with one exception.  On a
 *     resident handle made by spmm_create_csr without SPMM_REORDER and
 *     SPMM_RELABEL, a call that runs only A X products (spmm_apply,
 *     spmm_apply_host or spmm_apply_host_parts with transpose = 0) may
 *     overlap one that runs only A^T products (spmm_apply with transpose != 0,
 *     or spmm_pagerank): each orientation has its own task counter, scratch
 *     and hot-row buffer.  The host-buffer calls share the handle's group
 *     buffers, so two of them never overlap.  A host-buffer call that grows
 *     those buffers (the first, or one with wider groups) and a spmm_pagerank
 *     call that captures its graph (the first, or one with a new x, damping
 *     or iters) allocate, so they should not overlap anything on the handle.
 *     The device status word is per handle: a staging timeout in either call
 *     is reported by the first read of it (spmm_pagerank's own, or
 *     spmm_sync_status).  Separate handles never share state.
 *   - Memory: X and Y are caller-owned DEVICE pointers; Y is overwritten, not
 *     accumulated into; X and Y must not overlap.  Handles own device copies of
 *     A made at create time.
 *   - Index types: row pointers are int64 (nnz may exceed 2^31), column
 *     indices are int32 (n_cols < 2^31).
 */
#ifndef SPMM_H
#define SPMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmm_mat* spmm_mat_t;   /* opaque, owned by the library */

typedef enum {
    SPMM_F32 = 0,
    SPMM_BF16 = 1,
    SPMM_F16 = 2,
    SPMM_F64 = 3
} spmm_dtype;

typedef enum {
    SPMM_OK = 0,
    SPMM_ERR_ARG = -1,          /* a bad argument (null pointer, size, dtype, alignment) */
    SPMM_ERR_CUDA = -2,         /* a CUDA runtime call failed                            */
    SPMM_ERR_OOM = -3,          /* device or host allocation failed                      */
    SPMM_ERR_FORMAT = -4,       /* the sparse matrix is malformed                        */
    SPMM_ERR_TIMEOUT = -5,      /* a bounded device-side wait ran out                    */
    SPMM_ERR_UNSUPPORTED = -6,  /* a valid but unimplemented combination                 */
    SPMM_ERR_IO = -7            /* a file could not be opened, read or written           */
} spmm_status;

/* create flags */
#define SPMM_WANT_TRANSPOSE 0x1u   /* also build the transposed (CSC) copy for A^T X */
#define SPMM_HOST_STREAMING 0x2u   /* keep A in host memory and stream it per call (A X only) */
#define SPMM_REORDER 0x4u          /* relabel columns by decreasing degree (see spmm_create_csr) */
#define SPMM_FILE_DIRECT 0x8u      /* spmm_create_file: read with O_DIRECT (bypass the page cache) */
#define SPMM_RELABEL 0x10u         /* renumber the vertices of a square matrix by decreasing degree */

/* Tuning knobs of the warp-task plan (the GPU form of the paper's tile-row
 * batches, Section 3.4); a NULL pointer or a zero field selects the default.
 *   task_nnz   nonzeros per task of short rows; segment length of split
 *              rows                                            default 512, 32..512
 *   task_rows  rows per task of short rows                     default 64, 1..64
 *   long_row   rows with more nonzeros are split into segments
 *              combined in a fixed order (deterministic)       default 512, task_nnz..512
 *   short_max  rows with at most this many nonzeros are "short"
 *              (one lane group per row); longer rows get a
 *              whole warp                                      default 63, < task_nnz
 *   x_l2_policy  L2 cache policy of the X gathers: 0 = default
 *              (evict-last), 1 = evict-normal, 2 = evict-last; the
 *              streamed matrix is always read evict-first
 *   stream_slot_kib  streaming mode: staging slot size for column indices
 *              in KiB (two slots are used in turn)                 default 262144 (256 MiB)
 *   debug_fail_block streaming mode, for tests: 1 + the block before
 *              which the streamer reports an injected copy failure and
 *              drains (0 = never)
 *   compensated  1 = long rows and hub-row segments are summed with
 *              Neumaier's compensated float32 summation (each product's
 *              rounding error recovered with an FMA) and split rows'
 *              segment partials are combined the same way; 0 = plain
 *              float32 sums (default)
 *   short_runs  how lane groups share a run of short rows when an X row
 *              takes several lanes of at most 4 elements (k = 4, 16, 32,
 *              64 FP32; k = 8 BF16/FP16): 1 = each group sums whole rows
 *              in turn, 2 = the run's nonzeros are cut into equal pieces,
 *              one per group, and rows crossing pieces are joined in a
 *              fixed order; 0 or any other value = automatic: pieces when
 *              the plan's row-walk efficiency for this many lane groups
 *              (spmm_info.walk_eff) is below 0.5 and the row is on 4 or
 *              more lanes or its lanes hold at most 8 bytes, else whole
 *              rows.  Per orientation, like the plan.  Results differ
 *              between 1 and 2 only in the order of float32 additions.
 *   hot_cols   create only: the H most-referenced columns of each
 *              orientation (with >= 2 stored entries, most first) are
 *              "hot".  A second copy of the column indices names them by
 *              rank, and calls whose X rows take 4 bytes (k = 1 float32,
 *              k = 2 bf16/f16 with 4-byte aligned rows) copy their X rows
 *              into shared memory once per block and gather them from
 *              there (Section 3.4's cache blocking of the dense rows a tile
 *              reads).  Costs 4 bytes per stored entry plus 8 bytes per hot
 *              column of device memory per orientation.  0: default =
 *              automatic (H = 8192, for orientations with at least 2^20
 *              entries whose kernel has room for 4096 or more beside its
 *              staging buffers: pattern matrices); -1: none; > 0: at most
 *              that many, capped by the room in shared memory.  Results are
 *              the same sums in the same order as without.
 */
typedef struct {
    int32_t task_nnz;
    int32_t task_rows;
    int32_t long_row;
    int32_t short_max;
    int32_t x_l2_policy;
    int32_t stream_slot_kib;
    int32_t debug_fail_block;
    int32_t compensated;
    int32_t short_runs;
    int32_t hot_cols;
} spmm_opts;

/* Plan statistics reported by spmm_get_info. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    int64_t n_tasks;             /* warp tasks of the forward plan                  */
    int64_t n_split_rows;        /* rows split into segments                        */
    int64_t n_segments;          /* segment tasks (one partial result each)         */
    int64_t n_tasks_t;           /* the same three for the transposed plan (or 0)   */
    int64_t n_split_rows_t;
    int64_t n_segments_t;
    int64_t device_bytes;        /* device memory held by the handle                */
    int32_t value_dtype;         /* spmm_dtype of the stored values, -1 = pattern   */
    int32_t has_transpose;
    int32_t n_graphs;            /* graphs in a batched handle (1 otherwise)        */
    int32_t relabelled;          /* 1: made with SPMM_RELABEL                       */
    /* Row-walk efficiency of the forward plan's short-row runs for 2, 4, 8
     * and 16 lane groups per warp (X rows on 16, 8, 4 and 2 lanes): group g
     * takes rows g, g+G, ... of a run, one round is one row per group and
     * lasts as long as its longest row (in batches of 4 nonzeros, at least
     * one), and the efficiency is the batches summed over the batches the
     * rounds take (G x the longest); 1 if the plan has no short-row runs.
     * Low values mean idle groups, which equal pieces per group avoid
     * (spmm_opts.short_runs).  walk_eff_t: the same for the transposed plan
     * (or 0). */
    double walk_eff[4];
    double walk_eff_t[4];
    int64_t n_hot;               /* hot columns of the forward orientation (spmm_opts.hot_cols) */
    int64_t n_hot_t;             /* ... of the transposed orientation (or 0)        */
} spmm_info;

/*
 * spmm_create_csr -- build a handle from a CSR matrix in HOST memory
 * (Section 3.2 stores the matrix once in a compact format before any
 * multiplication; here the one-time step is validation, a copy to HBM, the
 * warp-task plan and, with SPMM_WANT_TRANSPOSE, a CSC copy for A^T X).
 *   out        receives the handle
 *   n_rows, n_cols  matrix shape, 0 <= n_rows, 1 <= n_cols < 2^31
 *   nnz        stored entries = row_ptr[n_rows]
 *   row_ptr    n_rows+1 int64, row_ptr[0] = 0, non-decreasing
 *   col_idx    nnz int32, 0 <= col < n_cols (any order within a row)
 *   values     nnz values of type vtype, or NULL for a pattern matrix (all 1)
 *   vtype      SPMM_F32, SPMM_BF16 or SPMM_F16 (ignored when values is NULL)
 *   flags      SPMM_WANT_TRANSPOSE, SPMM_HOST_STREAMING, SPMM_REORDER, SPMM_RELABEL
 *              (or'd), or 0
 *   opts       tuning knobs or NULL
 *   stream     stream for the copies; the call returns after they finish
 * Errors: SPMM_ERR_ARG (null/shape), SPMM_ERR_FORMAT (row_ptr not monotone,
 * wrong row_ptr[0] or row_ptr[n_rows], column out of range), SPMM_ERR_OOM,
 * SPMM_ERR_UNSUPPORTED (streaming with SPMM_WANT_TRANSPOSE, SPMM_REORDER or
 * SPMM_RELABEL), SPMM_ERR_CUDA; SPMM_ERR_ARG also for SPMM_RELABEL with a
 * non-square matrix or with SPMM_REORDER.  The input arrays are copied; the
 * caller keeps ownership.
 *
 * SPMM_REORDER (Section 5.1: the vertex order decides how well gathered rows
 * stay in cache): each orientation's columns are relabelled by decreasing
 * number of stored entries (ties in index order) inside the handle, so the
 * most-gathered rows of X share cache lines.  Callers still pass X and get Y
 * in the original order: every apply first copies X's rows into the new order
 * (one gather pass over X into a buffer of n_in * k elements that the handle
 * keeps and grows; growing waits for the device and cannot happen inside a
 * stream capture).  Rows and the entry order within a row are unchanged, so
 * results are bit-identical to a handle without the flag given the same X as
 * a contiguous (ldx = k), 16-byte-aligned array -- the layout of the
 * relabelled copy.  A strided or misaligned X can give another summation
 * order (the kernel's vector width follows X's alignment).  spmm_apply calls
 * on one SPMM_REORDER handle share its relabelled-X buffer and must not
 * overlap (on several streams at once).
 *
 * SPMM_RELABEL (Section 5.1 again, for square matrices): the handle stores
 * B = P A P^T, where P renumbers the vertices by decreasing total degree
 * (stored entries in the vertex's row plus those in its column; ties keep the
 * vertex order, spmm_relabel_order), and each row of B keeps its entries in
 * increasing new column order.  The most-gathered rows of X then share L2
 * lines and each warp task gathers from a narrower band of X (R-MAT scale 24:
 * 8-33% faster from k = 2 on, with the vectors in the new order).  Graphs
 * whose locality comes from clusters of similar degree rather than from hubs
 * lose it (a clustered block model ran 0.5-0.8x as fast at k = 8), so the
 * flag suits skewed degree distributions.
 *   Vectors in the new order ("the handle's order") go to
 * spmm_apply_relabelled at no extra cost.  spmm_apply keeps the input order
 * by gathering X's rows into the handle's order and Y's rows back (two
 * buffers the handle keeps and grows, n * k elements each; spmm_apply calls
 * on one such handle share them and must not overlap, as with SPMM_REORDER's
 * buffer).  spmm_pagerank, spmm_eigs, spmm_eigs_filtered, spmm_svds and
 * spmm_nmf take and return vectors in the input order and run in the
 * handle's order in between.  The new summation order within a row gives
 * other float32 roundings than a handle without the flag.  Not with
 * spmm_create_batched, spmm_apply_batched or the host-buffer calls
 * (spmm_apply_host, spmm_apply_host_parts: SPMM_ERR_UNSUPPORTED).
 *
 * Streaming mode (SPMM_HOST_STREAMING; Section 3.1 keeps the sparse matrix
 * outside memory and streams it while the dense matrices stay resident, and
 * Section 3.6 argues memory is better spent on the dense side): the matrix is
 * NOT copied.  The handle borrows row_ptr, col_idx and values, pins them with
 * cudaHostRegister unless they are already pinned, and every spmm_apply
 * streams them to HBM in blocks of whole warp tasks through two staging slots
 * (the copy of one block overlaps the multiplication of the previous one).
 * The caller must keep the arrays alive and unchanged until spmm_destroy.
 * Only Y = A X is available; X and Y stay in HBM.  Calls on one streaming
 * handle share its slots and must not overlap.
 */
int spmm_create_csr(spmm_mat_t* out, int64_t n_rows, int64_t n_cols, int64_t nnz,
                    const int64_t* row_ptr, const int32_t* col_idx, const void* values,
                    spmm_dtype vtype, uint32_t flags, const spmm_opts* opts, void* stream);

/*
 * spmm_create_tiles -- build a handle from the paper's tiled storage
 * (Section 3.2, SCSR + COO): the matrix is cut into tile x tile blocks
 * (tile <= 32768, so row and column numbers fit 15 bits).  In one tile's
 * data, every non-empty row with two or more entries is a header word
 * (0x8000 | row within the tile) followed by its column words (top bit clear,
 * column within the tile); then come the single-entry rows as (row, column)
 * word pairs (the coordinate section, which needs no end-of-row test).  The
 * storage of a tile with nnr non-empty rows and nnz entries of c value bytes
 * is 2*nnr + (2 + c)*nnz bytes.  Values follow the storage order.
 *   tile_row, tile_col  position of the tile in tile units
 *   n_scsr_words        16-bit words of the header/column section
 *   n_coo               single-entry rows stored as pairs after it
 *   data                n_scsr_words + 2*n_coo words (host)
 *   values              values in storage order (host), or NULL in every tile
 * The tiles are decoded on the host into CSR (a row's entries in tile order,
 * then storage order; repeated entries are kept and add up) and passed to
 * spmm_create_csr with the same vtype, flags, opts and stream.
 * Errors: SPMM_ERR_ARG (tile > 32768, NULL), SPMM_ERR_FORMAT (a column word
 * before any header, a header without columns, a top bit set in a coordinate
 * word, a row or column outside the tile or the matrix, values in some tiles
 * only), and those of spmm_create_csr.
 */
typedef struct {
    int64_t tile_row;
    int64_t tile_col;
    int64_t n_scsr_words;
    int64_t n_coo;
    const uint16_t* data;
    const void* values;
} spmm_tile_desc;

int spmm_create_tiles(spmm_mat_t* out, int64_t n_rows, int64_t n_cols, int32_t tile, int64_t n_tiles,
                      const spmm_tile_desc* tiles, spmm_dtype vtype, uint32_t flags, const spmm_opts* opts,
                      void* stream);

/*
 * spmm_create_batched -- one handle for a batch of independent graphs, stored
 * as one block-diagonal matrix: graph g owns the row block and the column
 * block that follow the blocks of graphs 0..g-1.  One spmm_apply on the
 * handle then runs every graph's warp tasks in a single persistent launch
 * (the GPU form of keeping many small multiplications busy at once); X and Y
 * are the graphs' dense matrices stacked in graph order (row offsets = the
 * running sums of n_cols for X and n_rows for Y, or the reverse for A^T X).
 * The paper has no counterpart: it multiplies one graph at a time, with one
 * task queue over its tile rows (Section 3.4); here one queue covers the
 * tasks of many graphs.
 *   n_graphs     number of graphs (>= 1)
 *   n_rows[g], n_cols[g]   shape of graph g
 *   row_ptrs[g], col_idxs[g]   host CSR of graph g (local column indices)
 *   values       NULL (pattern) or an array of n_graphs host value arrays of vtype
 *   flags, opts, stream    as for spmm_create_csr
 * Totals must stay below 2^31 rows and columns.  Errors as spmm_create_csr.
 */
int spmm_create_batched(spmm_mat_t* out, int32_t n_graphs, const int64_t* n_rows, const int64_t* n_cols,
                        const int64_t* const* row_ptrs, const int32_t* const* col_idxs,
                        const void* const* values, spmm_dtype vtype, uint32_t flags, const spmm_opts* opts,
                        void* stream);

/*
 * spmm_apply -- Y = A X (transpose = 0) or Y = A^T X (transpose = 1)
 * (Algorithm 1; A^T X is the W^T A / A H^T product of Section 4.3).
 *   X      device, row-major, rows = n_cols (A X) or n_rows (A^T X), leading
 *          dimension ldx >= k, element type xtype (F32, BF16 or F16)
 *   k      1..64 dense columns
 *   Y      device, row-major float32 (ytype must be SPMM_F32), rows = n_rows
 *          (A X) or n_cols (A^T X), leading dimension ldy >= k; only the first
 *          k columns of each row are written
 * Accumulation is float32 in a fixed order: repeated calls give bit-identical
 * results.  Asynchronous on `stream`; allocates nothing, except that a handle
 * made with SPMM_REORDER grows its relabelled-X buffer (SPMM_RELABEL: its X
 * and Y buffers) the first time a larger n * k is used (which waits for the
 * device), and a handle made by
 * spmm_create_file blocks the calling thread until every block of the matrix
 * has been read from its file.
 * Errors: SPMM_ERR_ARG (null, k out of range, ld < k, dtype, transpose without
 * SPMM_WANT_TRANSPOSE), SPMM_ERR_UNSUPPORTED (16-bit values with another X
 * type), SPMM_ERR_CUDA (launch failure); file handles also SPMM_ERR_IO and
 * SPMM_ERR_FORMAT (see spmm_create_file).
 */
int spmm_apply(spmm_mat_t A, const void* X, int64_t ldx, int32_t k, spmm_dtype xtype, void* Y,
               int64_t ldy, spmm_dtype ytype, int32_t transpose, void* stream);

/*
 * spmm_apply_relabelled -- spmm_apply with X and Y in the handle's vertex
 * order (SPMM_RELABEL): Y' = B X' with B = P A P^T, X' = P X, Y' = P Y, so a
 * computation that keeps its vectors in that order (convert them once with
 * spmm_relabel_rows) pays nothing for the relabelling.  Arguments, errors and
 * asynchrony as spmm_apply; allocates nothing.  On a handle made without
 * SPMM_RELABEL it is spmm_apply.  Section 5.1 shows that the vertex order
 * decides how well the dense rows' reads hit the cache; this is the product
 * of Section 3 on the reordered graph.
 */
int spmm_apply_relabelled(spmm_mat_t A, const void* X, int64_t ldx, int32_t k, spmm_dtype xtype, void* Y,
                          int64_t ldy, spmm_dtype ytype, int32_t transpose, void* stream);

/*
 * spmm_relabel_rows -- convert the n x k rows of a dense matrix between the
 * input vertex order and the handle's order (n = the handle's rows; square
 * handles only):
 *   to_handle_order != 0:  dst[v'] = src[old_of_new[v']]   (input -> handle)
 *   to_handle_order == 0:  dst[v]  = src[new_of_old[v]]    (handle -> input)
 * src, dst  device, row-major, leading dimensions ld_src, ld_dst >= k, element
 *           type dtype (F32, BF16, F16 or F64); they must not overlap
 * Without SPMM_RELABEL it copies.  Asynchronous on `stream`; allocates
 * nothing.  The permutation of a dense matrix's rows that goes with the
 * vertex reordering of Section 5.1.  Errors: SPMM_ERR_ARG (NULL, non-square
 * handle, k < 1, ld < k, dtype, src == dst), SPMM_ERR_CUDA.
 */
int spmm_relabel_rows(spmm_mat_t A, const void* src, int64_t ld_src, int32_t k, spmm_dtype dtype, void* dst,
                      int64_t ld_dst, int32_t to_handle_order, void* stream);

/*
 * spmm_get_relabel -- the handle's vertex order: old_of_new[v'] (host int32,
 * n entries) is the input vertex that is vertex v' of the handle; the
 * identity without SPMM_RELABEL (the vertex order of Section 5.1).
 * Synchronous.  Errors: SPMM_ERR_ARG (NULL), SPMM_ERR_CUDA.
 */
int spmm_get_relabel(spmm_mat_t A, int32_t* old_of_new);

/*
 * spmm_relabel_order -- host-only: the order SPMM_RELABEL gives an n x n CSR
 * matrix.  Vertex v has degree (row_ptr[v+1] - row_ptr[v]) + (entries with
 * column v); old_of_new lists the vertices by decreasing degree, equal degrees
 * in increasing vertex order.  No GPU is used.  Section 5.1 compares vertex
 * orders; this is the degree order, which gathers the hubs of a power-law
 * graph at the front.  Errors: SPMM_ERR_ARG (n out of range, NULL),
 * SPMM_ERR_FORMAT (row_ptr[0] != 0, decreasing row_ptr, column out of range),
 * SPMM_ERR_OOM.
 */
int spmm_relabel_order(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int32_t* old_of_new);

/*
 * spmm_apply_batched -- Y_i = A_i X_i (or A_i^T X_i) for n handles, each with
 * its own k_i, in one persistent launch per kernel instantiation the entries
 * need (Section 3.4's single task queue over many multiplications): entries
 * whose X rows share a vector width and chunking (for float32 X: k = 8, 12,
 * ..., 64; k = 2, 4, 6, ...; k = 1 and odd k up to 31) run in one launch, their warp tasks
 * numbered one after the other; the split rows of all entries are combined
 * by one more launch.  Up to 128 entries share a launch; more make more
 * launches.  The entries' arguments travel in the kernels' parameter space,
 * so the call allocates nothing.
 *   n        number of entries (>= 1)
 *   A[i]     resident handles (not streaming, not SPMM_REORDER), all
 *            different; with transpose, made with SPMM_WANT_TRANSPOSE
 *   X[i]     device, row-major with ld = k[i] (contiguous), rows = n_cols
 *            (A X) or n_rows (A^T X) of A[i], element type xtype
 *   Y[i]     device float32, row-major with ld = k[i], rows = n_rows (A X)
 *            or n_cols (A^T X) of A[i]; overwritten
 *   k[i]     1..64
 *   xtype    F32, BF16 or F16 for every entry
 * Each Y_i equals spmm_apply on its own handle within the tolerances of
 * spmm_apply (the same sums; short rows are always walked whole per lane
 * group and the shared-memory hot rows are not used, so rows on several
 * lanes may be added in another order).  Asynchronous on `stream`; calls
 * that share a handle must not overlap.
 * Errors: SPMM_ERR_ARG (NULL, k, repeated handle, transpose without
 * SPMM_WANT_TRANSPOSE), SPMM_ERR_UNSUPPORTED (streaming or relabelled handle,
 * 16-bit values with another X type), SPMM_ERR_CUDA.
 */
int spmm_apply_batched(int32_t n, const spmm_mat_t* A, const void* const* X, void* const* Y, const int32_t* k,
                       spmm_dtype xtype, int32_t transpose, void* stream);

/*
 * spmm_sync_status -- synchronise `stream` and report whether any call on A
 * since the last check hit a device-side timeout.  The kernels stage the
 * matrix with asynchronous copies and wait for them with a bound (2 s); a
 * wait that runs out marks the handle, leaves that call's output incomplete
 * and returns SPMM_ERR_TIMEOUT here (the mark is then cleared).  The paper
 * has no counterpart: this is the failure-detection side of the asynchronous
 * staging.
 */
int spmm_sync_status(spmm_mat_t A, void* stream);

/*
 * spmm_write_csr_file -- host-only: write a CSR matrix to `path` in the
 * library's file layout (the sparse matrix on storage, Section 3.1): a
 * 4096-byte header ("SPMMCSR1", int64 n_rows, n_cols, nnz, int32 vtype (-1 for
 * a pattern matrix), int32 0, int64 offsets of the three sections), then
 * int64 row_ptr[n_rows+1], int32 col_idx[nnz] and the values, each section
 * starting on a 4096-byte boundary.  Written to a temporary name and renamed.
 * Validates like spmm_create_csr.  Errors: SPMM_ERR_ARG, SPMM_ERR_FORMAT,
 * SPMM_ERR_IO.
 */
int spmm_write_csr_file(const char* path, int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                        const int32_t* col_idx, const void* values, spmm_dtype vtype);

/*
 * spmm_create_file -- a handle whose matrix stays in a file written by
 * spmm_write_csr_file: the semi-external mode of Section 3.1 (vertex-sized
 * data in memory, edge-sized data on storage, streamed for every product).
 * The row pointers are read once into pinned host memory and the warp-task
 * plan goes to HBM; every spmm_apply reads the column indices (and values) of
 * each block of whole tasks from the file with parallel preads into pinned
 * staging buffers and streams them through two HBM slots as in
 * SPMM_HOST_STREAMING, so reading block b+1 overlaps copying and multiplying
 * block b.  Every column index read is range-checked on the host before it
 * reaches the GPU.
 *   path    the file (kept open until spmm_destroy; it must not change)
 *   flags   0 or SPMM_FILE_DIRECT (O_DIRECT reads that bypass the page cache;
 *           SPMM_ERR_UNSUPPORTED where the file system refuses O_DIRECT)
 *   opts    tuning knobs or NULL (stream_slot_kib sets the block size)
 * A X only (no transpose).  spmm_apply on the handle blocks the calling thread
 * until the last block has been read; the multiplication finishes
 * asynchronously on the stream.  Errors at create: SPMM_ERR_IO (open/read),
 * SPMM_ERR_FORMAT (not such a file, bad row pointers), SPMM_ERR_OOM,
 * SPMM_ERR_CUDA; at apply: SPMM_ERR_IO (a read failed or the file was
 * truncated), SPMM_ERR_FORMAT (a column index out of range: the file changed).
 */
int spmm_create_file(spmm_mat_t* out, const char* path, uint32_t flags, const spmm_opts* opts, void* stream);

/*
 * spmm_vpart_cols -- host-only: the width of the vertical partitions
 * (column groups) that spmm_apply_host uses for a dense matrix of p columns
 * under a device-memory budget.  Section 3.3 splits dense matrices that do
 * not fit in memory into vertical partitions; Section 3.6 gives the rule:
 * spend the memory on as many input columns as fit, since each partition
 * costs one more pass over the sparse matrix.  Each column of a group costs
 * 2 * (n_in * sizeof(X element) + n_out * 4) bytes (X and Y double-buffered).
 *   n_in, n_out   rows of X and of Y
 *   p             columns of X and Y (>= 1)
 *   xtype         F32, BF16 or F16 (X element size)
 *   budget_bytes  device bytes available for the group buffers
 *   cols          out: min(p, 64, columns that fit)
 * Errors: SPMM_ERR_ARG; SPMM_ERR_OOM if not even one column fits.
 */
int spmm_vpart_cols(int64_t n_in, int64_t n_out, int32_t p, spmm_dtype xtype, int64_t budget_bytes,
                    int32_t* cols);

/*
 * spmm_apply_host -- Y = A X (or A^T X) with X and Y in HOST memory, in
 * vertical partitions (Section 3.3; the paper's external medium is SSD, here
 * it is host memory).  The p columns are processed in groups of g columns,
 * one pass over A per group: a 2-D copy of the group's columns to the device,
 * the SpMM in four runs of whole row tasks, and after each run a 2-D copy of
 * its rows of the result back into Y's columns.  Copy-in, multiply and
 * copy-out run on three streams with two device buffers for X and for Y, so
 * consecutive groups overlap, and a group's first rows leave while its last
 * rows multiply.
 *   A            handle (resident or streaming)
 *   X            host, row-major, n_in x p with leading dimension ldx >= p
 *                elements, element type xtype (F32, BF16 or F16); pinned
 *                memory (cudaHostAlloc / cudaHostRegister) gives full link
 *                speed, pageable memory works at a lower rate
 *   Y            host, float32 row-major n_out x p, leading dimension ldy >= p
 *   transpose    nonzero: Y = A^T X (needs SPMM_WANT_TRANSPOSE)
 *   group_cols   g in 1..64, or 0 to pick it with spmm_vpart_cols
 *   budget_bytes device-memory budget for the group buffers when group_cols
 *                is 0; 0 = 80% of the currently free device memory
 *   groups_out   out (may be NULL): number of groups = passes over A
 *   stream       the multiply runs on it, after the work already queued there
 * The device buffers, two copy streams and their events are kept by the
 * handle for later calls (freed by spmm_destroy); calls on one handle must not
 * overlap, except as stated under Concurrency above.  Returns when Y is
 * complete on the host.  The result equals
 * spmm_apply on the same columns.
 * Errors: SPMM_ERR_ARG, SPMM_ERR_UNSUPPORTED (value/X type mix),
 * SPMM_ERR_OOM (the budget holds no column), SPMM_ERR_CUDA.
 */
int spmm_apply_host(spmm_mat_t A, const void* X, int64_t ldx, int32_t p, spmm_dtype xtype, float* Y, int64_t ldy,
                    int32_t transpose, int32_t group_cols, int64_t budget_bytes, int32_t* groups_out,
                    void* stream);

/*
 * spmm_apply_host_parts -- as spmm_apply_host for a dense matrix stored as
 * vertical partitions, each in row-major order (Section 3.3's layout): part i
 * holds part_cols[i] columns (1..64) as one contiguous host array, so each
 * group moves with plain contiguous copies instead of strided ones.
 *   X_parts[i]   host, n_in x part_cols[i] elements of xtype, row-major, no padding
 *   Y_parts[i]   host, float32 n_out x part_cols[i], row-major, no padding
 *   n_parts      >= 1; one pass over A per part, in order
 * Other arguments, buffers, ordering and errors as spmm_apply_host.
 */
int spmm_apply_host_parts(spmm_mat_t A, const void* const* X_parts, float* const* Y_parts, const int32_t* part_cols,
                          int32_t n_parts, spmm_dtype xtype, int32_t transpose, void* stream);

/*
 * spmm_debug_wait_timeout -- diagnostic: run a one-warp kernel whose staging
 * wait can never complete (it announces a transfer it never issues), with a
 * bound of wait_ns nanoseconds, and report SPMM_ERR_TIMEOUT when the bound
 * ran out as intended (SPMM_OK would mean the timeout path is broken).
 * Synchronises `stream`; faults nothing.  The paper has no counterpart: it
 * checks the bound that every asynchronous copy's wait carries here.
 */
int spmm_debug_wait_timeout(uint64_t wait_ns, void* stream);

/*
 * spmm_plan_tasks -- host-only: build the warp-task plan spmm_create_csr
 * would build for this row-pointer array (no GPU work, no device memory):
 * the GPU form of Section 3.4's batches of tile rows, with Section 3.2's
 * special handling of rows by their number of entries.
 *   row_ptr   n_rows+1 int64 (host)
 *   opts      tuning knobs or NULL
 *   tasks     NULL, or room for *n_tasks + 1 descriptors of 4 int32 each:
 *             {r0, x, lo32(e0), hi32(e0)}; x >= 1: rows r0..r0+x-1 (short
 *             rows), x == 0: the long row r0, x < 0: a segment of split row r0
 *             writing partial slot -x-1; e0 = first nonzero; the last
 *             descriptor is a sentinel whose e0 is nnz
 *   n_tasks   in: capacity of `tasks` in descriptors (ignored if tasks is
 *             NULL); out: number of tasks (without the sentinel)
 *   n_split_rows, n_segments  out (may be NULL)
 * Errors: SPMM_ERR_ARG (null row_ptr or n_tasks, capacity too small),
 * SPMM_ERR_FORMAT (row_ptr not monotone or row_ptr[0] != 0).
 */
int spmm_plan_tasks(int64_t n_rows, const int64_t* row_ptr, const spmm_opts* opts, int32_t* tasks,
                    int64_t* n_tasks, int64_t* n_split_rows, int64_t* n_segments);

/*
 * spmm_plan_walk_eff -- host-only: the row-walk efficiency of the plan that
 * spmm_plan_tasks builds (spmm_info.walk_eff: for 2, 4, 8, 16 lane groups),
 * the statistic the automatic short_runs choice reads.  Section 3.4 balances
 * work over threads with small batches of rows; this measures how evenly a
 * run of short rows spreads over the lane groups of a warp when each group
 * takes whole rows.
 *   row_ptr   n_rows+1 int64 (host)
 *   opts      tuning knobs or NULL
 *   walk_eff  out: 4 doubles
 * Errors: SPMM_ERR_ARG (null pointer, bad n_rows), SPMM_ERR_FORMAT (row_ptr
 * not monotone or row_ptr[0] != 0), SPMM_ERR_OOM.
 */
int spmm_plan_walk_eff(int64_t n_rows, const int64_t* row_ptr, const spmm_opts* opts, double* walk_eff);

/*
 * spmm_plan_runs -- host-only: the runs of whole tasks into which the
 * host-buffer calls (spmm_apply_host, spmm_apply_host_parts) cut a product
 * of the plan spmm_plan_tasks builds, so that a run's rows of Y can be copied
 * out while the next run multiplies (they use 4 runs).  Section 3.4 overlaps
 * the I/O of one batch of tile rows with the multiplication of another; here
 * the overlapped I/O is the output's copy to host memory.  Run j ends at the
 * first task that starts at or after (j + 1) / max_runs of the stored entries
 * and begins a new row, so the segments of a split row stay in one run.
 *   row_ptr   n_rows+1 int64 (host)
 *   opts      tuning knobs or NULL
 *   max_runs  >= 1
 *   runs      out: room for max_runs x 6 int64 {t0, t1, r0, r1, s0, s1}: tasks
 *             t0..t1-1, rows r0..r1-1, split rows s0..s1-1 (in the order of
 *             the plan's split rows); consecutive runs meet, the first starts
 *             at 0 and the last ends at the task, row and split-row counts
 *   n_runs    out: number of runs (fewer than max_runs for small plans, 0 for
 *             a plan without tasks)
 * Errors: SPMM_ERR_ARG (null pointer, max_runs < 1, bad n_rows),
 * SPMM_ERR_FORMAT (row_ptr not monotone or row_ptr[0] != 0), SPMM_ERR_OOM.
 */
int spmm_plan_runs(int64_t n_rows, const int64_t* row_ptr, const spmm_opts* opts, int32_t max_runs, int64_t* runs,
                   int32_t* n_runs);

/*
 * spmm_apply_csr_static -- Y = A X without allocating device memory.  The
 * paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc (for example code inside a framework that hands out all device
 * memory from its own pool, or a loop that must not allocate after start-up)
 * and so cannot create a handle.  The caller passes the matrix, its plan, X
 * and Y in device buffers it owns; the kernels' scratch (partial sums of
 * split hub rows, the bounded-wait status word) comes from one static device
 * array of 4 MiB inside the library, which every GPU that loads the library
 * keeps until the process exits.
 *   n_rows, n_cols, nnz   matrix shape and stored entries
 *   row_ptr   device, n_rows+1 int64; must stay readable 16 bytes past its end
 *   col_idx   device, nnz int32; must stay readable 32 bytes past its end
 *   values    device, nnz values of type vtype, or NULL (pattern); readable
 *             32 bytes past its end.  F32 values, or BF16/F16 values with X of
 *             the same type.  (The kernel's bulk copies are widened to 16-byte
 *             boundaries; the extra bytes are read but not used.)
 *   tasks     device copy of the n_tasks + 1 descriptors (sentinel included)
 *             that spmm_plan_tasks returned for this row_ptr
 *   n_tasks, n_segments   as returned by spmm_plan_tasks; at most 16384
 *             segments (split hub-row pieces) fit the static scratch
 *   X, ldx, k, xtype, Y, ldy   as for spmm_apply (Y float32, device)
 * The result matches spmm_apply on a handle created from the same matrix and
 * options within the tolerances of spmm_apply (bit for bit where every
 * partial sum is exact): both use the same task kernel and lane geometry,
 * but this entry point always walks short rows whole per lane group and
 * never compensates, so rows spread over several lanes may be summed in
 * another order.  The first call on a device looks up the static array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call shares the array and it
 * keeps the last call's contents: calls whose work overlaps on the GPU race,
 * so order them on one stream or synchronise between them.  Each call clears
 * the array's status word; a timed-out staging wait, or a task whose
 * partial-sum slot lies beyond the 16384 slots (a task list that does not
 * belong to row_ptr), sets it and leaves part of Y unwritten -- the kernels
 * never write outside the array.  spmm_static_status reports it.
 * Asynchronous on `stream`.
 * Errors: SPMM_ERR_ARG (sizes, NULL, more than 16384 segments),
 * SPMM_ERR_UNSUPPORTED (value/X type mix), SPMM_ERR_CUDA.
 */
int spmm_apply_csr_static(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                          const int32_t* col_idx, const void* values, spmm_dtype vtype, const int32_t* tasks,
                          int64_t n_tasks, int64_t n_segments, const void* X, int64_t ldx, int32_t k,
                          spmm_dtype xtype, float* Y, int64_t ldy, void* stream);

/*
 * spmm_static_status -- the status of the most recent spmm_apply_csr_static
 * call on the current device, without allocating.  The paper has no
 * counterpart.  Synchronises `stream` (the stream the call was made on), then
 * reads the static array's status word with a 4-byte copy into host memory.
 * Returns SPMM_OK, SPMM_ERR_TIMEOUT (a staging wait ran out: Y incomplete),
 * SPMM_ERR_FORMAT (the task list named partial-sum slots beyond the static
 * array: the split rows of Y were not written) or SPMM_ERR_CUDA.  The word is
 * cleared by the next spmm_apply_csr_static call, not by this query.
 */
int spmm_static_status(void* stream);

/*
 * spmm_pagerank -- PageRank by power iteration (Section 4.1):
 *   x'(u) = (1-d)/N + d * sum_{v in B(u)} x(v)/L(v) + d * (sum_{L(v)=0} x(v)) / N
 * B(u) = in-neighbours of u, L(v) = out-degree of v; row v of A lists the
 * out-links of v; the rank of dangling vertices (L = 0) is spread uniformly.
 * Each iteration is one A^T product (k = 1, float32) plus a fused update with
 * FP64 reductions; all iterations run as one CUDA graph.
 *   A          square pattern handle (created without values) with SPMM_WANT_TRANSPOSE
 *   damping    d in [0, 1]
 *   iters      number of iterations (>= 0, no early stop)
 *   x          device float[N]: the ranks after `iters` iterations
 *   x0         device float[N] start vector, or NULL for 1/N
 *   residuals  host double[iters] or NULL: sum_u |x'(u) - x(u)| of each iteration (FP64)
 * Synchronises `stream` first, then runs on an internal stream and returns
 * when the ranks are ready.  The first call allocates a workspace (about 12
 * bytes per vertex) and an internal stream, and captures iterations
 * 2..iters as a CUDA graph; the handle keeps them until spmm_destroy, and a
 * later call with the same x, damping and iters only launches the graph
 * (another x, damping or iters is captured anew).  Calls on one handle must
 * not overlap, except with A X products as stated under Concurrency above.
 * Errors: SPMM_ERR_ARG (NULL, non-square, values present, no
 * transpose, bad d or iters), SPMM_ERR_TIMEOUT, SPMM_ERR_OOM, SPMM_ERR_CUDA.
 */
int spmm_pagerank(spmm_mat_t A, double damping, int32_t iters, float* x, const float* x0, double* residuals,
                  void* stream);

/*
 * spmm_nmf -- non-negative matrix factorisation A ~ W H by the multiplicative
 * updates of Section 4.3, H first, then W, for `steps` steps:
 *   Ht <- Ht o (A^T W) / (Ht (W^T W) + eps),   W <- W o (A Ht) / (W (Ht^T Ht) + eps)
 * H is stored transposed (Ht).  Each step is two SpMMs (A Ht and A^T W) plus
 * two k x k Gram matrices and two row-local updates; all steps run as one CUDA
 * graph.  On a batched handle every graph is factorised independently (its own
 * Grams and objective) while the SpMMs cover the whole batch in one launch.
 *   A          handle created with SPMM_WANT_TRANSPOSE (single or batched)
 *   k          rank, 1..64
 *   steps      number of H-then-W steps (>= 0)
 *   W          device float32, row-major (total rows) x k, contiguous (ld = k);
 *              in: initial factor (non-negative), out: factor after `steps`
 *   Ht         device float32, (total columns) x k, contiguous; in/out likewise
 *   ftype      SPMM_F32: the SpMMs read the float32 factors; SPMM_BF16: they read
 *              a bfloat16 copy (float32 accumulation); updates stay float32
 *   eps        added to every denominator (1e-12 keeps 0/0 at 0)
 *   objective  host double[n_graphs * (steps+1)] or NULL: for graph g,
 *              objective[g*(steps+1) + t] = ||A_g - W_g H_g||_F^2 before step t
 *              (t = steps: after the last), from ||A||^2 - 2 sum(W o A Ht)
 *              + tr((W^T W)(Ht^T Ht)) in FP64
 * Synchronises `stream`, runs on an internal stream, allocates its workspace.
 * Errors: SPMM_ERR_ARG, SPMM_ERR_UNSUPPORTED (16-bit values with the other
 * factor type), SPMM_ERR_TIMEOUT, SPMM_ERR_OOM, SPMM_ERR_CUDA.
 */
int spmm_nmf(spmm_mat_t A, int32_t k, int32_t steps, float* W, float* Ht, spmm_dtype ftype, double eps,
             double* objective, void* stream);

/*
 * spmm_eigs -- the nev largest (algebraic) eigenpairs of a symmetric matrix
 * S by a thick-restart block Krylov method (the symmetric form of the block
 * Krylov-Schur solver of Section 4.2, whose only sparse operation is the block
 * product S V).  The basis and S V are FP64; each expansion multiplies the
 * newest block by S with X in FP32 or BF16 (FP32 accumulation); Gram-Schmidt
 * (twice), CholQR2 and Rayleigh-Ritz are FP64; a restart keeps nev + block
 * Ritz vectors.
 *   S            square handle of a symmetric matrix (values F32, BF16 or none)
 *   nev          eigenpairs wanted
 *   block        block size (1..32)
 *   max_basis    basis size, nev + 2*block <= max_basis <= min(64, n)
 *   max_restarts restarts before giving up (the best pairs are returned)
 *   tol          stop when every wanted pair has ||S u - theta u||_2 <= tol (unit u)
 *   xtype        SPMM_F32 or SPMM_BF16: type of the block fed to the SpMM
 *   V0           device double[n * block], row-major start block (full rank)
 *   evals        host double[nev], descending
 *   evecs        device double[n * nev] row-major (unit columns), or NULL
 *   resid        host double[nev] residual norms, or NULL
 *   restarts_out host int32 restarts used, or NULL
 * Synchronises `stream`; runs on an internal stream; allocates its workspace
 * (about 6 * n * max_basis doubles).  Errors: SPMM_ERR_ARG (sizes, NULL,
 * rank-deficient start block), SPMM_ERR_UNSUPPORTED, SPMM_ERR_TIMEOUT,
 * SPMM_ERR_OOM, SPMM_ERR_CUDA.
 */
int spmm_eigs(spmm_mat_t S, int32_t nev, int32_t block, int32_t max_basis, int32_t max_restarts, double tol,
              spmm_dtype xtype, const double* V0, double* evals, double* evecs, double* resid,
              int32_t* restarts_out, void* stream);

/*
 * spmm_eigs_filtered -- the nev largest eigenpairs of a symmetric S by
 * Chebyshev-filtered subspace iteration: a block of `block` vectors is
 * multiplied by the degree-`degree` Chebyshev polynomial that stays within
 * [-1, 1] on [lower, cut] (cut = the block's smallest Ritz value) and grows
 * fastest above it, through `degree` block SpMMs (X in FP32 or BF16, FP32
 * accumulation, the three-term recurrence in FP32 scaled to stay O(1)), then
 * orthonormalised (CholQR2) and Rayleigh-Ritz projected with S in FP64.  Not
 * the paper's Krylov-Schur solver (spmm_eigs): the same products (Section 4.2's
 * only sparse operation is the block SpMM), arranged so that the FP64 work is
 * once per `degree` SpMMs, which converges on the clustered top spectrum of a
 * large normalised graph where the restarted Krylov method does not within
 * its restarts.  The filter steps of one iteration run as one CUDA graph.
 *   S            square handle of a symmetric matrix (values F32, BF16 or none)
 *   nev          eigenpairs wanted
 *   block        vectors filtered together, nev + 1 <= block <= min(64, n)
 *                (a few more than nev: the filter separates the wanted
 *                eigenvalues from the block's smallest Ritz value)
 *   degree       polynomial degree per iteration, 1..1000
 *   lower        a lower bound of S's spectrum (-1 for a normalised
 *                adjacency matrix D^-1/2 A D^-1/2)
 *   max_iters    filter iterations before giving up (best pairs returned)
 *   xtype        SPMM_F32 or SPMM_BF16: type of the block fed to the filter's
 *                SpMMs; the Rayleigh-Ritz product reads FP32 (BF16 with BF16
 *                values)
 *   tol, V0 (n x block), evals, evecs, resid   as for spmm_eigs
 *   iters_out    host int32 iterations used, or NULL
 * Synchronises `stream`; runs on an internal stream; allocates its workspace
 * (about 6 * n * block doubles and 4 * n * block floats).  Errors:
 * SPMM_ERR_ARG (sizes, NULL, rank-deficient start block, Ritz values not
 * above `lower`, a filtered block that lost rank), SPMM_ERR_UNSUPPORTED,
 * SPMM_ERR_TIMEOUT, SPMM_ERR_OOM, SPMM_ERR_CUDA.
 */
int spmm_eigs_filtered(spmm_mat_t S, int32_t nev, int32_t block, int32_t degree, double lower, int32_t max_iters,
                       double tol, spmm_dtype xtype, const double* V0, double* evals, double* evecs, double* resid,
                       int32_t* iters_out, void* stream);

/*
 * spmm_replan -- rebuild the warp-task plan of one orientation of a resident
 * handle for new tuning knobs (the matrix itself is not copied again).  The
 * paper sizes its tile-row batches from the cache size and the number of
 * dense columns (Section 3.4); here the batch shape is tunable per call site.
 *   opts        new knobs (NULL = defaults); transpose selects the A^T plan
 * Synchronises `stream`.  Errors: SPMM_ERR_ARG, SPMM_ERR_UNSUPPORTED
 * (streaming handles), SPMM_ERR_OOM, SPMM_ERR_CUDA.
 */
int spmm_replan(spmm_mat_t A, const spmm_opts* opts, int32_t transpose, void* stream);

/*
 * spmm_autotune -- time Y = A X (or A^T X) under candidate plans and leave
 * the handle on the fastest.  Each candidate is planned with spmm_replan,
 * warmed twice and timed `reps` times with CUDA events, L2 flushed before
 * every timed call.  X is filled inside with a fixed pattern of type xtype.
 *   candidates    caller's candidate knobs, or NULL for the built-in grid:
 *                 task_nnz {128,256,512} x short_max {7,15,31,63} x
 *                 x_l2_policy {1,2} (long_row 512), 24 candidates
 *   n_candidates  number of caller candidates (ignored when NULL)
 *   best_index    out: index of the fastest candidate
 *   times_ms      host double[number of candidates] or NULL: mean ms each
 * Synchronises `stream`; allocates its workspace.  Errors as spmm_replan.
 * The paper fixes its tile size and batch sizes by measurement (Sections 3.4,
 * 5.4); this measures the plan's knobs per matrix and call shape instead.
 */
int spmm_autotune(spmm_mat_t A, int32_t k, spmm_dtype xtype, int32_t transpose, const spmm_opts* candidates,
                  int32_t n_candidates, int32_t reps, int32_t* best_index, double* times_ms, void* stream);

/*
 * spmm_svds -- the nsv largest singular values of A (any shape) and their
 * right singular vectors, by the spmm_eigs method applied to A^T A without
 * forming it: each block product is A V (X in FP32 or BF16) followed by
 * A^T (A V) (the intermediate kept in FP32).  The paper computes singular
 * values of the directed Page graph with its eigensolver (Section 5.5.2).
 *   A           handle created with SPMM_WANT_TRANSPOSE
 *   V0          device double[n_cols * block] start block
 *   svals       host double[nsv], descending (square roots of the Ritz values)
 *   right_vecs  device double[n_cols * nsv] or NULL
 *   resid       host double[nsv] or NULL: ||A^T A v - s^2 v||_2
 *   other arguments and errors as spmm_eigs (max_basis <= min(64, n_cols))
 */
int spmm_svds(spmm_mat_t A, int32_t nsv, int32_t block, int32_t max_basis, int32_t max_restarts, double tol,
              spmm_dtype xtype, const double* V0, double* svals, double* right_vecs, double* resid,
              int32_t* restarts_out, void* stream);

/* spmm_get_info -- plan statistics of a handle (host call, no GPU work).
 * Bookkeeping of this library; the paper has no counterpart. */
int spmm_get_info(spmm_mat_t A, spmm_info* info);

/* spmm_destroy -- free a handle and its device memory (synchronises the
 * device work that uses it).  NULL is accepted and ignored.  Bookkeeping of
 * this library; the paper has no counterpart. */
int spmm_destroy(spmm_mat_t A);

/* spmm_last_error -- message of the last failing call on this thread
 * ("" if none).  The pointer stays valid until the thread's next call.
 * Bookkeeping of this library; the paper has no counterpart. */
const char* spmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPMM_H */
