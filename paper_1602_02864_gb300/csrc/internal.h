// internal.h -- types shared by the host side and the kernels of libspmm.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "spmm.h"

namespace spmm {

// An NVTX range for the scope of one call or step (visible in Nsight
// Systems timelines; free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Warp tasks, in natural row order, cover every row exactly once:
//   desc = int4 {r0, x, lo32(e0), hi32(e0)}, e0 = first nonzero of the task,
//   and the task's nonzero count is e0 of the next descriptor (a sentinel
//   descriptor closes the list).
//   x >= 1 : a run of x short rows r0 .. r0+x-1 (one lane group per row)
//   x == 0 : one long row r0 (all lane groups share its nonzeros)
//   x < 0  : one segment of a split hub row r0; its partial result goes to
//            slot -x-1 and combine.cu adds the segments in order.
//   split  = int4 {row, nseg, slot0, 0} for the combine pass.
constexpr int kWarpsPerBlock = 8;
constexpr int kMaxTaskNnz = 512;    // staged nonzeros per task (shared memory)
constexpr int kMaxTaskRows = 64;    // rows per short-row task
constexpr int kSlotStride = 64;     // floats allocated per partial-result slot (k <= 64; a call
                                    // with k columns packs slot s at s * k)
constexpr int kMaxK = 64;
constexpr uint64_t kWaitNs = 2000000000ull;   // bound of every device-side staging wait (2 s)
// bits of the device status word
constexpr int32_t kStatusTimeout = 1;     // a staging wait ran out; the call's results are incomplete
constexpr int32_t kStatusSlotRange = 2;   // a task named a partial slot beyond the scratch; its result is missing
// per-warp staging buffer (one of two): column indices, values, row pointers,
// each padded for 16-byte aligned bulk copies of an unaligned window
constexpr int kColBufInts = kMaxTaskNnz + 8;          // 2080 bytes
constexpr int kValBufBytes = (kMaxTaskNnz + 8) * 4;   // 2080 bytes
constexpr int kRpBufLongs = kMaxTaskRows + 4;         // 544 bytes

struct HostPlan {
    std::vector<int4> tasks;    // n_tasks + 1 (sentinel)
    std::vector<int4> splits;
    int64_t n_slots = 0;
    int64_t n_segments = 0;
    int64_t n_short = 0, n_long = 0;
    // row-walk efficiency of the short-row runs for 2, 4, 8, 16 lane groups
    // (spmm_info.walk_eff)
    double walk_eff[4] = {1.0, 1.0, 1.0, 1.0};
};

// A run of whole warp tasks t0 .. t1-1 covering rows r0 .. r1-1 (the
// segments of a split row are never in two runs), whose split rows are
// splits s0 .. s1-1.  The host-buffer calls multiply run by run and copy a
// run's rows of Y out while the next run multiplies.
struct RowBlock {
    int64_t t0, t1, r0, r1, s0, s1;
};
constexpr int kRowBlocks = 4;

// Device-side copy of one orientation (CSR of A, or CSR of A^T == CSC of A).
struct DevCSR {
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    int64_t* row_ptr = nullptr;     // padded by 2 entries (aligned bulk copies)
    int32_t* col_idx = nullptr;     // padded by 8 entries
    void* val = nullptr;            // padded by 8 entries
    int4* tasks = nullptr;          // n_tasks + 1
    int64_t n_tasks = 0;
    int4* splits = nullptr;
    int64_t n_splits = 0;
    int64_t n_segments = 0;
    float* partials = nullptr;      // scratch: n_slots x kSlotStride floats (slot s of a k-column call at s * k)
    float* partials_comp = nullptr; // compensation terms of the partials (compensated plans only)
    int64_t n_slots = 0;
    int32_t* perm = nullptr;        // SPMM_REORDER: original index of relabelled column c (n_cols)
    unsigned long long* task_ctr = nullptr;   // task counter of dynamically scheduled launches
    int32_t short_runs = 0;         // short-row runs over lane groups (spmm_opts.short_runs)
    // hot columns (hot.cu): col_hot is col_idx with ~slot for an entry in one
    // of the n_hot most-referenced columns, hot_cols[slot] that column; calls
    // with X rows of at most 4 bytes copy the hot rows of X into xh (packed,
    // kHotRowBytes each) and run the kernel variant that keeps them in
    // shared memory
    int32_t* col_hot = nullptr;     // padded by 8 entries, like col_idx
    int32_t* hot_cols = nullptr;
    int64_t n_hot = 0;
    void* xh = nullptr;
    double walk_eff[4] = {1.0, 1.0, 1.0, 1.0};   // HostPlan::walk_eff of the current plan
    std::vector<RowBlock> row_blocks;             // kRowBlocks runs of the current plan
};

// Streaming mode: the matrix stays in (pinned) host memory and flows to HBM
// in blocks of whole tasks, two staging slots used in turn.
struct StreamBlock {
    int64_t t0, t1;     // task range
    int64_t c0, c1;     // column-index / value range copied (c0 aligned down to 8)
    int64_t r0, r1;     // row-pointer range copied (r0 aligned down to 2)
};

// A CSR file opened by spmm_create_file (layout in filecsr.cpp).
constexpr int64_t kFileAlign = 4096;
struct FileCSR {
    int fd = -1;
    bool direct = false;               // opened with O_DIRECT
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    int32_t vtype = -1;
    int64_t off_rp = 0, off_ci = 0, off_val = 0;
};

struct Streamer {
    const int64_t* h_row_ptr = nullptr;
    const int32_t* h_col_idx = nullptr;
    const void* h_val = nullptr;
    bool reg_rp = false, reg_ci = false, reg_val = false;   // registered by the library
    std::vector<StreamBlock> blocks;
    int32_t* slot_col[2] = {nullptr, nullptr};
    void* slot_val[2] = {nullptr, nullptr};
    int64_t* slot_rp[2] = {nullptr, nullptr};
    int64_t slot_nnz = 0, slot_rows = 0;   // capacities
    cudaStream_t copy = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    int32_t fail_block = 0;                // test hook: 1 + block before which a copy "fails"
    int64_t bytes_per_apply = 0;           // host bytes streamed per call
    // file source (spmm_create_file): blocks are read into pinned staging first
    FileCSR file;
    int64_t* h_rp_owned = nullptr;         // pinned row pointers read from the file
    char* stage_col[2] = {nullptr, nullptr};
    char* stage_val[2] = {nullptr, nullptr};
    cudaEvent_t staged[2] = {nullptr, nullptr};   // the copies out of staging buffer i are done
    int32_t readers = 8;                   // parallel preads per block
};

struct Params {
    int32_t task_nnz = 512;     // nonzeros per short-row task
    int32_t task_rows = 64;     // rows per short-row task
    int32_t long_row = 512;     // rows longer than this are split
    int32_t short_max = 63;     // rows with more nonzeros are "long"
    int32_t x_evict_last = 1;   // L2 policy of the X gathers (1 = evict-last)
    int64_t slot_bytes = 256ll << 20;   // streaming staging slot (column indices)
    int32_t fail_block = 0;
    int32_t compensated = 0;            // compensated sums for long rows and hub segments
    int32_t short_runs = 0;             // 0 automatic, 1 row walk, 2 pieces per lane group
    int64_t hot_cols = -1;              // hot columns per orientation: -1 automatic, 0 none (create only)
};

}  // namespace spmm

namespace spmm {
// PageRank state kept by a handle after its first spmm_pagerank call: the
// workspace, an internal stream and the CUDA graph of iterations 2..iters,
// reused while (x, damping, iters) stay the same
struct PrCache {
    float *inv_deg = nullptr, *z = nullptr, *y = nullptr;
    double *part = nullptr, *scal = nullptr, *dres = nullptr;
    int32_t nblk = 0, dres_cap = 0;
    cudaStream_t s = nullptr;
    cudaGraphExec_t exec = nullptr;
    float* x = nullptr;
    double damping = -1.0;
    int32_t iters = -1;
    // SPMM_RELABEL: the ranks and the start vector in the handle's order
    float *xr = nullptr, *x0r = nullptr;
};
void pagerank_release(spmm_mat* A);
// drop the captured PageRank graph (the plan or a buffer it uses changed)
void pagerank_invalidate(spmm_mat* A);

// device buffers, streams and events of spmm_apply_host (created on first use)
struct HostIO {
    void* x[2] = {nullptr, nullptr};
    float* y[2] = {nullptr, nullptr};
    size_t x_bytes = 0, y_bytes = 0;     // size of each buffer
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev[8] = {};
};
}  // namespace spmm

struct spmm_mat {
    spmm::DevCSR fwd;
    spmm::DevCSR tr;
    bool has_tr = false;
    int32_t vtype = -1;       // spmm_dtype of values, -1 = pattern
    spmm::Params params;
    int64_t device_bytes = 0;
    int32_t* status = nullptr;  // device word: nonzero after a timed-out wait
    // batch layout (one graph for spmm_create_csr): graph g owns rows
    // row_off[g] .. row_off[g+1]-1 and columns col_off[g] .. col_off[g+1]-1
    std::vector<int64_t> row_off, col_off;
    std::vector<double> a2;     // ||A_g||_F^2 per graph
    bool streaming = false;
    spmm::Streamer st;
    spmm::HostIO hio;
    void* xperm = nullptr;      // SPMM_REORDER / SPMM_RELABEL: X with its rows in relabelled order (grow-only)
    size_t xperm_bytes = 0;
    // SPMM_RELABEL: the vertex order (device) and the result of spmm_apply
    // before its rows go back to the input order (grow-only)
    bool relabel = false;
    int32_t* rl_old_of_new = nullptr;
    int32_t* rl_new_of_old = nullptr;
    void* yperm = nullptr;
    size_t yperm_bytes = 0;
    spmm::PrCache pr;           // spmm_pagerank's workspace and graph (after its first call)
};

namespace spmm {

// plan.cpp
HostPlan build_plan(const int64_t* row_ptr, int64_t n_rows, const Params& p);
// at most nb runs of the plan's tasks with about equal stored entries
std::vector<RowBlock> cut_row_blocks(const HostPlan& plan, int nb);

// vpart.cu
void hostio_release(spmm_mat* A);

// filecsr.cpp
int file_open(const char* path, bool direct, FileCSR* f);
const char* file_read_range(int fd, bool direct, int64_t off, int64_t len, char* buf, int threads,
                            int64_t n_cols_check, std::string* err);

// stream.cu (file source)
int stream_file_setup(spmm_mat* A, cudaStream_t s);

// reorder.cu
void relabel_by_degree(int64_t n_cols, const int32_t* col_idx, int64_t nnz, std::vector<int32_t>& old_of_new,
                       std::vector<int32_t>& relabelled);
int reorder_reserve(spmm_mat* A, int64_t n_in, int32_t k, int32_t xtype, cudaStream_t s);
int reorder_x(spmm_mat* A, const DevCSR& d, const void* X, int64_t ldx, int32_t k, int32_t xtype, cudaStream_t s,
              const void** Xp);

// relabel.cu: the vertices of an n x n CSR by decreasing total degree
// (entries in the row plus entries in the column; ties in vertex order)
void relabel_order(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, std::vector<int32_t>& old_of_new);
// B = P A P^T on the host (each row's entries in increasing new column order)
int relabel_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const void* values, size_t vsize,
                const std::vector<int32_t>& old_of_new, std::vector<int32_t>& new_of_old, std::vector<int64_t>& rp,
                std::vector<int32_t>& ci, std::vector<char>& val);
// dst row r = src row idx[r] (idx == nullptr: row r); k elements of es bytes
cudaError_t gather_rows(const void* src, int64_t ld_src, const int32_t* idx, int64_t n, int32_t k, int es, void* dst,
                        int64_t ld_dst, cudaStream_t s);
// n x k rows between the input order and the handle's order (identity
// without SPMM_RELABEL)
cudaError_t relabel_rows_dev(const spmm_mat* A, const void* src, int64_t ld_src, int32_t k, int es, void* dst,
                             int64_t ld_dst, bool to_handle_order, cudaStream_t s);
// spmm_apply on an SPMM_RELABEL handle: X's rows into the handle's order, the
// product, Y's rows back
int apply_relabel_io(spmm_mat* A, int transpose, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y,
                     int64_t ldy, cudaStream_t s);

// hot.cu: rank the columns by stored entries (counts, or counted from
// col_idx when counts is null), keep the max_hot most-referenced ones that
// have at least two entries (hot_cols: slot -> column, most referenced
// first) and write col_idx with hot entries as ~slot to `encoded`; returns H
int64_t hot_select(int64_t n_cols, const int32_t* col_idx, int64_t nnz, const int64_t* counts, int64_t max_hot,
                   std::vector<int32_t>& hot_cols, std::vector<int32_t>& encoded);
// enqueue Xh[s, :] = X[hot_cols[s], :] (k elements of esize bytes) for the
// n_hot hot columns of d
cudaError_t hot_gather(const DevCSR& d, const void* X, int64_t ldx, int32_t k, int esize, cudaStream_t s);
// hot rows that fit the shared memory of the hot kernel variant beside its
// warps' staging buffers (value mode vmode, at most 4-byte rows); 0 if none
int64_t hot_capacity(int vmode);
// The hot variant runs one block of kHotWarps warps per SM (the warps of
// three blocks of the plain kernel) for calls whose X rows take exactly
// kHotRowBytes bytes.  Automatic hot columns: kHotAuto of them (32 KB of
// shared memory) for orientations of at least kHotMinNnz entries, when at
// least kHotAutoMin fit.  On R-MAT scale 24 (k = 1 float32, one block of 24
// warps) 4096 / 8192 / 16384 / 24576 hot rows took 0.859 / 0.828 / 0.845 /
// 1.320 ms against 0.923 ms without: every 32 KB taken from L1 costs L1 hits
// of the other gathers, and at 24576 L1 is almost gone.  With 16 warps the
// same sizes were slower than without; rows of 2 bytes (bf16 k = 1) were
// slower with any hot rows (1.04 against 0.87 ms), so they do not use them.
constexpr int kHotWarps = 24;
constexpr int kHotRowBytes = 4;
constexpr int64_t kHotAuto = 8192;
constexpr int64_t kHotAutoMin = 4096;
constexpr int64_t kHotMinNnz = 1 << 20;

// abi.cu
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int apply_dev(const spmm_mat* A, int transpose, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y,
              int64_t ldy, cudaStream_t s);
// apply_dev run by run (RowBlock): after a run's task kernel and the combine
// pass of its split rows, rows_done(r0, r1) enqueues what needs those rows of
// Y.  One run over all rows for streaming handles and plans without runs.
int apply_dev_runs(const spmm_mat* A, int transpose, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y,
                   int64_t ldy, cudaStream_t s, const std::function<int(int64_t, int64_t)>& rows_done);
// the task counter for a launch over rows of k elements of xtype (reset on s;
// nullptr for the static schedule) and the number of tasks per claim
unsigned long long* task_counter(const DevCSR& d, int32_t k, int32_t xtype, cudaStream_t s, cudaError_t* e,
                                 int32_t* chunk);
struct FwdArgs;
// Lane geometry of one call: VEC elements per lane load (the widest vector
// that divides k and keeps every X load and Y store aligned), CH column
// chunks, 2^lanes_log2 lanes per X row, nvec = k / VEC.
struct LaneGeometry {
    int vec = 1, ch = 1, lanes_log2 = 0, nvec = 1;
};
LaneGeometry lane_geometry(const void* X, int64_t ldx, int32_t k, int32_t xtype, const float* Y, int64_t ldy);
void set_geometry(FwdArgs& a, const void* X, int64_t ldx, int32_t k, int32_t xtype, const float* Y, int64_t ldy,
                  const DevCSR& d, int* vec_out, int* ch_out);
// automatic short_runs: pieces per lane group below this row-walk efficiency
constexpr double kPiecesBelowWalkEff = 0.5;
int value_mode(const spmm_mat* A, int32_t xtype);
cudaError_t launch_rows(const FwdArgs& a, int32_t xtype, int vmode, int vec, int ch, cudaStream_t s);

// stream.cu
int stream_setup(spmm_mat* A, const int64_t* row_ptr, const int32_t* col_idx, const void* values, size_t vsize,
                 cudaStream_t s);
int stream_apply(const spmm_mat* A, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y, int64_t ldy,
                 cudaStream_t s);
void stream_release(spmm_mat* A);

// Arguments of the task kernel (one instantiation per x type / value type /
// vector width / column chunks).
struct FwdArgs {
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const void* val;
    const int4* tasks;
    int64_t n_tasks;
    float* partials;
    int64_t n_slots;      // slots in `partials`: a segment task whose slot is not below this
                          // writes nothing and sets kStatusSlotRange in *status
    const void* X;
    int64_t ldx;
    float* Y;
    int64_t ldy;
    int32_t k;
    int32_t lanes_log2;   // log2(lanes per nonzero)
    int32_t nvec;         // k / VEC vectors per X row
    int32_t* status;      // status bits (kStatusTimeout, kStatusSlotRange), or-ed in by the kernels
    uint64_t wait_ns;     // bound of every staging wait
    int32_t x_evict_last; // gather X with the L2 evict-last policy
    int32_t compensated;  // long rows / hub segments: compensated summation
    float* partials_comp; // compensation term of each segment partial (compensated only)
    // Dynamic scheduling: after its first task (static, one per warp), a warp
    // claims the next task_chunk tasks, from W + task_chunk * atomicAdd(task_ctr,
    // 1) on (W = warps in the grid); the counter is zero at launch.  nullptr:
    // tasks t, t + W, t + 2W, ...
    unsigned long long* task_ctr = nullptr;
    int32_t task_chunk = 1;
    // short-row runs over rows of several lanes: 1 = merge-based pieces per
    // lane group, 0 = each group walks whole rows
    int32_t merge_groups = 0;
    // hot variant: a negative column index c names row ~c of the hot rows,
    // hot_bytes (a multiple of 16) of them packed at Xh, copied into shared
    // memory at the start of each block
    const void* Xh = nullptr;
    int64_t hot_bytes = 0;
};

// One launch over the tasks of several matrices (spmm_apply_batched): the
// entries' arguments travel in the kernel's parameter space (no device
// allocation); the tasks of entry e are numbers off[e] .. off[e+1]-1 of the
// launch.  g holds the launch-wide fields: n_tasks (all entries), task_ctr,
// task_chunk, status, wait_ns.
constexpr int kMaxBatch = 128;
struct MultiArgs {
    FwdArgs g;
    int32_t n;
    int64_t off[kMaxBatch + 1];
    FwdArgs ent[kMaxBatch];
};
static_assert(sizeof(MultiArgs) <= 32000, "kernel parameter space holds at most 32764 bytes");

// Launches from a handle are scheduled dynamically.  Tasks over wide X rows
// (at least kWideRowBytes bytes) vary a lot in time (gathers that miss L2)
// and are claimed one at a time (R-MAT scale 24, FP32: k = 4 1.95 -> 1.92 ms,
// k = 16 3.97 -> 3.22 ms against the static stride).  Narrow-row tasks are
// short, and claiming them one at a time made the counter's atomics the
// bottleneck (k = 1 1.11 -> 1.38 ms), so they are claimed kNarrowTaskChunk at
// a time.  With three blocks per SM, 30 PageRank iterations took 34.4 / 30.8 /
// 30.0 / 30.2 / 30.5 ms claiming 2 / 4 / 8 / 16 / 32 tasks (BF16 k = 1 1.08 /
// 0.94 / 0.89 / 0.88 / 0.89 ms).
constexpr int kWideRowBytes = 16;
#ifndef SPMM_NARROW_TASK_CHUNK
#define SPMM_NARROW_TASK_CHUNK 8
#endif
constexpr int kNarrowTaskChunk = SPMM_NARROW_TASK_CHUNK;

// rows_*.cu: launch the task kernel for one X dtype.  vmode: 0 pattern,
// 1 f32 values, 2 bf16 values, 3 f16 values.  Returns a cudaError_t.
cudaError_t launch_rows_f32(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
cudaError_t launch_rows_bf16(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
cudaError_t launch_rows_f16(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
// one lane per X row (ch == 1, lanes_log2 == 0); called by the three above
cudaError_t launch_rows_f32_one(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
cudaError_t launch_rows_bf16_one(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
cudaError_t launch_rows_f16_one(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
// merge-based short-row runs over lane groups (ch == 1, FwdArgs::merge_groups)
cudaError_t launch_rows_f32_mg(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
cudaError_t launch_rows_bf16_mg(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
cudaError_t launch_rows_f16_mg(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s);
// one lane per X row of at most 4 bytes with the hot rows in shared memory
// (FwdArgs::Xh set)
cudaError_t launch_rows_f32_hot(const FwdArgs& a, int vmode, int vec, cudaStream_t s);
cudaError_t launch_rows_bf16_hot(const FwdArgs& a, int vmode, int vec, cudaStream_t s);
cudaError_t launch_rows_f16_hot(const FwdArgs& a, int vmode, int vec, cudaStream_t s);

// rows_multi_*.cu: one launch of the generic task kernel over the entries of
// M (same X type, value mode, vector width, chunks and compensation)
cudaError_t launch_rows_multi_f32(const MultiArgs& M, int vmode, int vec, int ch, bool comp, cudaStream_t s);
cudaError_t launch_rows_multi_bf16(const MultiArgs& M, int vmode, int vec, int ch, bool comp, cudaStream_t s);
cudaError_t launch_rows_multi_f16(const MultiArgs& M, int vmode, int vec, int ch, bool comp, cudaStream_t s);

// combine.cu: the split rows of several matrices in one launch
// (spmm_apply_batched); launch_combine_multi fills off[] and lanes_log2
struct CombineEntry {
    const int4* splits;
    int64_t n_splits;
    const float* partials;
    const float* pcomp;     // compensation terms, or null
    float* Y;
    int64_t ldy;
    int32_t k, lanes_log2;
};
struct CombineMulti {
    int32_t n;
    int64_t off[kMaxBatch + 1];
    CombineEntry ent[kMaxBatch];
};
cudaError_t launch_combine_multi(CombineMulti& m, cudaStream_t s);

// combine.cu: Y[row] = sum of the split row's partials in a fixed order.
cudaError_t launch_combine(const int4* splits, int64_t n_splits, const float* partials, float* Y,
                           int64_t ldy, int32_t k, cudaStream_t s, const float* partials_comp = nullptr);

// status.cu: a kernel whose staging wait can never complete, to exercise
// the bounded-wait error path.
cudaError_t launch_wait_selftest(int32_t* status, uint64_t wait_ns, cudaStream_t s);

}  // namespace spmm
