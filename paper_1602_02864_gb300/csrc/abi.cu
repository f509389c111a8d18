// abi.cu -- the extern "C" entry points declared in include/spmm.h.
//
// spmm_create_csr validates the CSR input on the host, builds the warp-task
// plan (plan.cpp), copies the matrix and the plan to HBM, and optionally
// builds the transposed copy (a stable counting sort by column, so the
// transposed rows list their entries in increasing original-row order).
// spmm_apply only launches kernels: it allocates nothing and never
// synchronises the host.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace spmm {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SPMM_ERR_OOM : SPMM_ERR_CUDA;
}

static size_t dtype_size(int32_t t) {
    switch (t) {
        case SPMM_F32: return 4;
        case SPMM_BF16: return 2;
        case SPMM_F16: return 2;
        case SPMM_F64: return 8;
        default: return 0;
    }
}

static void free_dev(DevCSR& d) {
    cudaFree(d.row_ptr);
    cudaFree(d.col_idx);
    cudaFree(d.val);
    cudaFree(d.tasks);
    cudaFree(d.splits);
    cudaFree(d.partials);
    cudaFree(d.partials_comp);
    cudaFree(d.perm);
    cudaFree(d.task_ctr);
    cudaFree(d.col_hot);
    cudaFree(d.hot_cols);
    cudaFree(d.xh);
    d = DevCSR{};
}

// Copy count elements to a new device array with `pad` zeroed elements after
// them (the task kernel widens its bulk copies to 16-byte boundaries).
template <typename T>
static cudaError_t upload(T** dst, const T* src, size_t count, size_t pad, cudaStream_t s, int64_t* bytes) {
    *dst = nullptr;
    if (count + pad == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dst, (count + pad) * sizeof(T));
    if (e != cudaSuccess) { *dst = nullptr; return e; }
    *bytes += (int64_t)((count + pad) * sizeof(T));
    if (pad && (e = cudaMemsetAsync(*dst + count, 0, pad * sizeof(T), s)) != cudaSuccess) return e;
    if (count == 0) return cudaSuccess;
    return cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s);
}

// Copy one orientation (host CSR) and its plan to the device.
// With `reorder`, the columns are relabelled by decreasing count of stored
// entries (the device keeps the original index of each new label).  Hot
// columns (hot.cu): p.hot_cols -1 = automatic (kHotAuto), 0 = none, > 0 = at
// most that many, never more than fit the hot variant's shared memory;
// col_counts, if given, are the stored entries per column.
static int build_orientation(DevCSR& d, int64_t n_rows, int64_t n_cols, const int64_t* row_ptr,
                             const int32_t* col_idx, const void* val, size_t vsize, const Params& p,
                             bool reorder, const int64_t* col_counts, cudaStream_t s, int64_t* bytes) {
    d.n_rows = n_rows;
    d.n_cols = n_cols;
    d.short_runs = p.short_runs;
    d.nnz = row_ptr[n_rows];
    HostPlan plan = build_plan(row_ptr, n_rows, p);
    std::copy(plan.walk_eff, plan.walk_eff + 4, d.walk_eff);
    d.row_blocks = cut_row_blocks(plan, kRowBlocks);
    cudaError_t e;
    if ((e = upload(&d.row_ptr, row_ptr, (size_t)n_rows + 1, 2, s, bytes)) != cudaSuccess)
        return cuda_fail(e, "row_ptr");
    const int64_t cap = hot_capacity(val ? 1 : 0);
    const int64_t want_hot = p.hot_cols >= 0 ? std::min(p.hot_cols, cap)
                             : (d.nnz >= kHotMinNnz && cap >= kHotAutoMin) ? std::min(kHotAuto, cap)
                                                                           : 0;
    std::vector<int32_t> old_of_new, relabelled, hot, encoded;
    const int32_t* cols = col_idx;
    try {
        if (reorder) {
            relabel_by_degree(n_cols, col_idx, d.nnz, old_of_new, relabelled);
            cols = relabelled.data();
            col_counts = nullptr;   // counted again under the new labels
        }
        if (want_hot > 0) hot_select(n_cols, cols, d.nnz, col_counts, want_hot, hot, encoded);
    } catch (const std::bad_alloc&) {
        set_error("create: out of host memory for the column relabelling");
        return SPMM_ERR_OOM;
    }
    if (reorder && (e = upload(&d.perm, old_of_new.data(), (size_t)n_cols, 0, s, bytes)) != cudaSuccess)
        return cuda_fail(e, "col_idx");
    if ((e = upload(&d.col_idx, cols, (size_t)d.nnz, 8, s, bytes)) != cudaSuccess) return cuda_fail(e, "col_idx");
    if (!hot.empty()) {
        if ((e = upload(&d.col_hot, encoded.data(), (size_t)d.nnz, 8, s, bytes)) != cudaSuccess ||
            (e = upload(&d.hot_cols, hot.data(), hot.size(), 0, s, bytes)) != cudaSuccess)
            return cuda_fail(e, "hot columns");
        const size_t xb = (hot.size() * kHotRowBytes + 15) & ~(size_t)15;
        if ((e = cudaMalloc(&d.xh, xb)) != cudaSuccess) {
            d.xh = nullptr;
            return cuda_fail(e, "hot rows of X");
        }
        *bytes += (int64_t)xb;
        d.n_hot = (int64_t)hot.size();
    }
    // the host vectors are freed on return: finish their copies first
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "col_idx");
    if (val) {
        if ((e = upload((char**)&d.val, (const char*)val, (size_t)d.nnz * vsize, 8 * vsize, s, bytes)) != cudaSuccess)
            return cuda_fail(e, "values");
    }
    if ((e = upload(&d.tasks, plan.tasks.data(), plan.tasks.size(), 0, s, bytes)) != cudaSuccess)
        return cuda_fail(e, "tasks");
    d.n_tasks = (int64_t)plan.tasks.size() - 1;   // the last descriptor is the sentinel
    if ((e = upload(&d.splits, plan.splits.data(), plan.splits.size(), 0, s, bytes)) != cudaSuccess)
        return cuda_fail(e, "splits");
    d.n_splits = (int64_t)plan.splits.size();
    d.n_segments = plan.n_segments;
    d.n_slots = plan.n_slots;
    if ((e = cudaMalloc((void**)&d.task_ctr, sizeof(unsigned long long))) != cudaSuccess) {
        d.task_ctr = nullptr;
        return cuda_fail(e, "task counter");
    }
    *bytes += (int64_t)sizeof(unsigned long long);
    if (d.n_slots > 0) {
        size_t pb = (size_t)d.n_slots * kSlotStride * sizeof(float);
        if ((e = cudaMalloc((void**)&d.partials, pb)) != cudaSuccess) { d.partials = nullptr; return cuda_fail(e, "partials"); }
        *bytes += (int64_t)pb;
        if (p.compensated) {
            if ((e = cudaMalloc((void**)&d.partials_comp, pb)) != cudaSuccess) {
                d.partials_comp = nullptr;
                return cuda_fail(e, "partials");
            }
            *bytes += (int64_t)pb;
        }
    }
    // the plan vectors die with this frame: finish the copies first
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "create sync");
    return SPMM_OK;
}

// Defaults for zero fields, then clamp into the ranges the kernels assume
// (every task's nonzeros fit the staging buffers).
static Params resolve_params(const spmm_opts* opts) {
    Params prm;
    if (opts) {
        if (opts->task_nnz > 0) prm.task_nnz = opts->task_nnz;
        if (opts->task_rows > 0) prm.task_rows = opts->task_rows;
        if (opts->long_row > 0) prm.long_row = opts->long_row;
        if (opts->short_max > 0) prm.short_max = opts->short_max;
        if (opts->x_l2_policy == 1) prm.x_evict_last = 0;
        if (opts->x_l2_policy == 2) prm.x_evict_last = 1;
        if (opts->stream_slot_kib > 0) prm.slot_bytes = (int64_t)opts->stream_slot_kib << 10;
        if (opts->debug_fail_block > 0) prm.fail_block = opts->debug_fail_block;
        prm.compensated = opts->compensated ? 1 : 0;
        prm.short_runs = (opts->short_runs == 1 || opts->short_runs == 2) ? opts->short_runs : 0;
        if (opts->hot_cols != 0) prm.hot_cols = opts->hot_cols < 0 ? 0 : opts->hot_cols;
    }
    prm.task_nnz = std::min(std::max(prm.task_nnz, 32), kMaxTaskNnz);
    prm.task_rows = std::min(std::max(prm.task_rows, 1), kMaxTaskRows);
    prm.long_row = std::min(std::max(prm.long_row, prm.task_nnz), kMaxTaskNnz);
    prm.short_max = std::min(std::max(prm.short_max, 1), prm.task_nnz - 1);
    return prm;
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_plan_tasks(int64_t n_rows, const int64_t* row_ptr, const spmm_opts* opts, int32_t* tasks,
                               int64_t* n_tasks, int64_t* n_split_rows, int64_t* n_segments) {
    if (!row_ptr || !n_tasks || n_rows < 0 || n_rows >= (int64_t)1 << 31) {
        set_error("spmm_plan_tasks: bad argument");
        return SPMM_ERR_ARG;
    }
    if (row_ptr[0] != 0) { set_error("spmm_plan_tasks: row_ptr[0] != 0"); return SPMM_ERR_FORMAT; }
    for (int64_t i = 0; i < n_rows; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) { set_error("spmm_plan_tasks: row_ptr decreases"); return SPMM_ERR_FORMAT; }
    HostPlan plan;
    try {
        plan = build_plan(row_ptr, n_rows, resolve_params(opts));
    } catch (const std::bad_alloc&) {
        set_error("spmm_plan_tasks: out of host memory");
        return SPMM_ERR_OOM;
    }
    const int64_t nt = (int64_t)plan.tasks.size() - 1;
    if (tasks) {
        if (*n_tasks < nt) { set_error("spmm_plan_tasks: tasks capacity too small"); return SPMM_ERR_ARG; }
        std::memcpy(tasks, plan.tasks.data(), plan.tasks.size() * sizeof(int4));
    }
    *n_tasks = nt;
    if (n_split_rows) *n_split_rows = (int64_t)plan.splits.size();
    if (n_segments) *n_segments = plan.n_segments;
    return SPMM_OK;
}

extern "C" int spmm_plan_walk_eff(int64_t n_rows, const int64_t* row_ptr, const spmm_opts* opts, double* walk_eff) {
    if (!row_ptr || !walk_eff || n_rows < 0 || n_rows >= (int64_t)1 << 31) {
        set_error("spmm_plan_walk_eff: bad argument");
        return SPMM_ERR_ARG;
    }
    if (row_ptr[0] != 0) { set_error("spmm_plan_walk_eff: row_ptr[0] != 0"); return SPMM_ERR_FORMAT; }
    for (int64_t i = 0; i < n_rows; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) { set_error("spmm_plan_walk_eff: row_ptr decreases"); return SPMM_ERR_FORMAT; }
    try {
        const HostPlan plan = build_plan(row_ptr, n_rows, resolve_params(opts));
        std::copy(plan.walk_eff, plan.walk_eff + 4, walk_eff);
    } catch (const std::bad_alloc&) {
        set_error("spmm_plan_walk_eff: out of host memory");
        return SPMM_ERR_OOM;
    }
    return SPMM_OK;
}

extern "C" int spmm_plan_runs(int64_t n_rows, const int64_t* row_ptr, const spmm_opts* opts, int32_t max_runs,
                              int64_t* runs, int32_t* n_runs) {
    if (!row_ptr || !runs || !n_runs || max_runs < 1 || n_rows < 0 || n_rows >= (int64_t)1 << 31) {
        set_error("spmm_plan_runs: bad argument");
        return SPMM_ERR_ARG;
    }
    if (row_ptr[0] != 0) { set_error("spmm_plan_runs: row_ptr[0] != 0"); return SPMM_ERR_FORMAT; }
    for (int64_t i = 0; i < n_rows; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) { set_error("spmm_plan_runs: row_ptr decreases"); return SPMM_ERR_FORMAT; }
    try {
        const HostPlan plan = build_plan(row_ptr, n_rows, resolve_params(opts));
        const std::vector<RowBlock> rb = cut_row_blocks(plan, max_runs);
        for (size_t j = 0; j < rb.size(); ++j) {
            const RowBlock& b = rb[j];
            const int64_t v[6] = {b.t0, b.t1, b.r0, b.r1, b.s0, b.s1};
            std::copy(v, v + 6, runs + 6 * j);
        }
        *n_runs = (int32_t)rb.size();
    } catch (const std::bad_alloc&) {
        set_error("spmm_plan_runs: out of host memory");
        return SPMM_ERR_OOM;
    }
    return SPMM_OK;
}

extern "C" const char* spmm_last_error(void) { return g_error.c_str(); }

namespace spmm {

// Host value of stored entry p (for ||A||^2 of each graph).
// f(chunk, lo, hi) for `chunks` equal pieces of [0, n), on up to
// hardware_concurrency host threads.
template <class F>
static void parallel_chunks(int64_t n, int chunks, F&& f) {
    const int nt = std::max(1, std::min<int>(chunks, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int c; (c = next.fetch_add(1)) < chunks;) f(c, n * c / chunks, n * (c + 1) / chunks);
    };
    if (nt == 1 || n < (1 << 20)) {
        worker();
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
}

static double host_value(const void* v, int32_t vtype, int64_t p) {
    if (!v) return 1.0;
    if (vtype == SPMM_F32) return (double)static_cast<const float*>(v)[p];
    const uint16_t b = static_cast<const uint16_t*>(v)[p];
    if (vtype == SPMM_BF16) {
        const uint32_t u = (uint32_t)b << 16;
        float f;
        std::memcpy(&f, &u, 4);
        return (double)f;
    }
    __half_raw hr;
    hr.x = b;
    return (double)__half2float(__half(hr));
}

// Validate a host CSR, copy it and its plan(s) to the device.  Graph offsets
// (for batched handles) are filled in by the caller.
static int create_impl(spmm_mat** out, int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                       const int32_t* col_idx, const void* values, spmm_dtype vtype, uint32_t flags,
                       const spmm_opts* opts, cudaStream_t s, const char* who) {
    const std::string w(who);
    if (!out) { set_error(w + ": out is NULL"); return SPMM_ERR_ARG; }
    if (n_rows < 0 || n_rows >= (int64_t)1 << 31 || n_cols < 1 || n_cols >= (int64_t)1 << 31 || nnz < 0) {
        set_error(w + ": need 0 <= n_rows < 2^31, 1 <= n_cols < 2^31, nnz >= 0");
        return SPMM_ERR_ARG;
    }
    if (!row_ptr || (nnz > 0 && !col_idx)) { set_error(w + ": row_ptr/col_idx is NULL"); return SPMM_ERR_ARG; }
    if (flags & ~(SPMM_WANT_TRANSPOSE | SPMM_HOST_STREAMING | SPMM_REORDER | SPMM_RELABEL)) {
        set_error(w + ": unknown flag bits");
        return SPMM_ERR_ARG;
    }
    if ((flags & SPMM_HOST_STREAMING) && (flags & (SPMM_WANT_TRANSPOSE | SPMM_REORDER | SPMM_RELABEL))) {
        set_error(w + ": the streaming mode computes A X only, without relabelling "
                      "(no SPMM_WANT_TRANSPOSE, SPMM_REORDER or SPMM_RELABEL)");
        return SPMM_ERR_UNSUPPORTED;
    }
    const bool reorder = (flags & SPMM_REORDER) != 0;
    const bool relabel = (flags & SPMM_RELABEL) != 0;
    if (relabel && reorder) {
        set_error(w + ": SPMM_RELABEL and SPMM_REORDER exclude each other");
        return SPMM_ERR_ARG;
    }
    if (relabel && n_rows != n_cols) {
        set_error(w + ": SPMM_RELABEL renumbers the vertices of a square matrix");
        return SPMM_ERR_ARG;
    }
    size_t vsize = 0;
    if (values) {
        if (vtype != SPMM_F32 && vtype != SPMM_BF16 && vtype != SPMM_F16) {
            set_error(w + ": values must be F32, BF16 or F16");
            return SPMM_ERR_ARG;
        }
        vsize = dtype_size(vtype);
    }
    // ---- validate the CSR structure
    if (row_ptr[0] != 0) { set_error(w + ": row_ptr[0] != 0"); return SPMM_ERR_FORMAT; }
    if (row_ptr[n_rows] != nnz) { set_error(w + ": row_ptr[n_rows] != nnz"); return SPMM_ERR_FORMAT; }
    for (int64_t i = 0; i < n_rows; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) {
            set_error(w + ": row_ptr decreases at row " + std::to_string(i));
            return SPMM_ERR_FORMAT;
        }
    // column range and ||A||_F^2 in 64 fixed chunks on host threads (the chunk
    // sums are added in chunk order, so the norm does not depend on the thread
    // count); the first bad entry is reported
    constexpr int kChunks = 64;
    std::vector<int64_t> bad(kChunks, -1);
    std::vector<double> a2c(kChunks, 0.0);
    parallel_chunks(nnz, kChunks, [&](int c, int64_t lo, int64_t hi) {
        double acc = 0.0;
        for (int64_t p = lo; p < hi; ++p) {
            if (col_idx[p] < 0 || (int64_t)col_idx[p] >= n_cols) {
                bad[c] = p;
                return;
            }
            if (values) {
                const double v = host_value(values, vtype, p);
                acc += v * v;
            }
        }
        a2c[c] = values ? acc : (double)(hi - lo);
    });
    for (int c = 0; c < kChunks; ++c)
        if (bad[c] >= 0) {
            set_error(w + ": column index out of range at entry " + std::to_string(bad[c]));
            return SPMM_ERR_FORMAT;
        }
    double a2 = 0.0;
    for (int c = 0; c < kChunks; ++c) a2 += a2c[c];
    const Params prm = resolve_params(opts);
    // SPMM_RELABEL: from here on the matrix is B = P A P^T
    std::vector<int32_t> rl_old_of_new, rl_new_of_old, rl_ci;
    std::vector<int64_t> rl_rp;
    std::vector<char> rl_val;
    if (relabel) {
        int rrc = SPMM_OK;
        try {
            relabel_order(n_rows, row_ptr, col_idx, rl_old_of_new);
            rrc = relabel_csr(n_rows, row_ptr, col_idx, values, vsize, rl_old_of_new, rl_new_of_old, rl_rp, rl_ci,
                              rl_val);
        } catch (const std::bad_alloc&) {
            rrc = SPMM_ERR_OOM;
        }
        if (rrc != SPMM_OK) {
            set_error(w + ": out of host memory for the relabelled matrix");
            return rrc;
        }
        row_ptr = rl_rp.data();
        col_idx = rl_ci.data();
        if (values) values = rl_val.data();
    }

    spmm_mat* A = new (std::nothrow) spmm_mat();
    if (!A) { set_error(w + ": out of host memory"); return SPMM_ERR_OOM; }
    A->params = prm;
    A->vtype = values ? (int32_t)vtype : -1;
    A->row_off = {0, n_rows};
    A->col_off = {0, n_cols};
    A->a2 = {a2};
    cudaError_t se = cudaMalloc((void**)&A->status, sizeof(int32_t));
    if (se == cudaSuccess) se = cudaMemsetAsync(A->status, 0, sizeof(int32_t), s);
    if (se != cudaSuccess) {
        cudaFree(A->status);
        delete A;
        return cuda_fail(se, (w + ": status word").c_str());
    }
    int rc;
    if (flags & SPMM_HOST_STREAMING) {
        A->streaming = true;
        A->fwd.n_rows = n_rows;
        A->fwd.n_cols = n_cols;
        A->fwd.nnz = nnz;
        rc = stream_setup(A, row_ptr, col_idx, values, vsize, s);
        if (rc != SPMM_OK) {
            stream_release(A);
            free_dev(A->fwd);
            cudaFree(A->status);
            delete A;
            return rc;
        }
        *out = A;
        return SPMM_OK;
    }
    rc = build_orientation(A->fwd, n_rows, n_cols, row_ptr, col_idx, values, vsize, prm, reorder, nullptr, s,
                           &A->device_bytes);
    if (rc == SPMM_OK && (flags & SPMM_WANT_TRANSPOSE)) {
        // CSR of A^T by a stable counting sort on the column index.
        std::vector<int64_t> tptr((size_t)n_cols + 1, 0);
        std::vector<int32_t> tidx;
        std::vector<char> tval;
        try {
            tidx.resize((size_t)nnz);
            if (values) tval.resize((size_t)nnz * vsize);
        } catch (const std::bad_alloc&) {
            rc = SPMM_ERR_OOM;
            set_error(w + ": out of host memory for the transpose");
        }
        if (rc == SPMM_OK) {
            for (int64_t p = 0; p < nnz; ++p) tptr[(size_t)col_idx[p] + 1]++;
            for (int64_t c = 0; c < n_cols; ++c) tptr[c + 1] += tptr[c];
            std::vector<int64_t> pos(tptr.begin(), tptr.end() - 1);
            for (int64_t i = 0; i < n_rows; ++i)
                for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                    int64_t q = pos[(size_t)col_idx[p]]++;
                    tidx[(size_t)q] = (int32_t)i;
                    if (values) std::memcpy(&tval[(size_t)q * vsize], (const char*)values + p * vsize, vsize);
                }
            // the columns of A^T are the rows of A: their entry counts are A's row lengths
            std::vector<int64_t> outdeg((size_t)n_rows);
            for (int64_t i = 0; i < n_rows; ++i) outdeg[(size_t)i] = row_ptr[i + 1] - row_ptr[i];
            rc = build_orientation(A->tr, n_cols, n_rows, tptr.data(), tidx.data(), values ? tval.data() : nullptr,
                                   vsize, prm, reorder, outdeg.data(), s, &A->device_bytes);
            A->has_tr = (rc == SPMM_OK);
        }
    }
    if (rc == SPMM_OK && relabel) {
        const size_t pb = (size_t)n_rows * sizeof(int32_t);
        cudaError_t e = cudaMalloc((void**)&A->rl_old_of_new, pb);
        if (e == cudaSuccess) e = cudaMalloc((void**)&A->rl_new_of_old, pb);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(A->rl_old_of_new, rl_old_of_new.data(), pb, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(A->rl_new_of_old, rl_new_of_old.data(), pb, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, (w + ": vertex order").c_str());
        } else {
            A->relabel = true;
            A->device_bytes += 2 * (int64_t)pb;
        }
    }
    if (rc != SPMM_OK) {
        free_dev(A->fwd);
        free_dev(A->tr);
        cudaFree(A->rl_old_of_new);
        cudaFree(A->rl_new_of_old);
        cudaFree(A->status);
        delete A;
        return rc;
    }
    *out = A;
    return SPMM_OK;
}

extern "C" int spmm_create_file(spmm_mat_t* out, const char* path, uint32_t flags, const spmm_opts* opts,
                                void* stream) {
    set_error("");
    if (!out || !path) { set_error("spmm_create_file: NULL argument"); return SPMM_ERR_ARG; }
    if (flags & ~SPMM_FILE_DIRECT) {
        set_error("spmm_create_file: only SPMM_FILE_DIRECT is accepted (A X only, no relabelling)");
        return SPMM_ERR_UNSUPPORTED;
    }
    FileCSR f;
    int rc = file_open(path, (flags & SPMM_FILE_DIRECT) != 0, &f);
    if (rc != SPMM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    spmm_mat* A = new (std::nothrow) spmm_mat();
    if (!A) {
        ::close(f.fd);
        set_error("spmm_create_file: out of host memory");
        return SPMM_ERR_OOM;
    }
    A->params = resolve_params(opts);
    A->vtype = f.vtype;
    A->row_off = {0, f.n_rows};
    A->col_off = {0, f.n_cols};
    A->a2 = {0.0};
    A->streaming = true;
    A->fwd.n_rows = f.n_rows;
    A->fwd.n_cols = f.n_cols;
    A->fwd.nnz = f.nnz;
    A->st.file = f;
    auto fail = [&](int code) {
        stream_release(A);   // closes the file
        free_dev(A->fwd);
        cudaFree(A->status);
        delete A;
        return code;
    };
    cudaError_t e;
    if ((e = cudaMalloc((void**)&A->status, sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemsetAsync(A->status, 0, sizeof(int32_t), s)) != cudaSuccess)
        return fail(cuda_fail(e, "spmm_create_file: status word"));
    // row pointers: read once into pinned memory and validated
    const int64_t rp_bytes = (f.n_rows + 1) * 8;
    char* rp_buf = nullptr;
    if ((e = cudaHostAlloc((void**)&rp_buf, (size_t)rp_bytes + 2 * kFileAlign, cudaHostAllocDefault)) != cudaSuccess)
        return fail(cuda_fail(e, "spmm_create_file: row pointers"));
    std::string err;
    const char* rp = file_read_range(f.fd, f.direct, f.off_rp, rp_bytes, rp_buf, 8, 0, &err);
    if (!rp) {
        cudaFreeHost(rp_buf);
        set_error("spmm_create_file: " + err);
        return fail(SPMM_ERR_IO);
    }
    // keep the row pointers at the start of their own pinned buffer
    if (rp != rp_buf) std::memmove(rp_buf, rp, (size_t)rp_bytes);
    A->st.h_rp_owned = reinterpret_cast<int64_t*>(rp_buf);
    const int64_t* row_ptr = A->st.h_rp_owned;
    if (row_ptr[0] != 0 || row_ptr[f.n_rows] != f.nnz) {
        set_error("spmm_create_file: row_ptr[0] != 0 or row_ptr[n_rows] != nnz");
        return fail(SPMM_ERR_FORMAT);
    }
    for (int64_t i = 0; i < f.n_rows; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) {
            set_error("spmm_create_file: row_ptr decreases at row " + std::to_string(i));
            return fail(SPMM_ERR_FORMAT);
        }
    const size_t vsize = f.vtype < 0 ? 0 : dtype_size((spmm_dtype)f.vtype);
    if ((rc = stream_setup(A, row_ptr, nullptr, nullptr, vsize, s)) != SPMM_OK) return fail(rc);
    if ((rc = stream_file_setup(A, s)) != SPMM_OK) return fail(rc);
    *out = A;
    return SPMM_OK;
}

int create_from_host_csr(spmm_mat** out, int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                         const int32_t* col_idx, const void* values, spmm_dtype vtype, uint32_t flags,
                         const spmm_opts* opts, cudaStream_t s, const char* who) {
    return create_impl(out, n_rows, n_cols, nnz, row_ptr, col_idx, values, vtype, flags, opts, s, who);
}

}  // namespace spmm

extern "C" int spmm_create_csr(spmm_mat_t* out, int64_t n_rows, int64_t n_cols, int64_t nnz,
                               const int64_t* row_ptr, const int32_t* col_idx, const void* values,
                               spmm_dtype vtype, uint32_t flags, const spmm_opts* opts, void* stream) {
    set_error("");
    return create_impl(out, n_rows, n_cols, nnz, row_ptr, col_idx, values, vtype, flags, opts,
                       (cudaStream_t)stream, "spmm_create_csr");
}

extern "C" int spmm_create_batched(spmm_mat_t* out, int32_t n_graphs, const int64_t* n_rows, const int64_t* n_cols,
                                   const int64_t* const* row_ptrs, const int32_t* const* col_idxs,
                                   const void* const* values, spmm_dtype vtype, uint32_t flags,
                                   const spmm_opts* opts, void* stream) {
    set_error("");
    if (!out || n_graphs < 1 || !n_rows || !n_cols || !row_ptrs || !col_idxs) {
        set_error("spmm_create_batched: NULL argument or n_graphs < 1");
        return SPMM_ERR_ARG;
    }
    if (flags & SPMM_RELABEL) {
        set_error("spmm_create_batched: SPMM_RELABEL is for single square matrices (relabel each graph's "
                  "vertices before batching)");
        return SPMM_ERR_UNSUPPORTED;
    }
    const size_t vsize = values ? dtype_size(vtype) : 0;
    std::vector<int64_t> roff((size_t)n_graphs + 1, 0), coff((size_t)n_graphs + 1, 0);
    int64_t nnz = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        if (n_rows[g] < 0 || n_cols[g] < 1 || !row_ptrs[g] || (values && !values[g])) {
            set_error("spmm_create_batched: bad size or NULL array for graph " + std::to_string(g));
            return SPMM_ERR_ARG;
        }
        const int64_t* rp = row_ptrs[g];
        if (rp[0] != 0) { set_error("spmm_create_batched: row_ptr[0] != 0 in graph " + std::to_string(g)); return SPMM_ERR_FORMAT; }
        for (int64_t i = 0; i < n_rows[g]; ++i)
            if (rp[i + 1] < rp[i]) {
                set_error("spmm_create_batched: row_ptr decreases in graph " + std::to_string(g));
                return SPMM_ERR_FORMAT;
            }
        const int64_t z = rp[n_rows[g]];
        if (z > 0 && !col_idxs[g]) { set_error("spmm_create_batched: col_idx is NULL"); return SPMM_ERR_ARG; }
        for (int64_t p = 0; p < z; ++p)
            if (col_idxs[g][p] < 0 || col_idxs[g][p] >= n_cols[g]) {
                set_error("spmm_create_batched: column index out of range in graph " + std::to_string(g));
                return SPMM_ERR_FORMAT;
            }
        roff[g + 1] = roff[g] + n_rows[g];
        coff[g + 1] = coff[g] + n_cols[g];
        nnz += z;
    }
    if (roff[n_graphs] >= (int64_t)1 << 31 || coff[n_graphs] >= (int64_t)1 << 31) {
        set_error("spmm_create_batched: more than 2^31 rows or columns in the batch");
        return SPMM_ERR_ARG;
    }
    // block-diagonal CSR of the whole batch
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<char> va;
    try {
        rp.resize((size_t)roff[n_graphs] + 1);
        ci.resize((size_t)nnz);
        if (values) va.resize((size_t)nnz * vsize);
    } catch (const std::bad_alloc&) {
        set_error("spmm_create_batched: out of host memory");
        return SPMM_ERR_OOM;
    }
    int64_t e = 0;
    std::vector<double> a2((size_t)n_graphs, 0.0);
    rp[0] = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        const int64_t z = row_ptrs[g][n_rows[g]];
        for (int64_t i = 0; i < n_rows[g]; ++i) rp[(size_t)(roff[g] + i + 1)] = e + row_ptrs[g][i + 1];
        for (int64_t p = 0; p < z; ++p) ci[(size_t)(e + p)] = (int32_t)(col_idxs[g][p] + coff[g]);
        if (values) std::memcpy(&va[(size_t)e * vsize], values[g], (size_t)z * vsize);
        for (int64_t p = 0; p < z; ++p) {
            const double v = values ? host_value(values[g], vtype, p) : 1.0;
            a2[(size_t)g] += v * v;
        }
        e += z;
    }
    spmm_mat* A = nullptr;
    const int rc = create_impl(&A, roff[n_graphs], coff[n_graphs], nnz, rp.data(), ci.data(),
                               values ? va.data() : nullptr, vtype, flags, opts, (cudaStream_t)stream,
                               "spmm_create_batched");
    if (rc != SPMM_OK) return rc;
    A->row_off = roff;
    A->col_off = coff;
    A->a2 = a2;
    *out = A;
    return SPMM_OK;
}

namespace spmm {

// The task counter of a launch (reset on s) and the tasks claimed at a time.
unsigned long long* task_counter(const DevCSR& d, int32_t k, int32_t xtype, cudaStream_t s, cudaError_t* e,
                                 int32_t* chunk) {
    *e = cudaSuccess;
    *chunk = (int64_t)k * (int64_t)dtype_size((spmm_dtype)xtype) >= kWideRowBytes ? 1 : kNarrowTaskChunk;
    if (!d.task_ctr) return nullptr;
    *e = cudaMemsetAsync(d.task_ctr, 0, sizeof(unsigned long long), s);
    return *e == cudaSuccess ? d.task_ctr : nullptr;
}

LaneGeometry lane_geometry(const void* X, int64_t ldx, int32_t k, int32_t xtype, const float* Y, int64_t ldy) {
    const int esize = (int)dtype_size(xtype);
    const uintptr_t xa = (uintptr_t)X, ya = (uintptr_t)Y;
    LaneGeometry g;
    int vec = 16 / esize;
    for (; vec > 1; vec >>= 1) {
        const int yv = std::min(vec, 4);
        if (k % vec == 0 && ldx % vec == 0 && xa % (uintptr_t)(vec * esize) == 0 && ldy % yv == 0 &&
            ya % (uintptr_t)(yv * 4) == 0)
            break;
    }
    // A whole 16-byte X row on one lane (k = 4 FP32, k = 8 BF16/FP16) measured
    // slower than two lanes of 8 bytes (BF16 k = 8: 2.27 -> 2.08 ms on R-MAT
    // scale 24), so such rows get two lanes.
    if (vec * esize == 16 && k == vec) vec >>= 1;
    g.vec = vec;
    g.nvec = k / vec;
    g.ch = g.nvec > 32 ? 2 : 1;
    const int per = (g.nvec + g.ch - 1) / g.ch;
    while ((1 << g.lanes_log2) < per) ++g.lanes_log2;
    return g;
}

void set_geometry(FwdArgs& a, const void* X, int64_t ldx, int32_t k, int32_t xtype, const float* Y, int64_t ldy,
                  const DevCSR& d, int* vec_out, int* ch_out) {
    const int esize = (int)dtype_size(xtype);
    const LaneGeometry gm = lane_geometry(X, ldx, k, xtype, Y, ldy);
    const int vec = gm.vec, ch = gm.ch, lg = gm.lanes_log2, nvec = gm.nvec;
    a.X = X;
    a.ldx = ldx;
    a.Y = const_cast<float*>(Y);
    a.ldy = ldy;
    a.k = k;
    a.lanes_log2 = lg;
    a.nvec = nvec;
    // Short-row runs over lane groups: equal pieces per group (merge_groups)
    // or whole rows per group.  Pieces win where the row walk would leave
    // groups idle behind the longest row of each round (plan statistic
    // walk_eff below 0.5: R-MAT, FP32 k = 16 2.79 -> 2.70 ms, k = 32
    // 4.38 -> 4.18) and lose where rows have similar lengths (Chung-Lu batch
    // k = 16 0.88 -> 1.19 ms, SBM k = 64 10.9 -> 13.0).  32-byte rows on two
    // lanes keep the walk (R-MAT k = 8 2.21 -> 2.33 with pieces); lanes of 8
    // 16-bit elements spill in the pieces path, which is not built for them.
    const bool pieces_ok = ch == 1 && lg >= 1 && lg <= 4 && vec <= 4;
    a.merge_groups = d.short_runs == 2 ? pieces_ok
                     : d.short_runs == 1 ? false
                                         : pieces_ok && (lg >= 2 || vec * esize <= 8) &&
                                               d.walk_eff[4 - lg] < kPiecesBelowWalkEff;
    *vec_out = vec;
    *ch_out = ch;
}

int value_mode(const spmm_mat* A, int32_t xtype) {
    int vmode = 0;
    if (A->vtype == SPMM_F32) vmode = 1;
    else if (A->vtype == SPMM_BF16) vmode = 2;
    else if (A->vtype == SPMM_F16) vmode = 3;
    if ((vmode == 2 && xtype != SPMM_BF16) || (vmode == 3 && xtype != SPMM_F16)) return -1;
    return vmode;
}

cudaError_t launch_rows(const FwdArgs& a, int32_t xtype, int vmode, int vec, int ch, cudaStream_t s) {
    if (xtype == SPMM_F32) return launch_rows_f32(a, vmode, vec, ch, s);
    if (xtype == SPMM_BF16) return launch_rows_bf16(a, vmode, vec, ch, s);
    return launch_rows_f16(a, vmode, vec, ch, s);
}

// The product on a resident handle: one run over all tasks (rows_done ==
// nullptr), or each of d.row_blocks followed by rows_done on its rows.
static int apply_resident(const spmm_mat* A, int transpose, const void* X, int64_t ldx, int32_t k, int32_t xtype,
                          float* Y, int64_t ldy, cudaStream_t s,
                          const std::function<int(int64_t, int64_t)>* rows_done) {
    const DevCSR& d = transpose ? A->tr : A->fwd;
    const int vmode = value_mode(A, xtype);
    if (vmode < 0) {
        set_error("spmm_apply: 16-bit values need X of the same 16-bit type (or use F32 values)");
        return SPMM_ERR_UNSUPPORTED;
    }
    if (d.perm) {   // relabelled columns: gather X's rows into the new order first
        const void* Xp = nullptr;
        const int rc = reorder_x(const_cast<spmm_mat*>(A), d, X, ldx, k, xtype, s, &Xp);
        if (rc != SPMM_OK) return rc;
        X = Xp;
        ldx = k;
    }
    FwdArgs a;
    int vec = 1, ch = 1;
    set_geometry(a, X, ldx, k, xtype, Y, ldy, d, &vec, &ch);
    const int esize = (int)dtype_size(xtype);
    a.col_idx = d.col_idx;
    if (d.n_hot > 0 && k * esize == kHotRowBytes && ch == 1 && a.lanes_log2 == 0) {
        // one lane per 4-byte X row: the hot variant, fed with the packed hot
        // rows of X and the column indices that name them
        const cudaError_t eh = hot_gather(d, X, ldx, k, esize, s);
        if (eh != cudaSuccess) return cuda_fail(eh, "spmm_apply: hot rows");
        a.col_idx = d.col_hot;
        a.Xh = d.xh;
        a.hot_bytes = (d.n_hot * k * esize + 15) & ~(int64_t)15;
    }
    a.row_ptr = d.row_ptr;
    a.val = d.val;
    a.partials = d.partials;
    a.n_slots = d.n_slots;
    a.status = A->status;
    a.wait_ns = kWaitNs;
    a.x_evict_last = A->params.x_evict_last;
    a.compensated = d.partials_comp != nullptr || (A->params.compensated && d.n_slots == 0);
    a.partials_comp = d.partials_comp;
    const RowBlock all{0, d.n_tasks, 0, d.n_rows, 0, d.n_splits};
    const bool by_runs = rows_done && d.row_blocks.size() > 1;
    const size_t n_runs = by_runs ? d.row_blocks.size() : 1;
    for (size_t j = 0; j < n_runs; ++j) {
        const RowBlock& b = by_runs ? d.row_blocks[j] : all;
        cudaError_t ec = cudaSuccess;
        a.task_ctr = task_counter(d, k, xtype, s, &ec, &a.task_chunk);
        if (ec != cudaSuccess) return cuda_fail(ec, "spmm_apply: task counter");
        a.tasks = d.tasks + b.t0;
        a.n_tasks = b.t1 - b.t0;
        cudaError_t e = launch_rows(a, xtype, vmode, vec, ch, s);
        if (e != cudaSuccess) return cuda_fail(e, "spmm_apply: task kernel");
        e = launch_combine(d.splits + b.s0, b.s1 - b.s0, d.partials, Y, ldy, k, s, d.partials_comp);
        if (e != cudaSuccess) return cuda_fail(e, "spmm_apply: combine kernel");
        if (rows_done) {
            const int rc = (*rows_done)(b.r0, b.r1);
            if (rc != SPMM_OK) return rc;
        }
    }
    return SPMM_OK;
}

// Enqueue Y = A X (or A^T X) for a validated handle; shared by spmm_apply and
// the applications built on it.
int apply_dev(const spmm_mat* A, int transpose, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y,
              int64_t ldy, cudaStream_t s) {
    NvtxRange range(transpose ? "spmm_apply A^T X" : "spmm_apply A X");
    if (A->streaming && !transpose) return stream_apply(A, X, ldx, k, xtype, Y, ldy, s);
    if ((transpose ? A->tr : A->fwd).n_rows == 0) return SPMM_OK;
    return apply_resident(A, transpose, X, ldx, k, xtype, Y, ldy, s, nullptr);
}

int apply_dev_runs(const spmm_mat* A, int transpose, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y,
                   int64_t ldy, cudaStream_t s, const std::function<int(int64_t, int64_t)>& rows_done) {
    NvtxRange range(transpose ? "spmm_apply A^T X (runs)" : "spmm_apply A X (runs)");
    const DevCSR& d = transpose ? A->tr : A->fwd;
    if (d.n_rows == 0) return SPMM_OK;
    if (A->streaming && !transpose) {
        const int rc = stream_apply(A, X, ldx, k, xtype, Y, ldy, s);
        return rc != SPMM_OK ? rc : rows_done(0, d.n_rows);
    }
    return apply_resident(A, transpose, X, ldx, k, xtype, Y, ldy, s, &rows_done);
}

}  // namespace spmm

extern "C" int spmm_apply(spmm_mat_t A, const void* X, int64_t ldx, int32_t k, spmm_dtype xtype, void* Y,
                          int64_t ldy, spmm_dtype ytype, int32_t transpose, void* stream) {
    if (!A) { set_error("spmm_apply: A is NULL"); return SPMM_ERR_ARG; }
    if (k < 1 || k > kMaxK) { set_error("spmm_apply: k must be in 1..64"); return SPMM_ERR_ARG; }
    if (ldx < k || ldy < k) { set_error("spmm_apply: ldx and ldy must be >= k"); return SPMM_ERR_ARG; }
    if (ytype != SPMM_F32) { set_error("spmm_apply: Y must be F32"); return SPMM_ERR_ARG; }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16 && xtype != SPMM_F16) {
        set_error("spmm_apply: X must be F32, BF16 or F16");
        return SPMM_ERR_ARG;
    }
    if (transpose && !A->has_tr) {
        set_error("spmm_apply: transpose needs SPMM_WANT_TRANSPOSE at create");
        return SPMM_ERR_ARG;
    }
    const DevCSR& d = transpose ? A->tr : A->fwd;
    if (d.n_rows == 0) return SPMM_OK;
    if (!X || !Y) { set_error("spmm_apply: X or Y is NULL"); return SPMM_ERR_ARG; }
    if (A->relabel) return apply_relabel_io(A, transpose, X, ldx, k, (int32_t)xtype, (float*)Y, ldy, (cudaStream_t)stream);
    return apply_dev(A, transpose, X, ldx, k, (int32_t)xtype, (float*)Y, ldy, (cudaStream_t)stream);
}

extern "C" int spmm_apply_relabelled(spmm_mat_t A, const void* X, int64_t ldx, int32_t k, spmm_dtype xtype, void* Y,
                                     int64_t ldy, spmm_dtype ytype, int32_t transpose, void* stream) {
    if (!A) { set_error("spmm_apply_relabelled: A is NULL"); return SPMM_ERR_ARG; }
    if (!A->relabel) return spmm_apply(A, X, ldx, k, xtype, Y, ldy, ytype, transpose, stream);
    if (k < 1 || k > kMaxK) { set_error("spmm_apply_relabelled: k must be in 1..64"); return SPMM_ERR_ARG; }
    if (ldx < k || ldy < k) { set_error("spmm_apply_relabelled: ldx and ldy must be >= k"); return SPMM_ERR_ARG; }
    if (ytype != SPMM_F32) { set_error("spmm_apply_relabelled: Y must be F32"); return SPMM_ERR_ARG; }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16 && xtype != SPMM_F16) {
        set_error("spmm_apply_relabelled: X must be F32, BF16 or F16");
        return SPMM_ERR_ARG;
    }
    if (transpose && !A->has_tr) {
        set_error("spmm_apply_relabelled: transpose needs SPMM_WANT_TRANSPOSE at create");
        return SPMM_ERR_ARG;
    }
    if (A->fwd.n_rows == 0) return SPMM_OK;
    if (!X || !Y) { set_error("spmm_apply_relabelled: X or Y is NULL"); return SPMM_ERR_ARG; }
    return apply_dev(A, transpose, X, ldx, k, (int32_t)xtype, (float*)Y, ldy, (cudaStream_t)stream);
}

extern "C" int spmm_get_info(spmm_mat_t A, spmm_info* info) {
    if (!A || !info) { set_error("spmm_get_info: NULL argument"); return SPMM_ERR_ARG; }
    std::memset(info, 0, sizeof(*info));
    info->n_rows = A->fwd.n_rows;
    info->n_cols = A->fwd.n_cols;
    info->nnz = A->fwd.nnz;
    info->n_tasks = A->fwd.n_tasks;
    info->n_split_rows = A->fwd.n_splits;
    info->n_segments = A->fwd.n_segments;
    if (A->has_tr) {
        info->n_tasks_t = A->tr.n_tasks;
        info->n_split_rows_t = A->tr.n_splits;
        info->n_segments_t = A->tr.n_segments;
    }
    info->device_bytes = A->device_bytes;
    info->value_dtype = A->vtype;
    info->has_transpose = A->has_tr ? 1 : 0;
    info->n_graphs = (int32_t)(A->row_off.size() - 1);
    info->relabelled = A->relabel ? 1 : 0;
    info->n_hot = A->fwd.n_hot;
    info->n_hot_t = A->has_tr ? A->tr.n_hot : 0;
    for (int i = 0; i < 4; ++i) {
        info->walk_eff[i] = A->fwd.walk_eff[i];
        info->walk_eff_t[i] = A->has_tr ? A->tr.walk_eff[i] : 0.0;
    }
    return SPMM_OK;
}

extern "C" int spmm_destroy(spmm_mat_t A) {
    if (!A) return SPMM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (A->streaming) stream_release(A);
    hostio_release(A);
    pagerank_release(A);
    cudaFree(A->xperm);
    cudaFree(A->yperm);
    cudaFree(A->rl_old_of_new);
    cudaFree(A->rl_new_of_old);
    free_dev(A->fwd);
    free_dev(A->tr);
    cudaFree(A->status);
    delete A;
    if (e != cudaSuccess) return cuda_fail(e, "spmm_destroy: pending device work failed");
    return SPMM_OK;
}

extern "C" int spmm_sync_status(spmm_mat_t A, void* stream) {
    if (!A) { set_error("spmm_sync_status: A is NULL"); return SPMM_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "spmm_sync_status: stream");
    int32_t st = 0;
    if ((e = cudaMemcpy(&st, A->status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "spmm_sync_status: read status");
    if (st != 0) {
        cudaMemset(A->status, 0, sizeof(int32_t));
        if (st & kStatusTimeout) {
            set_error("spmm_sync_status: a device-side staging wait timed out; results of the calls since the "
                      "last check are incomplete");
            return SPMM_ERR_TIMEOUT;
        }
        set_error("spmm_sync_status: a task named a partial slot beyond the scratch; results of the calls "
                  "since the last check are incomplete");
        return SPMM_ERR_FORMAT;
    }
    return SPMM_OK;
}

extern "C" int spmm_debug_wait_timeout(uint64_t wait_ns, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* st = nullptr;
    cudaError_t e = cudaMalloc((void**)&st, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "spmm_debug_wait_timeout: alloc");
    int32_t h = 0;
    if ((e = cudaMemsetAsync(st, 0, sizeof(int32_t), s)) == cudaSuccess &&
        (e = launch_wait_selftest(st, wait_ns, s)) == cudaSuccess &&
        (e = cudaMemcpyAsync(&h, st, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) == cudaSuccess)
        e = cudaStreamSynchronize(s);
    cudaFree(st);
    if (e != cudaSuccess) return cuda_fail(e, "spmm_debug_wait_timeout");
    if (h != 0) {
        set_error("spmm_debug_wait_timeout: the wait ran out as intended");
        return SPMM_ERR_TIMEOUT;
    }
    return SPMM_OK;
}

// ------------------------------------------------------------------ re-planning and autotuning
namespace spmm {

// Rebuild the task plan of one orientation for new parameters; the matrix
// itself stays where it is.
static int replan_orientation(DevCSR& d, const Params& p, cudaStream_t s, int64_t* bytes) {
    std::vector<int64_t> rp;
    try {
        rp.resize((size_t)d.n_rows + 1);
    } catch (const std::bad_alloc&) {
        set_error("replan: out of host memory");
        return SPMM_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(rp.data(), d.row_ptr, rp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "replan: row pointers");
    HostPlan plan = build_plan(rp.data(), d.n_rows, p);
    int4 *tasks = nullptr, *splits = nullptr;
    float *partials = nullptr, *pcomp = nullptr;
    int64_t added = 0;
    const size_t pb = (size_t)plan.n_slots * kSlotStride * sizeof(float);
    if ((e = upload(&tasks, plan.tasks.data(), plan.tasks.size(), 0, s, &added)) != cudaSuccess ||
        (e = upload(&splits, plan.splits.data(), plan.splits.size(), 0, s, &added)) != cudaSuccess ||
        (plan.n_slots > 0 && (e = cudaMalloc((void**)&partials, pb)) != cudaSuccess) ||
        (plan.n_slots > 0 && p.compensated && (e = cudaMalloc((void**)&pcomp, pb)) != cudaSuccess)) {
        cudaFree(tasks);
        cudaFree(splits);
        cudaFree(partials);
        return cuda_fail(e, "replan: upload");
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "replan: sync");
    *bytes -= (int64_t)((d.n_tasks + 1) * sizeof(int4) + d.n_splits * sizeof(int4) +
                        d.n_slots * kSlotStride * sizeof(float) * (d.partials_comp ? 2 : 1));
    *bytes += added + (int64_t)(pb * (pcomp ? 2 : 1));
    cudaFree(d.tasks);
    cudaFree(d.splits);
    cudaFree(d.partials);
    cudaFree(d.partials_comp);
    d.partials_comp = pcomp;
    d.tasks = tasks;
    d.n_tasks = (int64_t)plan.tasks.size() - 1;
    d.splits = splits;
    d.n_splits = (int64_t)plan.splits.size();
    d.n_segments = plan.n_segments;
    d.partials = partials;
    d.n_slots = plan.n_slots;
    std::copy(plan.walk_eff, plan.walk_eff + 4, d.walk_eff);
    d.row_blocks = cut_row_blocks(plan, kRowBlocks);
    d.short_runs = p.short_runs;
    return SPMM_OK;
}

__global__ void fill_x_kernel(void* X, int64_t n, int xtype) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)((i * 2654435761ull) % 1000ull) * 1e-3f - 0.5f;
        if (xtype == SPMM_F32) static_cast<float*>(X)[i] = v;
        else if (xtype == SPMM_BF16) static_cast<__nv_bfloat16*>(X)[i] = __float2bfloat16(v);
        else static_cast<__half*>(X)[i] = __float2half(v);
    }
}

}  // namespace spmm

extern "C" int spmm_replan(spmm_mat_t A, const spmm_opts* opts, int32_t transpose, void* stream) {
    if (!A) { set_error("spmm_replan: A is NULL"); return SPMM_ERR_ARG; }
    if (A->streaming) { set_error("spmm_replan: not available for streaming handles"); return SPMM_ERR_UNSUPPORTED; }
    if (transpose && !A->has_tr) { set_error("spmm_replan: no transposed copy"); return SPMM_ERR_ARG; }
    const Params p = resolve_params(opts);
    pagerank_invalidate(A);   // its graph holds the old plan's task list and scratch
    const int rc = replan_orientation(transpose ? A->tr : A->fwd, p, (cudaStream_t)stream, &A->device_bytes);
    if (rc == SPMM_OK) {
        // the L2 policy and compensation are launch parameters shared by both orientations
        A->params.x_evict_last = p.x_evict_last;
        A->params.compensated = p.compensated;
        const int64_t hot_cols = A->params.hot_cols;   // fixed at create (the stored column indices)
        if (!transpose) A->params = p;
        A->params.hot_cols = hot_cols;
    }
    return rc;
}

extern "C" int spmm_autotune(spmm_mat_t A, int32_t k, spmm_dtype xtype, int32_t transpose,
                             const spmm_opts* candidates, int32_t n_candidates, int32_t reps, int32_t* best_index,
                             double* times_ms, void* stream) {
    if (!A || !best_index) { set_error("spmm_autotune: NULL argument"); return SPMM_ERR_ARG; }
    if (k < 1 || k > kMaxK || reps < 1 || (candidates && n_candidates < 1)) {
        set_error("spmm_autotune: need 1 <= k <= 64, reps >= 1, n_candidates >= 1");
        return SPMM_ERR_ARG;
    }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16 && xtype != SPMM_F16) {
        set_error("spmm_autotune: X must be F32, BF16 or F16");
        return SPMM_ERR_ARG;
    }
    if (A->streaming) { set_error("spmm_autotune: not available for streaming handles"); return SPMM_ERR_UNSUPPORTED; }
    if (transpose && !A->has_tr) { set_error("spmm_autotune: no transposed copy"); return SPMM_ERR_ARG; }
    // built-in search space: task size x short-row limit x L2 policy of X
    std::vector<spmm_opts> grid;
    if (candidates) {
        grid.assign(candidates, candidates + n_candidates);
    } else {
        for (int tn : {128, 256, 512})
            for (int sm : {7, 15, 31, 63})
                for (int pol : {1, 2}) {
                    if (sm >= tn) continue;
                    spmm_opts o{};
                    o.task_nnz = tn;
                    o.short_max = sm;
                    o.long_row = 512;
                    o.x_l2_policy = pol;
                    grid.push_back(o);
                }
    }
    const DevCSR& d = transpose ? A->tr : A->fwd;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t esz = xtype == SPMM_F32 ? 4 : 2;
    void* X = nullptr;
    float* Y = nullptr;
    void* flush = nullptr;
    const size_t flush_bytes = 256u << 20;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SPMM_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&X, (size_t)std::max<int64_t>(d.n_cols, 1) * k * esz)) != cudaSuccess ||
        (e = cudaMalloc((void**)&Y, (size_t)std::max<int64_t>(d.n_rows, 1) * k * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&flush, flush_bytes)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
        (e = cudaEventCreate(&e1)) != cudaSuccess) {
        rc = cuda_fail(e, "spmm_autotune: workspace");
    }
    int best = -1;
    double best_ms = 0.0;
    if (rc == SPMM_OK) {
        fill_x_kernel<<<1024, 256, 0, s>>>(X, d.n_cols * k, xtype);
        for (size_t c = 0; c < grid.size() && rc == SPMM_OK; ++c) {
            if ((rc = spmm_replan(A, &grid[c], transpose, stream)) != SPMM_OK) break;
            for (int w = 0; w < 2 && rc == SPMM_OK; ++w) rc = apply_dev(A, transpose, X, k, k, xtype, Y, k, s);
            double total = 0.0;
            for (int r = 0; r < reps && rc == SPMM_OK; ++r) {
                cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);   // evict the previous call from L2
                cudaEventRecord(e0, s);
                rc = apply_dev(A, transpose, X, k, k, xtype, Y, k, s);
                cudaEventRecord(e1, s);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_fail(e, "spmm_autotune: timing"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (rc != SPMM_OK) break;
            const double mean = total / reps;
            if (times_ms) times_ms[c] = mean;
            if (best < 0 || mean < best_ms) { best = (int)c; best_ms = mean; }
        }
        if (rc == SPMM_OK && best >= 0) rc = spmm_replan(A, &grid[(size_t)best], transpose, stream);
    }
    if (rc == SPMM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_fail(e, "spmm_autotune: sync");
    cudaFree(X);
    cudaFree(Y);
    cudaFree(flush);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc == SPMM_OK) *best_index = best;
    return rc;
}
