// stream.cu -- streaming mode: the matrix stays in host memory.
//
// The paper keeps the sparse matrix on SSDs and streams tile rows into memory
// while the dense matrices stay in RAM (Section 3.1); its executor reads tile
// rows asynchronously and multiplies each one when it has arrived (Algorithm
// 1), and the amount of memory to give each side follows Section 3.6 (spend
// memory on the dense matrix, stream the sparse one).  Here the matrix stays
// in the caller's host memory (pinned by the library if it is not already),
// X and Y stay in HBM, and the matrix flows over the host link in blocks of
// whole warp tasks.  Two staging slots alternate: the copy of block b+1 runs
// on a copy stream while the task kernel works on block b; events order each
// slot's reuse.  The task list, split table and partials live in HBM as in
// the resident mode, so results are identical to it.
//
// The same pipeline serves a matrix kept in a file (spmm_create_file): each
// block's column indices and values are first read from the file into one of
// two pinned staging buffers, and the copy to HBM starts from there.
#include <unistd.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <thread>

#include "internal.h"

namespace spmm {

// Cut the task list into blocks whose column-index range fits a slot.
static void cut_blocks(const std::vector<int4>& tasks, int64_t n_rows, int64_t slot_nnz, std::vector<StreamBlock>& out,
                       int64_t* max_nnz, int64_t* max_rows) {
    auto e0 = [&](size_t t) { return ((int64_t)(uint32_t)tasks[t].z) | ((int64_t)tasks[t].w << 32); };
    const size_t nt = tasks.size() - 1;   // last descriptor is the sentinel
    *max_nnz = 0;
    *max_rows = 0;
    size_t t = 0;
    while (t < nt) {
        StreamBlock b;
        b.t0 = (int64_t)t;
        const int64_t c0 = e0(t) & ~(int64_t)7;
        const int64_t r0 = (int64_t)tasks[t].x & ~(int64_t)1;
        int64_t rmax = tasks[t].x;
        size_t u = t;
        while (u < nt) {
            const int64_t end_nnz = e0(u + 1);
            if (u > t && end_nnz - c0 > slot_nnz) break;
            const int32_t x = tasks[u].y;
            rmax = std::max<int64_t>(rmax, (int64_t)tasks[u].x + (x > 0 ? x : 1));
            ++u;
        }
        b.t1 = (int64_t)u;
        b.c0 = c0;
        b.c1 = e0(u);
        b.r0 = r0;
        b.r1 = std::min<int64_t>(n_rows + 1, rmax + 2);   // the kernel's row-pointer window reads up to r0+x+1
        *max_nnz = std::max(*max_nnz, b.c1 - b.c0);
        *max_rows = std::max(*max_rows, b.r1 - b.r0);
        out.push_back(b);
        t = u;
    }
}

static cudaError_t pin(const void* p, size_t bytes, bool* registered) {
    *registered = false;
    if (!p || bytes == 0) return cudaSuccess;
    // memory that is page-locked already (cudaHostAlloc, or registered by the
    // caller) is used as it is
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost) return cudaSuccess;
    cudaGetLastError();
    cudaError_t e = cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterDefault);
    if (e == cudaErrorHostMemoryAlreadyRegistered) {
        cudaGetLastError();
        return cudaSuccess;
    }
    if (e == cudaSuccess) *registered = true;
    return e;
}

int stream_setup(spmm_mat* A, const int64_t* row_ptr, const int32_t* col_idx, const void* values, size_t vsize,
                 cudaStream_t s) {
    Streamer& S = A->st;
    DevCSR& d = A->fwd;
    const int64_t n = d.n_rows, nnz = d.nnz;
    S.h_row_ptr = row_ptr;
    S.h_col_idx = col_idx;
    S.h_val = values;
    S.fail_block = A->params.fail_block;
    HostPlan plan = build_plan(row_ptr, n, A->params);
    d.short_runs = A->params.short_runs;
    std::copy(plan.walk_eff, plan.walk_eff + 4, d.walk_eff);
    const int64_t slot_nnz = std::max<int64_t>(A->params.slot_bytes / 4, 2 * kMaxTaskNnz + 16);
    int64_t max_nnz = 0, max_rows = 0;
    cut_blocks(plan.tasks, n, slot_nnz, S.blocks, &max_nnz, &max_rows);
    S.slot_nnz = max_nnz + 16;
    S.slot_rows = max_rows + 4;
    cudaError_t e;
    int64_t* bytes = &A->device_bytes;
    auto dmalloc = [&](void** p, size_t b) {
        cudaError_t r = cudaMalloc(p, b);
        if (r == cudaSuccess) *bytes += (int64_t)b;
        return r;
    };
    if (!S.h_rp_owned && (e = pin(row_ptr, (size_t)(n + 1) * 8, &S.reg_rp)) != cudaSuccess)
        return cuda_fail(e, "streaming: pin row_ptr");
    if ((e = pin(col_idx, (size_t)nnz * 4, &S.reg_ci)) != cudaSuccess) return cuda_fail(e, "streaming: pin col_idx");
    if ((e = pin(values, (size_t)nnz * vsize, &S.reg_val)) != cudaSuccess) return cuda_fail(e, "streaming: pin values");
    for (int i = 0; i < 2; ++i) {
        if ((e = dmalloc((void**)&S.slot_col[i], (size_t)S.slot_nnz * 4)) != cudaSuccess ||
            (e = dmalloc((void**)&S.slot_rp[i], (size_t)S.slot_rows * 8)) != cudaSuccess ||
            (vsize > 0 && (e = dmalloc(&S.slot_val[i], (size_t)S.slot_nnz * vsize)) != cudaSuccess))
            return cuda_fail(e, "streaming: staging slots");
    }
    if ((e = cudaStreamCreateWithFlags(&S.copy, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "streaming: copy stream");
    for (int i = 0; i < 2; ++i) {
        if ((e = cudaEventCreateWithFlags(&S.copied[i], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&S.freed[i], cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "streaming: events");
        if ((e = cudaEventRecord(S.freed[i], S.copy)) != cudaSuccess) return cuda_fail(e, "streaming: events");
    }
    // the plan in HBM, as in the resident mode
    if ((e = cudaMalloc((void**)&d.tasks, plan.tasks.size() * sizeof(int4))) != cudaSuccess)
        return cuda_fail(e, "streaming: tasks");
    *bytes += (int64_t)(plan.tasks.size() * sizeof(int4));
    cudaMemcpyAsync(d.tasks, plan.tasks.data(), plan.tasks.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    d.n_tasks = (int64_t)plan.tasks.size() - 1;
    if (!plan.splits.empty()) {
        if ((e = cudaMalloc((void**)&d.splits, plan.splits.size() * sizeof(int4))) != cudaSuccess)
            return cuda_fail(e, "streaming: splits");
        *bytes += (int64_t)(plan.splits.size() * sizeof(int4));
        cudaMemcpyAsync(d.splits, plan.splits.data(), plan.splits.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    }
    d.n_splits = (int64_t)plan.splits.size();
    d.n_segments = plan.n_segments;
    d.n_slots = plan.n_slots;
    if ((e = cudaMalloc((void**)&d.task_ctr, sizeof(unsigned long long))) != cudaSuccess) {
        d.task_ctr = nullptr;
        return cuda_fail(e, "streaming: task counter");
    }
    *bytes += (int64_t)sizeof(unsigned long long);
    if (d.n_slots > 0) {
        if ((e = cudaMalloc((void**)&d.partials, (size_t)d.n_slots * kSlotStride * sizeof(float))) != cudaSuccess)
            return cuda_fail(e, "streaming: partials");
        *bytes += (int64_t)d.n_slots * kSlotStride * sizeof(float);
        if (A->params.compensated) {
            if ((e = cudaMalloc((void**)&d.partials_comp, (size_t)d.n_slots * kSlotStride * sizeof(float))) !=
                cudaSuccess)
                return cuda_fail(e, "streaming: partials");
            *bytes += (int64_t)d.n_slots * kSlotStride * sizeof(float);
        }
    }
    S.bytes_per_apply = nnz * 4 + (int64_t)(nnz * vsize) + (n + 1) * 8;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "streaming: set-up");
    return SPMM_OK;
}

// File source: pinned staging buffers for one block of column indices and
// values each (widened to the file alignment at both ends), used in turn.
int stream_file_setup(spmm_mat* A, cudaStream_t s) {
    Streamer& S = A->st;
    const size_t vsize = S.file.vtype < 0 ? 0 : (S.file.vtype == SPMM_F32 ? 4 : 2);
    cudaError_t e;
    for (int i = 0; i < 2; ++i) {
        if ((e = cudaHostAlloc((void**)&S.stage_col[i], (size_t)S.slot_nnz * 4 + 2 * kFileAlign,
                               cudaHostAllocDefault)) != cudaSuccess ||
            (vsize && (e = cudaHostAlloc((void**)&S.stage_val[i], (size_t)S.slot_nnz * vsize + 2 * kFileAlign,
                                         cudaHostAllocDefault)) != cudaSuccess))
            return cuda_fail(e, "spmm_create_file: staging buffers");
        if ((e = cudaEventCreateWithFlags(&S.staged[i], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventRecord(S.staged[i], S.copy)) != cudaSuccess)
            return cuda_fail(e, "spmm_create_file: events");
    }
    const int hc = (int)std::thread::hardware_concurrency();
    S.readers = std::max(1, std::min(16, hc > 0 ? hc : 8));
    (void)s;
    return SPMM_OK;
}

int stream_apply(const spmm_mat* A, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y, int64_t ldy,
                 cudaStream_t s) {
    const Streamer& S = A->st;
    const DevCSR& d = A->fwd;
    if (d.n_rows == 0) return SPMM_OK;
    const int vmode = value_mode(A, xtype);
    if (vmode < 0) {
        set_error("spmm_apply: 16-bit values need X of the same 16-bit type (or use F32 values)");
        return SPMM_ERR_UNSUPPORTED;
    }
    const size_t vsize = vmode == 0 ? 0 : (vmode == 1 ? 4 : 2);
    FwdArgs a;
    int vec = 1, ch = 1;
    set_geometry(a, X, ldx, k, xtype, Y, ldy, d, &vec, &ch);
    a.partials = d.partials;
    a.n_slots = d.n_slots;
    a.status = A->status;
    a.wait_ns = kWaitNs;
    a.x_evict_last = A->params.x_evict_last;
    a.compensated = d.partials_comp != nullptr || (A->params.compensated && d.n_slots == 0);
    a.partials_comp = d.partials_comp;
    int rc = SPMM_OK;
    cudaError_t e = cudaSuccess;
    for (size_t bi = 0; bi < S.blocks.size(); ++bi) {
        NvtxRange brange("spmm_apply stream block");
        const StreamBlock& b = S.blocks[bi];
        const int slot = (int)(bi & 1);
        if (S.fail_block > 0 && (size_t)(S.fail_block - 1) == bi) {
            set_error("spmm_apply (streaming): injected copy failure before block " + std::to_string(bi));
            rc = SPMM_ERR_CUDA;
            break;
        }
        const int32_t* src_col = S.h_col_idx ? S.h_col_idx + b.c0 : nullptr;
        const char* src_val = S.h_val ? static_cast<const char*>(S.h_val) + b.c0 * vsize : nullptr;
        if (S.file.fd >= 0) {
            // read the block from the file into staging buffer `slot` once the
            // copies out of it (block bi-2) are done; the GPU meanwhile copies
            // and multiplies block bi-1
            if ((e = cudaEventSynchronize(S.staged[slot])) != cudaSuccess) break;
            std::string err;
            src_col = reinterpret_cast<const int32_t*>(
                file_read_range(S.file.fd, S.file.direct, S.file.off_ci + b.c0 * 4, (b.c1 - b.c0) * 4,
                                S.stage_col[slot], S.readers, S.file.n_cols, &err));
            if (src_col && vmode)
                src_val = file_read_range(S.file.fd, S.file.direct, S.file.off_val + b.c0 * (int64_t)vsize,
                                          (b.c1 - b.c0) * (int64_t)vsize, S.stage_val[slot], S.readers, 0, &err);
            if (!src_col || (vmode && !src_val)) {
                set_error("spmm_apply (file): block " + std::to_string(bi) + ": " + err);
                rc = err.rfind("column", 0) == 0 ? SPMM_ERR_FORMAT : SPMM_ERR_IO;
                break;
            }
        }
        // copy block bi into its slot once the kernel that last read the slot is done
        if ((e = cudaStreamWaitEvent(S.copy, S.freed[slot], 0)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(S.slot_col[slot], src_col, (size_t)(b.c1 - b.c0) * 4, cudaMemcpyHostToDevice,
                                 S.copy)) != cudaSuccess)
            break;
        if (vmode && (e = cudaMemcpyAsync(S.slot_val[slot], src_val, (size_t)(b.c1 - b.c0) * vsize,
                                          cudaMemcpyHostToDevice, S.copy)) != cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(S.slot_rp[slot], S.h_row_ptr + b.r0, (size_t)(b.r1 - b.r0) * 8,
                                 cudaMemcpyHostToDevice, S.copy)) != cudaSuccess)
            break;
        if ((e = cudaEventRecord(S.copied[slot], S.copy)) != cudaSuccess) break;
        if (S.file.fd >= 0 && (e = cudaEventRecord(S.staged[slot], S.copy)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(s, S.copied[slot], 0)) != cudaSuccess) break;
        // rebased views: global index i of the block lives at slot offset i - c0 (or i - r0)
        a.col_idx = S.slot_col[slot] - b.c0;
        a.val = vmode ? static_cast<const void*>(static_cast<const char*>(S.slot_val[slot]) - b.c0 * vsize) : nullptr;
        a.row_ptr = S.slot_rp[slot] - b.r0;
        a.tasks = d.tasks + b.t0;
        a.n_tasks = b.t1 - b.t0;
        a.task_ctr = task_counter(d, k, xtype, s, &e, &a.task_chunk);
        if (e != cudaSuccess) break;
        if ((e = launch_rows(a, xtype, vmode, vec, ch, s)) != cudaSuccess) break;
        if ((e = cudaEventRecord(S.freed[slot], s)) != cudaSuccess) break;
    }
    if (rc == SPMM_OK && e == cudaSuccess)
        e = launch_combine(d.splits, d.n_splits, d.partials, Y, ldy, k, s, d.partials_comp);
    if (rc != SPMM_OK || e != cudaSuccess) {
        // drain what was enqueued before reporting, so the slots are idle again
        cudaStreamSynchronize(S.copy);
        cudaStreamSynchronize(s);
        if (rc == SPMM_OK) rc = cuda_fail(e, "spmm_apply (streaming)");
    }
    return rc;
}

void stream_release(spmm_mat* A) {
    Streamer& S = A->st;
    if (S.copy) cudaStreamSynchronize(S.copy);
    for (int i = 0; i < 2; ++i) {
        cudaFree(S.slot_col[i]);
        cudaFree(S.slot_val[i]);
        cudaFree(S.slot_rp[i]);
        if (S.copied[i]) cudaEventDestroy(S.copied[i]);
        if (S.freed[i]) cudaEventDestroy(S.freed[i]);
    }
    if (S.copy) cudaStreamDestroy(S.copy);
    if (S.reg_rp) cudaHostUnregister(const_cast<int64_t*>(S.h_row_ptr));
    if (S.reg_ci) cudaHostUnregister(const_cast<int32_t*>(S.h_col_idx));
    if (S.reg_val) cudaHostUnregister(const_cast<void*>(S.h_val));
    for (int i = 0; i < 2; ++i) {
        cudaFreeHost(S.stage_col[i]);
        cudaFreeHost(S.stage_val[i]);
        if (S.staged[i]) cudaEventDestroy(S.staged[i]);
    }
    cudaFreeHost(S.h_rp_owned);
    if (S.file.fd >= 0) ::close(S.file.fd);
    S = Streamer{};
}

}  // namespace spmm
