// vpart.cu -- Y = A X with X and Y in host memory, in vertical partitions.
//
// Section 3.3: when the dense matrices do not fit in memory they are split
// into vertical partitions (column groups), each kept in row-major order, and
// the SpMM runs once per partition -- one pass over the sparse matrix each.
// Section 3.6: the memory should go to as many input columns as fit, since
// every extra partition is one more pass over A.
//
// Here the memory is HBM, the external medium is host memory, and a partition
// is a group of g columns of X (and the same columns of Y).  Per group:
// a 2-D copy of its columns host -> device (copy-in stream), the task kernel
// on the caller's stream in a few runs of whole tasks (RowBlock), and after
// each run a 2-D copy of its rows of the result device -> host (copy-out
// stream), so a group's result leaves while the rest of it multiplies.  X and
// Y have two device buffers each, so the copy-in of group i+1 and the
// copy-out of group i-1 run while group i multiplies.  The buffers, streams
// and events stay with the handle for later calls.
//
// spmm_apply_host takes ordinary row-major X and Y (any leading dimension) and
// copies each group's columns with strided 2-D copies; spmm_apply_host_parts
// takes the paper's layout, each vertical partition a contiguous row-major
// array, and so moves each group with contiguous copies.
#include <algorithm>
#include <vector>

#include "internal.h"

using namespace spmm;

namespace {

int64_t xbytes_of(int32_t xtype) { return xtype == SPMM_F32 ? 4 : 2; }

// device bytes one column of a group costs: two X buffers and two Y buffers
int64_t bytes_per_col(int64_t n_in, int64_t n_out, int32_t xtype) {
    return 2 * (n_in * xbytes_of(xtype) + n_out * 4);
}

}  // namespace

extern "C" int spmm_vpart_cols(int64_t n_in, int64_t n_out, int32_t p, spmm_dtype xtype, int64_t budget_bytes,
                               int32_t* cols) {
    if (!cols || n_in < 0 || n_out < 0 || p < 1 || budget_bytes < 0 ||
        (xtype != SPMM_F32 && xtype != SPMM_BF16 && xtype != SPMM_F16)) {
        set_error("spmm_vpart_cols: need cols != NULL, n_in, n_out >= 0, p >= 1, budget >= 0, X F32/BF16/F16");
        return SPMM_ERR_ARG;
    }
    const int64_t per = std::max<int64_t>(1, bytes_per_col(n_in, n_out, xtype));
    const int64_t fit = budget_bytes / per;
    if (fit < 1) {
        set_error("spmm_vpart_cols: the budget (" + std::to_string(budget_bytes) + " bytes) holds no column (" +
                  std::to_string(per) + " bytes per column, double-buffered X and Y)");
        return SPMM_ERR_OOM;
    }
    *cols = (int32_t)std::min<int64_t>({fit, (int64_t)p, (int64_t)kMaxK});
    return SPMM_OK;
}

namespace spmm {

// grow-only device buffers and the copy streams/events of spmm_apply_host
static int hostio_setup(spmm_mat* A, size_t xb, size_t yb) {
    HostIO& h = A->hio;
    cudaError_t e;
    if (!h.s_in) {
        if ((e = cudaStreamCreateWithFlags(&h.s_in, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&h.s_out, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "spmm_apply_host: streams");
        for (auto& ev : h.ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "spmm_apply_host: events");
    }
    if (xb > h.x_bytes || yb > h.y_bytes) {
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "spmm_apply_host: pending work");
        for (int b = 0; b < 2; ++b) {
            cudaFree(h.x[b]);
            cudaFree(h.y[b]);
            h.x[b] = nullptr;
            h.y[b] = nullptr;
        }
        h.x_bytes = h.y_bytes = 0;
        for (int b = 0; b < 2; ++b) {
            if ((e = cudaMalloc(&h.x[b], std::max<size_t>(xb, 16))) != cudaSuccess ||
                (e = cudaMalloc((void**)&h.y[b], std::max<size_t>(yb, 16))) != cudaSuccess) {
                for (int c = 0; c < 2; ++c) {
                    cudaFree(h.x[c]);
                    cudaFree(h.y[c]);
                    h.x[c] = nullptr;
                    h.y[c] = nullptr;
                }
                cudaGetLastError();
                return cuda_fail(e, "spmm_apply_host: device buffers");
            }
        }
        h.x_bytes = xb;
        h.y_bytes = yb;
    }
    return SPMM_OK;
}

void hostio_release(spmm_mat* A) {
    HostIO& h = A->hio;
    for (int b = 0; b < 2; ++b) {
        cudaFree(h.x[b]);
        cudaFree(h.y[b]);
    }
    for (auto& ev : h.ev)
        if (ev) cudaEventDestroy(ev);
    if (h.s_in) cudaStreamDestroy(h.s_in);
    if (h.s_out) cudaStreamDestroy(h.s_out);
    h = HostIO{};
}

}  // namespace spmm

namespace {

struct Group {
    const char* x;       // host, first element of the group's columns
    size_t x_pitch;      // bytes between rows
    float* y;
    size_t y_pitch;
    int32_t w;           // columns
};

int check_common(const spmm_mat* A, spmm_dtype xtype, int32_t transpose, const char* who) {
    if (!A) { set_error(std::string(who) + ": A is NULL"); return SPMM_ERR_ARG; }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16 && xtype != SPMM_F16) {
        set_error(std::string(who) + ": X must be F32, BF16 or F16");
        return SPMM_ERR_ARG;
    }
    if (transpose && !A->has_tr) {
        set_error(std::string(who) + ": transpose needs SPMM_WANT_TRANSPOSE at create");
        return SPMM_ERR_ARG;
    }
    if (value_mode(A, xtype) < 0) {
        set_error(std::string(who) + ": 16-bit values need X of the same 16-bit type (or use F32 values)");
        return SPMM_ERR_UNSUPPORTED;
    }
    if (A->relabel) {
        set_error(std::string(who) + ": handles with SPMM_RELABEL take device buffers (spmm_apply)");
        return SPMM_ERR_UNSUPPORTED;
    }
    return SPMM_OK;
}

// rows x width bytes between pitched buffers; one plain copy when both sides
// are contiguous (a 2-D copy moves row by row, which for narrow rows is far
// slower than the link)
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows,
                      cudaMemcpyKind kind, cudaStream_t s) {
    if (dpitch == width && spitch == width) return cudaMemcpyAsync(dst, src, width * rows, kind, s);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, kind, s);
}

// The group pipeline: copy-in on s_in, multiply on s, copy-out on s_out, two
// device buffers each for X and Y.  Returns when every group's Y is on the host.
int run_groups(spmm_mat* A, const std::vector<Group>& groups, int32_t xtype, int32_t transpose, cudaStream_t s) {
    const int64_t n_in = transpose ? A->fwd.n_rows : A->fwd.n_cols;
    const int64_t n_out = transpose ? A->fwd.n_cols : A->fwd.n_rows;
    const int64_t xe = xbytes_of(xtype);
    int32_t wmax = 0;
    for (const Group& gr : groups) wmax = std::max(wmax, gr.w);
    int rc;
    if ((rc = hostio_setup(A, (size_t)(n_in * wmax * xe), (size_t)(n_out * wmax * 4))) != SPMM_OK) return rc;
    HostIO& h = A->hio;
    // events: 0,1 X ready; 2,3 X free; 4,5 Y ready; 6,7 Y free (per buffer)
    cudaEvent_t *x_ready = h.ev, *x_free = h.ev + 2, *y_ready = h.ev + 4, *y_free = h.ev + 6;
    cudaError_t e = cudaSuccess;
    // the copy streams start after the work already queued on the caller's stream
    if ((e = cudaEventRecord(x_free[0], s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h.s_in, x_free[0], 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h.s_out, x_free[0], 0)) != cudaSuccess)
        return cuda_fail(e, "spmm_apply_host: order");
    const int n_groups = (int)groups.size();
    for (int i = 0; i < n_groups; ++i) {
        const int b = i & 1;
        const Group& gr = groups[i];
        const int32_t w = gr.w;
        // copy-in of group i (buffer b is free once group i-2 has multiplied)
        if (i >= 2 && (e = cudaStreamWaitEvent(h.s_in, x_free[b], 0)) != cudaSuccess) break;
        if (n_in > 0 && (e = copy_rows(h.x[b], (size_t)(w * xe), gr.x, gr.x_pitch, (size_t)(w * xe), (size_t)n_in,
                                       cudaMemcpyHostToDevice, h.s_in)) != cudaSuccess)
            break;
        if ((e = cudaEventRecord(x_ready[b], h.s_in)) != cudaSuccess) break;
        // multiply (Y buffer b is free once group i-2 has been copied out),
        // run by run: each run's rows of Y leave while the next run multiplies
        if ((e = cudaStreamWaitEvent(s, x_ready[b], 0)) != cudaSuccess) break;
        if (i >= 2 && (e = cudaStreamWaitEvent(s, y_free[b], 0)) != cudaSuccess) break;
        // copy-out of rows r0 .. r1-1 of group i (the wait takes the event's
        // latest record, so one event serves every run)
        auto rows_out = [&](int64_t r0, int64_t r1) -> int {
            cudaError_t ce = cudaEventRecord(y_ready[b], s);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h.s_out, y_ready[b], 0);
            if (ce == cudaSuccess && r1 > r0)
                ce = copy_rows(reinterpret_cast<char*>(gr.y) + (size_t)r0 * gr.y_pitch, gr.y_pitch,
                               h.y[b] + (size_t)r0 * w, (size_t)(w * 4), (size_t)(w * 4), (size_t)(r1 - r0),
                               cudaMemcpyDeviceToHost, h.s_out);
            return ce == cudaSuccess ? SPMM_OK : cuda_fail(ce, "spmm_apply_host: copy-out");
        };
        if (n_in > 0) {
            if ((rc = apply_dev_runs(A, transpose, h.x[b], w, w, xtype, h.y[b], w, s, rows_out)) != SPMM_OK)
                return rc;
        } else if ((e = cudaMemsetAsync(h.y[b], 0, (size_t)(n_out * w * 4), s)) != cudaSuccess ||
                   (rc = rows_out(0, n_out)) != SPMM_OK) {
            if (rc != SPMM_OK) return rc;
            break;
        }
        if ((e = cudaEventRecord(x_free[b], s)) != cudaSuccess) break;
        if ((e = cudaEventRecord(y_free[b], h.s_out)) != cudaSuccess) break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "spmm_apply_host: group pipeline");
    // the caller's stream continues after the last copy-out; Y is complete on return
    if ((e = cudaStreamWaitEvent(s, y_free[(n_groups - 1) & 1], 0)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h.s_out)) != cudaSuccess)
        return cuda_fail(e, "spmm_apply_host: finish");
    return SPMM_OK;
}

}  // namespace

extern "C" int spmm_apply_host(spmm_mat_t A, const void* X, int64_t ldx, int32_t p, spmm_dtype xtype, float* Y,
                               int64_t ldy, int32_t transpose, int32_t group_cols, int64_t budget_bytes,
                               int32_t* groups_out, void* stream) {
    int rc;
    NvtxRange range("spmm_apply_host");
    if ((rc = check_common(A, xtype, transpose, "spmm_apply_host")) != SPMM_OK) return rc;
    if (p < 1 || ldx < p || ldy < p || group_cols < 0 || group_cols > kMaxK || budget_bytes < 0) {
        set_error("spmm_apply_host: need p >= 1, ldx >= p, ldy >= p, 0 <= group_cols <= 64, budget >= 0");
        return SPMM_ERR_ARG;
    }
    const int64_t n_in = transpose ? A->fwd.n_rows : A->fwd.n_cols;
    const int64_t n_out = transpose ? A->fwd.n_cols : A->fwd.n_rows;
    if (groups_out) *groups_out = 0;
    if (n_out == 0) return SPMM_OK;
    if (!X || !Y) { set_error("spmm_apply_host: X or Y is NULL"); return SPMM_ERR_ARG; }
    int32_t g = group_cols;
    if (g == 0) {
        int64_t budget = budget_bytes;
        if (budget == 0) {
            size_t fr = 0, tot = 0;
            cudaError_t e = cudaMemGetInfo(&fr, &tot);
            if (e != cudaSuccess) return cuda_fail(e, "spmm_apply_host: memory info");
            budget = (int64_t)(fr / 10 * 8);      // leave a fifth of the free memory
            // buffers already held by this handle count as free
            budget += (int64_t)(2 * (A->hio.x_bytes + A->hio.y_bytes));
        }
        if ((rc = spmm_vpart_cols(n_in, n_out, p, xtype, budget, &g)) != SPMM_OK) return rc;
    }
    g = std::min(g, p);
    const int64_t xe = xbytes_of(xtype);
    std::vector<Group> groups;
    for (int32_t c0 = 0; c0 < p; c0 += g)
        groups.push_back(Group{static_cast<const char*>(X) + (size_t)c0 * xe, (size_t)(ldx * xe), Y + c0,
                               (size_t)(ldy * 4), std::min(g, p - c0)});
    if ((rc = run_groups(A, groups, xtype, transpose, (cudaStream_t)stream)) != SPMM_OK) return rc;
    if (groups_out) *groups_out = (int32_t)groups.size();
    return SPMM_OK;
}

extern "C" int spmm_apply_host_parts(spmm_mat_t A, const void* const* X_parts, float* const* Y_parts,
                                     const int32_t* part_cols, int32_t n_parts, spmm_dtype xtype, int32_t transpose,
                                     void* stream) {
    NvtxRange range("spmm_apply_host_parts");
    int rc;
    if ((rc = check_common(A, xtype, transpose, "spmm_apply_host_parts")) != SPMM_OK) return rc;
    if (n_parts < 1 || !X_parts || !Y_parts || !part_cols) {
        set_error("spmm_apply_host_parts: need n_parts >= 1 and the three arrays");
        return SPMM_ERR_ARG;
    }
    const int64_t n_out = transpose ? A->fwd.n_cols : A->fwd.n_rows;
    const int64_t xe = xbytes_of(xtype);
    std::vector<Group> groups;
    for (int32_t i = 0; i < n_parts; ++i) {
        const int32_t w = part_cols[i];
        if (w < 1 || w > kMaxK || !X_parts[i] || !Y_parts[i]) {
            set_error("spmm_apply_host_parts: part " + std::to_string(i) + " needs 1..64 columns and both pointers");
            return SPMM_ERR_ARG;
        }
        groups.push_back(Group{static_cast<const char*>(X_parts[i]), (size_t)(w * xe), Y_parts[i], (size_t)(w * 4), w});
    }
    if (n_out == 0) return SPMM_OK;
    return run_groups(A, groups, xtype, transpose, (cudaStream_t)stream);
}
