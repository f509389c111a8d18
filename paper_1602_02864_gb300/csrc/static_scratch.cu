// static_scratch.cu -- Y = A X for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework
// that owns all device memory through its own pool, or a real-time loop that
// must not allocate after start-up.  They already hold the matrix, X and Y in
// their own device buffers, but cannot create a handle (creating one copies
// the matrix and allocates the hub-row scratch).  spmm_apply_csr_static runs
// the same task kernel on the caller's arrays and takes its scratch -- the
// partial sums of split hub rows and the status word of the bounded waits --
// from one file-scope __device__ array of fixed size instead.
//
// The array is shared by every call on a device and keeps the previous
// call's contents; nothing in it needs to start at zero except the status
// word, which each call clears.  Calls whose kernels overlap on the GPU race
// on the array, so calls must be ordered (one stream, or synchronised).
#include <algorithm>
#include <mutex>

#include "internal.h"

namespace spmm {

constexpr int64_t kStaticSlots = 16384;   // split-row segments per call (4 MiB)
constexpr int64_t kStaticFloats = kStaticSlots * kSlotStride + 64;   // + status word, padded

static __device__ __align__(256) float g_static_scratch[kStaticFloats];

constexpr int kMaxDevices = 64;
static float* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the static scratch on the current device, looked up once
// per device (a host-side name of a __device__ array is not its address).
static cudaError_t static_scratch_address(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Adds each split row's partials in segment order.  The split table is not
// available here, so the last segment task of a row finds its first slot
// from the task list: every segment but the last has the same length, so the
// number of earlier segments is (e0_last - row_start) / (e0_last - e0_prev).
// A row whose slots would fall outside [0, max_slots) -- a task list that does
// not belong to row_ptr -- is left unwritten and sets kStatusSlotRange.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
combine_from_tasks_kernel(const int4* __restrict__ tasks, int64_t n_tasks, const int64_t* __restrict__ row_ptr,
                          const float* __restrict__ partials, int64_t max_slots, float* __restrict__ Y, int64_t ldy,
                          int32_t k, int32_t* status) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + w;
    if (t >= n_tasks) return;
    const int4 d = tasks[t];
    if (d.y >= 0) return;                               // not a segment
    const int4 dn = tasks[t + 1];
    if (dn.y < 0 && dn.x == d.x) return;                // not the row's last segment
    const int4 dp = t > 0 ? tasks[t - 1] : d;           // a split row has >= 2 segments
    const int64_t e0 = ((int64_t)(uint32_t)d.z) | ((int64_t)d.w << 32);
    const int64_t ep = ((int64_t)(uint32_t)dp.z) | ((int64_t)dp.w << 32);
    const int64_t last = -(int64_t)d.y - 1;
    const int64_t before = (t > 0 && dp.y < 0 && dp.x == d.x && e0 > ep) ? (e0 - row_ptr[d.x]) / (e0 - ep) : -1;
    const int64_t first = last - before;
    if (before < 1 || first < 0 || last >= max_slots) {
        if (lane == 0) atomicOr(status, kStatusSlotRange);
        return;
    }
    for (int c = lane; c < k; c += 32) {
        float acc = 0.f;
        for (int64_t q = first; q <= last; ++q) acc += __ldcg(partials + q * k + c);
        Y[(int64_t)d.x * ldy + c] = acc;
    }
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_apply_csr_static(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                                     const int32_t* col_idx, const void* values, spmm_dtype vtype,
                                     const int32_t* tasks, int64_t n_tasks, int64_t n_segments, const void* X,
                                     int64_t ldx, int32_t k, spmm_dtype xtype, float* Y, int64_t ldy,
                                     void* stream) {
    if (n_rows < 0 || n_rows >= (int64_t)1 << 31 || n_cols < 1 || n_cols >= (int64_t)1 << 31 || nnz < 0 ||
        n_tasks < 0 || n_segments < 0) {
        set_error("spmm_apply_csr_static: bad sizes");
        return SPMM_ERR_ARG;
    }
    if (n_segments > kStaticSlots) {
        set_error("spmm_apply_csr_static: the plan has " + std::to_string(n_segments) +
                  " split-row segments; the static scratch holds at most " + std::to_string(kStaticSlots) +
                  " (use spmm_create_csr / spmm_apply, or a plan with a larger long_row)");
        return SPMM_ERR_ARG;
    }
    if (k < 1 || k > kMaxK || ldx < k || ldy < k) {
        set_error("spmm_apply_csr_static: need 1 <= k <= 64, ldx >= k, ldy >= k");
        return SPMM_ERR_ARG;
    }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16 && xtype != SPMM_F16) {
        set_error("spmm_apply_csr_static: X must be F32, BF16 or F16");
        return SPMM_ERR_ARG;
    }
    int vmode = 0;
    if (values) {
        if (vtype == SPMM_F32) vmode = 1;
        else if (vtype == SPMM_BF16 && xtype == SPMM_BF16) vmode = 2;
        else if (vtype == SPMM_F16 && xtype == SPMM_F16) vmode = 3;
        else {
            set_error("spmm_apply_csr_static: values must be F32, or 16-bit of the same type as X");
            return SPMM_ERR_UNSUPPORTED;
        }
    }
    if (n_rows == 0 || n_tasks == 0) return SPMM_OK;
    if (!row_ptr || !tasks || !X || !Y || (nnz > 0 && !col_idx)) {
        set_error("spmm_apply_csr_static: NULL pointer");
        return SPMM_ERR_ARG;
    }
    float* scratch = nullptr;
    cudaError_t e = static_scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_error(std::string("spmm_apply_csr_static: static scratch address: ") + cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    int32_t* status = reinterpret_cast<int32_t*>(scratch + kStaticSlots * kSlotStride);
    cudaStream_t s = (cudaStream_t)stream;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int32_t), s)) != cudaSuccess) {
        set_error(std::string("spmm_apply_csr_static: clear status: ") + cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    // the same lane geometry as spmm_apply; short-row runs walk whole rows
    // per lane group and nothing is compensated, so the sums of rows on
    // several lanes may be added in another order than on a handle
    const LaneGeometry gm = lane_geometry(X, ldx, k, xtype, Y, ldy);
    FwdArgs a;
    a.row_ptr = row_ptr;
    a.col_idx = col_idx;
    a.val = values;
    a.tasks = reinterpret_cast<const int4*>(tasks);
    a.n_tasks = n_tasks;
    a.partials = scratch;
    a.n_slots = kStaticSlots;
    a.X = X;
    a.ldx = ldx;
    a.Y = Y;
    a.ldy = ldy;
    a.k = k;
    a.lanes_log2 = gm.lanes_log2;
    a.nvec = gm.nvec;
    a.status = status;
    a.wait_ns = kWaitNs;
    a.x_evict_last = 1;
    a.compensated = 0;
    a.partials_comp = nullptr;
    const int vec = gm.vec, ch = gm.ch;
    if (xtype == SPMM_F32) e = launch_rows_f32(a, vmode, vec, ch, s);
    else if (xtype == SPMM_BF16) e = launch_rows_bf16(a, vmode, vec, ch, s);
    else e = launch_rows_f16(a, vmode, vec, ch, s);
    if (e != cudaSuccess) {
        set_error(std::string("spmm_apply_csr_static: task kernel: ") + cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    if (n_segments > 0) {
        const dim3 grid((unsigned)((n_tasks + kWarpsPerBlock - 1) / kWarpsPerBlock));
        combine_from_tasks_kernel<<<grid, kWarpsPerBlock * 32, 0, s>>>(a.tasks, n_tasks, row_ptr, scratch,
                                                                       kStaticSlots, Y, ldy, k, status);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            set_error(std::string("spmm_apply_csr_static: combine kernel: ") + cudaGetErrorString(e));
            return SPMM_ERR_CUDA;
        }
    }
    return SPMM_OK;
}

extern "C" int spmm_static_status(void* stream) {
    float* scratch = nullptr;
    cudaError_t e = static_scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_error(std::string("spmm_static_status: static scratch address: ") + cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    const int32_t* status = reinterpret_cast<const int32_t*>(scratch + kStaticSlots * kSlotStride);
    int32_t st = 0;
    if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess ||
        (e = cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        set_error(std::string("spmm_static_status: ") + cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    if (st & kStatusTimeout) {
        set_error("spmm_static_status: a staging wait of the last call timed out; its Y is incomplete");
        return SPMM_ERR_TIMEOUT;
    }
    if (st & kStatusSlotRange) {
        set_error("spmm_static_status: the last call's task list named a partial slot beyond the static "
                  "scratch (tasks not planned for this row_ptr?); its split rows are missing from Y");
        return SPMM_ERR_FORMAT;
    }
    return SPMM_OK;
}
