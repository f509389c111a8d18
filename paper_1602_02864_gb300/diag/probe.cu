// probe.cu -- measured rates of random row gathers on this GPU.
//
// The SpMM's cost is dominated by gathering one X row per nonzero from
// effectively random addresses, so the bound that matters is the rate of
// random row reads, from L2 when X fits there and from DRAM when it does not,
// rather than the copy bandwidth that the algorithmic-byte roofline divides
// by.  This diagnostic gathers rows of row_bytes (4..256) at uniformly random
// row indices (a multiplicative hash, so every index lies inside the table)
// from a table of table_bytes, with eight loads in flight per lane, and
// reports rows and bytes per second.
//
// spmm_probe_gather_cols replays a matrix's own column-index stream instead:
// one row of a zero table (n_cols rows of row_bytes) per stored entry, in
// storage order, with nothing else of the SpMM (no values, row pointers,
// reductions or stores).  On a power-law graph the hot columns stay in L2,
// so this, not the uniform probe, is the reference rate for that matrix.  It is
// not a bound: its plain gathers keep the hot columns in L2 worse than the
// SpMM's task order does, and from 8-column X rows on the SpMM runs faster.
#include "internal.h"
#include "spmm_probe.h"

namespace spmm {

__device__ __forceinline__ uint32_t probe_hash(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
    return x;
}

// lanes = row_bytes / 4 rounded up to a power of two (<= 64 -> 16-byte loads
// by row_bytes/16 lanes when row_bytes >= 16, 4-byte loads otherwise)
__global__ void probe_gather_kernel(const float* __restrict__ table, uint32_t rows_mask, int row_floats, int lg,
                                    int64_t per_group, float* __restrict__ sink) {
    const int lanes = 1 << lg;
    const int lane = threadIdx.x & 31, li = lane & (lanes - 1);
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> lg;
    float acc = 0.f;
    if (row_floats >= 4) {
        const float4* t4 = reinterpret_cast<const float4*>(table);
        const int vec_per_row = row_floats >> 2;
        for (int64_t i = 0; i < per_group; i += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t r = probe_hash((uint32_t)(group * 1315423911u + (i + u) * 2654435761u)) & rows_mask;
                v[u] = __ldg(t4 + (int64_t)r * vec_per_row + li);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u].x + v[u].y + v[u].z + v[u].w;
        }
    } else {
        for (int64_t i = 0; i < per_group; i += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t r = probe_hash((uint32_t)(group * 1315423911u + (i + u) * 2654435761u)) & rows_mask;
                v[u] = __ldg(table + (int64_t)r * row_floats + (li < row_floats ? li : 0));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u];
        }
    }
    if (acc == 1234.5f) sink[0] = acc;        // keeps the loads alive
}

// groups of `lanes` lanes; each group gathers the row of every ngroups-th
// column index (8 in flight), lane li loading vector li of the row
template <typename V>
__global__ void probe_cols_kernel(const int32_t* __restrict__ col, int64_t nnz, const V* __restrict__ table,
                                  int vec_per_row, int lg, float* __restrict__ sink) {
    const int lane = threadIdx.x & 31, li = lane & ((1 << lg) - 1);
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> lg;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) >> lg;
    const int lv = li < vec_per_row ? li : 0;
    float acc = 0.f;
    for (int64_t b = group; b < nnz; b += 8 * ngroups) {
        int32_t c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t e = b + u * ngroups;
            c[u] = e < nnz ? __ldcs(col + e) : -1;
        }
        V v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c[u] >= 0) v[u] = __ldg(table + (int64_t)c[u] * vec_per_row + lv);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c[u] >= 0) {
                const float* f = reinterpret_cast<const float*>(&v[u]);
#pragma unroll
                for (int j = 0; j < (int)(sizeof(V) / 4); ++j) acc += f[j];
            }
    }
    if (acc == 1234.5f) sink[0] = acc;        // keeps the loads alive
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_probe_gather_cols(spmm_mat_t A, int32_t transpose, int32_t row_bytes, double* rows_per_s,
                                      double* bytes_per_s, void* stream) {
    if (!A || !rows_per_s || !bytes_per_s || row_bytes < 4 || row_bytes > 256 || row_bytes % 4) {
        set_error("spmm_probe_gather_cols: need a handle and row_bytes a multiple of 4 in 4..256");
        return SPMM_ERR_ARG;
    }
    if (A->streaming) {
        set_error("spmm_probe_gather_cols: the column indices of a streaming handle are not resident");
        return SPMM_ERR_UNSUPPORTED;
    }
    if (transpose && !A->has_tr) {
        set_error("spmm_probe_gather_cols: transpose needs SPMM_WANT_TRANSPOSE at create");
        return SPMM_ERR_ARG;
    }
    const DevCSR& M = transpose ? A->tr : A->fwd;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int width = row_bytes % 16 == 0 ? 16 : row_bytes % 8 == 0 ? 8 : 4;
    const int vec_per_row = row_bytes / width;
    int lg = 0;
    while ((1 << lg) < vec_per_row) ++lg;
    const size_t tbytes = (size_t)std::max<int64_t>(M.n_cols, 1) * row_bytes;
    void* table = nullptr;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SPMM_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&table, tbytes)) != cudaSuccess || (e = cudaMalloc((void**)&sink, 64)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        rc = cuda_fail(e, "spmm_probe_gather_cols: workspace");
    } else {
        cudaMemsetAsync(table, 0, tbytes, s);
        const int threads = 512, blocks = sms * 4, reps = 5;
        auto launch = [&]() {
            if (width == 16)
                probe_cols_kernel<float4><<<blocks, threads, 0, s>>>(M.col_idx, M.nnz, (const float4*)table,
                                                                      vec_per_row, lg, sink);
            else if (width == 8)
                probe_cols_kernel<float2><<<blocks, threads, 0, s>>>(M.col_idx, M.nnz, (const float2*)table,
                                                                      vec_per_row, lg, sink);
            else
                probe_cols_kernel<float><<<blocks, threads, 0, s>>>(M.col_idx, M.nnz, (const float*)table,
                                                                     vec_per_row, lg, sink);
        };
        launch();
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
            rc = cuda_fail(e, "spmm_probe_gather_cols: run");
        } else {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double sec = ms * 1e-3 / reps;
            *rows_per_s = (double)M.nnz / sec;
            *bytes_per_s = (double)M.nnz * (row_bytes + 4) / sec;
        }
    }
    cudaFree(table);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

extern "C" int spmm_probe_gather(int64_t table_bytes, int32_t row_bytes, double* rows_per_s, double* bytes_per_s,
                                 void* stream) {
    if (!rows_per_s || !bytes_per_s || row_bytes < 4 || row_bytes > 256 || (row_bytes & (row_bytes - 1)) ||
        table_bytes < 4096 || table_bytes > ((int64_t)64 << 30)) {
        set_error("spmm_probe_gather: need row_bytes a power of two in 4..256 and 4 KiB <= table_bytes <= 64 GiB");
        return SPMM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // rows: the largest power of two that fits the table
    int64_t rows = 1;
    while (rows * 2 * row_bytes <= table_bytes) rows *= 2;
    const int row_floats = row_bytes / 4;
    const int lanes = row_floats >= 4 ? row_floats / 4 : 1;
    int lg = 0;
    while ((1 << lg) < lanes) ++lg;
    float *table = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SPMM_OK;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&table, (size_t)(rows * row_bytes))) != cudaSuccess ||
        (e = cudaMalloc((void**)&sink, 64)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
        (e = cudaEventCreate(&e1)) != cudaSuccess) {
        rc = cuda_fail(e, "spmm_probe_gather: workspace");
    } else {
        cudaMemsetAsync(table, 0, (size_t)(rows * row_bytes), s);
        const int threads = 512, blocks = sms * 4;
        const int64_t groups = (int64_t)blocks * threads / lanes;
        int64_t per = (int64_t)(4e9 / ((double)groups * row_bytes));
        per = std::max<int64_t>(8, per / 8 * 8);
        probe_gather_kernel<<<blocks, threads, 0, s>>>(table, (uint32_t)(rows - 1), row_floats, lg, 8, sink);
        cudaEventRecord(e0, s);
        probe_gather_kernel<<<blocks, threads, 0, s>>>(table, (uint32_t)(rows - 1), row_floats, lg, per, sink);
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
            rc = cuda_fail(e, "spmm_probe_gather: run");
        } else {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double n = (double)groups * (double)per;
            *rows_per_s = n / (ms * 1e-3);
            *bytes_per_s = n * row_bytes / (ms * 1e-3);
        }
    }
    cudaFree(table);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}
