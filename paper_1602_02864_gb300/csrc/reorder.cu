// reorder.cu -- SPMM_REORDER: columns relabelled by decreasing degree.
//
// Section 5.1 shows that the vertex order decides how well the gathered rows
// of the dense matrix stay in cache.  With SPMM_REORDER a handle relabels the
// columns of each orientation by decreasing count of stored entries (ties
// keep the original order), so the rows of X that most entries gather sit
// together at the front of X and share L2 sectors and lines.  Rows keep their
// order and each row keeps its stored entry order, so every output element is
// the same sum in the same order: the results are bit-identical to those of a
// handle without the flag given X as a contiguous, aligned array (the layout
// of the relabelled copy; the kernel's vector width follows X's alignment).
// Each apply first gathers X's rows into the new order (one pass over X) in a
// buffer the handle keeps.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace spmm {

void relabel_by_degree(int64_t n_cols, const int32_t* col_idx, int64_t nnz, std::vector<int32_t>& old_of_new,
                       std::vector<int32_t>& relabelled) {
    std::vector<int64_t> cnt((size_t)n_cols, 0);
    for (int64_t p = 0; p < nnz; ++p) cnt[(size_t)col_idx[p]]++;
    int64_t maxc = 0;
    for (int64_t c = 0; c < n_cols; ++c) maxc = std::max(maxc, cnt[(size_t)c]);
    old_of_new.resize((size_t)n_cols);
    std::vector<int32_t> new_of_old((size_t)n_cols);
    if (maxc <= 4 * n_cols + 1024) {
        // counting sort on (maxc - count); a stable pass keeps ties in id order
        std::vector<int64_t> start((size_t)maxc + 2, 0);
        for (int64_t c = 0; c < n_cols; ++c) start[(size_t)(maxc - cnt[(size_t)c]) + 1]++;
        for (int64_t b = 0; b <= maxc; ++b) start[(size_t)b + 1] += start[(size_t)b];
        for (int64_t c = 0; c < n_cols; ++c) {
            const int64_t nw = start[(size_t)(maxc - cnt[(size_t)c])]++;
            old_of_new[(size_t)nw] = (int32_t)c;
        }
    } else {
        for (int64_t c = 0; c < n_cols; ++c) old_of_new[(size_t)c] = (int32_t)c;
        std::stable_sort(old_of_new.begin(), old_of_new.end(),
                         [&](int32_t a, int32_t b) { return cnt[(size_t)a] > cnt[(size_t)b]; });
    }
    for (int64_t nw = 0; nw < n_cols; ++nw) new_of_old[(size_t)old_of_new[(size_t)nw]] = (int32_t)nw;
    relabelled.resize((size_t)nnz);
    for (int64_t p = 0; p < nnz; ++p) relabelled[(size_t)p] = new_of_old[(size_t)col_idx[p]];
}

// Xp[r, :] = X[perm[r], :] in units of V (vpr units per row)
template <typename V>
__global__ void permute_rows_kernel(const V* __restrict__ X, int64_t ldx_v, const int32_t* __restrict__ perm,
                                    int64_t n, int vpr, V* __restrict__ Xp) {
    const int64_t total = n * vpr;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / vpr;
        const int v = (int)(t - r * vpr);
        Xp[t] = __ldg(X + (int64_t)__ldg(perm + r) * ldx_v + v);
    }
}

int reorder_reserve(spmm_mat* A, int64_t n_in, int32_t k, int32_t xtype, cudaStream_t s) {
    const size_t need = (size_t)std::max<int64_t>(n_in, 1) * (size_t)k * (xtype == SPMM_F32 ? 4 : 2);
    if (need <= A->xperm_bytes) return SPMM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "reorder: capture status");
    if (cs != cudaStreamCaptureStatusNone) {
        set_error("reorder: the relabelled-X buffer must grow, which cannot happen during stream capture "
                  "(apply once with this k before capturing)");
        return SPMM_ERR_UNSUPPORTED;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "reorder: pending work");
    pagerank_invalidate(A);   // its graph writes the old buffer
    cudaFree(A->xperm);
    A->xperm = nullptr;
    A->xperm_bytes = 0;
    if ((e = cudaMalloc(&A->xperm, need)) != cudaSuccess) {
        A->xperm = nullptr;
        return cuda_fail(e, "reorder: relabelled-X buffer");
    }
    A->xperm_bytes = need;
    A->device_bytes += (int64_t)need;
    return SPMM_OK;
}

int reorder_x(spmm_mat* A, const DevCSR& d, const void* X, int64_t ldx, int32_t k, int32_t xtype, cudaStream_t s,
              const void** Xp) {
    const int64_t n = d.n_cols;
    int rc = reorder_reserve(A, n, k, xtype, s);
    if (rc != SPMM_OK) return rc;
    const int es = xtype == SPMM_F32 ? 4 : 2;
    const int64_t row_b = (int64_t)k * es, ld_b = ldx * es;
    int vb = 16;
    while (vb > 2 && (row_b % vb || ld_b % vb || (uintptr_t)X % vb)) vb >>= 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int vpr = (int)(row_b / vb);
    const int64_t total = n * vpr;
    const int threads = 256;
    const int64_t want = (total + threads - 1) / threads;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
    switch (vb) {
        case 16:
            permute_rows_kernel<uint4><<<blocks, threads, 0, s>>>(static_cast<const uint4*>(X), ld_b / 16, d.perm, n,
                                                                 vpr, static_cast<uint4*>(A->xperm));
            break;
        case 8:
            permute_rows_kernel<uint2><<<blocks, threads, 0, s>>>(static_cast<const uint2*>(X), ld_b / 8, d.perm, n,
                                                                 vpr, static_cast<uint2*>(A->xperm));
            break;
        case 4:
            permute_rows_kernel<uint32_t><<<blocks, threads, 0, s>>>(static_cast<const uint32_t*>(X), ld_b / 4,
                                                                    d.perm, n, vpr, static_cast<uint32_t*>(A->xperm));
            break;
        default:
            permute_rows_kernel<uint16_t><<<blocks, threads, 0, s>>>(static_cast<const uint16_t*>(X), ld_b / 2,
                                                                    d.perm, n, vpr, static_cast<uint16_t*>(A->xperm));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "reorder: permute kernel");
    *Xp = A->xperm;
    return SPMM_OK;
}

}  // namespace spmm
