// relabel.cu -- SPMM_RELABEL: the vertices of a square matrix renumbered by
// decreasing degree, rows and columns alike.
//
// Section 5.1 shows that the order of the vertices decides how well the rows
// of the dense matrix that the multiplication gathers stay in cache.  With
// SPMM_RELABEL the handle stores B = P A P^T, where P numbers the vertices by
// decreasing total degree (stored entries in the vertex's row plus entries in
// its column; ties in vertex order), and each row of B keeps its entries in
// increasing (new) column order.  The most-gathered rows of X then sit
// together at the front of X and share L2 lines, and the rows of a warp task
// gather from a narrower band of X.  Vectors that stay in the new order for a
// whole computation pay nothing for it (spmm_apply_relabelled; the iterative
// applications permute their vectors once on entry and once on exit);
// spmm_apply keeps the original order by gathering X's rows into the new
// order and Y's rows back, one pass over each.
//
// old_of_new[v'] is the original vertex of new vertex v'; new_of_old is its
// inverse.  A vector in the input order is brought into the handle's order by
// dst[v'] = src[old_of_new[v']] and back by dst[v] = src[new_of_old[v]].
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.h"

namespace spmm {

void relabel_order(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, std::vector<int32_t>& old_of_new) {
    const int64_t nnz = row_ptr[n];
    std::vector<int64_t> deg((size_t)n);
    for (int64_t v = 0; v < n; ++v) deg[(size_t)v] = row_ptr[v + 1] - row_ptr[v];
    for (int64_t p = 0; p < nnz; ++p) deg[(size_t)col_idx[p]]++;
    int64_t maxd = 0;
    for (int64_t v = 0; v < n; ++v) maxd = std::max(maxd, deg[(size_t)v]);
    old_of_new.resize((size_t)n);
    if (maxd <= 4 * n + 1024) {
        // counting sort on (maxd - degree); the stable pass keeps ties in vertex order
        std::vector<int64_t> start((size_t)maxd + 2, 0);
        for (int64_t v = 0; v < n; ++v) start[(size_t)(maxd - deg[(size_t)v]) + 1]++;
        for (int64_t b = 0; b <= maxd; ++b) start[(size_t)b + 1] += start[(size_t)b];
        for (int64_t v = 0; v < n; ++v) old_of_new[(size_t)start[(size_t)(maxd - deg[(size_t)v])]++] = (int32_t)v;
    } else {
        for (int64_t v = 0; v < n; ++v) old_of_new[(size_t)v] = (int32_t)v;
        std::stable_sort(old_of_new.begin(), old_of_new.end(),
                         [&](int32_t a, int32_t b) { return deg[(size_t)a] > deg[(size_t)b]; });
    }
}

int relabel_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const void* values, size_t vsize,
                const std::vector<int32_t>& old_of_new, std::vector<int32_t>& new_of_old, std::vector<int64_t>& rp,
                std::vector<int32_t>& ci, std::vector<char>& val) {
    const int64_t nnz = row_ptr[n];
    try {
        new_of_old.resize((size_t)n);
        rp.assign((size_t)n + 1, 0);
        ci.resize((size_t)nnz);
        if (values) val.resize((size_t)nnz * vsize);
    } catch (const std::bad_alloc&) {
        return SPMM_ERR_OOM;
    }
    for (int64_t v = 0; v < n; ++v) new_of_old[(size_t)old_of_new[(size_t)v]] = (int32_t)v;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t u = old_of_new[(size_t)v];
        rp[(size_t)v + 1] = rp[(size_t)v] + (row_ptr[u + 1] - row_ptr[u]);
    }
    // rows on host threads, in chunks of about equal entries; each row's
    // entries in increasing new column order (equal columns keep their order)
    const int nt = std::max(1, std::min<int>(32, (int)std::thread::hardware_concurrency()));
    const int chunks = nnz < (1 << 20) ? 1 : 8 * nt;
    std::vector<int64_t> bound((size_t)chunks + 1, n);
    bound[0] = 0;
    for (int c = 1; c < chunks; ++c)
        bound[(size_t)c] = std::upper_bound(rp.begin(), rp.end(), nnz * c / chunks) - rp.begin() - 1;
    for (int c = 1; c <= chunks; ++c) bound[(size_t)c] = std::max(bound[(size_t)c], bound[(size_t)c - 1]);
    std::atomic<int> next{0};
    auto worker = [&]() {
        std::vector<std::pair<int32_t, int64_t>> e;
        for (int c; (c = next.fetch_add(1)) < chunks;) {
            for (int64_t v = bound[(size_t)c]; v < bound[(size_t)c + 1]; ++v) {
                const int64_t u = old_of_new[(size_t)v];
                const int64_t p0 = row_ptr[u], p1 = row_ptr[u + 1];
                e.clear();
                for (int64_t p = p0; p < p1; ++p) e.emplace_back(new_of_old[(size_t)col_idx[p]], p);
                std::sort(e.begin(), e.end());
                int64_t q = rp[(size_t)v];
                for (const auto& x : e) {
                    ci[(size_t)q] = x.first;
                    if (values) std::memcpy(&val[(size_t)q * vsize], (const char*)values + x.second * vsize, vsize);
                    ++q;
                }
            }
        }
    };
    if (chunks == 1) {
        worker();
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
        for (auto& t : pool) t.join();
    }
    return SPMM_OK;
}

// dst row r = src row idx[r] (idx == nullptr: row r), n rows of vpr units V
template <typename V>
__global__ void gather_rows_kernel(const V* __restrict__ src, int64_t ld_src, const int32_t* __restrict__ idx,
                                   int64_t n, int vpr, V* __restrict__ dst, int64_t ld_dst) {
    const int64_t total = n * vpr;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / vpr;
        const int u = (int)(t - r * vpr);
        const int64_t sr = idx ? (int64_t)__ldg(idx + r) : r;
        dst[r * ld_dst + u] = __ldg(src + sr * ld_src + u);
    }
}

cudaError_t gather_rows(const void* src, int64_t ld_src, const int32_t* idx, int64_t n, int32_t k, int es, void* dst,
                        int64_t ld_dst, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t row_b = (int64_t)k * es, lds_b = ld_src * es, ldd_b = ld_dst * es;
    int vb = 16;
    while (vb > 2 && (row_b % vb || lds_b % vb || ldd_b % vb || (uintptr_t)src % vb || (uintptr_t)dst % vb)) vb >>= 1;
    if (row_b % vb || lds_b % vb || ldd_b % vb || (uintptr_t)src % vb || (uintptr_t)dst % vb) vb = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int vpr = (int)(row_b / vb);
    const int threads = 256;
    const int64_t want = (n * vpr + threads - 1) / threads;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(sms, 1) * 16));
#define SPMM_GATHER(V, B)                                                                                    \
    gather_rows_kernel<V><<<blocks, threads, 0, s>>>(static_cast<const V*>(src), lds_b / B, idx, n, vpr,     \
                                                     static_cast<V*>(dst), ldd_b / B)
    switch (vb) {
        case 16: SPMM_GATHER(uint4, 16); break;
        case 8: SPMM_GATHER(uint2, 8); break;
        case 4: SPMM_GATHER(uint32_t, 4); break;
        case 2: SPMM_GATHER(uint16_t, 2); break;
        default: SPMM_GATHER(unsigned char, 1); break;
    }
#undef SPMM_GATHER
    return cudaGetLastError();
}

cudaError_t relabel_rows_dev(const spmm_mat* A, const void* src, int64_t ld_src, int32_t k, int es, void* dst,
                             int64_t ld_dst, bool to_handle_order, cudaStream_t s) {
    const int32_t* idx = A->relabel ? (to_handle_order ? A->rl_old_of_new : A->rl_new_of_old) : nullptr;
    return gather_rows(src, ld_src, idx, A->fwd.n_rows, k, es, dst, ld_dst, s);
}

// grow-only device buffer (not during a stream capture)
static int grow(void** buf, size_t* have, size_t need, int64_t* device_bytes, cudaStream_t s, const char* what) {
    if (need <= *have) return SPMM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (cs != cudaStreamCaptureStatusNone) {
        set_error(std::string(what) + ": the buffer must grow, which cannot happen during stream capture "
                                      "(apply once with this k before capturing)");
        return SPMM_ERR_UNSUPPORTED;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, what);
    cudaFree(*buf);
    *device_bytes -= (int64_t)*have;
    *buf = nullptr;
    *have = 0;
    if ((e = cudaMalloc(buf, need)) != cudaSuccess) {
        *buf = nullptr;
        return cuda_fail(e, what);
    }
    *have = need;
    *device_bytes += (int64_t)need;
    return SPMM_OK;
}

int apply_relabel_io(spmm_mat* A, int transpose, const void* X, int64_t ldx, int32_t k, int32_t xtype, float* Y,
                     int64_t ldy, cudaStream_t s) {
    const int64_t n = A->fwd.n_rows;
    const int es = xtype == SPMM_F32 ? 4 : 2;
    int rc = grow(&A->xperm, &A->xperm_bytes, (size_t)std::max<int64_t>(n, 1) * k * es, &A->device_bytes, s,
                  "spmm_apply (relabelled handle): X buffer");
    if (rc == SPMM_OK)
        rc = grow(&A->yperm, &A->yperm_bytes, (size_t)std::max<int64_t>(n, 1) * k * 4, &A->device_bytes, s,
                  "spmm_apply (relabelled handle): Y buffer");
    if (rc != SPMM_OK) return rc;
    cudaError_t e = relabel_rows_dev(A, X, ldx, k, es, A->xperm, k, true, s);
    if (e != cudaSuccess) return cuda_fail(e, "spmm_apply (relabelled handle): X rows");
    rc = apply_dev(A, transpose, A->xperm, k, k, xtype, static_cast<float*>(A->yperm), k, s);
    if (rc != SPMM_OK) return rc;
    e = relabel_rows_dev(A, A->yperm, k, k, 4, Y, ldy, false, s);
    if (e != cudaSuccess) return cuda_fail(e, "spmm_apply (relabelled handle): Y rows");
    return SPMM_OK;
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_relabel_order(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int32_t* old_of_new) {
    set_error("");
    if (n < 1 || n >= (int64_t)1 << 31 || !row_ptr || !old_of_new || (row_ptr[n] > 0 && !col_idx)) {
        set_error("spmm_relabel_order: need 1 <= n < 2^31 and non-NULL arrays");
        return SPMM_ERR_ARG;
    }
    if (row_ptr[0] != 0) { set_error("spmm_relabel_order: row_ptr[0] != 0"); return SPMM_ERR_FORMAT; }
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) {
            set_error("spmm_relabel_order: row_ptr decreases at row " + std::to_string(i));
            return SPMM_ERR_FORMAT;
        }
    for (int64_t p = 0; p < row_ptr[n]; ++p)
        if (col_idx[p] < 0 || (int64_t)col_idx[p] >= n) {
            set_error("spmm_relabel_order: column index out of range at entry " + std::to_string(p));
            return SPMM_ERR_FORMAT;
        }
    std::vector<int32_t> o;
    try {
        relabel_order(n, row_ptr, col_idx, o);
    } catch (const std::bad_alloc&) {
        set_error("spmm_relabel_order: out of host memory");
        return SPMM_ERR_OOM;
    }
    std::memcpy(old_of_new, o.data(), (size_t)n * sizeof(int32_t));
    return SPMM_OK;
}

extern "C" int spmm_get_relabel(spmm_mat_t A, int32_t* old_of_new) {
    if (!A || !old_of_new) { set_error("spmm_get_relabel: NULL argument"); return SPMM_ERR_ARG; }
    const int64_t n = A->fwd.n_rows;
    if (!A->relabel) {
        for (int64_t v = 0; v < n; ++v) old_of_new[v] = (int32_t)v;
        return SPMM_OK;
    }
    const cudaError_t e = cudaMemcpy(old_of_new, A->rl_old_of_new, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPMM_OK : cuda_fail(e, "spmm_get_relabel");
}

extern "C" int spmm_relabel_rows(spmm_mat_t A, const void* src, int64_t ld_src, int32_t k, spmm_dtype dtype,
                                 void* dst, int64_t ld_dst, int32_t to_handle_order, void* stream) {
    if (!A || !src || !dst) { set_error("spmm_relabel_rows: NULL argument"); return SPMM_ERR_ARG; }
    if (A->fwd.n_rows != A->fwd.n_cols) {
        set_error("spmm_relabel_rows: the handle's matrix is not square, so it has no vertex order");
        return SPMM_ERR_ARG;
    }
    if (k < 1 || ld_src < k || ld_dst < k) { set_error("spmm_relabel_rows: need k >= 1 and ld >= k"); return SPMM_ERR_ARG; }
    if (dtype != SPMM_F32 && dtype != SPMM_BF16 && dtype != SPMM_F16 && dtype != SPMM_F64) {
        set_error("spmm_relabel_rows: dtype must be F32, BF16, F16 or F64");
        return SPMM_ERR_ARG;
    }
    if (src == dst) { set_error("spmm_relabel_rows: src and dst must not alias"); return SPMM_ERR_ARG; }
    const int es = dtype == SPMM_F64 ? 8 : (dtype == SPMM_F32 ? 4 : 2);
    const cudaError_t e = relabel_rows_dev(A, src, ld_src, k, es, dst, ld_dst,
                                           to_handle_order != 0, (cudaStream_t)stream);
    return e == cudaSuccess ? SPMM_OK : cuda_fail(e, "spmm_relabel_rows");
}
