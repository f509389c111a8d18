// hot.cu -- the most-referenced columns of an orientation and their compact
// copy of X.
//
// The paper's largest compute gain comes from keeping the dense rows a tile
// touches in cache (Section 3.4, Algorithm 1's tiles; Section 5.4 cache
// blocking).  On a power-law graph most stored entries point at a few
// columns.  At create, each orientation ranks its columns by stored entries
// and keeps a second copy of its column indices in which an entry of one of
// the H most-referenced columns ("hot" columns) is ~slot, slot = the
// column's rank (0 = most referenced).  A call whose X rows take 4 bytes
// (k = 1 float32, k = 2 bf16/f16) first copies the H hot rows of X into a
// packed buffer; the hot variant (one block of 24 warps per SM) copies that
// buffer into shared memory once per block and gathers hot rows from there,
// so only the other gathers use the L1-to-L2 request path, which bounds the
// k = 1 product (78% busy on R-MAT).  The 8192 hottest columns take 21% of
// R-MAT scale 24's entries; the product runs 10% faster with them (the
// shared memory they take is L1 that the other gathers lose).  The sums and
// their order are unchanged: only the address a row is read from differs.
#include <algorithm>
#include <functional>
#include <numeric>
#include <thread>
#include <vector>

#include "rows_kernel.cuh"

namespace spmm {

int64_t hot_capacity(int vmode) {
    int dev = 0, opt = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&opt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    const int64_t stage = (int64_t)kHotWarps * (vmode ? Layout<1>::kWarp : Layout<0>::kWarp);
    const int64_t room = (int64_t)opt - stage - 16;
    return room > 0 ? (room / kHotRowBytes) & ~(int64_t)3 : 0;
}

static void parallel_for_chunks(int64_t n, const std::function<void(int64_t, int64_t)>& f) {
    const int nt = std::max(1, std::min<int>(32, (int)std::thread::hardware_concurrency()));
    if (nt == 1 || n < (1 << 20)) {
        f(0, n);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt); });
    for (auto& th : pool) th.join();
}

int64_t hot_select(int64_t n_cols, const int32_t* col_idx, int64_t nnz, const int64_t* counts_in, int64_t max_hot,
                   std::vector<int32_t>& hot_cols, std::vector<int32_t>& encoded) {
    hot_cols.clear();
    if (max_hot <= 0 || nnz == 0) return 0;
    std::vector<int64_t> cnt;
    if (counts_in) {
        cnt.assign(counts_in, counts_in + n_cols);
    } else {
        cnt.assign((size_t)n_cols, 0);
        for (int64_t p = 0; p < nnz; ++p) ++cnt[(size_t)col_idx[p]];
    }
    // columns with at least two entries, most entries first, ties by id
    std::vector<int32_t> cand;
    cand.reserve((size_t)n_cols);
    for (int64_t c = 0; c < n_cols; ++c)
        if (cnt[(size_t)c] >= 2) cand.push_back((int32_t)c);
    const int64_t H = std::min<int64_t>(max_hot, (int64_t)cand.size());
    if (H == 0) return 0;
    auto hotter = [&](int32_t a, int32_t b) {
        return cnt[(size_t)a] != cnt[(size_t)b] ? cnt[(size_t)a] > cnt[(size_t)b] : a < b;
    };
    if (H < (int64_t)cand.size()) std::nth_element(cand.begin(), cand.begin() + H, cand.end(), hotter);
    cand.resize((size_t)H);
    std::sort(cand.begin(), cand.end(), hotter);
    hot_cols.assign(cand.begin(), cand.end());
    std::vector<int32_t> slot((size_t)n_cols, -1);
    for (int64_t s = 0; s < H; ++s) slot[(size_t)hot_cols[(size_t)s]] = (int32_t)s;
    encoded.resize((size_t)nnz);
    parallel_for_chunks(nnz, [&](int64_t lo, int64_t hi) {
        for (int64_t p = lo; p < hi; ++p) {
            const int32_t c = col_idx[p];
            const int32_t s = slot[(size_t)c];
            encoded[(size_t)p] = s >= 0 ? ~s : c;
        }
    });
    return H;
}

// Xh[s, 0:k] = X[hot_cols[s], 0:k], W-byte words (W divides the row bytes,
// X's address and its row stride in bytes).
template <typename W>
__global__ void hot_gather_kernel(const char* __restrict__ X, int64_t ldx_bytes, const int32_t* __restrict__ hot_cols,
                                  int64_t n_hot, int words_per_row, W* __restrict__ Xh) {
    const int64_t total = n_hot * words_per_row;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / words_per_row;
        const int w = (int)(i - s * words_per_row);
        const int64_t c = hot_cols[s];
        Xh[i] = __ldg(reinterpret_cast<const W*>(X + c * ldx_bytes) + w);
    }
}

cudaError_t hot_gather(const DevCSR& d, const void* X, int64_t ldx, int32_t k, int esize, cudaStream_t s) {
    if (d.n_hot <= 0) return cudaSuccess;
    const int64_t row_bytes = (int64_t)k * esize, ld_bytes = ldx * esize;
    const uintptr_t xa = (uintptr_t)X;
    int w = 16;
    while (w > esize && (row_bytes % w || ld_bytes % w || xa % w)) w >>= 1;
    const int wpr = (int)(row_bytes / w);
    const int64_t total = d.n_hot * wpr;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (total + 255) / 256;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    const char* Xc = static_cast<const char*>(X);
    switch (w) {
        case 16: hot_gather_kernel<uint4><<<grid, 256, 0, s>>>(Xc, ld_bytes, d.hot_cols, d.n_hot, wpr, (uint4*)d.xh); break;
        case 8: hot_gather_kernel<uint2><<<grid, 256, 0, s>>>(Xc, ld_bytes, d.hot_cols, d.n_hot, wpr, (uint2*)d.xh); break;
        case 4: hot_gather_kernel<uint32_t><<<grid, 256, 0, s>>>(Xc, ld_bytes, d.hot_cols, d.n_hot, wpr, (uint32_t*)d.xh); break;
        default: hot_gather_kernel<uint16_t><<<grid, 256, 0, s>>>(Xc, ld_bytes, d.hot_cols, d.n_hot, wpr, (uint16_t*)d.xh); break;
    }
    return cudaGetLastError();
}

}  // namespace spmm
