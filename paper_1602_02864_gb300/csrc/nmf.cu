// nmf.cu -- non-negative matrix factorisation on the SpMM path (Section 4.3).
//
// The multiplicative update rules of Section 4.3 (Lee and Seung), H first,
// then W, with H stored transposed (Ht, one row per column of A):
//   Ht <- Ht o (A^T W) / (Ht (W^T W) + eps)
//   W  <- W  o (A Ht)  / (W (Ht^T Ht) + eps)
// The two sparse products run through the task kernel (A^T W on the
// transposed copy), so every step is two SpMMs plus two k x k Gram matrices
// and two row-local updates.  The objective ||A - W H||_F^2 is tracked
// without forming W H:  ||A||^2 - 2 sum(W o (A Ht)) + tr((W^T W)(Ht^T Ht)).
//
// Batched handles (spmm_create_batched) hold one block-diagonal matrix, so
// the SpMMs cover every graph at once while the Grams, updates and objective
// are kept per graph: rows are cut into chunks that never cross a graph
// boundary, each chunk gives FP64 partial sums, and a per-graph pass adds the
// partials in chunk order (deterministic).  Gram products are summed in FP32
// over tiles of 32 rows and the tile sums in FP64 (the GPU's FP64 rate is low).
// All steps are captured into one CUDA graph.
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"

namespace spmm {

constexpr int kNmfThreads = 256;
constexpr int kChunkRows = 2048;
constexpr int kTileRows = 32;

// Fixed-order block sum of a double; result valid in thread 0.
__device__ __forceinline__ double nmf_block_sum(double v, double* sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    __syncthreads();
    return s;
}

// partial[c][r*k + s] = sum over the chunk's rows of M[i][r] * M[i][s]
__global__ void __launch_bounds__(kNmfThreads)
gram_partial_kernel(const float* __restrict__ M, int k, const int4* __restrict__ chunks, double* __restrict__ partial) {
    __shared__ float tile[kTileRows * kMaxK];
    const int4 ch = chunks[blockIdx.x];        // {graph, begin, end, 0}
    const int kk = k * k;
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    for (int64_t r0 = ch.y; r0 < ch.z; r0 += kTileRows) {
        const int rows = (int)min((int64_t)kTileRows, (int64_t)ch.z - r0);
        for (int i = threadIdx.x; i < rows * k; i += blockDim.x) tile[i] = M[r0 * k + i];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int e = threadIdx.x + j * kNmfThreads;
            if (e < kk) {
                const int r = e / k, s = e % k;
                float f = 0.f;
                for (int t = 0; t < rows; ++t) f = fmaf(tile[t * k + r], tile[t * k + s], f);
                acc[j] += (double)f;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int e = threadIdx.x + j * kNmfThreads;
        if (e < kk) partial[(int64_t)blockIdx.x * kk + e] = acc[j];
    }
}

// G[g] = sum of graph g's chunk partials, in chunk order
__global__ void gram_reduce_kernel(const double* __restrict__ partial, const int2* __restrict__ graph_chunks, int k,
                                   double* __restrict__ G) {
    const int g = blockIdx.x;
    const int2 gc = graph_chunks[g];           // {first chunk, chunk count}
    const int kk = k * k;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < gc.y; ++c) s += partial[(int64_t)(gc.x + c) * kk + e];
        G[(int64_t)g * kk + e] = s;
    }
}

// M[i][a] <- M[i][a] * Num[i][a] / (sum_q M[i][q] G[q][a] + eps), row by row
__global__ void __launch_bounds__(kNmfThreads)
nmf_update_kernel(float* __restrict__ M, const float* __restrict__ Num, const double* __restrict__ G, int k,
                  const int4* __restrict__ chunks, float eps) {
    __shared__ float g_s[kMaxK * kMaxK];
    __shared__ float row_s[kNmfThreads];
    const int4 ch = chunks[blockIdx.x];
    const int kk = k * k;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) g_s[e] = (float)G[(int64_t)ch.x * kk + e];
    const int rows_per = kNmfThreads / k;      // rows handled per pass
    const int lr = threadIdx.x / k, a = threadIdx.x % k;
    __syncthreads();
    for (int64_t r0 = ch.y; r0 < ch.z; r0 += rows_per) {
        const int64_t i = r0 + lr;
        const bool on = lr < rows_per && i < ch.z;
        if (on) row_s[lr * k + a] = M[i * k + a];
        __syncthreads();
        if (on) {
            float den = 0.f;
            for (int q = 0; q < k; ++q) den = fmaf(row_s[lr * k + q], g_s[q * k + a], den);
            M[i * k + a] = row_s[lr * k + a] * (Num[i * k + a] / (den + eps));
        }
        __syncthreads();
    }
}

// partial[c] = sum over the chunk's rows of sum_a W[i][a] * AH[i][a]
__global__ void __launch_bounds__(kNmfThreads)
nmf_cross_kernel(const float* __restrict__ W, const float* __restrict__ AH, int k, const int4* __restrict__ chunks,
                 double* __restrict__ partial) {
    __shared__ double sh[32];
    const int4 ch = chunks[blockIdx.x];
    double acc = 0.0;
    for (int64_t i = ch.y + threadIdx.x; i < ch.z; i += blockDim.x) {
        float f = 0.f;
        for (int a = 0; a < k; ++a) f = fmaf(W[i * k + a], AH[i * k + a], f);
        acc += (double)f;
    }
    const double s = nmf_block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// obj[g] = ||A_g||^2 - 2 * sum(cross partials of g) + tr(GW_g GH_g)
__global__ void nmf_objective_kernel(const double* __restrict__ cross, const int2* __restrict__ graph_chunks,
                                     const double* __restrict__ GW, const double* __restrict__ GH,
                                     const double* __restrict__ a2, int k, double* __restrict__ obj, int64_t stride) {
    __shared__ double sh[32];
    const int g = blockIdx.x;
    const int kk = k * k;
    double q = 0.0;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
        const int r = e / k, s = e % k;
        q += GW[(int64_t)g * kk + r * k + s] * GH[(int64_t)g * kk + s * k + r];
    }
    const double quad = nmf_block_sum(q, sh);
    if (threadIdx.x == 0) {
        const int2 gc = graph_chunks[g];
        double c = 0.0;
        for (int i = 0; i < gc.y; ++i) c += cross[gc.x + i];
        obj[(int64_t)g * stride] = a2[g] - 2.0 * c + quad;
    }
}

// ---- ranks k = 8, 16, 32, 64 with 16-byte aligned factors: the same sums
// organised for the memory system (the kernels above stage 32 or 16 rows at a
// time behind block barriers and wait on every global load).

// Gram partials, register-blocked: thread t owns the 4 x 4 block ob of the
// K x K Gram (OB = (K/4)^2 blocks) and the rows rg, rg + RG, ... (RG =
// 256 / OB row groups) of each tile of T = 4096 / K rows.  Tiles are staged
// in shared memory from float4 loads issued one tile ahead (double buffer,
// one barrier per tile); products are summed in FP32 over at most
// kGramPromote rows per thread, then added to FP64; at the end the row
// groups' FP64 blocks are added in row-group order behind one barrier.
constexpr int kGramPromote = 128;

template <int K>
__global__ void __launch_bounds__(kNmfThreads, 3)
gram_partial_blocked_kernel(const float* __restrict__ M, const int4* __restrict__ chunks,
                            double* __restrict__ partial) {
    constexpr int NB = K / 4, OB = NB * NB, RG = kNmfThreads / OB;
    constexpr int T = 4096 / K;                    // rows per tile (4096 floats)
    constexpr int TV = T * K / 4;                  // float4 per tile
    constexpr int PV = TV / kNmfThreads;           // float4 per thread per tile
    static_assert(TV % kNmfThreads == 0 && RG >= 1 && T % RG == 0, "tile shape");
    __shared__ __align__(16) float tile[2][4096];
    const int4 ch = chunks[blockIdx.x];
    const int t = threadIdx.x, ob = t % OB, rg = t / OB;
    const int rb = (ob / NB) * 4, sb = (ob % NB) * 4;
    float a32[16];
    double a64[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a32[j] = 0.f, a64[j] = 0.0;
    int since = 0;
    const int64_t r_begin = ch.y, r_end = ch.z;
    const int64_t ntiles = (r_end - r_begin + T - 1) / T;
    float4 pre[PV];
    auto load = [&](int64_t ti) {
        const int64_t r0 = r_begin + ti * T;
        const int64_t nv = min((int64_t)T, r_end - r0) * (K / 4);   // float4 of real rows
        const float4* src = reinterpret_cast<const float4*>(M + r0 * K);
#pragma unroll
        for (int p = 0; p < PV; ++p) {
            const int v = t + p * kNmfThreads;
            pre[p] = v < nv ? __ldg(src + v) : make_float4(0.f, 0.f, 0.f, 0.f);   // rows past the end add 0
        }
    };
    if (ntiles > 0) load(0);
    for (int64_t ti = 0; ti < ntiles; ++ti) {
        float* tb = tile[ti & 1];
#pragma unroll
        for (int p = 0; p < PV; ++p) reinterpret_cast<float4*>(tb)[t + p * kNmfThreads] = pre[p];
        __syncthreads();
        if (ti + 1 < ntiles) load(ti + 1);
        for (int r = rg; r < T; r += RG) {
            const float4 x = *reinterpret_cast<const float4*>(tb + r * K + rb);
            const float4 y = *reinterpret_cast<const float4*>(tb + r * K + sb);
            const float xr[4] = {x.x, x.y, x.z, x.w}, yr[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a32[i * 4 + j] = fmaf(xr[i], yr[j], a32[i * 4 + j]);
            if (++since == kGramPromote) {
#pragma unroll
                for (int j = 0; j < 16; ++j) a64[j] += (double)a32[j], a32[j] = 0.f;
                since = 0;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) a64[j] += (double)a32[j];
    // every row group's FP64 block into shared memory (RG x K x K doubles =
    // 32 KB, the tiles' space), then each element added over the row groups
    // in row-group order
    static_assert(RG * K * K * (int)sizeof(double) == (int)sizeof(tile), "row-group blocks fill the tiles' space");
    double* red = reinterpret_cast<double*>(&tile[0][0]);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) red[rg * K * K + (rb + i) * K + sb + j] = a64[i * 4 + j];
    __syncthreads();
    for (int e = t; e < K * K; e += kNmfThreads) {
        double sum = 0.0;
        for (int g = 0; g < RG; ++g) sum += red[g * K * K + e];
        partial[(int64_t)blockIdx.x * K * K + e] = sum;
    }
}

// The update of nmf_update_kernel, warp by warp: a row sits on L = min(K, 32)
// lanes (E = K / L elements each); den is formed with the row's elements
// passed by shuffles, in the same order and the same FP32 operations as
// nmf_update_kernel, four row groups in flight per warp; no block barrier
// after the Gram is staged.
template <int K>
__global__ void __launch_bounds__(kNmfThreads)
nmf_update_warp_kernel(float* __restrict__ M, const float* __restrict__ Num, const double* __restrict__ G,
                       const int4* __restrict__ chunks, float eps) {
    constexpr int L = K < 32 ? K : 32, E = K / L, RPW = 32 / L, U = 4;
    __shared__ float g_s[K * K];
    const int4 ch = chunks[blockIdx.x];
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) g_s[e] = (float)G[(int64_t)ch.x * K * K + e];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = lane / L, li = lane % L;
    const int nw = blockDim.x >> 5;
    for (int64_t base = ch.y + (int64_t)warp * RPW * U; base < ch.z; base += (int64_t)nw * RPW * U) {
        float m[U][E], num[U][E];
        bool on[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * RPW + sub;
            on[u] = i < ch.z;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                m[u][e] = on[u] ? M[i * K + li + e * L] : 0.f;
                num[u][e] = on[u] ? Num[i * K + li + e * L] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float den[E];
#pragma unroll
            for (int e = 0; e < E; ++e) den[e] = 0.f;
#pragma unroll
            for (int e2 = 0; e2 < E; ++e2)
                for (int q = 0; q < L; ++q) {
                    const float mq = __shfl_sync(0xffffffffu, m[u][e2], q, L);
#pragma unroll
                    for (int e = 0; e < E; ++e) den[e] = fmaf(mq, g_s[(q + e2 * L) * K + li + e * L], den[e]);
                }
            if (on[u]) {
                const int64_t i = base + u * RPW + sub;
#pragma unroll
                for (int e = 0; e < E; ++e) M[i * K + li + e * L] = m[u][e] * (num[u][e] / (den[e] + eps));
            }
        }
    }
}

// nmf_cross_kernel as one flat dot product over the chunk's elements (its rows
// are contiguous): float4 loads, four products in FP32, FP64 per thread,
// then the fixed-order block sum.
__global__ void __launch_bounds__(kNmfThreads)
nmf_cross_flat_kernel(const float* __restrict__ W, const float* __restrict__ AH, int k,
                      const int4* __restrict__ chunks, double* __restrict__ partial) {
    __shared__ double sh[32];
    const int4 ch = chunks[blockIdx.x];
    const int64_t e0 = (int64_t)ch.y * k, nv = ((int64_t)ch.z - ch.y) * k / 4;
    const float4* w4 = reinterpret_cast<const float4*>(W + e0);
    const float4* a4 = reinterpret_cast<const float4*>(AH + e0);
    double acc = 0.0;
#pragma unroll 4
    for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
        const float4 w = __ldg(w4 + v), a = __ldg(a4 + v);
        acc += (double)fmaf(w.w, a.w, fmaf(w.z, a.z, fmaf(w.y, a.y, w.x * a.x)));
    }
    const double s = nmf_block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// Chunks of at most kChunkRows rows that never cross a graph boundary.
static void make_chunks(const std::vector<int64_t>& off, std::vector<int4>& chunks, std::vector<int2>& per_graph) {
    chunks.clear();
    per_graph.clear();
    for (size_t g = 0; g + 1 < off.size(); ++g) {
        const int first = (int)chunks.size();
        for (int64_t r = off[g]; r < off[g + 1]; r += kChunkRows)
            chunks.push_back(make_int4((int)g, (int)r, (int)std::min(off[g + 1], r + kChunkRows), 0));
        if (off[g + 1] == off[g]) chunks.push_back(make_int4((int)g, (int)off[g], (int)off[g], 0));
        per_graph.push_back(make_int2(first, (int)chunks.size() - first));
    }
}

}  // namespace spmm

using namespace spmm;

static int nmf_impl(spmm_mat_t A, int32_t k, int32_t steps, float* W, float* Ht, spmm_dtype ftype, double eps,
                    double* objective, void* stream) {
    if (!A || !W || !Ht) { set_error("spmm_nmf: NULL argument"); return SPMM_ERR_ARG; }
    NvtxRange range("spmm_nmf");
    if (k < 1 || k > kMaxK || steps < 0 || !(eps >= 0.0)) {
        set_error("spmm_nmf: need 1 <= k <= 64, steps >= 0, eps >= 0");
        return SPMM_ERR_ARG;
    }
    if (!A->has_tr) { set_error("spmm_nmf: needs SPMM_WANT_TRANSPOSE at create (W^T A)"); return SPMM_ERR_ARG; }
    if (ftype != SPMM_F32 && ftype != SPMM_BF16) { set_error("spmm_nmf: ftype must be F32 or BF16"); return SPMM_ERR_ARG; }
    if (ftype == SPMM_BF16 && (A->vtype == SPMM_F16)) {
        set_error("spmm_nmf: F16 values need F32 factors");
        return SPMM_ERR_UNSUPPORTED;
    }
    if (ftype == SPMM_F32 && (A->vtype == SPMM_BF16 || A->vtype == SPMM_F16)) {
        set_error("spmm_nmf: 16-bit values need factors of the same type");
        return SPMM_ERR_UNSUPPORTED;
    }
    const int ng = (int)A->row_off.size() - 1;
    const int64_t nr = A->fwd.n_rows, nc = A->fwd.n_cols;
    std::vector<int4> chW, chH;
    std::vector<int2> gW, gH;
    make_chunks(A->row_off, chW, gW);
    make_chunks(A->col_off, chH, gH);
    const int kk = k * k;
    const int64_t ostride = (int64_t)steps + 1;
    cudaStream_t user = (cudaStream_t)stream;
    // workspace
    int4 *dchW = nullptr, *dchH = nullptr;
    int2 *dgW = nullptr, *dgH = nullptr;
    double *part = nullptr, *GW = nullptr, *GH = nullptr, *cross = nullptr, *da2 = nullptr, *dobj = nullptr;
    float *AtW = nullptr, *AH = nullptr;
    __nv_bfloat16* fb = nullptr;     // bf16 copy of the factor fed to the SpMM
    cudaStream_t s = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = SPMM_OK;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err, const char* what) { rc = cuda_fail(err, what); };
    const size_t nch = std::max(chW.size(), chH.size());
    do {
        if ((e = cudaStreamSynchronize(user)) != cudaSuccess) { fail(e, "spmm_nmf: stream"); break; }
        if ((e = cudaMalloc((void**)&dchW, chW.size() * sizeof(int4))) != cudaSuccess ||
            (e = cudaMalloc((void**)&dchH, chH.size() * sizeof(int4))) != cudaSuccess ||
            (e = cudaMalloc((void**)&dgW, gW.size() * sizeof(int2))) != cudaSuccess ||
            (e = cudaMalloc((void**)&dgH, gH.size() * sizeof(int2))) != cudaSuccess ||
            (e = cudaMalloc((void**)&part, nch * kk * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&GW, (size_t)ng * kk * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&GH, (size_t)ng * kk * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&cross, chW.size() * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&da2, (size_t)ng * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&dobj, (size_t)ng * ostride * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&AtW, (size_t)std::max<int64_t>(nc, 1) * k * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&AH, (size_t)std::max<int64_t>(nr, 1) * k * sizeof(float))) != cudaSuccess ||
            (ftype == SPMM_BF16 &&
             (e = cudaMalloc((void**)&fb, (size_t)std::max(nr, nc) * k * sizeof(__nv_bfloat16))) != cudaSuccess)) {
            fail(e, "spmm_nmf: workspace");
            break;
        }
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) { fail(e, "spmm_nmf: stream"); break; }
        cudaMemcpyAsync(dchW, chW.data(), chW.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dchH, chH.data(), chH.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dgW, gW.data(), gW.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dgH, gH.data(), gH.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
        if ((e = cudaMemcpyAsync(da2, A->a2.data(), (size_t)ng * sizeof(double), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess) { fail(e, "spmm_nmf: upload"); break; }
        const unsigned nbW = (unsigned)chW.size(), nbH = (unsigned)chH.size();
        const float feps = (float)eps;
        const int spmm_x = ftype == SPMM_BF16 ? SPMM_BF16 : SPMM_F32;
        // one SpMM with the factor as X (converted to bf16 first if asked)
        auto spmm = [&](int transpose, const float* F, int64_t frows, float* out) -> int {
            const void* X = F;
            if (ftype == SPMM_BF16) {
                to_bf16_kernel<<<1216, 256, 0, s>>>(F, fb, frows * k);
                X = fb;
            }
            return apply_dev(A, transpose, X, k, k, spmm_x, out, k, s);
        };
        // ranks 8, 16, 32, 64 with 16-byte aligned factors take the blocked Gram,
        // the warp-level update and the flat cross term
        const bool blocked = (k == 8 || k == 16 || k == 32 || k == 64) && ((uintptr_t)W & 15) == 0 &&
                             ((uintptr_t)Ht & 15) == 0;
        auto gram = [&](const float* M, bool wside, double* G) {
            const unsigned nb = wside ? nbW : nbH;
            const int4* chs = wside ? dchW : dchH;
            if (!blocked) gram_partial_kernel<<<nb, kNmfThreads, 0, s>>>(M, k, chs, part);
            else if (k == 8) gram_partial_blocked_kernel<8><<<nb, kNmfThreads, 0, s>>>(M, chs, part);
            else if (k == 16) gram_partial_blocked_kernel<16><<<nb, kNmfThreads, 0, s>>>(M, chs, part);
            else if (k == 32) gram_partial_blocked_kernel<32><<<nb, kNmfThreads, 0, s>>>(M, chs, part);
            else gram_partial_blocked_kernel<64><<<nb, kNmfThreads, 0, s>>>(M, chs, part);
            gram_reduce_kernel<<<ng, kNmfThreads, 0, s>>>(part, wside ? dgW : dgH, k, G);
        };
        auto update = [&](float* M, const float* Num, const double* G, bool wside) {
            const unsigned nb = wside ? nbW : nbH;
            const int4* chs = wside ? dchW : dchH;
            if (!blocked) nmf_update_kernel<<<nb, kNmfThreads, 0, s>>>(M, Num, G, k, chs, feps);
            else if (k == 8) nmf_update_warp_kernel<8><<<nb, kNmfThreads, 0, s>>>(M, Num, G, chs, feps);
            else if (k == 16) nmf_update_warp_kernel<16><<<nb, kNmfThreads, 0, s>>>(M, Num, G, chs, feps);
            else if (k == 32) nmf_update_warp_kernel<32><<<nb, kNmfThreads, 0, s>>>(M, Num, G, chs, feps);
            else nmf_update_warp_kernel<64><<<nb, kNmfThreads, 0, s>>>(M, Num, G, chs, feps);
        };
        auto record_objective = [&](int t) {
            if (blocked) nmf_cross_flat_kernel<<<nbW, kNmfThreads, 0, s>>>(W, AH, k, dchW, cross);
            else nmf_cross_kernel<<<nbW, kNmfThreads, 0, s>>>(W, AH, k, dchW, cross);
            nmf_objective_kernel<<<ng, kNmfThreads, 0, s>>>(cross, dgW, GW, GH, da2, k, dobj + t, ostride);
        };
        // initial objective (outside the graph; also warms the SpMM launch set-up)
        gram(W, true, GW);
        gram(Ht, false, GH);
        if ((rc = spmm(0, Ht, nc, AH)) != SPMM_OK) break;
        record_objective(0);
        if ((rc = spmm(1, W, nr, AtW)) != SPMM_OK) break;        // warm the transposed launch
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "spmm_nmf: init"); break; }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "spmm_nmf: init sync"); break; }
        if (steps > 0) {
            if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
                fail(e, "spmm_nmf: capture");
                break;
            }
            for (int32_t t = 0; t < steps && rc == SPMM_OK; ++t) {
                // H step: Ht <- Ht o (A^T W) / (Ht (W^T W) + eps); GW holds W^T W
                if ((rc = spmm(1, W, nr, AtW)) != SPMM_OK) break;
                update(Ht, AtW, GW, false);
                gram(Ht, false, GH);
                // W step: W <- W o (A Ht) / (W (Ht^T Ht) + eps)
                if ((rc = spmm(0, Ht, nc, AH)) != SPMM_OK) break;
                update(W, AH, GH, true);
                gram(W, true, GW);
                record_objective(t + 1);
            }
            cudaError_t ec = cudaStreamEndCapture(s, &graph);
            if (rc != SPMM_OK) break;
            if (ec != cudaSuccess) { fail(ec, "spmm_nmf: end capture"); break; }
            if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) { fail(e, "spmm_nmf: instantiate"); break; }
            if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) { fail(e, "spmm_nmf: launch"); break; }
        }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "spmm_nmf: run"); break; }
        int32_t st = 0;
        if ((e = cudaMemcpy(&st, A->status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fail(e, "spmm_nmf: status");
            break;
        }
        if (st != 0) {
            cudaMemset(A->status, 0, sizeof(int32_t));
            set_error("spmm_nmf: a device-side staging wait timed out; the factors are incomplete");
            rc = SPMM_ERR_TIMEOUT;
            break;
        }
        if (objective &&
            (e = cudaMemcpy(objective, dobj, (size_t)ng * ostride * sizeof(double), cudaMemcpyDeviceToHost)) !=
                cudaSuccess) {
            fail(e, "spmm_nmf: objective");
            break;
        }
    } while (0);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (s) cudaStreamDestroy(s);
    cudaFree(dchW); cudaFree(dchH); cudaFree(dgW); cudaFree(dgH); cudaFree(part); cudaFree(GW); cudaFree(GH);
    cudaFree(cross); cudaFree(da2); cudaFree(dobj); cudaFree(AtW); cudaFree(AH); cudaFree(fb);
    return rc;
}

// SPMM_RELABEL: W and Ht (n x k each) go into the handle's vertex order and
// come back once per call; the steps run in between.
extern "C" int spmm_nmf(spmm_mat_t A, int32_t k, int32_t steps, float* W, float* Ht, spmm_dtype ftype, double eps,
                        double* objective, void* stream) {
    if (!A || !A->relabel || !W || !Ht || k < 1 || k > kMaxK)
        return nmf_impl(A, k, steps, W, Ht, ftype, eps, objective, stream);
    const int64_t n = A->fwd.n_rows;
    cudaStream_t s = (cudaStream_t)stream;
    float *wr = nullptr, *hr = nullptr;
    cudaError_t e = cudaMalloc((void**)&wr, (size_t)n * k * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&hr, (size_t)n * k * sizeof(float));
    if (e == cudaSuccess) e = relabel_rows_dev(A, W, k, k, 4, wr, k, true, s);
    if (e == cudaSuccess) e = relabel_rows_dev(A, Ht, k, k, 4, hr, k, true, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int rc = e == cudaSuccess ? nmf_impl(A, k, steps, wr, hr, ftype, eps, objective, stream)
                              : cuda_fail(e, "spmm_nmf: factors into the handle's order");
    if (rc == SPMM_OK) {
        e = relabel_rows_dev(A, wr, k, k, 4, W, k, false, s);
        if (e == cudaSuccess) e = relabel_rows_dev(A, hr, k, k, 4, Ht, k, false, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "spmm_nmf: factors into the input order");
    }
    cudaFree(wr);
    cudaFree(hr);
    return rc;
}
