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
        auto gram = [&](const float* M, bool wside, double* G) {
            gram_partial_kernel<<<wside ? nbW : nbH, kNmfThreads, 0, s>>>(M, k, wside ? dchW : dchH, part);
            gram_reduce_kernel<<<ng, kNmfThreads, 0, s>>>(part, wside ? dgW : dgH, k, G);
        };
        auto record_objective = [&](int t) {
            nmf_cross_kernel<<<nbW, kNmfThreads, 0, s>>>(W, AH, k, dchW, cross);
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
                nmf_update_kernel<<<nbH, kNmfThreads, 0, s>>>(Ht, AtW, GW, k, dchH, feps);
                gram(Ht, false, GH);
                // W step: W <- W o (A Ht) / (W (Ht^T Ht) + eps)
                if ((rc = spmm(0, Ht, nc, AH)) != SPMM_OK) break;
                nmf_update_kernel<<<nbW, kNmfThreads, 0, s>>>(W, AH, GH, k, dchW, feps);
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
