// pagerank.cu -- PageRank power iteration on the SpMM path (paper Section 4.1).
//
// Update rule (Section 4.1): PR(u) = (1-d)/N + d * sum_{v in B(u)} PR(v)/L(v),
// with B(u) the in-neighbours of u and L(v) the out-degree of v; the rank of
// dangling vertices (L = 0) is spread uniformly, so the ranks keep summing to 1.
// Row v of A lists the out-links of v, so the in-neighbour sum is the product
// with the transposed matrix: y = A^T z with z[v] = x[v] / L(v).
//
// One iteration = the task kernel on A^T (k = 1, float32) + one fused
// elementwise kernel (new ranks, the next z = x' * (1/L), FP64 per-block
// partial sums of the L1 change and of the dangling mass) + a one-block kernel
// adding the partials in a fixed order.  Iterations 2..iters are one CUDA
// graph; the handle keeps it with the workspace, so a later call with the
// same x, damping and iteration count only launches it.  Ranks are float32;
// every reduction is FP64 and run-to-run deterministic.
#include <vector>

#include "internal.h"

namespace spmm {

constexpr int kPrThreads = 256;

// Fixed-order block sum of a double (xor tree inside warps, then warp sums
// added in warp order by thread 0).  Result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
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

// inv[v] = 1/L(v) as float (0 marks a dangling vertex, L = 0); x = x0 or 1/N.
__global__ void pr_init_kernel(const int64_t* __restrict__ row_ptr, int64_t n, float* __restrict__ inv,
                               float* __restrict__ x, const float* __restrict__ x0) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t L = row_ptr[i + 1] - row_ptr[i];
        inv[i] = L > 0 ? 1.0f / (float)L : 0.f;
        x[i] = x0 ? x0[i] : (float)(1.0 / (double)n);
    }
}

// One rank update of element i (float32): x' = base + d*y; returns |x' - x|,
// writes z' = x' / L and adds x' to dang for a dangling vertex.
__device__ __forceinline__ float pr_elem(float y, float& x, float inv, float base, float d, float& z, float& dang) {
    const float xn = fmaf(d, y, base);
    const float r = fabsf(xn - x);
    x = xn;
    z = xn * inv;
    if (inv == 0.f) dang += xn;
    return r;
}

// z = x / L (0 where L = 0); per-block partial of the dangling mass.
__global__ void pr_scale_kernel(const float* __restrict__ x, const float* __restrict__ inv, int64_t n,
                                float* __restrict__ z, double* __restrict__ part_dang) {
    __shared__ double sh[32];
    double dang = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float xi = x[i], iv = inv[i];
        z[i] = xi * iv;
        if (iv == 0.f) dang += (double)xi;
    }
    const double s = block_sum(dang, sh);
    if (threadIdx.x == 0) part_dang[blockIdx.x] = s;
}

// x' = (1-d)/N + d*D/N + d*y, with D the dangling mass of x (scal[0]);
// partials of sum |x' - x| and of the dangling mass of x'; z' = x' / L.
// Float4 accesses; the per-element arithmetic is float32 and every group of
// four is added to FP64 per-thread sums, then to FP64 block partials.
__global__ void pr_update_kernel(const float* __restrict__ y, float* __restrict__ x, const float* __restrict__ inv,
                                 int64_t n, double d, const double* __restrict__ scal, float* __restrict__ z,
                                 double* __restrict__ part_res, double* __restrict__ part_dang) {
    __shared__ double sh[32];
    const float base = (float)((1.0 - d) / (double)n + d * scal[0] / (double)n);
    const float df = (float)d;
    double res = 0.0, dang = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)z) | ((uintptr_t)inv)) & 15) == 0;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = n >> 2;
        for (int64_t i = tid; i < n4; i += stride) {
            const float4 y4 = reinterpret_cast<const float4*>(y)[i];
            float4 x4 = reinterpret_cast<const float4*>(x)[i];
            const float4 v4 = reinterpret_cast<const float4*>(inv)[i];
            float4 z4;
            float dg = 0.f, r = 0.f;
            r += pr_elem(y4.x, x4.x, v4.x, base, df, z4.x, dg);
            r += pr_elem(y4.y, x4.y, v4.y, base, df, z4.y, dg);
            r += pr_elem(y4.z, x4.z, v4.z, base, df, z4.z, dg);
            r += pr_elem(y4.w, x4.w, v4.w, base, df, z4.w, dg);
            reinterpret_cast<float4*>(x)[i] = x4;
            reinterpret_cast<float4*>(z)[i] = z4;
            res += (double)r;
            dang += (double)dg;
        }
        done = n4 << 2;
    }
    for (int64_t i = done + tid; i < n; i += stride) {   // tail (or unaligned buffers)
        float xi = x[i], zi, dg = 0.f;
        res += (double)pr_elem(y[i], xi, inv[i], base, df, zi, dg);
        x[i] = xi;
        z[i] = zi;
        dang += (double)dg;
    }
    const double s1 = block_sum(res, sh);
    const double s2 = block_sum(dang, sh);
    if (threadIdx.x == 0) {
        part_res[blockIdx.x] = s1;
        part_dang[blockIdx.x] = s2;
    }
}

// scal[0] = sum of the dangling partials; res_out (if given) = sum of the
// residual partials; both in block order.
__global__ void pr_reduce_kernel(const double* __restrict__ part_dang, const double* __restrict__ part_res,
                                 int nparts, double* __restrict__ scal, double* __restrict__ res_out) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        a += part_dang[i];
        if (res_out) b += part_res[i];
    }
    const double sa = block_sum(a, sh);
    const double sb = block_sum(b, sh);
    if (threadIdx.x == 0) {
        scal[0] = sa;
        if (res_out) *res_out = sb;
    }
}

}  // namespace spmm

using namespace spmm;

namespace spmm {

void pagerank_release(spmm_mat* A) {
    PrCache& c = A->pr;
    if (c.exec) cudaGraphExecDestroy(c.exec);
    if (c.s) cudaStreamDestroy(c.s);
    cudaFree(c.inv_deg);
    cudaFree(c.z);
    cudaFree(c.y);
    cudaFree(c.part);
    cudaFree(c.scal);
    cudaFree(c.dres);
    cudaFree(c.xr);
    cudaFree(c.x0r);
    c = PrCache{};
}

void pagerank_invalidate(spmm_mat* A) {
    PrCache& c = A->pr;
    if (c.exec) cudaGraphExecDestroy(c.exec);
    c.exec = nullptr;
    c.x = nullptr;
    c.damping = -1.0;
    c.iters = -1;
}

// The workspace of an n-vertex PageRank with room for `iters` residuals.
static cudaError_t pr_reserve(PrCache& c, int64_t n, int32_t iters, int nblk) {
    cudaError_t e = cudaSuccess;
    if (!c.inv_deg) {
        if ((e = cudaMalloc((void**)&c.inv_deg, n * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&c.z, n * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&c.y, n * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&c.part, 2 * (size_t)nblk * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&c.scal, 8 * sizeof(double))) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking)) != cudaSuccess)
            return e;
        c.nblk = nblk;
    }
    if (iters > c.dres_cap) {
        cudaFree(c.dres);
        c.dres = nullptr;
        c.dres_cap = 0;
        if ((e = cudaMalloc((void**)&c.dres, (size_t)iters * sizeof(double))) != cudaSuccess) return e;
        c.dres_cap = iters;
        if (c.exec) {                          // its residual pointers are gone
            cudaGraphExecDestroy(c.exec);
            c.exec = nullptr;
            c.iters = -1;
        }
    }
    return e;
}

}  // namespace spmm

extern "C" int spmm_pagerank(spmm_mat_t A, double damping, int32_t iters, float* x, const float* x0,
                             double* residuals, void* stream) {
    if (!A || !x) { set_error("spmm_pagerank: NULL argument"); return SPMM_ERR_ARG; }
    if (A->fwd.n_rows != A->fwd.n_cols || A->fwd.n_rows < 1) {
        set_error("spmm_pagerank: the matrix must be square and non-empty");
        return SPMM_ERR_ARG;
    }
    if (!A->has_tr) { set_error("spmm_pagerank: needs SPMM_WANT_TRANSPOSE at create"); return SPMM_ERR_ARG; }
    if (A->vtype != -1) {
        set_error("spmm_pagerank: PageRank walks the graph pattern; create the handle without values");
        return SPMM_ERR_ARG;
    }
    if (iters < 0 || !(damping >= 0.0 && damping <= 1.0)) {
        set_error("spmm_pagerank: need iters >= 0 and 0 <= damping <= 1");
        return SPMM_ERR_ARG;
    }
    const int64_t n = A->fwd.n_rows;
    cudaStream_t user = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "spmm_pagerank: device query");
    PrCache& c = A->pr;
    int rc = SPMM_OK;
    NvtxRange range("spmm_pagerank");
    auto fail = [&](cudaError_t err, const char* what) { rc = cuda_fail(err, what); };
    do {
        if ((e = cudaStreamSynchronize(user)) != cudaSuccess) { fail(e, "spmm_pagerank: stream"); break; }
        if ((e = pr_reserve(c, n, iters, sms * 8)) != cudaSuccess) {
            fail(e, "spmm_pagerank: workspace");
            pagerank_release(A);
            break;
        }
        const int nblk = c.nblk;
        cudaStream_t s = c.s;
        // SPMM_RELABEL: the iterations run on the ranks in the handle's vertex
        // order, in a buffer the handle keeps (so the captured graph stays
        // valid); the start vector comes in and the ranks go out once
        float* const x_user = x;
        if (A->relabel) {
            if (!c.xr && (e = cudaMalloc((void**)&c.xr, (size_t)n * sizeof(float))) != cudaSuccess) {
                fail(e, "spmm_pagerank: relabelled ranks");
                break;
            }
            if (x0) {
                if (!c.x0r && (e = cudaMalloc((void**)&c.x0r, (size_t)n * sizeof(float))) != cudaSuccess) {
                    fail(e, "spmm_pagerank: relabelled start vector");
                    break;
                }
                if ((e = relabel_rows_dev(A, x0, 1, 1, 4, c.x0r, 1, true, s)) != cudaSuccess) {
                    fail(e, "spmm_pagerank: start vector into the handle's order");
                    break;
                }
                x0 = c.x0r;
            }
            x = c.xr;
        }
        // set-up outside the graph: 1/L, the start vector, z and its dangling mass
        pr_init_kernel<<<nblk, kPrThreads, 0, s>>>(A->fwd.row_ptr, n, c.inv_deg, x, x0);
        pr_scale_kernel<<<nblk, kPrThreads, 0, s>>>(x, c.inv_deg, n, c.z, c.part);
        pr_reduce_kernel<<<1, kPrThreads, 0, s>>>(c.part, nullptr, nblk, c.scal, nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "spmm_pagerank: init"); break; }
        if (iters > 0) {
            // the first iteration runs outside the graph, so the task kernel's
            // one-time launch set-up (attributes, occupancy) happens before capture
            if ((rc = apply_dev(A, 1, c.z, 1, 1, SPMM_F32, c.y, 1, s)) != SPMM_OK) break;
            pr_update_kernel<<<nblk, kPrThreads, 0, s>>>(c.y, x, c.inv_deg, n, damping, c.scal, c.z, c.part + nblk,
                                                         c.part);
            pr_reduce_kernel<<<1, kPrThreads, 0, s>>>(c.part, c.part + nblk, nblk, c.scal, c.dres);
            if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "spmm_pagerank: first iteration"); break; }
        }
        if (iters > 1) {
            // iterations 2..iters: one graph, captured on the first call with
            // this x, damping and iteration count and relaunched after that
            if (!(c.exec && c.x == x && c.damping == damping && c.iters == iters)) {
                if (c.exec) {
                    cudaGraphExecDestroy(c.exec);
                    c.exec = nullptr;
                }
                c.iters = -1;
                if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "spmm_pagerank: first iteration"); break; }
                if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
                    fail(e, "spmm_pagerank: capture");
                    break;
                }
                for (int32_t t = 1; t < iters && rc == SPMM_OK; ++t) {
                    rc = apply_dev(A, 1, c.z, 1, 1, SPMM_F32, c.y, 1, s);
                    if (rc != SPMM_OK) break;
                    pr_update_kernel<<<nblk, kPrThreads, 0, s>>>(c.y, x, c.inv_deg, n, damping, c.scal, c.z,
                                                                 c.part + nblk, c.part);
                    pr_reduce_kernel<<<1, kPrThreads, 0, s>>>(c.part, c.part + nblk, nblk, c.scal, c.dres + t);
                }
                cudaGraph_t graph = nullptr;
                cudaError_t ec = cudaStreamEndCapture(s, &graph);
                if (rc == SPMM_OK && ec != cudaSuccess) fail(ec, "spmm_pagerank: end capture");
                if (rc == SPMM_OK && (e = cudaGraphInstantiate(&c.exec, graph, 0)) != cudaSuccess) {
                    c.exec = nullptr;
                    fail(e, "spmm_pagerank: instantiate");
                }
                if (graph) cudaGraphDestroy(graph);
                if (rc != SPMM_OK) break;
                c.x = x;
                c.damping = damping;
                c.iters = iters;
            }
            if ((e = cudaGraphLaunch(c.exec, s)) != cudaSuccess) { fail(e, "spmm_pagerank: launch"); break; }
        }
        if (A->relabel && (e = relabel_rows_dev(A, x, 1, 1, 4, x_user, 1, false, s)) != cudaSuccess) {
            fail(e, "spmm_pagerank: ranks into the input order");
            break;
        }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "spmm_pagerank: run"); break; }
        int32_t st = 0;
        if ((e = cudaMemcpy(&st, A->status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fail(e, "spmm_pagerank: status");
            break;
        }
        if (st != 0) {
            cudaMemset(A->status, 0, sizeof(int32_t));
            set_error("spmm_pagerank: a device-side staging wait timed out; the ranks are incomplete");
            rc = SPMM_ERR_TIMEOUT;
            break;
        }
        if (residuals && iters > 0 &&
            (e = cudaMemcpy(residuals, c.dres, (size_t)iters * sizeof(double), cudaMemcpyDeviceToHost)) !=
                cudaSuccess) {
            fail(e, "spmm_pagerank: residuals");
            break;
        }
    } while (0);
    return rc;
}
