// eigs.cu -- block eigensolver on the SpMM path (paper Section 4.2).
//
// Section 4.2 runs a block Krylov-Schur eigensolver whose only sparse
// operation is the block product S V.  This is a thick-restart block Krylov
// method for a symmetric S (for symmetric matrices Krylov-Schur restarting is
// thick-restart Lanczos): the basis V and S V are held in FP64; every
// expansion multiplies the newest block by S through the task kernel (X =
// the block in FP32 or BF16, FP32 accumulation, converted back to FP64);
// orthogonalisation is block classical Gram-Schmidt applied twice followed by
// CholQR2, all in FP64 and on the device (the b x b Cholesky factor and its
// inverse by one small kernel), so the expansions of a cycle are captured as
// one CUDA graph; the Rayleigh-Ritz problem T = V^T (S V) is solved on the
// host in FP64 by cyclic Jacobi once per restart; a restart keeps the best
// nev + block Ritz vectors and their images, and the next expansion starts
// from S applied to the kept Ritz vectors (whose components orthogonal to V
// are the residuals).
//
// Tall-skinny FP64 kernels: C = A^T B (chunked partials added in a fixed
// order) and Out = beta Out + alpha A C (one thread per output element).
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"

namespace spmm {

constexpr int kEigThreads = 256;
constexpr int kEigMaxBasis = 64;
constexpr int kTsTile = 16;

// partial[c][r*q + s] = sum over chunk rows i of A[i][r] * B[i][s]
__global__ void __launch_bounds__(kEigThreads)
ts_tn_partial_kernel(const double* __restrict__ A, int64_t lda, int p, const double* __restrict__ B, int64_t ldb,
                     int q, int64_t n, int64_t chunk, double* __restrict__ partial) {
    __shared__ double ta[kTsTile * kEigMaxBasis];
    __shared__ double tb[kTsTile * kEigMaxBasis];
    const int pq = p * q;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    for (int64_t r0 = i0; r0 < i1; r0 += kTsTile) {
        const int rows = (int)min((int64_t)kTsTile, i1 - r0);
        for (int t = threadIdx.x; t < rows * p; t += blockDim.x) ta[t] = A[(r0 + t / p) * lda + t % p];
        for (int t = threadIdx.x; t < rows * q; t += blockDim.x) tb[t] = B[(r0 + t / q) * ldb + t % q];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int e = threadIdx.x + j * kEigThreads;
            if (e < pq) {
                const int r = e / q, s = e % q;
                double f = 0.0;
                for (int t = 0; t < rows; ++t) f = fma(ta[t * p + r], tb[t * q + s], f);
                acc[j] += f;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int e = threadIdx.x + j * kEigThreads;
        if (e < pq) partial[(int64_t)blockIdx.x * pq + e] = acc[j];
    }
}

__global__ void ts_reduce_kernel(const double* __restrict__ partial, int nparts, int pq, double* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < pq; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nparts; ++c) s += partial[(int64_t)c * pq + e];
        out[e] = s;
    }
}

// Out[i][j] = beta * Out[i][j] + alpha * sum_r A[i][r] * C[r][j]   (C is p x q, row-major)
__global__ void __launch_bounds__(kEigThreads)
ts_nn_kernel(const double* __restrict__ A, int64_t lda, int p, const double* __restrict__ C, int q, double* Out,
             int64_t ldo, int64_t n, double alpha, double beta) {
    __shared__ double cs[kEigMaxBasis * kEigMaxBasis];
    for (int t = threadIdx.x; t < p * q; t += blockDim.x) cs[t] = C[t];
    __syncthreads();
    const int64_t total = n * q;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / q;
        const int j = (int)(t % q);
        double s = 0.0;
        for (int r = 0; r < p; ++r) s = fma(A[i * lda + r], cs[r * q + j], s);
        Out[i * ldo + j] = (beta == 0.0 ? 0.0 : beta * Out[i * ldo + j]) + alpha * s;
    }
}

// strided FP64 block -> contiguous FP32 or BF16 (SpMM input)
__global__ void f64_to_x_kernel(const double* __restrict__ src, int64_t lds, int b, int64_t n, void* dst, int bf16) {
    const int64_t total = n * b;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[(t / b) * lds + t % b];
        if (bf16) static_cast<__nv_bfloat16*>(dst)[t] = __double2bfloat16(v);
        else static_cast<float*>(dst)[t] = (float)v;
    }
}

// contiguous FP32 (SpMM output) -> strided FP64 block
__global__ void f32_to_f64_kernel(const float* __restrict__ src, int b, int64_t n, double* dst, int64_t ldd) {
    const int64_t total = n * b;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        dst[(t / b) * ldd + t % b] = (double)src[t];
}

// strided FP64 copy of an n x b block
__global__ void copy_block_kernel(const double* __restrict__ src, int64_t lds, int b, int64_t n, double* dst,
                                  int64_t ldd) {
    const int64_t total = n * b;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        dst[(t / b) * ldd + t % b] = src[(t / b) * lds + t % b];
}

// residual block R = AU - U diag(theta)
__global__ void residual_kernel(const double* __restrict__ AU, const double* __restrict__ U, const double* theta,
                                int q, int64_t n, double* R) {
    const int64_t total = n * q;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        R[t] = AU[t] - theta[t % q] * U[t];
}

// Chebyshev filter step (FP32): Yn = alpha * SY + beta * Yc + gamma * Yp,
// coefficients (alpha, beta, gamma) read from device memory so one captured
// graph serves every filter interval
__global__ void cheb_step_kernel(const float* __restrict__ SY, const float* __restrict__ Yc,
                                 const float* __restrict__ Yp, float* __restrict__ Yn, int64_t total,
                                 const float* __restrict__ coef) {
    const float al = coef[0], be = coef[1], ga = coef[2];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        Yn[t] = fmaf(al, SY[t], fmaf(be, Yc[t], Yp ? ga * Yp[t] : 0.f));
}

// contiguous FP32 -> BF16 (the SpMM input of a BF16 filter step)
__global__ void f32_to_bf16_kernel(const float* __restrict__ src, int64_t total, __nv_bfloat16* __restrict__ dst) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = __float2bfloat16(src[t]);
}

// Block Cholesky G = R^T R (R upper, b x b row-major, b <= 32) and its inverse
// Rinv = R^-1 (upper), by one block of 32 threads: the pivots in turn (thread
// 0), each pivot's row of R across the threads, then column c of the inverse
// by back substitution in thread c.  A pivot that is not safely positive
// (below 1e-24 x trace) marks *flag and leaves the identity in Rinv, so the
// kernels queued after it keep running on finite numbers until the host
// reads the flag.
__global__ void chol_inv_kernel(const double* __restrict__ G, int b, double* __restrict__ Rinv,
                                int32_t* __restrict__ flag) {
    __shared__ double R[32 * 32];
    __shared__ int bad;
    const int t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int e = t; e < b * b; e += blockDim.x) R[e] = 0.0;
    __syncthreads();
    double tr = 0.0;
    for (int i = 0; i < b; ++i) tr += G[i * b + i];
    for (int j = 0; j < b; ++j) {
        if (t == 0) {
            double d = G[j * b + j];
            for (int k = 0; k < j; ++k) d -= R[k * b + j] * R[k * b + j];
            if (!(d > 1e-24 * (tr > 0 ? tr : 1.0))) bad = 1;
            R[j * b + j] = bad ? 1.0 : sqrt(d);
        }
        __syncthreads();
        if (bad) break;
        const double rjj = R[j * b + j];
        for (int i = j + 1 + t; i < b; i += blockDim.x) {
            double s = G[j * b + i];
            for (int k = 0; k < j; ++k) s -= R[k * b + j] * R[k * b + i];
            R[j * b + i] = s / rjj;
        }
        __syncthreads();
    }
    if (bad) {
        for (int e = t; e < b * b; e += blockDim.x) Rinv[e] = (e / b == e % b) ? 1.0 : 0.0;
        if (t == 0) *flag = 1;
        return;
    }
    for (int c = t; c < b; c += blockDim.x) {
        double x[32];
        x[c] = 1.0 / R[c * b + c];
        for (int i = c - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= c; ++k) s += R[i * b + k] * x[k];
            x[i] = -s / R[i * b + i];
        }
        for (int i = 0; i < b; ++i) Rinv[i * b + c] = i <= c ? x[i] : 0.0;
    }
}

// ---------------------------------------------------------------- host linear algebra
// Cholesky G = R^T R (R upper); false if a pivot is not safely positive.
static bool cholesky_upper(int b, const std::vector<double>& G, std::vector<double>& R) {
    R.assign((size_t)b * b, 0.0);
    double tr = 0.0;
    for (int i = 0; i < b; ++i) tr += G[(size_t)i * b + i];
    for (int j = 0; j < b; ++j) {
        double d = G[(size_t)j * b + j];
        for (int k = 0; k < j; ++k) d -= R[(size_t)k * b + j] * R[(size_t)k * b + j];
        if (!(d > 1e-24 * (tr > 0 ? tr : 1.0))) return false;
        const double rjj = std::sqrt(d);
        R[(size_t)j * b + j] = rjj;
        for (int i = j + 1; i < b; ++i) {
            double s = G[(size_t)j * b + i];
            for (int k = 0; k < j; ++k) s -= R[(size_t)k * b + j] * R[(size_t)k * b + i];
            R[(size_t)j * b + i] = s / rjj;
        }
    }
    return true;
}

// inverse of an upper-triangular b x b matrix
static std::vector<double> upper_inverse(int b, const std::vector<double>& R) {
    std::vector<double> X((size_t)b * b, 0.0);
    for (int j = 0; j < b; ++j) {
        X[(size_t)j * b + j] = 1.0 / R[(size_t)j * b + j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= j; ++k) s += R[(size_t)i * b + k] * X[(size_t)k * b + j];
            X[(size_t)i * b + j] = -s / R[(size_t)i * b + i];
        }
    }
    return X;
}

// cyclic Jacobi eigen-decomposition of a symmetric m x m matrix (destroyed);
// column c of V is the eigenvector of evals[c]
static void jacobi_eigh(int m, std::vector<double>& M, std::vector<double>& evals, std::vector<double>& V) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double x = M[(size_t)i * m + j];
                tot += x * x;
                if (i != j) off += x * x;
            }
        if (off == 0.0 || off <= 1e-30 * tot) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = M[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double theta = (M[(size_t)q * m + q] - M[(size_t)p * m + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < m; ++r) {
                    const double a = M[(size_t)r * m + p], b = M[(size_t)r * m + q];
                    M[(size_t)r * m + p] = c * a - s * b;
                    M[(size_t)r * m + q] = s * a + c * b;
                }
                for (int r = 0; r < m; ++r) {
                    const double a = M[(size_t)p * m + r], b = M[(size_t)q * m + r];
                    M[(size_t)p * m + r] = c * a - s * b;
                    M[(size_t)q * m + r] = s * a + c * b;
                }
                for (int r = 0; r < m; ++r) {
                    const double a = V[(size_t)r * m + p], b = V[(size_t)r * m + q];
                    V[(size_t)r * m + p] = c * a - s * b;
                    V[(size_t)r * m + q] = s * a + c * b;
                }
            }
    }
    evals.resize(m);
    for (int i = 0; i < m; ++i) evals[i] = M[(size_t)i * m + i];
}

namespace {

struct Eig {
    const spmm_mat* A;
    int64_t n;
    int m, b;
    int xtype;
    int op = 0;              // 0: S V;  1: A^T (A V)
    float* T1 = nullptr;     // A V (op 1), n_rows x b
    cudaStream_t s;
    double *V = nullptr, *AV = nullptr, *W = nullptr, *W2 = nullptr, *part = nullptr, *small = nullptr;
    double *U = nullptr, *AU = nullptr, *theta = nullptr;
    double* small2 = nullptr;   // b x b inverse Cholesky factor (device-side CholQR)
    int32_t* flags = nullptr;   // breakdown flag of each expansion of a cycle (device)
    float* Yf = nullptr;
    void* Xs = nullptr;
    int64_t chunk = 0;
    int nchunks = 0;
    int grid = 0;

    cudaError_t tn(const double* Am, int64_t lda, int p, const double* Bm, int64_t ldb, int q, std::vector<double>& out) {
        ts_tn_partial_kernel<<<nchunks, kEigThreads, 0, s>>>(Am, lda, p, Bm, ldb, q, n, chunk, part);
        ts_reduce_kernel<<<(p * q + 255) / 256, 256, 0, s>>>(part, nchunks, p * q, small);
        out.resize((size_t)p * q);
        cudaError_t e = cudaMemcpyAsync(out.data(), small, (size_t)p * q * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    }
    cudaError_t nn(const double* Am, int64_t lda, int p, const std::vector<double>& C, int q, double* Out, int64_t ldo,
                   double alpha, double beta) {
        cudaError_t e = cudaMemcpyAsync(small, C.data(), (size_t)p * q * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        ts_nn_kernel<<<grid, kEigThreads, 0, s>>>(Am, lda, p, small, q, Out, ldo, n, alpha, beta);
        // small is reused by the next call: finish this one first
        return cudaStreamSynchronize(s);
    }
    // Y = S * block (block: n x b FP64 with leading dimension ld) into out (ld m)
    int apply_block(const double* blk, int64_t ld, double* out, int64_t ldo) {
        f64_to_x_kernel<<<grid, kEigThreads, 0, s>>>(blk, ld, b, n, Xs, xtype == SPMM_BF16);
        int rc;
        if (op == 0) {
            rc = apply_dev(A, 0, Xs, b, b, xtype, Yf, b, s);
        } else {   // A^T (A V): the intermediate stays float32
            rc = apply_dev(A, 0, Xs, b, b, xtype, T1, b, s);
            if (rc == SPMM_OK) rc = apply_dev(A, 1, T1, b, b, SPMM_F32, Yf, b, s);
        }
        if (rc != SPMM_OK) return rc;
        f32_to_f64_kernel<<<grid, kEigThreads, 0, s>>>(Yf, b, n, out, ldo);
        return SPMM_OK;
    }
    // C = A^T B into device memory, and Out = beta Out + alpha A C with C in
    // device memory: the tall-skinny products with no host round trip
    void tn_dev(const double* Am, int64_t lda, int p, const double* Bm, int64_t ldb, int q, double* out) {
        ts_tn_partial_kernel<<<nchunks, kEigThreads, 0, s>>>(Am, lda, p, Bm, ldb, q, n, chunk, part);
        ts_reduce_kernel<<<(p * q + 255) / 256, 256, 0, s>>>(part, nchunks, p * q, out);
    }
    void nn_dev(const double* Am, int64_t lda, int p, const double* C, int q, double* Out, int64_t ldo, double alpha,
                double beta) {
        ts_nn_kernel<<<grid, kEigThreads, 0, s>>>(Am, lda, p, C, q, Out, ldo, n, alpha, beta);
    }
    // orthonormalise() on the device only: CGS2 against V[:, :cur], then
    // CholQR2 with the Cholesky factor inverted by chol_inv_kernel; a
    // breakdown marks flags[slot] instead of returning
    void orthonormalize_dev(int cur, int slot) {
        for (int pass = 0; pass < 2 && cur > 0; ++pass) {
            tn_dev(V, m, cur, W, b, b, small);
            nn_dev(V, m, cur, small, b, W, b, -1.0, 1.0);
        }
        for (int pass = 0; pass < 2; ++pass) {
            tn_dev(W, b, b, W, b, b, small);
            chol_inv_kernel<<<1, 32, 0, s>>>(small, b, small2, flags + slot);
            nn_dev(W, b, b, small2, b, W2, b, 1.0, 0.0);
            std::swap(W, W2);
        }
    }
    // n_exp expansions of the basis from column cur0, the first from the
    // image AV[:, seed0] and each next one from the image of the block before;
    // every step stays on the device (a breakdown in expansion x marks
    // flags[x]), so a cycle can be captured as one graph
    int expand_cycle(int cur0, int seed0, int n_exp) {
        cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)n_exp * sizeof(int32_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "spmm_eigs: flags");
        int cur = cur0, seed = seed0;
        for (int x = 0; x < n_exp; ++x) {
            copy_block_kernel<<<grid, kEigThreads, 0, s>>>(AV + seed, m, b, n, W, b);
            orthonormalize_dev(cur, x);
            copy_block_kernel<<<grid, kEigThreads, 0, s>>>(W, b, b, n, V + cur, m);
            const int rc = apply_block(V + cur, m, AV + cur, m);
            if (rc != SPMM_OK) return rc;
            seed = cur;
            cur += b;
        }
        e = cudaGetLastError();
        return e == cudaSuccess ? SPMM_OK : cuda_fail(e, "spmm_eigs: expansion");
    }
    // orthonormalise W (n x b) against V[:, :cur] twice, then CholQR2; false on breakdown
    bool orthonormalize(int cur, cudaError_t& e) {
        std::vector<double> C, G, R;
        for (int pass = 0; pass < 2 && cur > 0; ++pass) {
            if ((e = tn(V, m, cur, W, b, b, C)) != cudaSuccess) return false;
            if ((e = nn(V, m, cur, C, b, W, b, -1.0, 1.0)) != cudaSuccess) return false;
        }
        for (int pass = 0; pass < 2; ++pass) {
            if ((e = tn(W, b, b, W, b, b, G)) != cudaSuccess) return false;
            if (!cholesky_upper(b, G, R)) return false;
            const std::vector<double> Ri = upper_inverse(b, R);
            if ((e = nn(W, b, b, Ri, b, W2, b, 1.0, 0.0)) != cudaSuccess) return false;
            std::swap(W, W2);
        }
        return true;
    }
};

}  // namespace

}  // namespace spmm

using namespace spmm;

static int eigs_impl(spmm_mat_t S, int op, int32_t nev, int32_t block, int32_t max_basis, int32_t max_restarts,
                     double tol, spmm_dtype xtype, const double* V0, double* evals, double* evecs, double* resid,
                     int32_t* restarts_out, void* stream) {
    if (!S || !V0 || !evals) { set_error("spmm_eigs: NULL argument"); return SPMM_ERR_ARG; }
    NvtxRange range(op ? "spmm_svds" : "spmm_eigs");
    const int64_t n = op ? S->fwd.n_cols : S->fwd.n_rows;
    if (op == 0 && (S->fwd.n_cols != n || n < 1)) { set_error("spmm_eigs: the matrix must be square"); return SPMM_ERR_ARG; }
    if (op == 1 && !S->has_tr) { set_error("spmm_svds: needs SPMM_WANT_TRANSPOSE at create"); return SPMM_ERR_ARG; }
    if (block < 1 || block > 32 || nev < 1 || nev > block + 32 || max_basis > kEigMaxBasis ||
        max_basis < nev + 2 * block || max_basis > n || max_restarts < 0 || !(tol > 0.0)) {
        set_error("spmm_eigs: need 1 <= block <= 32, nev + 2*block <= max_basis <= min(64, n), max_restarts >= 0, "
                  "tol > 0");
        return SPMM_ERR_ARG;
    }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16) { set_error("spmm_eigs: xtype must be F32 or BF16"); return SPMM_ERR_ARG; }
    if (S->vtype == SPMM_F16 || (S->vtype == SPMM_BF16 && xtype != SPMM_BF16)) {
        set_error("spmm_eigs: 16-bit values need X of the same type (use F32 values)");
        return SPMM_ERR_UNSUPPORTED;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    Eig E;
    E.A = S;
    E.n = n;
    E.m = max_basis;
    E.b = block;
    E.xtype = xtype;
    E.op = op;
    E.grid = std::max(1, sms * 8);
    E.chunk = std::max<int64_t>(1024, (n + 1023) / 1024);
    E.nchunks = (int)((n + E.chunk - 1) / E.chunk);
    const int m = max_basis, b = block;
    const int keep = std::min(nev + b, m - b);
    int rc = SPMM_OK;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err, const char* what) { rc = cuda_fail(err, what); };
    do {
        if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess) { fail(e, "spmm_eigs: stream"); break; }
        if ((e = cudaStreamCreateWithFlags(&E.s, cudaStreamNonBlocking)) != cudaSuccess) { fail(e, "spmm_eigs: stream"); break; }
        const size_t nm = (size_t)n * m * sizeof(double);
        if ((e = cudaMalloc((void**)&E.V, nm)) != cudaSuccess || (e = cudaMalloc((void**)&E.AV, nm)) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.U, nm)) != cudaSuccess || (e = cudaMalloc((void**)&E.AU, nm)) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.W, (size_t)n * m * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.W2, (size_t)n * m * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.part, (size_t)E.nchunks * m * m * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.small, (size_t)m * m * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.small2, (size_t)b * b * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.flags, (size_t)kEigMaxBasis * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.theta, (size_t)m * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.Yf, (size_t)n * b * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&E.Xs, (size_t)n * b * sizeof(float))) != cudaSuccess ||
            (op && (e = cudaMalloc((void**)&E.T1, (size_t)std::max<int64_t>(S->fwd.n_rows, 1) * b * sizeof(float))) !=
                       cudaSuccess)) {
            fail(e, "spmm_eigs: workspace");
            break;
        }
        // start block
        copy_block_kernel<<<E.grid, kEigThreads, 0, E.s>>>(V0, b, b, n, E.W, b);
        if (!E.orthonormalize(0, e)) {
            if (e != cudaSuccess) fail(e, "spmm_eigs: orthonormalise");
            else { set_error("spmm_eigs: the start block is rank-deficient"); rc = SPMM_ERR_ARG; }
            break;
        }
        copy_block_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.W, b, b, n, E.V, m);
        if ((rc = E.apply_block(E.V, m, E.AV, m)) != SPMM_OK) break;
        int cur = b, seed = 0, restarts = 0;
        std::vector<double> T, th, Y, Rn;
        bool done = false;
        // Every cycle after the first restart expands the same columns from
        // the same seeds, so that expansion phase is captured as one CUDA
        // graph the second time it comes (the first run happens eagerly, so
        // any buffer the product grows is grown outside the capture).
        int g_cur0 = -1, g_n = -1, seen_cur0 = -1, seen_n = -1;
        cudaGraphExec_t gexec = nullptr;
        std::vector<int32_t> hflags(kEigMaxBasis);
        while (!done) {
            // ---- expand the basis block by block (device only)
            const int cur0 = cur, n_exp = (m - cur) / b;
            if (n_exp > 0) {
                if (gexec && g_cur0 == cur0 && g_n == n_exp && seed == 0) {
                    if ((e = cudaGraphLaunch(gexec, E.s)) != cudaSuccess) { fail(e, "spmm_eigs: expansion graph"); break; }
                } else if (seed == 0 && seen_cur0 == cur0 && seen_n == n_exp) {
                    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
                    if ((e = cudaStreamBeginCapture(E.s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
                        fail(e, "spmm_eigs: capture");
                        break;
                    }
                    rc = E.expand_cycle(cur0, 0, n_exp);
                    cudaGraph_t graph = nullptr;
                    const cudaError_t ec = cudaStreamEndCapture(E.s, &graph);
                    if (rc == SPMM_OK && ec != cudaSuccess) fail(ec, "spmm_eigs: end capture");
                    if (rc == SPMM_OK && (e = cudaGraphInstantiate(&gexec, graph, 0)) != cudaSuccess) {
                        gexec = nullptr;
                        fail(e, "spmm_eigs: instantiate");
                    }
                    if (graph) cudaGraphDestroy(graph);
                    if (rc != SPMM_OK) break;
                    g_cur0 = cur0;
                    g_n = n_exp;
                    if ((e = cudaGraphLaunch(gexec, E.s)) != cudaSuccess) { fail(e, "spmm_eigs: expansion graph"); break; }
                } else {
                    if ((rc = E.expand_cycle(cur0, seed, n_exp)) != SPMM_OK) break;
                    if (seed == 0) {
                        seen_cur0 = cur0;
                        seen_n = n_exp;
                    }
                }
                // the first expansion that broke down (its span was invariant) ends the basis
                if ((e = cudaMemcpyAsync(hflags.data(), E.flags, (size_t)n_exp * sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, E.s)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(E.s)) != cudaSuccess) {
                    fail(e, "spmm_eigs: expansion flags");
                    break;
                }
                int x = 0;
                while (x < n_exp && hflags[(size_t)x] == 0) ++x;
                cur = cur0 + x * b;
            }
            // ---- Rayleigh-Ritz on span(V[:, :cur])
            if ((e = E.tn(E.V, m, cur, E.AV, m, cur, T)) != cudaSuccess) { fail(e, "spmm_eigs: projection"); break; }
            for (int i = 0; i < cur; ++i)
                for (int j = i + 1; j < cur; ++j) {
                    const double a = 0.5 * (T[(size_t)i * cur + j] + T[(size_t)j * cur + i]);
                    T[(size_t)i * cur + j] = a;
                    T[(size_t)j * cur + i] = a;
                }
            jacobi_eigh(cur, T, th, Y);
            std::vector<int> order(cur);
            for (int i = 0; i < cur; ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return th[x] > th[y]; });
            const int kp = std::min(keep, cur);
            std::vector<double> Yk((size_t)cur * kp), thk(kp);
            for (int c = 0; c < kp; ++c) {
                thk[c] = th[order[c]];
                for (int r = 0; r < cur; ++r) Yk[(size_t)r * kp + c] = Y[(size_t)r * cur + order[c]];
            }
            if ((e = E.nn(E.V, m, cur, Yk, kp, E.U, kp, 1.0, 0.0)) != cudaSuccess ||
                (e = E.nn(E.AV, m, cur, Yk, kp, E.AU, kp, 1.0, 0.0)) != cudaSuccess) {
                fail(e, "spmm_eigs: Ritz vectors");
                break;
            }
            // residual norms of the Ritz pairs
            cudaMemcpyAsync(E.theta, thk.data(), kp * sizeof(double), cudaMemcpyHostToDevice, E.s);
            residual_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.AU, E.U, E.theta, kp, n, E.W2);
            if ((e = E.tn(E.W2, kp, kp, E.W2, kp, kp, Rn)) != cudaSuccess) { fail(e, "spmm_eigs: residuals"); break; }
            double worst = 0.0;
            for (int i = 0; i < nev; ++i) worst = std::max(worst, std::sqrt(std::max(0.0, Rn[(size_t)i * kp + i])));
            if (worst <= tol || restarts >= max_restarts) {
                for (int i = 0; i < nev; ++i) {
                    evals[i] = thk[i];
                    if (resid) resid[i] = std::sqrt(std::max(0.0, Rn[(size_t)i * kp + i]));
                }
                if (evecs) copy_block_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.U, kp, nev, n, evecs, nev);
                if (restarts_out) *restarts_out = restarts;
                done = true;
                break;
            }
            // ---- thick restart: keep the best kp Ritz vectors and their images
            copy_block_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.U, kp, kp, n, E.V, m);
            copy_block_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.AU, kp, kp, n, E.AV, m);
            cur = kp;
            seed = 0;
            ++restarts;
        }
        if (gexec) cudaGraphExecDestroy(gexec);
        if (rc != SPMM_OK) break;
        if ((e = cudaStreamSynchronize(E.s)) != cudaSuccess) { fail(e, "spmm_eigs: run"); break; }
        int32_t st = 0;
        if ((e = cudaMemcpy(&st, S->status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fail(e, "spmm_eigs: status");
            break;
        }
        if (st != 0) {
            cudaMemset(S->status, 0, sizeof(int32_t));
            set_error("spmm_eigs: a device-side staging wait timed out; the result is incomplete");
            rc = SPMM_ERR_TIMEOUT;
        }
    } while (0);
    if (E.s) {
        cudaStreamSynchronize(E.s);
        cudaStreamDestroy(E.s);
    }
    cudaFree(E.V); cudaFree(E.AV); cudaFree(E.U); cudaFree(E.AU); cudaFree(E.W); cudaFree(E.W2);
    cudaFree(E.part); cudaFree(E.small); cudaFree(E.theta); cudaFree(E.Yf); cudaFree(E.Xs); cudaFree(E.T1);
    cudaFree(E.small2); cudaFree(E.flags);
    return rc;
}

// SPMM_RELABEL: the start block (n x block) goes into the handle's vertex
// order and the vectors (n x nvec) come back, once per call; run(V0, vecs)
// solves with the pointers it is given.  Other handles call run directly.
template <class F>
static int in_handle_order(spmm_mat_t A, int32_t block, const double* V0, int32_t nvec, double* vecs, void* stream,
                           const char* who, F run) {
    if (!A || !A->relabel || !V0 || block < 1 || block > 64 || nvec < 1 || nvec > 64) return run(V0, vecs);
    const int64_t n = A->fwd.n_rows;
    cudaStream_t s = (cudaStream_t)stream;
    double *v0r = nullptr, *vr = nullptr;
    cudaError_t e = cudaMalloc((void**)&v0r, (size_t)n * block * sizeof(double));
    if (e == cudaSuccess && vecs) e = cudaMalloc((void**)&vr, (size_t)n * nvec * sizeof(double));
    if (e == cudaSuccess) e = relabel_rows_dev(A, V0, block, block, 8, v0r, block, true, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int rc = e == cudaSuccess ? run(v0r, vr) : cuda_fail(e, who);
    if (rc == SPMM_OK && vecs) {
        e = relabel_rows_dev(A, vr, nvec, nvec, 8, vecs, nvec, false, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, who);
    }
    cudaFree(v0r);
    cudaFree(vr);
    return rc;
}

extern "C" int spmm_eigs(spmm_mat_t S, int32_t nev, int32_t block, int32_t max_basis, int32_t max_restarts,
                         double tol, spmm_dtype xtype, const double* V0, double* evals, double* evecs,
                         double* resid, int32_t* restarts_out, void* stream) {
    return in_handle_order(S, block, V0, nev, evecs, stream, "spmm_eigs: vectors and the handle's order",
                           [&](const double* v0, double* vec) {
                               return eigs_impl(S, 0, nev, block, max_basis, max_restarts, tol, xtype, v0, evals,
                                                vec, resid, restarts_out, stream);
                           });
}

extern "C" int spmm_svds(spmm_mat_t A, int32_t nsv, int32_t block, int32_t max_basis, int32_t max_restarts,
                         double tol, spmm_dtype xtype, const double* V0, double* svals, double* right_vecs,
                         double* resid, int32_t* restarts_out, void* stream) {
    const int rc = in_handle_order(A, block, V0, nsv, right_vecs, stream, "spmm_svds: vectors and the handle's order",
                                   [&](const double* v0, double* vec) {
                                       return eigs_impl(A, 1, nsv, block, max_basis, max_restarts, tol, xtype, v0,
                                                        svals, vec, resid, restarts_out, stream);
                                   });
    if (rc == SPMM_OK)
        for (int i = 0; i < nsv; ++i) svals[i] = std::sqrt(std::max(0.0, svals[i]));
    return rc;
}

// ---------------------------------------------------------------- filtered subspace iteration
// The block of s vectors U is multiplied by the Chebyshev polynomial of degree
// d that is bounded by 1 on [lower, cut] and grows fastest above it (cut = the
// smallest Ritz value of the block, so every wanted direction is amplified
// against the rest), in FP32 through d block SpMMs; the filtered block is then
// orthonormalised (CholQR2) and Rayleigh-Ritz projected with S (one more SpMM)
// in FP64.  The three-term recurrence is scaled to stay O(1) at the largest
// Ritz value (Zhou and Saad's scaled Chebyshev filter):
//   e = (cut - lower) / 2, c = (cut + lower) / 2, s1 = e / (top - c)
//   Y1 = (s1 / e) (S - c) Y0
//   Y{j+1} = (2 s{j+1} / e) (S - c) Yj - sj s{j+1} Y{j-1},  s{j+1} = 1 / (2 / s1 - sj)
// The d filter steps run as one CUDA graph, captured on the first iteration
// and relaunched with new coefficients.
static int eigs_filtered_impl(spmm_mat_t S, int32_t nev, int32_t block, int32_t degree, double lower,
                              int32_t max_iters, double tol, spmm_dtype xtype, const double* V0, double* evals,
                              double* evecs, double* resid, int32_t* iters_out, void* stream) {
    if (!S || !V0 || !evals) { set_error("spmm_eigs_filtered: NULL argument"); return SPMM_ERR_ARG; }
    NvtxRange range("spmm_eigs_filtered");
    const int64_t n = S->fwd.n_rows;
    if (S->fwd.n_cols != n || n < 1) { set_error("spmm_eigs_filtered: the matrix must be square"); return SPMM_ERR_ARG; }
    if (nev < 1 || block < nev + 1 || block > kEigMaxBasis || block > n || degree < 1 || degree > 1000 ||
        max_iters < 0 || !(tol > 0.0) || !std::isfinite(lower)) {
        set_error("spmm_eigs_filtered: need nev + 1 <= block <= min(64, n), 1 <= degree <= 1000, max_iters >= 0, "
                  "tol > 0, a finite lower bound");
        return SPMM_ERR_ARG;
    }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16) { set_error("spmm_eigs_filtered: xtype must be F32 or BF16"); return SPMM_ERR_ARG; }
    if (S->vtype == SPMM_F16 || (S->vtype == SPMM_BF16 && xtype != SPMM_BF16)) {
        set_error("spmm_eigs_filtered: 16-bit values need X of the same type (use F32 values)");
        return SPMM_ERR_UNSUPPORTED;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int b = block;
    Eig E;
    E.A = S;
    E.n = n;
    E.m = b;
    E.b = b;
    // the Rayleigh-Ritz product S U reads U in FP32 (xtype is the filter's
    // SpMM input): with BF16 there, the residuals could not fall below BF16's
    // rounding of U
    E.xtype = S->vtype == SPMM_BF16 ? SPMM_BF16 : SPMM_F32;
    E.grid = std::max(1, sms * 8);
    E.chunk = std::max<int64_t>(1024, (n + 1023) / 1024);
    E.nchunks = (int)((n + E.chunk - 1) / E.chunk);
    float* Yc[3] = {nullptr, nullptr, nullptr};
    float* coef = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = SPMM_OK;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err, const char* what) { rc = cuda_fail(err, what); };
    const int64_t nb = n * b;
    do {
        if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess) { fail(e, "spmm_eigs_filtered: stream"); break; }
        if ((e = cudaStreamCreateWithFlags(&E.s, cudaStreamNonBlocking)) != cudaSuccess) { fail(e, "spmm_eigs_filtered: stream"); break; }
        const size_t nm = (size_t)nb * sizeof(double);
        if ((e = cudaMalloc((void**)&E.V, nm)) != cudaSuccess || (e = cudaMalloc((void**)&E.AV, nm)) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.U, nm)) != cudaSuccess || (e = cudaMalloc((void**)&E.AU, nm)) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.W, nm)) != cudaSuccess || (e = cudaMalloc((void**)&E.W2, nm)) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.part, (size_t)E.nchunks * b * b * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.small, (size_t)b * b * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.theta, (size_t)b * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&E.Yf, (size_t)nb * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&E.Xs, (size_t)nb * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&Yc[0], (size_t)nb * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&Yc[1], (size_t)nb * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&Yc[2], (size_t)nb * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&coef, (size_t)degree * 3 * sizeof(float))) != cudaSuccess) {
            fail(e, "spmm_eigs_filtered: workspace");
            break;
        }
        // U = orthonormalised start block; SU = S U; Rayleigh-Ritz
        copy_block_kernel<<<E.grid, kEigThreads, 0, E.s>>>(V0, b, b, n, E.W, b);
        if (!E.orthonormalize(0, e)) {
            if (e != cudaSuccess) fail(e, "spmm_eigs_filtered: orthonormalise");
            else { set_error("spmm_eigs_filtered: the start block is rank-deficient"); rc = SPMM_ERR_ARG; }
            break;
        }
        std::swap(E.V, E.W);                        // V = U (ld b)
        std::vector<double> T, th, Y, Rn, thk((size_t)b), best_res((size_t)b, 0.0);
        int it = 0;
        for (;; ++it) {
            if ((rc = E.apply_block(E.V, b, E.AV, b)) != SPMM_OK) break;
            if ((e = E.tn(E.V, b, b, E.AV, b, b, T)) != cudaSuccess) { fail(e, "spmm_eigs_filtered: projection"); break; }
            for (int i = 0; i < b; ++i)
                for (int j = i + 1; j < b; ++j) {
                    const double a = 0.5 * (T[(size_t)i * b + j] + T[(size_t)j * b + i]);
                    T[(size_t)i * b + j] = a;
                    T[(size_t)j * b + i] = a;
                }
            jacobi_eigh(b, T, th, Y);
            std::vector<int> order(b);
            for (int i = 0; i < b; ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return th[x] > th[y]; });
            std::vector<double> Yk((size_t)b * b);
            for (int c = 0; c < b; ++c) {
                thk[c] = th[order[c]];
                for (int r = 0; r < b; ++r) Yk[(size_t)r * b + c] = Y[(size_t)r * b + order[c]];
            }
            // Ritz vectors and their images; residual norms
            if ((e = E.nn(E.V, b, b, Yk, b, E.U, b, 1.0, 0.0)) != cudaSuccess ||
                (e = E.nn(E.AV, b, b, Yk, b, E.AU, b, 1.0, 0.0)) != cudaSuccess) {
                fail(e, "spmm_eigs_filtered: Ritz vectors");
                break;
            }
            std::swap(E.V, E.U);
            std::swap(E.AV, E.AU);
            cudaMemcpyAsync(E.theta, thk.data(), b * sizeof(double), cudaMemcpyHostToDevice, E.s);
            residual_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.AV, E.V, E.theta, b, n, E.W2);
            if ((e = E.tn(E.W2, b, b, E.W2, b, b, Rn)) != cudaSuccess) { fail(e, "spmm_eigs_filtered: residuals"); break; }
            double worst = 0.0;
            for (int i = 0; i < b; ++i) best_res[i] = std::sqrt(std::max(0.0, Rn[(size_t)i * b + i]));
            for (int i = 0; i < nev; ++i) worst = std::max(worst, best_res[i]);
            if (worst <= tol || it >= max_iters) break;
            // ---- filter the block: coefficients for this interval
            const double cut = thk[b - 1], top = thk[0];
            if (!(cut > lower) || !(top > cut)) {
                set_error("spmm_eigs_filtered: the block's Ritz values do not lie above the lower bound "
                          "(give a lower bound of the spectrum, or a larger block)");
                rc = SPMM_ERR_ARG;
                break;
            }
            const double ee = 0.5 * (cut - lower), cc = 0.5 * (cut + lower), s1 = ee / (top - cc);
            std::vector<float> cf((size_t)degree * 3);
            double sj = s1;
            for (int j = 0; j < degree; ++j) {
                double al, be, ga;
                if (j == 0) {
                    al = s1 / ee;
                    be = -al * cc;
                    ga = 0.0;
                } else {
                    const double sn = 1.0 / (2.0 / s1 - sj);
                    al = 2.0 * sn / ee;
                    be = -al * cc;
                    ga = -sj * sn;
                    sj = sn;
                }
                cf[(size_t)j * 3] = (float)al;
                cf[(size_t)j * 3 + 1] = (float)be;
                cf[(size_t)j * 3 + 2] = (float)ga;
            }
            if ((e = cudaMemcpyAsync(coef, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice, E.s)) !=
                cudaSuccess) {
                fail(e, "spmm_eigs_filtered: coefficients");
                break;
            }
            // Y0 = U in FP32
            f64_to_x_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.V, b, b, n, Yc[0], 0);
            if (!exec) {
                // steps 1..d on rotating buffers: Y{j} in Yc[j % 3]
                cudaGraph_t graph = nullptr;
                if ((e = cudaStreamBeginCapture(E.s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
                    fail(e, "spmm_eigs_filtered: capture");
                    break;
                }
                for (int j = 0; j < degree && rc == SPMM_OK; ++j) {
                    float* yc = Yc[j % 3];
                    float* yp = j > 0 ? Yc[(j + 2) % 3] : nullptr;
                    float* yn = Yc[(j + 1) % 3];
                    const void* X = yc;
                    if (xtype == SPMM_BF16) {
                        f32_to_bf16_kernel<<<E.grid, kEigThreads, 0, E.s>>>(yc, nb, static_cast<__nv_bfloat16*>(E.Xs));
                        X = E.Xs;
                    }
                    rc = apply_dev(S, 0, X, b, b, xtype, E.Yf, b, E.s);
                    if (rc == SPMM_OK)
                        cheb_step_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.Yf, yc, yp, yn, nb, coef + (size_t)j * 3);
                }
                const cudaError_t ec = cudaStreamEndCapture(E.s, &graph);
                if (rc == SPMM_OK && ec != cudaSuccess) fail(ec, "spmm_eigs_filtered: end capture");
                if (rc == SPMM_OK && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
                    exec = nullptr;
                    fail(e, "spmm_eigs_filtered: instantiate");
                }
                if (graph) cudaGraphDestroy(graph);
                if (rc != SPMM_OK) break;
            }
            if ((e = cudaGraphLaunch(exec, E.s)) != cudaSuccess) { fail(e, "spmm_eigs_filtered: filter"); break; }
            // the filtered block, orthonormalised, is the next U
            f32_to_f64_kernel<<<E.grid, kEigThreads, 0, E.s>>>(Yc[degree % 3], b, n, E.W, b);
            if (!E.orthonormalize(0, e)) {
                if (e != cudaSuccess) fail(e, "spmm_eigs_filtered: orthonormalise");
                else {
                    set_error("spmm_eigs_filtered: the filtered block lost rank (lower the degree)");
                    rc = SPMM_ERR_ARG;
                }
                break;
            }
            std::swap(E.V, E.W);
        }
        if (rc != SPMM_OK) break;
        for (int i = 0; i < nev; ++i) {
            evals[i] = thk[i];
            if (resid) resid[i] = best_res[i];
        }
        if (evecs) copy_block_kernel<<<E.grid, kEigThreads, 0, E.s>>>(E.V, b, nev, n, evecs, nev);
        if (iters_out) *iters_out = it;
        if ((e = cudaStreamSynchronize(E.s)) != cudaSuccess) { fail(e, "spmm_eigs_filtered: run"); break; }
        int32_t st = 0;
        if ((e = cudaMemcpy(&st, S->status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fail(e, "spmm_eigs_filtered: status");
            break;
        }
        if (st != 0) {
            cudaMemset(S->status, 0, sizeof(int32_t));
            set_error("spmm_eigs_filtered: a device-side staging wait timed out; the result is incomplete");
            rc = SPMM_ERR_TIMEOUT;
        }
    } while (0);
    if (E.s) {
        cudaStreamSynchronize(E.s);
        cudaStreamDestroy(E.s);
    }
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(E.V); cudaFree(E.AV); cudaFree(E.U); cudaFree(E.AU); cudaFree(E.W); cudaFree(E.W2);
    cudaFree(E.part); cudaFree(E.small); cudaFree(E.theta); cudaFree(E.Yf); cudaFree(E.Xs);
    cudaFree(Yc[0]); cudaFree(Yc[1]); cudaFree(Yc[2]); cudaFree(coef);
    return rc;
}

extern "C" int spmm_eigs_filtered(spmm_mat_t S, int32_t nev, int32_t block, int32_t degree, double lower,
                                  int32_t max_iters, double tol, spmm_dtype xtype, const double* V0, double* evals,
                                  double* evecs, double* resid, int32_t* iters_out, void* stream) {
    return in_handle_order(S, block, V0, nev, evecs, stream, "spmm_eigs_filtered: vectors and the handle's order",
                           [&](const double* v0, double* vec) {
                               return eigs_filtered_impl(S, nev, block, degree, lower, max_iters, tol, xtype, v0,
                                                         evals, vec, resid, iters_out, stream);
                           });
}
