// combine.cu -- second pass for split (hub) rows: Y[row, :] = sum of the row's
// segment partials, added in segment order so the result is the same on
// every run.  One warp per split row; lanes cover the k columns; eight
// partial loads are issued before they are added.
#include "internal.h"

namespace spmm {

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
combine_kernel(const int4* __restrict__ splits, int64_t n_splits, const float* __restrict__ partials,
               float* __restrict__ Y, int64_t ldy, int32_t k, const float* __restrict__ pcomp) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + w;
    if (s >= n_splits) return;
    const int4 sp = splits[s];                 // {row, nseg, slot0, 0}
    if (pcomp) {                               // Neumaier summation of (sum, compensation) partials
        for (int c = lane; c < k; c += 32) {
            const int64_t base = (int64_t)sp.z * kSlotStride + c;
            float acc = 0.f, cmp = 0.f;
            for (int q = 0; q < sp.y; ++q) {
                const float x = __ldcg(partials + base + (int64_t)q * kSlotStride);
                const float t = acc + x;
                cmp += ((fabsf(acc) >= fabsf(x)) ? (acc - t) + x : (x - t) + acc) +
                       __ldcg(pcomp + base + (int64_t)q * kSlotStride);
                acc = t;
            }
            Y[(int64_t)sp.x * ldy + c] = acc + cmp;
        }
        return;
    }
    for (int c = lane; c < k; c += 32) {
        const float* p = partials + (int64_t)sp.z * kSlotStride + c;
        float acc = 0.f;
        int q = 0;
        for (; q + 8 <= sp.y; q += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (int64_t)(q + u) * kSlotStride);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u];
        }
        for (; q < sp.y; ++q) acc += __ldcg(p + (int64_t)q * kSlotStride);
        Y[(int64_t)sp.x * ldy + c] = acc;
    }
}

cudaError_t launch_combine(const int4* splits, int64_t n_splits, const float* partials, float* Y,
                           int64_t ldy, int32_t k, cudaStream_t s, const float* partials_comp) {
    if (n_splits <= 0) return cudaSuccess;
    const dim3 block(kWarpsPerBlock * 32);
    const dim3 grid((unsigned)((n_splits + kWarpsPerBlock - 1) / kWarpsPerBlock));
    combine_kernel<<<grid, block, 0, s>>>(splits, n_splits, partials, Y, ldy, k, partials_comp);
    return cudaGetLastError();
}

}  // namespace spmm
