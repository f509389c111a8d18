// combine.cu -- second pass for split (hub) rows: Y[row, :] = sum of the row's
// segment partials, added in a fixed order so the result is the same on every
// run.  The partials of a call with k columns are packed k floats per slot
// (slot s at s * k), so a small k reads only the floats it needs.
#include "internal.h"

namespace spmm {

// One warp per split row.  With k < 32 the warp is cut into SG = 32 / L
// segment groups of L lanes (L the smallest power of two >= k): group g adds
// segments g, g + SG, ... in order, then the groups' sums are added by a
// fixed xor-shuffle tree, so the result is the same on every run.
// Compensated partials are added in segment order by one group (SG = 1).
__device__ __forceinline__ void combine_row(const int4 sp, const float* __restrict__ partials, float* __restrict__ Y,
                                            int64_t ldy, int32_t k, int32_t lanes_log2,
                                            const float* __restrict__ pcomp, int lane) {
    if (pcomp) {                               // Neumaier summation of (sum, compensation) partials
        for (int c = lane; c < k; c += 32) {
            const int64_t base = (int64_t)sp.z * k + c;
            float acc = 0.f, cmp = 0.f;
            for (int q = 0; q < sp.y; ++q) {
                const float x = __ldcg(partials + base + (int64_t)q * k);
                const float t = acc + x;
                cmp += ((fabsf(acc) >= fabsf(x)) ? (acc - t) + x : (x - t) + acc) +
                       __ldcg(pcomp + base + (int64_t)q * k);
                acc = t;
            }
            Y[(int64_t)sp.x * ldy + c] = acc + cmp;
        }
        return;
    }
    const int L = 1 << lanes_log2, SG = 32 >> lanes_log2;
    const int g = lane >> lanes_log2, li = lane & (L - 1);
    for (int c0 = 0; c0 < k; c0 += L) {        // one pass unless k > 32
        const int c = c0 + li;
        const float* p = partials + (int64_t)sp.z * k + c;
        float acc = 0.f;
        if (c < k) {
            int q = g;
            for (; q + 7 * SG < sp.y; q += 8 * SG) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (int64_t)(q + u * SG) * k);
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += v[u];
            }
            for (; q < sp.y; q += SG) acc += __ldcg(p + (int64_t)q * k);
        }
        for (int off = L; off < 32; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (g == 0 && c < k) Y[(int64_t)sp.x * ldy + c] = acc;
    }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
combine_kernel(const int4* __restrict__ splits, int64_t n_splits, const float* __restrict__ partials,
               float* __restrict__ Y, int64_t ldy, int32_t k, int32_t lanes_log2, const float* __restrict__ pcomp) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + w;
    if (s >= n_splits) return;                 // whole warps
    combine_row(splits[s], partials, Y, ldy, k, lanes_log2, pcomp, lane);
}

// the split rows of several matrices (spmm_apply_batched): warp s takes split
// row s of the concatenated lists, entry e owning rows off[e] .. off[e+1]-1
__global__ void __launch_bounds__(kWarpsPerBlock * 32) combine_multi_kernel(const __grid_constant__ CombineMulti m) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + w;
    if (s >= m.off[m.n]) return;
    int lo = 0, hi = m.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m.off[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    const CombineEntry& E = m.ent[lo];
    combine_row(E.splits[s - m.off[lo]], E.partials, E.Y, E.ldy, E.k, E.lanes_log2, E.pcomp, lane);
}

static int combine_lanes_log2(int32_t k) {
    int lg = 0;
    while ((1 << lg) < k && lg < 5) ++lg;
    return lg;
}

cudaError_t launch_combine_multi(CombineMulti& m, cudaStream_t s) {
    m.off[0] = 0;
    for (int e = 0; e < m.n; ++e) {
        m.ent[e].lanes_log2 = combine_lanes_log2(m.ent[e].k);
        m.off[e + 1] = m.off[e] + m.ent[e].n_splits;
    }
    if (m.off[m.n] <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((m.off[m.n] + kWarpsPerBlock - 1) / kWarpsPerBlock));
    combine_multi_kernel<<<grid, kWarpsPerBlock * 32, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_combine(const int4* splits, int64_t n_splits, const float* partials, float* Y,
                           int64_t ldy, int32_t k, cudaStream_t s, const float* partials_comp) {
    if (n_splits <= 0) return cudaSuccess;
    const int lg = combine_lanes_log2(k);
    const dim3 block(kWarpsPerBlock * 32);
    const dim3 grid((unsigned)((n_splits + kWarpsPerBlock - 1) / kWarpsPerBlock));
    combine_kernel<<<grid, block, 0, s>>>(splits, n_splits, partials, Y, ldy, k, lg, partials_comp);
    return cudaGetLastError();
}

}  // namespace spmm
