// rows_kernel.cuh -- the SpMM task kernel, Y = A X for one CSR orientation.
//
// Section 3.4 / Algorithm 1 of the paper: a nonzero a_ij scales the whole
// dense row X[j, :] into output row i, the row operation is vectorised (AVX
// in the paper, 16-byte lane loads here), and each output row has a single
// owner.
//
// Persistent warps walk the task list (plan.cpp), claiming their next tasks
// from an atomic counter (one task at a time for wide X rows, a few for narrow
// ones; FwdArgs::task_ctr), or, without a counter, with a stride of the grid's
// warp count.  Each warp stages a task's column indices, values and row
// pointers into shared memory with bulk asynchronous copies (cp.async.bulk,
// completion on an mbarrier) one task ahead, so the copy of task i+1 overlaps
// the gathers of task i -- the GPU form of the paper's asynchronous tile-row
// reads (Algorithm 1: read the tile rows asynchronously, multiply once they
// have arrived).  Every wait on a copy is bounded; on timeout the warp sets a
// status word, waits (bounded) for its other copy and exits.
//
// A warp is cut into G = 32 / LANES lane groups; LANES lanes cover one X row
// (each lane VEC consecutive elements, CH chunks of them).
//   short-row task: group g owns rows g, g+G, ... of the run and sums each
//                   row's nonzeros in order (with one lane per X row, k = 1
//                   takes the flat path and rows of up to 8 bytes the
//                   merge-based path; the MG instantiations cut the run
//                   into equal pieces per lane group instead: all three
//                   are described at their branches);
//   long row / hub segment: group g takes nonzeros g, g+G, g+2G, ...; the
//                   groups' partial sums are added by a fixed xor-shuffle
//                   tree; a segment writes its sum to a partial slot.
// All summation orders are fixed, so repeated calls give identical results.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>
#include <type_traits>

#include "internal.h"

namespace spmm {

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared; both addresses 16-byte aligned, bytes % 16
// == 0.  `policy` is an L2 cache policy (the streamed matrix is marked
// evict-first so it does not push the gathered X rows out of L2).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// read-only global loads with an L2 cache policy
__device__ __forceinline__ float4 ldg_f4(const float* p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ldg_f2(const float* p, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldg_f1(const float* p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint4 ldg_u4(const void* p, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ldg_u2(const void* p, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ldg_u1(const void* p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ldg_u16(const void* p, uint64_t pol) {
    unsigned short v;
    asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of `bar`; false if it did not complete within limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// ------------------------------------------------------- element loading --
template <typename XT>
__device__ __forceinline__ float bits_to_f32(uint32_t b);
template <>
__device__ __forceinline__ float bits_to_f32<__nv_bfloat16>(uint32_t b) {
    return __uint_as_float(b << 16);
}
template <>
__device__ __forceinline__ float bits_to_f32<__half>(uint32_t b) {
    return __half2float(__ushort_as_half((unsigned short)b));
}

// VEC consecutive elements of X held as loaded (16-bit types stay packed two
// per 32-bit word until they are used, which halves the registers that hold
// loads in flight).  p is aligned to VEC * sizeof(XT).
template <typename XT, int VEC>
struct XVec {
    static_assert(sizeof(XT) == 2, "16-bit element path");
    static constexpr int kWords = (VEC + 1) / 2;
    uint32_t w[kWords];
    __device__ __forceinline__ void load(const XT* p, uint64_t pol) {
        if constexpr (VEC == 8) {
            uint4 v = ldg_u4(p, pol);
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
        } else if constexpr (VEC == 4) {
            uint2 v = ldg_u2(p, pol);
            w[0] = v.x; w[1] = v.y;
        } else if constexpr (VEC == 2) {
            w[0] = ldg_u1(p, pol);
        } else {
            w[0] = ldg_u16(p, pol);
        }
    }
    __device__ __forceinline__ float get(int i) const {
        return bits_to_f32<XT>((i & 1) ? (w[i >> 1] >> 16) : (w[i >> 1] & 0xffffu));
    }
    // the same elements from shared memory (VEC <= 2: rows of at most 4 bytes)
    __device__ __forceinline__ void load_sh(const XT* p) {
        static_assert(VEC <= 2, "shared-memory rows of at most 4 bytes");
        if constexpr (VEC == 2) w[0] = *reinterpret_cast<const uint32_t*>(p);
        else w[0] = *reinterpret_cast<const unsigned short*>(p);
    }
};

template <int VEC>
struct XVec<float, VEC> {
    float f[VEC];
    __device__ __forceinline__ void load(const float* p, uint64_t pol) {
        if constexpr (VEC == 4) {
            float4 v = ldg_f4(p, pol);
            f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
        } else if constexpr (VEC == 2) {
            float2 v = ldg_f2(p, pol);
            f[0] = v.x; f[1] = v.y;
        } else {
            f[0] = ldg_f1(p, pol);
        }
    }
    __device__ __forceinline__ float get(int i) const { return f[i]; }
    __device__ __forceinline__ void load_sh(const float* p) {
        static_assert(VEC == 1, "shared-memory rows of at most 4 bytes");
        f[0] = *p;
    }
};

// Store VEC floats to an address aligned to min(VEC, 4) * 4 bytes.
template <int VEC>
__device__ __forceinline__ void store_y(float* p, const float (&v)[VEC]) {
    if constexpr (VEC >= 4) {
#pragma unroll
        for (int i = 0; i < VEC; i += 4)
            __stcs(reinterpret_cast<float4*>(p + i), make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
    } else if constexpr (VEC == 2) {
        __stcs(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
    } else {
        __stcs(p, v[0]);
    }
}

// value of staged entry i (shared memory, raw bytes of the stored type)
template <int VMODE>
__device__ __forceinline__ float staged_val(const unsigned char* v, int i) {
    if constexpr (VMODE == 1) return reinterpret_cast<const float*>(v)[i];
    if constexpr (VMODE == 2) return __uint_as_float((uint32_t)reinterpret_cast<const unsigned short*>(v)[i] << 16);
    if constexpr (VMODE == 3) return __half2float(__ushort_as_half(reinterpret_cast<const unsigned short*>(v)[i]));
    return 1.0f;
}

template <int VMODE>
struct Layout {
    static constexpr int kValBytes = VMODE == 0 ? 0 : (VMODE == 1 ? 4 : 2);
    static constexpr int kColOff = 0;
    static constexpr int kValOff = kColBufInts * 4;
    static constexpr int kRpOff = kValOff + (VMODE ? kValBufBytes : 0);
    static constexpr int kBuf = kRpOff + kRpBufLongs * 8;       // bytes per staging buffer
    static constexpr int kWarp = 2 * kBuf + 16;                 // two buffers + two mbarriers
    static constexpr int kBlock = kWarpsPerBlock * kWarp;
    static_assert(kBuf % 16 == 0 && kWarp % 16 == 0, "16-byte aligned staging buffers");
};

struct Staged {
    const int32_t* col;         // col[i] = column of nonzero e0 + i
    const unsigned char* val;   // raw value bytes, entry i = nonzero e0 + i
    const int64_t* rp;          // rp[j] = row_ptr[r0 + j] (short-row tasks)
};

__device__ __forceinline__ int64_t desc_e0(const int4 d) {
    return ((int64_t)(uint32_t)d.z) | ((int64_t)d.w << 32);
}

// Issue the bulk copies of one task into staging buffer `buf` (lane 0 only).
// Windows are widened to 16-byte boundaries; the arrays are padded on the
// device so the widened end stays inside the allocation.
template <int VMODE>
__device__ __forceinline__ void issue_task(const FwdArgs& a, const int4 d0, const int4 d1, unsigned char* buf,
                                           uint64_t* bar, uint64_t pol) {
    using Lay = Layout<VMODE>;
    const int64_t e0 = desc_e0(d0), e1 = desc_e0(d1);
    const int64_t cs = e0 & ~(int64_t)3, ce = (e1 + 3) & ~(int64_t)3;
    const uint32_t cbytes = (uint32_t)((ce - cs) * 4);
    uint32_t vbytes = 0, rbytes = 0;
    int64_t vs = 0, rs = 0;
    if constexpr (VMODE != 0) {
        constexpr int epb = 16 / Lay::kValBytes;
        vs = e0 & ~(int64_t)(epb - 1);
        const int64_t ve = (e1 + epb - 1) & ~(int64_t)(epb - 1);
        vbytes = (uint32_t)((ve - vs) * Lay::kValBytes);
    }
    if (d0.y > 0) {
        rs = (int64_t)d0.x & ~(int64_t)1;
        const int64_t re = ((int64_t)d0.x + d0.y + 2) & ~(int64_t)1;
        rbytes = (uint32_t)((re - rs) * 8);
    }
    mbar_arrive_expect_tx(bar, cbytes + vbytes + rbytes);
    if (cbytes) bulk_g2s(buf + Lay::kColOff, a.col_idx + cs, cbytes, bar, pol);
    if constexpr (VMODE != 0)
        if (vbytes)
            bulk_g2s(buf + Lay::kValOff, reinterpret_cast<const unsigned char*>(a.val) + vs * Lay::kValBytes, vbytes,
                     bar, pol);
    if (rbytes) bulk_g2s(buf + Lay::kRpOff, a.row_ptr + rs, rbytes, bar, pol);
}

#ifndef SPMM_UNROLL_BYTES
#define SPMM_UNROLL_BYTES 64      // X bytes in flight per lane
#endif
#ifndef SPMM_K1_FLAT
#define SPMM_K1_FLAT 1            // k = 1 short-row runs: flat gather through shared memory
#endif
#ifndef SPMM_FLAT_UF
#define SPMM_FLAT_UF 8            // k = 1 flat path: nonzeros gathered per lane per round
#endif
#ifndef SPMM_MERGE
#define SPMM_MERGE 1              // one lane per X row: merge-based short-row runs
#endif

#ifndef SPMM_MIN_BLOCKS
#define SPMM_MIN_BLOCKS 3         // resident blocks per SM the register budget targets (80 registers)
#endif

// Resident blocks per SM that the register budget of an instantiation targets.
// Three blocks (80 registers a thread) measured faster than four (64) for
// every path but the pattern group merge over rows on 8 or more lanes
// (R-MAT scale 24, FP32: k = 1 1.10 -> 0.93 ms, k = 8 2.23 -> 1.92, 30
// PageRank iterations 35.9 -> 31.6 ms; k = 32 4.20 -> 4.34, k = 64
// 7.59 -> 7.91), which keeps four in its own variant (MG == 2).
template <int VMODE, int MG>
constexpr int min_blocks() {
    return (MG == 2 && VMODE == 0) ? 4 : SPMM_MIN_BLOCKS;
}

// ONE: one lane per X row (k == VEC, CH == 1); the lane geometry is then a
// compile-time constant and short-row runs take the flat (k = 1) or, for X
// rows of up to 8 bytes, the merge-based path.  MG != 0: several lanes per X
// row (CH == 1) and short-row runs merge-based over lane groups, with 3
// blocks per SM and 4 nonzeros in flight per group (MG == 1) or 4 blocks and
// 2 in flight (MG == 2).
// Warps per block: kWarpsPerBlock, or kHotWarps in one block per SM for the
// instantiations that keep the hot rows of X in shared memory (HOT).
template <bool HOT>
constexpr int warps_per_block() {
    return HOT ? kHotWarps : kWarpsPerBlock;
}

// HOT: one lane per X row of at most 4 bytes; a negative column index c
// names row ~c of the hot rows of X, which the block copies into shared
// memory (after its warps' staging buffers) before its first task, so those
// gathers leave the L1-to-L2 request path alone (hot.cu).
// MULTI: the tasks of several matrices (MultiArgs M, spmm_apply_batched),
// numbered one after the other; every task takes the matrix, X, Y, k and
// lane geometry of its own entry.  ga holds the launch-wide fields (task
// count, counter, status, wait bound).
template <typename XT, int VMODE, int VEC, int CH, bool COMP, bool ONE, int MG, bool HOT, bool MULTI>
__device__ __forceinline__ void rows_run(const FwdArgs& ga, const MultiArgs* M) {
    static_assert(!MULTI || (!ONE && MG == 0 && !HOT), "batched launches use the generic row walk");
    static_assert(!ONE || CH == 1, "one lane per row needs CH == 1");
    static_assert(MG == 0 || (!ONE && CH == 1), "merge over lane groups needs several lanes and CH == 1");
    static_assert(!HOT || (ONE && MG == 0 && VEC * sizeof(XT) <= 4), "hot rows in shared memory: <= 4-byte rows");
    constexpr int WPB = warps_per_block<HOT>();
    constexpr bool kFlat = ONE && VEC == 1 && SPMM_K1_FLAT;
    // merge-based runs pay off for X rows of up to 8 bytes; for 16-byte rows
    // (mostly gathered from DRAM) the row-per-lane walk measured faster
    constexpr bool kMerge = ONE && !kFlat && SPMM_MERGE && VEC * sizeof(XT) <= 8;
    // the same over lane groups, for rows that need several lanes (MG)
    constexpr bool kMergeG = MG != 0;
    using Lay = Layout<VMODE>;
    // nonzeros in flight per lane group
    constexpr int kBytes = VEC * CH * (int)sizeof(XT);
    constexpr int kU = SPMM_UNROLL_BYTES / kBytes;
    constexpr int U = kU < 2 ? 2 : (kU > 8 ? 8 : kU);
#ifndef SPMM_MERGE_UNROLL
#define SPMM_MERGE_UNROLL 2
#endif
    constexpr int UM = U < SPMM_MERGE_UNROLL ? U : SPMM_MERGE_UNROLL;   // merge path: nonzeros in flight per lane
#ifndef SPMM_MERGE_WIDE_UNROLL
#define SPMM_MERGE_WIDE_UNROLL 4
#endif
    // merge over lane groups: nonzeros in flight per group (4 spill at 64
    // registers, and with staged values at 80)
    constexpr int kUW = (MG == 1 && VMODE == 0) ? SPMM_MERGE_WIDE_UNROLL : 2;
    constexpr int UW = U < kUW ? U : kUW;
    extern __shared__ __align__(128) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wb = smem + w * Lay::kWarp;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wb + 2 * Lay::kBuf);
    const FwdArgs& a = ga;      // launch-wide fields (and, unless MULTI, the matrix's)
    const XT* hs = nullptr;     // hot rows of X in shared memory (HOT)
    if constexpr (HOT) {
        // one bulk copy of the packed hot rows, before any warp leaves
        uint64_t* hbar = reinterpret_cast<uint64_t*>(smem + WPB * Lay::kWarp);
        hs = reinterpret_cast<const XT*>(smem + WPB * Lay::kWarp + 16);
        if (threadIdx.x == 0) {
            mbar_init(hbar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(hbar, (uint32_t)a.hot_bytes);
            bulk_g2s(const_cast<XT*>(hs), a.Xh, (uint32_t)a.hot_bytes, hbar, policy_evict_last());
        }
        if (!mbar_wait_bounded(hbar, 0, a.wait_ns)) {
            if (threadIdx.x == 0) atomicOr(a.status, kStatusTimeout);
            // the copy may still be in flight: wait for it (bounded) before leaving
            mbar_wait_bounded(hbar, 0, a.wait_ns);
            return;
        }
    }

    const int64_t W = (int64_t)gridDim.x * WPB;
    int64_t t = (int64_t)blockIdx.x * WPB + w;
    if (t >= a.n_tasks) return;
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // the entry of task t (MULTI: a binary search of the entries' first tasks)
    // and its two descriptors
    auto fetch = [&](int64_t tt, int4& x0, int4& x1) -> int {
        if constexpr (MULTI) {
            int lo = 0, hi = M->n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (M->off[mid] <= tt) lo = mid;
                else hi = mid - 1;
            }
            const int64_t tl = tt - M->off[lo];
            x0 = M->ent[lo].tasks[tl];
            x1 = M->ent[lo].tasks[tl + 1];
            return lo;
        } else {
            x0 = a.tasks[tt];
            x1 = a.tasks[tt + 1];
            return 0;
        }
    };
    auto entry = [&](int e) -> const FwdArgs& {
        if constexpr (MULTI) return M->ent[e];
        else return a;
    };

    // lane geometry (of the current task's entry when MULTI)
    int lg = 0, LANES = 1, G = 32, g = 0, li = 0;
    bool act[CH];
    const XT* xb = nullptr;
    const uint64_t apol = policy_evict_first();
    uint64_t xpol = 0;
    const FwdArgs* cur = &a;    // the entry of the task being computed
    auto set_geometry = [&](const FwdArgs& E) {
        lg = ONE ? 0 : E.lanes_log2;
        LANES = 1 << lg;
        G = 32 >> lg;
        g = lane >> lg;
        li = lane & (LANES - 1);
#pragma unroll
        for (int c = 0; c < CH; ++c) act[c] = (li + c * LANES) < E.nvec;
        xb = reinterpret_cast<const XT*>(E.X) + (int64_t)li * VEC;
        xpol = E.x_evict_last ? policy_evict_last() : policy_evict_normal();
        cur = &E;
    };
    // load the X row of column index c (elements off.. of this lane's part)
    auto gather = [&](auto& xv, int64_t c, int off) {
        if constexpr (HOT) {
            if (c < 0) {
                xv.load_sh(hs + (int64_t)(~c) * VEC);
                return;
            }
        }
        xv.load(xb + c * cur->ldx + off, xpol);
    };
    int4 d0, d1;
    int ed = fetch(t, d0, d1);
    set_geometry(entry(ed));
    if (lane == 0) issue_task<VMODE>(entry(ed), d0, d1, wb, &bars[0], apol);
    // the next task: static stride, or the next of a chunk claimed from the
    // counter by lane 0
    int64_t cnext = 0, cend = 0;
    auto next_task = [&](int64_t cur) -> int64_t {
        if (!a.task_ctr) return cur + W;
        if (cnext < cend) return cnext++;
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(a.task_ctr, 1ull);
        cnext = W + (int64_t)__shfl_sync(0xffffffffu, v, 0) * a.task_chunk;
        cend = cnext + a.task_chunk;
        return cnext++;
    };
    int64_t tn = next_task(t);
    int4 n0 = make_int4(0, 0, 0, 0), n1 = n0;
    int en = 0;
    if (tn < a.n_tasks) en = fetch(tn, n0, n1);
    uint32_t phase = 0;     // bit b = parity to wait for on buffer b
    int b = 0;

    for (;;) {
        // stage the next task into the other buffer (its readers are done)
        if (tn < a.n_tasks) {
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async();
                issue_task<VMODE>(entry(en), n0, n1, wb + (b ^ 1) * Lay::kBuf, &bars[b ^ 1], apol);
            }
        }
        // prefetch the descriptor after next
        const int64_t tnn = tn < a.n_tasks ? next_task(tn) : a.n_tasks;
        int4 m0 = make_int4(0, 0, 0, 0), m1 = m0;
        int em = 0;
        if (tnn < a.n_tasks) em = fetch(tnn, m0, m1);

        if (!mbar_wait_bounded(&bars[b], (phase >> b) & 1u, a.wait_ns)) {
            if (lane == 0) atomicOr(a.status, kStatusTimeout);
            if (tn < a.n_tasks) mbar_wait_bounded(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u, a.wait_ns);
            return;
        }
        phase ^= 1u << b;

        // ---- compute task (d0, d1) from buffer b
        if constexpr (MULTI) {
            if (cur != &entry(ed)) set_geometry(entry(ed));
        }
        {
            const FwdArgs& a = *cur;   // the task's entry (the launch's matrix unless MULTI)
            const unsigned char* buf = wb + b * Lay::kBuf;
            const int64_t e0 = desc_e0(d0);
            const int n = (int)(desc_e0(d1) - e0);
            Staged st;
            st.col = reinterpret_cast<const int32_t*>(buf + Lay::kColOff) + (e0 & 3);
            if constexpr (VMODE != 0) {
                constexpr int epb = 16 / Lay::kValBytes;
                st.val = buf + Lay::kValOff + (e0 & (epb - 1)) * Lay::kValBytes;
            } else {
                st.val = nullptr;
            }
            st.rp = reinterpret_cast<const int64_t*>(buf + Lay::kRpOff) + (d0.x & 1);

            if (kFlat && d0.y > 0) {
                // k = 1, run of short rows: every lane gathers the task's
                // nonzeros as one flat array (lane, lane+32, ...) and writes each
                // product over its staged column index; then lane j adds the
                // products of rows j, j+32 in nonzero order from shared memory.
                const int nr = d0.y;
                int32_t* prod = const_cast<int32_t*>(st.col);
                constexpr int UF = SPMM_FLAT_UF;
                for (int base = 0; base < n; base += 32 * UF) {
                    float xv[UF], av[UF];
#pragma unroll
                    for (int u = 0; u < UF; ++u) {
                        const int idx = base + lane + 32 * u;
                        if (idx < n) {
                            const int64_t cidx = st.col[idx];
                            av[u] = staged_val<VMODE>(st.val, idx);
                            XVec<XT, 1> t1;
                            gather(t1, cidx, 0);
                            xv[u] = t1.get(0);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < UF; ++u) {
                        const int idx = base + lane + 32 * u;
                        if (idx < n) prod[idx] = __float_as_int(av[u] * xv[u]);
                    }
                }
                __syncwarp();
                for (int j = lane; j < nr; j += 32) {
                    const int s = (int)(st.rp[j] - e0), e = (int)(st.rp[j + 1] - e0);
                    float acc = 0.f;
                    for (int i = s; i < e; i += 4) {          // four loads in flight, added in order
                        const float p0 = __int_as_float(prod[i]);
                        const float p1 = i + 1 < e ? __int_as_float(prod[i + 1]) : 0.f;
                        const float p2 = i + 2 < e ? __int_as_float(prod[i + 2]) : 0.f;
                        const float p3 = i + 3 < e ? __int_as_float(prod[i + 3]) : 0.f;
                        acc += p0;
                        if (i + 1 < e) acc += p1;
                        if (i + 2 < e) acc += p2;
                        if (i + 3 < e) acc += p3;
                    }
                    __stcs(a.Y + (int64_t)(d0.x + j) * a.ldy, acc);
                }
                fence_proxy_async();   // the products were written where the next copy lands
            } else if (kMerge && d0.y > 0) {
                // run of short rows, one lane per X row (merge-based): the task's
                // nonzeros are cut into 32 equal contiguous pieces, lane l taking
                // piece l, so every lane gathers about n/32 rows of X whatever
                // the row lengths.  A lane walks its piece in order and stores
                // the rows that lie wholly inside it.  A row that crosses piece
                // boundaries leaves a tail partial in each lane it continues out
                // of and a head partial in the lane where it ends; a segmented
                // scan (shfl_up) over the lanes' tails, keyed by row,
                // adds the tails, and the ending lane adds its head last.
                const int nr = d0.y;
                for (int j = lane; j < nr; j += 32)       // rows without nonzeros
                    if (st.rp[j] == st.rp[j + 1]) {
                        float z[VEC];
#pragma unroll
                        for (int v = 0; v < VEC; ++v) z[v] = 0.f;
                        store_y<VEC>(a.Y + (int64_t)(d0.x + j) * a.ldy, z);
                    }
                const int per = (n + 31) >> 5;
                const int cs = min(n, lane * per), ce = min(n, cs + per);
                float tail[VEC], head[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) tail[v] = 0.f, head[v] = 0.f;
                int key = -1 - lane;                      // tail row, or a key no other lane has
                int hrow = -1;                            // head row
                if (cs < ce) {
                    // r: the row holding nonzero cs (largest r with rp[r] <= e0 + cs)
                    int lo = 0, hi = nr - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((int)(st.rp[mid] - e0) <= cs) lo = mid;
                        else hi = mid - 1;
                    }
                    int r = lo;
                    int rs = (int)(st.rp[r] - e0), re = (int)(st.rp[r + 1] - e0);
                    float acc[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
                    for (int i = cs; i < ce; i += UM) {
                        XVec<XT, VEC> xv[UM];
                        float av[UM];
#pragma unroll
                        for (int u = 0; u < UM; ++u)
                            if (i + u < ce) {
                                const int64_t cidx = st.col[i + u];
                                av[u] = staged_val<VMODE>(st.val, i + u);
                                gather(xv[u], cidx, 0);
                            }
#pragma unroll
                        for (int u = 0; u < UM; ++u)
                            if (i + u < ce) {
                                while (i + u >= re) {             // row r ended inside the piece
                                    if (rs < re) {
                                        if (rs >= cs) {
                                            store_y<VEC>(a.Y + (int64_t)(d0.x + r) * a.ldy, acc);
                                        } else {
                                            hrow = r;
#pragma unroll
                                            for (int v = 0; v < VEC; ++v) head[v] = acc[v];
                                        }
                                    }
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
                                    ++r;
                                    rs = re;
                                    re = (int)(st.rp[r + 1] - e0);
                                }
#pragma unroll
                                for (int v = 0; v < VEC; ++v) acc[v] = fmaf(av[u], xv[u].get(v), acc[v]);
                            }
                    }
                    // the row holding nonzero ce - 1
                    if (re > ce) {
                        key = r;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) tail[v] = acc[v];
                    } else if (rs >= cs) {
                        store_y<VEC>(a.Y + (int64_t)(d0.x + r) * a.ldy, acc);
                    } else {
                        hrow = r;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) head[v] = acc[v];
                    }
                }
                // segmented inclusive scan of the tails (a row's tails sit in
                // consecutive lanes, so equal keys bound a segment)
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int kup = __shfl_up_sync(0xffffffffu, key, off);
                    float up[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) up[v] = __shfl_up_sync(0xffffffffu, tail[v], off);
                    if (lane >= off && kup == key)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) tail[v] += up[v];
                }
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    const float prev = __shfl_up_sync(0xffffffffu, tail[v], 1);
                    head[v] = prev + head[v];
                }
                if (hrow >= 0) store_y<VEC>(a.Y + (int64_t)(d0.x + hrow) * a.ldy, head);
            } else if (kMergeG && d0.y > 0) {
                // run of short rows, LANES lanes per X row (merge-based over lane
                // groups): the task's nonzeros are cut into G equal contiguous
                // pieces, group g taking piece g, so every group gathers about
                // n/G rows of X whatever the row lengths.  As in the one-lane
                // case, a row crossing pieces is finished by a segmented scan
                // over the groups' tails (shfl_up by multiples of LANES, so lane
                // li of a group meets lane li of the others) and its head.
                const int nr = d0.y;
                for (int j = g; j < nr; j += G)           // rows without nonzeros
                    if (st.rp[j] == st.rp[j + 1] && act[0]) {
                        float z[VEC];
#pragma unroll
                        for (int v = 0; v < VEC; ++v) z[v] = 0.f;
                        store_y<VEC>(a.Y + (int64_t)(d0.x + j) * a.ldy + li * VEC, z);
                    }
                const int per = (n + G - 1) / G;
                const int cs = min(n, g * per), ce = min(n, cs + per);
                float tail[VEC], head[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) tail[v] = 0.f, head[v] = 0.f;
                int key = -1 - g;                         // tail row, or a key no other group has
                int hrow = -1;                            // head row
                if (cs < ce) {
                    int lo = 0, hi = nr - 1;              // the row holding nonzero cs
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((int)(st.rp[mid] - e0) <= cs) lo = mid;
                        else hi = mid - 1;
                    }
                    int r = lo;
                    int rs = (int)(st.rp[r] - e0), re = (int)(st.rp[r + 1] - e0);
                    float acc[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
                    for (int i = cs; i < ce; i += UW) {
                        XVec<XT, VEC> xv[UW];
                        float av[UW];
#pragma unroll
                        for (int u = 0; u < UW; ++u)
                            if (i + u < ce) {
                                const int64_t cidx = st.col[i + u];
                                av[u] = staged_val<VMODE>(st.val, i + u);
                                if (act[0]) gather(xv[u], cidx, 0);
                            }
#pragma unroll
                        for (int u = 0; u < UW; ++u)
                            if (i + u < ce) {
                                while (i + u >= re) {             // row r ended inside the piece
                                    if (rs < re) {
                                        if (rs >= cs) {
                                            if (act[0]) store_y<VEC>(a.Y + (int64_t)(d0.x + r) * a.ldy + li * VEC, acc);
                                        } else {
                                            hrow = r;
#pragma unroll
                                            for (int v = 0; v < VEC; ++v) head[v] = acc[v];
                                        }
                                    }
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
                                    ++r;
                                    rs = re;
                                    re = (int)(st.rp[r + 1] - e0);
                                }
                                if (act[0]) {
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) acc[v] = fmaf(av[u], xv[u].get(v), acc[v]);
                                }
                            }
                    }
                    if (re > ce) {                        // the row holding nonzero ce - 1
                        key = r;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) tail[v] = acc[v];
                    } else if (rs >= cs) {
                        if (act[0]) store_y<VEC>(a.Y + (int64_t)(d0.x + r) * a.ldy + li * VEC, acc);
                    } else {
                        hrow = r;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) head[v] = acc[v];
                    }
                }
                for (int off = 1; off < G; off <<= 1) {
                    const int kup = __shfl_up_sync(0xffffffffu, key, off * LANES);
                    float up[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) up[v] = __shfl_up_sync(0xffffffffu, tail[v], off * LANES);
                    if (g >= off && kup == key)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) tail[v] += up[v];
                }
#pragma unroll
                for (int v = 0; v < VEC; ++v) head[v] += __shfl_up_sync(0xffffffffu, tail[v], LANES);
                if (hrow >= 0 && act[0]) store_y<VEC>(a.Y + (int64_t)(d0.x + hrow) * a.ldy + li * VEC, head);
            } else if (!kFlat && !kMerge && !kMergeG && d0.y > 0) {
                // run of short rows: lane group g owns rows g, g+G, ...
                const int nr = d0.y;
                for (int j = g; j < nr; j += G) {
                    const int s = (int)(st.rp[j] - e0), e = (int)(st.rp[j + 1] - e0);
                    float acc[CH][VEC];
#pragma unroll
                    for (int c = 0; c < CH; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;
                    for (int i = s; i < e; i += U) {
                        XVec<XT, VEC> xv[U][CH];
                        float av[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (i + u < e) {
                                const int64_t cidx = st.col[i + u];
                                av[u] = staged_val<VMODE>(st.val, i + u);
#pragma unroll
                                for (int c = 0; c < CH; ++c)
                                    if (act[c]) gather(xv[u][c], cidx, c * LANES * VEC);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            if (i + u < e) {
#pragma unroll
                                for (int c = 0; c < CH; ++c)
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) acc[c][v] = fmaf(av[u], xv[u][c].get(v), acc[c][v]);
                            }
                    }
                    float* dst = a.Y + (int64_t)(d0.x + j) * a.ldy;
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (act[c]) store_y<VEC>(dst + (li + c * LANES) * VEC, acc[c]);
                }
            } else if (COMP) {
                // one long row or hub segment, compensated: Neumaier summation of
                // the products, whose own rounding error fmaf recovers exactly
                float acc[CH][VEC], cmp[CH][VEC];
#pragma unroll
                for (int c = 0; c < CH; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f, cmp[c][v] = 0.f;
                for (int i = g; i < n; i += G * U) {
                    XVec<XT, VEC> xv[U][CH];
                    float av[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int idx = i + u * G;
                        if (idx < n) {
                            const int64_t cidx = st.col[idx];
                            av[u] = staged_val<VMODE>(st.val, idx);
#pragma unroll
                            for (int c = 0; c < CH; ++c)
                                if (act[c]) gather(xv[u][c], cidx, c * LANES * VEC);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (i + u * G < n) {
#pragma unroll
                            for (int c = 0; c < CH; ++c)
#pragma unroll
                                for (int v = 0; v < VEC; ++v) {
                                    const float x = xv[u][c].get(v);
                                    const float p = av[u] * x;
                                    const float pe = fmaf(av[u], x, -p);       // exact product error
                                    const float t = acc[c][v] + p;
                                    const float e = (fabsf(acc[c][v]) >= fabsf(p)) ? (acc[c][v] - t) + p
                                                                                   : (p - t) + acc[c][v];
                                    cmp[c][v] += e + pe;
                                    acc[c][v] = t;
                                }
                        }
                }
                for (int off = LANES; off < 32; off <<= 1)
#pragma unroll
                    for (int c = 0; c < CH; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const float s2 = __shfl_xor_sync(0xffffffffu, acc[c][v], off);
                            const float c2 = __shfl_xor_sync(0xffffffffu, cmp[c][v], off);
                            const float t = acc[c][v] + s2;
                            const float e = (fabsf(acc[c][v]) >= fabsf(s2)) ? (acc[c][v] - t) + s2
                                                                            : (s2 - t) + acc[c][v];
                            cmp[c][v] += c2 + e;
                            acc[c][v] = t;
                        }
                if (g == 0) {
                    if (d0.y == 0) {                   // whole row: one rounding of sum + compensation
#pragma unroll
                        for (int c = 0; c < CH; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[c][v] += cmp[c][v];
                        float* dst = a.Y + (int64_t)d0.x * a.ldy;
#pragma unroll
                        for (int c = 0; c < CH; ++c)
                            if (act[c]) store_y<VEC>(dst + (li + c * LANES) * VEC, acc[c]);
                    } else if ((int64_t)(-d0.y - 1) < a.n_slots) {   // segment: keep the pair for the combine pass
                        const int64_t slot = (int64_t)(-d0.y - 1) * a.k;
#pragma unroll
                        for (int c = 0; c < CH; ++c)
                            if (act[c]) {
                                store_y<VEC>(a.partials + slot + (li + c * LANES) * VEC, acc[c]);
                                store_y<VEC>(a.partials_comp + slot + (li + c * LANES) * VEC, cmp[c]);
                            }
                    } else if (lane == 0) {                // a slot beyond the scratch: write nothing
                        atomicOr(a.status, kStatusSlotRange);
                    }
                }
            } else {
                // one long row or one hub segment: nonzeros g, g+G, ... per group
                float acc[CH][VEC];
#pragma unroll
                for (int c = 0; c < CH; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;
                for (int i = g; i < n; i += G * U) {
                    XVec<XT, VEC> xv[U][CH];
                    float av[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int idx = i + u * G;
                        if (idx < n) {
                            const int64_t cidx = st.col[idx];
                            av[u] = staged_val<VMODE>(st.val, idx);
#pragma unroll
                            for (int c = 0; c < CH; ++c)
                                if (act[c]) gather(xv[u][c], cidx, c * LANES * VEC);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (i + u * G < n) {
#pragma unroll
                            for (int c = 0; c < CH; ++c)
#pragma unroll
                                for (int v = 0; v < VEC; ++v) acc[c][v] = fmaf(av[u], xv[u][c].get(v), acc[c][v]);
                        }
                }
                for (int off = LANES; off < 32; off <<= 1)
#pragma unroll
                    for (int c = 0; c < CH; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[c][v] += __shfl_xor_sync(0xffffffffu, acc[c][v], off);
                if (d0.y < 0 && (int64_t)(-d0.y - 1) >= a.n_slots) {   // a slot beyond the scratch
                    if (lane == 0) atomicOr(a.status, kStatusSlotRange);
                } else if (g == 0) {
                    float* dst = (d0.y == 0) ? a.Y + (int64_t)d0.x * a.ldy
                                             : a.partials + (int64_t)(-d0.y - 1) * a.k;
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (act[c]) store_y<VEC>(dst + (li + c * LANES) * VEC, acc[c]);
                }
            }
        }
        if (tn >= a.n_tasks) break;
        d0 = n0; d1 = n1; ed = en;
        n0 = m0; n1 = m1; en = em;
        tn = tnn;
        b ^= 1;
    }
}

template <typename XT, int VMODE, int VEC, int CH, bool COMP, bool ONE, int MG = 0, bool HOT = false>
__global__ void __launch_bounds__(warps_per_block<HOT>() * 32, (HOT ? 1 : min_blocks<VMODE, MG>()))
    rows_kernel(const __grid_constant__ FwdArgs a) {
    rows_run<XT, VMODE, VEC, CH, COMP, ONE, MG, HOT, false>(a, nullptr);
}

// the tasks of up to kMaxBatch matrices in one launch (spmm_apply_batched);
// two blocks per SM, so the per-task lane geometry fits in registers
template <typename XT, int VMODE, int VEC, int CH, bool COMP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2) rows_kernel_multi(const __grid_constant__ MultiArgs m) {
    rows_run<XT, VMODE, VEC, CH, COMP, false, 0, false, true>(m.g, &m);
}

template <typename XT, int VMODE, int VEC, int CH, bool COMP, bool ONE, int MG = 0, bool HOT = false>
cudaError_t launch_one(const FwdArgs& a, cudaStream_t s) {
    using Lay = Layout<VMODE>;
    constexpr int WPB = warps_per_block<HOT>();
    constexpr int kStage = WPB * Lay::kWarp;      // staging buffers of the block's warps
    // per instantiation, computed once (thread-safe; a failure is reported to
    // every caller)
    static std::once_flag once;
    static int blocks_per_sm = 0, num_sms = 0, max_smem = 0;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [] {
        cudaError_t e = cudaSuccess;
        int dev = 0, nb = 0, sms = 0, opt = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&opt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        // the hot variant asks for the whole opt-in shared memory (its hot rows fill what the staging leaves)
        const int want = HOT ? opt : kStage;
        if (e == cudaSuccess && want > 48 * 1024)
            e = cudaFuncSetAttribute(rows_kernel<XT, VMODE, VEC, CH, COMP, ONE, MG, HOT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rows_kernel<XT, VMODE, VEC, CH, COMP, ONE, MG, HOT>,
                                                              WPB * 32, want);
        setup = e;
        num_sms = sms;
        max_smem = opt;
        blocks_per_sm = nb > 0 ? nb : 1;
    });
    if (setup != cudaSuccess) return setup;
    size_t smem = kStage;
    if constexpr (HOT) {
        smem += 16 + (size_t)a.hot_bytes;
        if (smem > (size_t)max_smem || a.hot_bytes <= 0 || a.hot_bytes % 16) return cudaErrorInvalidValue;
    }
    const int64_t want = (a.n_tasks + WPB - 1) / WPB;
    const int64_t cap = (int64_t)blocks_per_sm * num_sms;
    const dim3 grid((unsigned)(want < cap ? want : cap));
    rows_kernel<XT, VMODE, VEC, CH, COMP, ONE, MG, HOT><<<grid, WPB * 32, smem, s>>>(a);
    return cudaGetLastError();
}

// One launch over the entries of M (generic row walk, three blocks per SM).
template <typename XT, int VMODE, int VEC, int CH, bool COMP>
cudaError_t launch_multi_one(const MultiArgs& m, cudaStream_t s) {
    using Lay = Layout<VMODE>;
    static std::once_flag once;
    static int blocks_per_sm = 0, num_sms = 0;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [] {
        cudaError_t e = cudaSuccess;
        int dev = 0, nb = 0, sms = 0;
        if (Lay::kBlock > 48 * 1024)
            e = cudaFuncSetAttribute(rows_kernel_multi<XT, VMODE, VEC, CH, COMP>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kBlock);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rows_kernel_multi<XT, VMODE, VEC, CH, COMP>,
                                                              kWarpsPerBlock * 32, Lay::kBlock);
        setup = e;
        num_sms = sms;
        blocks_per_sm = nb > 0 ? nb : 1;
    });
    if (setup != cudaSuccess) return setup;
    const int64_t want = (m.g.n_tasks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t cap = (int64_t)blocks_per_sm * num_sms;
    const dim3 grid((unsigned)(want < cap ? want : cap));
    rows_kernel_multi<XT, VMODE, VEC, CH, COMP><<<grid, kWarpsPerBlock * 32, Lay::kBlock, s>>>(m);
    return cudaGetLastError();
}

template <typename XT>
cudaError_t launch_rows_multi_t(const MultiArgs& m, int vmode, int vec, int ch, bool comp, cudaStream_t s) {
    if (m.g.n_tasks <= 0) return cudaSuccess;
#define SPMM_LAUNCH_MULTI(VM, V, C)                                                      \
    if (vmode == VM && vec == V && ch == C)                                              \
        return comp ? launch_multi_one<XT, VM, V, C, true>(m, s) : launch_multi_one<XT, VM, V, C, false>(m, s);
    if constexpr (sizeof(XT) == 4) {
        SPMM_LAUNCH_MULTI(0, 4, 1) SPMM_LAUNCH_MULTI(0, 2, 1) SPMM_LAUNCH_MULTI(0, 1, 1) SPMM_LAUNCH_MULTI(0, 1, 2)
        SPMM_LAUNCH_MULTI(1, 4, 1) SPMM_LAUNCH_MULTI(1, 2, 1) SPMM_LAUNCH_MULTI(1, 1, 1) SPMM_LAUNCH_MULTI(1, 1, 2)
    } else {
        constexpr int VM3 = std::is_same<XT, __half>::value ? 3 : 2;
        SPMM_LAUNCH_MULTI(0, 8, 1) SPMM_LAUNCH_MULTI(0, 4, 1) SPMM_LAUNCH_MULTI(0, 2, 1) SPMM_LAUNCH_MULTI(0, 1, 1)
        SPMM_LAUNCH_MULTI(0, 1, 2)
        SPMM_LAUNCH_MULTI(1, 8, 1) SPMM_LAUNCH_MULTI(1, 4, 1) SPMM_LAUNCH_MULTI(1, 2, 1) SPMM_LAUNCH_MULTI(1, 1, 1)
        SPMM_LAUNCH_MULTI(1, 1, 2)
        SPMM_LAUNCH_MULTI(VM3, 8, 1) SPMM_LAUNCH_MULTI(VM3, 4, 1) SPMM_LAUNCH_MULTI(VM3, 2, 1)
        SPMM_LAUNCH_MULTI(VM3, 1, 1) SPMM_LAUNCH_MULTI(VM3, 1, 2)
    }
#undef SPMM_LAUNCH_MULTI
    return cudaErrorInvalidValue;
}

// One lane per X row of at most 4 bytes, hot rows in shared memory.
template <typename XT>
cudaError_t launch_rows_hot_t(const FwdArgs& a, int vmode, int vec, cudaStream_t s) {
    if (a.n_tasks <= 0) return cudaSuccess;
#define SPMM_LAUNCH_HOT(VM, V)                                                           \
    if (vmode == VM && vec == V)                                                         \
        return a.compensated ? launch_one<XT, VM, V, 1, true, true, 0, true>(a, s)       \
                             : launch_one<XT, VM, V, 1, false, true, 0, true>(a, s);
    if constexpr (sizeof(XT) == 4) {
        SPMM_LAUNCH_HOT(0, 1) SPMM_LAUNCH_HOT(1, 1)
    } else {
        constexpr int VM3 = std::is_same<XT, __half>::value ? 3 : 2;
        SPMM_LAUNCH_HOT(0, 1) SPMM_LAUNCH_HOT(0, 2) SPMM_LAUNCH_HOT(1, 1) SPMM_LAUNCH_HOT(1, 2)
        SPMM_LAUNCH_HOT(VM3, 1) SPMM_LAUNCH_HOT(VM3, 2)
    }
#undef SPMM_LAUNCH_HOT
    return cudaErrorInvalidValue;
}

template <typename XT, bool ONE, int MG = 0>
cudaError_t launch_rows_t(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s) {
    static_assert(!(ONE && MG), "one lane per row has no lane groups");
    if (a.n_tasks <= 0) return cudaSuccess;
#define SPMM_LAUNCH(VM, V, C)                                                            \
    if (vmode == VM && vec == V && ch == C)                                              \
        return a.compensated ? launch_one<XT, VM, V, C, true, ONE, MG>(a, s)             \
                             : launch_one<XT, VM, V, C, false, ONE, MG>(a, s);
    if constexpr (MG == 2) {     // float pattern rows of 4-element lanes only
        if constexpr (sizeof(XT) == 4) { SPMM_LAUNCH(0, 4, 1) }
    } else if constexpr (MG == 1) {   // CH == 1, at most 4 elements per lane
        if constexpr (sizeof(XT) == 4) {
            SPMM_LAUNCH(0, 4, 1) SPMM_LAUNCH(0, 2, 1) SPMM_LAUNCH(0, 1, 1)
            SPMM_LAUNCH(1, 4, 1) SPMM_LAUNCH(1, 2, 1) SPMM_LAUNCH(1, 1, 1)
        } else {
            constexpr int VM3 = std::is_same<XT, __half>::value ? 3 : 2;
            SPMM_LAUNCH(0, 4, 1) SPMM_LAUNCH(0, 2, 1) SPMM_LAUNCH(0, 1, 1)
            SPMM_LAUNCH(1, 4, 1) SPMM_LAUNCH(1, 2, 1) SPMM_LAUNCH(1, 1, 1)
            SPMM_LAUNCH(VM3, 4, 1) SPMM_LAUNCH(VM3, 2, 1) SPMM_LAUNCH(VM3, 1, 1)
        }
    } else if constexpr (ONE) {  // CH == 1 only
        if constexpr (sizeof(XT) == 4) {
            SPMM_LAUNCH(0, 4, 1) SPMM_LAUNCH(0, 2, 1) SPMM_LAUNCH(0, 1, 1)
            SPMM_LAUNCH(1, 4, 1) SPMM_LAUNCH(1, 2, 1) SPMM_LAUNCH(1, 1, 1)
        } else {
            constexpr int VM3 = std::is_same<XT, __half>::value ? 3 : 2;  // own-type values
            SPMM_LAUNCH(0, 8, 1) SPMM_LAUNCH(0, 4, 1) SPMM_LAUNCH(0, 2, 1) SPMM_LAUNCH(0, 1, 1)
            SPMM_LAUNCH(1, 8, 1) SPMM_LAUNCH(1, 4, 1) SPMM_LAUNCH(1, 2, 1) SPMM_LAUNCH(1, 1, 1)
            SPMM_LAUNCH(VM3, 8, 1) SPMM_LAUNCH(VM3, 4, 1) SPMM_LAUNCH(VM3, 2, 1) SPMM_LAUNCH(VM3, 1, 1)
        }
    } else {
        if constexpr (sizeof(XT) == 4) {
            SPMM_LAUNCH(0, 4, 1) SPMM_LAUNCH(0, 2, 1) SPMM_LAUNCH(0, 1, 1) SPMM_LAUNCH(0, 1, 2)
            SPMM_LAUNCH(1, 4, 1) SPMM_LAUNCH(1, 2, 1) SPMM_LAUNCH(1, 1, 1) SPMM_LAUNCH(1, 1, 2)
        } else {
            constexpr int VM3 = std::is_same<XT, __half>::value ? 3 : 2;
            SPMM_LAUNCH(0, 8, 1) SPMM_LAUNCH(0, 4, 1) SPMM_LAUNCH(0, 2, 1) SPMM_LAUNCH(0, 1, 1) SPMM_LAUNCH(0, 1, 2)
            SPMM_LAUNCH(1, 8, 1) SPMM_LAUNCH(1, 4, 1) SPMM_LAUNCH(1, 2, 1) SPMM_LAUNCH(1, 1, 1) SPMM_LAUNCH(1, 1, 2)
            SPMM_LAUNCH(VM3, 8, 1) SPMM_LAUNCH(VM3, 4, 1) SPMM_LAUNCH(VM3, 2, 1) SPMM_LAUNCH(VM3, 1, 1)
            SPMM_LAUNCH(VM3, 1, 2)
        }
    }
#undef SPMM_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace spmm
