// rmat_cuda.cu -- synth.c's R-MAT generator on the GPU, for graphs whose edge
// list is too large to sort on the host (2^29 vertices, 2^34 edges).
//
// Edge e makes exactly the draws synth_rmat_edges makes (Philox4x32-10 with
// counter (e, level / 4, 0, DOM_EDGE) and the same key), so both produce the
// same edge multiset.  The edges are bucketed by row block (the top
// `block_bits` bits of the source) into one 64-bit key array, key =
// source << scale | destination; the caller sorts and deduplicates each
// block's range, which yields the CSR rows of that block in order.  No SpMM
// arithmetic lives here.
#include <stdint.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u
#define DOM_EDGE 0x45444745u

namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        const uint32_t hi0 = __umulhi(PHILOX_M0, c[0]), lo0 = PHILOX_M0 * c[0];
        const uint32_t hi1 = __umulhi(PHILOX_M1, c[2]), lo1 = PHILOX_M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// the key synth.c derives from (seed, seed2 = 0)
__device__ __forceinline__ void draw4(uint64_t seed, uint64_t idx, uint32_t sub, uint32_t out[4]) {
    out[0] = (uint32_t)idx; out[1] = (uint32_t)(idx >> 32); out[2] = sub; out[3] = DOM_EDGE;
    philox4x32_10(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Row and column of edge e after its first `levels` levels (bits from the top).
__device__ __forceinline__ void rmat_edge(int scale, int levels, uint64_t e, double t0, double t1, double t2,
                                          uint64_t seed, uint32_t* row, uint32_t* col) {
    uint32_t r = 0, c = 0, w[4];
    for (int l = 0; l < levels; ++l) {
        if ((l & 3) == 0) draw4(seed, e, (uint32_t)(l >> 2), w);
        const double u = (double)w[l & 3] * (1.0 / 4294967296.0);
        const int q = (u < t0) ? 0 : (u < t1) ? 1 : (u < t2) ? 2 : 3;
        r |= (uint32_t)(q >> 1) << (scale - 1 - l);
        c |= (uint32_t)(q & 1) << (scale - 1 - l);
    }
    *row = r;
    *col = c;
}

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int kChunk = kThreads * kPerThread;

__global__ void __launch_bounds__(kThreads) block_count_kernel(int scale, int64_t n_edges, double t0, double t1,
                                                               double t2, uint64_t seed, int bb,
                                                               unsigned long long* hist) {
    extern __shared__ unsigned int sh[];
    const int nb = 1 << bb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r, c;
        rmat_edge(scale, bb, (uint64_t)e, t0, t1, t2, seed, &r, &c);
        atomicAdd(&sh[r >> (scale - bb)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// Per chunk of kChunk edges: rank each edge within its bin in shared memory,
// reserve the bins' ranges with one global atomic each, then write the keys.
// base has nb + 1 entries (base[nb] = n_edges); a write outside its bin's
// range is skipped and counted in *overflow (it cannot happen when the counts
// came from block_count_kernel with the same arguments).
__global__ void __launch_bounds__(kThreads) block_fill_kernel(int scale, int64_t n_edges, double t0, double t1,
                                                              double t2, uint64_t seed, int bb,
                                                              const unsigned long long* base,
                                                              unsigned long long* cursor, uint64_t* keys,
                                                              unsigned long long* overflow) {
    extern __shared__ unsigned char smem[];
    const int nb = 1 << bb;
    unsigned int* cnt = reinterpret_cast<unsigned int*>(smem);                                  // nb
    unsigned long long* start = reinterpret_cast<unsigned long long*>(smem + ((nb * 4 + 15) & ~15));   // nb
    const int64_t n_chunks = (n_edges + kChunk - 1) / kChunk;
    for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        uint64_t key[kPerThread];
        uint32_t bin[kPerThread], rank[kPerThread];
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const int64_t e = ch * kChunk + (int64_t)j * kThreads + threadIdx.x;
            bin[j] = 0xffffffffu;
            if (e < n_edges) {
                uint32_t r, c;
                rmat_edge(scale, scale, (uint64_t)e, t0, t1, t2, seed, &r, &c);
                key[j] = ((uint64_t)r << scale) | c;
                bin[j] = r >> (scale - bb);
                rank[j] = atomicAdd(&cnt[bin[j]], 1u);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
            if (cnt[i]) start[i] = base[i] + atomicAdd(&cursor[i], (unsigned long long)cnt[i]);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPerThread; ++j)
            if (bin[j] != 0xffffffffu) {
                const unsigned long long pos = start[bin[j]] + rank[j];
                if (pos < base[bin[j] + 1]) keys[pos] = key[j];
                else atomicAdd(overflow, 1ull);
            }
        __syncthreads();
    }
}

}  // namespace

extern "C" int synth_rmat_block_count(int32_t scale, int64_t n_edges, double t0, double t1, double t2,
                                      uint64_t seed, int32_t block_bits, unsigned long long* hist, void* stream) {
    if (scale < 1 || scale > 31 || block_bits < 0 || block_bits > 12 || block_bits > scale || n_edges < 0) return -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t sh = (size_t)4 << block_bits;
    block_count_kernel<<<sms * 8, kThreads, sh, (cudaStream_t)stream>>>(scale, n_edges, t0, t1, t2, seed, block_bits,
                                                                        hist);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int synth_rmat_block_fill(int32_t scale, int64_t n_edges, double t0, double t1, double t2,
                                     uint64_t seed, int32_t block_bits, const unsigned long long* base,
                                     unsigned long long* cursor, uint64_t* keys, unsigned long long* overflow,
                                     void* stream) {
    if (scale < 1 || scale > 31 || block_bits < 0 || block_bits > 12 || block_bits > scale || n_edges < 0) return -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = 1 << block_bits;
    const size_t sh = (size_t)(((nb * 4 + 15) & ~15) + nb * 8);
    if (sh > 48 * 1024 &&
        cudaFuncSetAttribute(block_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) != cudaSuccess)
        return -2;
    block_fill_kernel<<<sms * 8, kThreads, sh, (cudaStream_t)stream>>>(scale, n_edges, t0, t1, t2, seed, block_bits,
                                                                       base, cursor, keys, overflow);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Page-locked host memory for generated arrays that will be streamed to the
// GPU (allocated pinned, so no later registration of a large range is needed).
extern "C" void* synth_host_alloc(uint64_t bytes) {
    void* p = nullptr;
    if (cudaHostAlloc(&p, bytes ? bytes : 1, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

extern "C" void synth_host_free(void* p) { cudaFreeHost(p); }
