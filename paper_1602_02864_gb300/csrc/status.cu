// status.cu -- a kernel whose staging wait can never complete: it announces a
// 16-byte transfer on an mbarrier but issues none, so its bounded wait runs
// out and sets the status word.  Nothing is in flight when it returns.  Used
// to check the timeout path of the bounded waits without faulting the GPU.
#include "rows_kernel.cuh"

namespace spmm {

__global__ void wait_selftest_kernel(int32_t* status, uint64_t wait_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
    __syncwarp();
    if (!mbar_wait_bounded(&bar, 0, wait_ns) && threadIdx.x == 0) atomicExch(status, 1);
}

cudaError_t launch_wait_selftest(int32_t* status, uint64_t wait_ns, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(status, wait_ns);
    return cudaGetLastError();
}

}  // namespace spmm
