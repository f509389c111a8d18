// rows_bf16_hot.cu -- row-task kernel instantiations for __nv_bfloat16 X with one lane
// per X row of at most 4 bytes and the hot rows of X in shared memory, in
// their own translation unit so they compile in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_bf16_hot(const FwdArgs& a, int vmode, int vec, cudaStream_t s) {
    return launch_rows_hot_t<__nv_bfloat16>(a, vmode, vec, s);
}

}  // namespace spmm
