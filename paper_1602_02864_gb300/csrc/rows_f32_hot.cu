// rows_f32_hot.cu -- row-task kernel instantiations for float X with one lane
// per X row of at most 4 bytes and the hot rows of X in shared memory, in
// their own translation unit so they compile in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_f32_hot(const FwdArgs& a, int vmode, int vec, cudaStream_t s) {
    return launch_rows_hot_t<float>(a, vmode, vec, s);
}

}  // namespace spmm
