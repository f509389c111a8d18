// rows_bf16_one.cu -- row-task kernel instantiations for __nv_bfloat16 X with one
// lane per X row (k equal to the vector width), in their own translation unit
// so they compile in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_bf16_one(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s) {
    return launch_rows_t<__nv_bfloat16, true>(a, vmode, vec, ch, s);
}

}  // namespace spmm
