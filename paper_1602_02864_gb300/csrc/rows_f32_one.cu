// rows_f32_one.cu -- row-task kernel instantiations for float X with one
// lane per X row (k equal to the vector width), in their own translation unit
// so they compile in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_f32_one(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s) {
    return launch_rows_t<float, true>(a, vmode, vec, ch, s);
}

}  // namespace spmm
