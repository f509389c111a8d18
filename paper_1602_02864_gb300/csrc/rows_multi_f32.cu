// rows_multi_f32.cu -- the task kernel over several matrices in one launch
// (spmm_apply_batched) for float X, in its own translation unit so it
// compiles in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_multi_f32(const MultiArgs& M, int vmode, int vec, int ch, bool comp, cudaStream_t s) {
    return launch_rows_multi_t<float>(M, vmode, vec, ch, comp, s);
}

}  // namespace spmm
