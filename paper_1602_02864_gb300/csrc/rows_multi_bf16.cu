// rows_multi_bf16.cu -- the task kernel over several matrices in one launch
// (spmm_apply_batched) for __nv_bfloat16 X, in its own translation unit so it
// compiles in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_multi_bf16(const MultiArgs& M, int vmode, int vec, int ch, bool comp, cudaStream_t s) {
    return launch_rows_multi_t<__nv_bfloat16>(M, vmode, vec, ch, comp, s);
}

}  // namespace spmm
