// rows_multi_f16.cu -- the task kernel over several matrices in one launch
// (spmm_apply_batched) for __half X, in its own translation unit so it
// compiles in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_multi_f16(const MultiArgs& M, int vmode, int vec, int ch, bool comp, cudaStream_t s) {
    return launch_rows_multi_t<__half>(M, vmode, vec, ch, comp, s);
}

}  // namespace spmm
