// rows_f16_mg.cu -- row-task kernel instantiations for __half X whose short-row
// runs are split into equal pieces per lane group (merge-based), in their own
// translation unit so they compile in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_f16_mg(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s) {
    return launch_rows_t<__half, false, 1>(a, vmode, vec, ch, s);
}

}  // namespace spmm
