// rows_f32_mg.cu -- row-task kernel instantiations for float X whose short-row
// runs are split into equal pieces per lane group (merge-based), in their own
// translation unit so they compile in parallel with the others.
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_f32_mg(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s) {
    // pattern rows on 8 or more lanes of 4 elements (k = 32, 64) run faster
    // with 4 resident blocks and 2 nonzeros in flight per lane group
    if (vmode == 0 && vec == 4 && a.lanes_log2 >= 3) return launch_rows_t<float, false, 2>(a, vmode, vec, ch, s);
    return launch_rows_t<float, false, 1>(a, vmode, vec, ch, s);
}

}  // namespace spmm
