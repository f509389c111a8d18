// rows_f16.cu -- row-task kernel instantiations for __half X (split per dtype so
// the translation units compile in parallel).
#include "rows_kernel.cuh"

namespace spmm {

cudaError_t launch_rows_f16(const FwdArgs& a, int vmode, int vec, int ch, cudaStream_t s) {
    if (a.Xh && ch == 1 && a.lanes_log2 == 0) return launch_rows_f16_hot(a, vmode, vec, s);
    if (ch == 1 && a.lanes_log2 == 0) return launch_rows_f16_one(a, vmode, vec, ch, s);
    if (a.merge_groups) return launch_rows_f16_mg(a, vmode, vec, ch, s);
    return launch_rows_t<__half, false>(a, vmode, vec, ch, s);
}

}  // namespace spmm
