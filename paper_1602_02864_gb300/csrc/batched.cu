// batched.cu -- spmm_apply_batched: Y_i = A_i X_i (or A_i^T X_i) for several
// handles, each with its own k, in as few launches as their kernels allow.
//
// The paper's executor keeps one global queue of tile-row tasks (Section
// 3.4) so that many small multiplications keep every thread busy.  Here the
// entries whose X rows share a kernel instantiation (X type, value mode,
// vector width, column chunks, compensation) form one group, and one
// persistent launch of the task kernel runs the tasks of every entry of the
// group, numbered one after the other: a warp finds its task's entry, then
// takes that entry's matrix, X, Y, k and lane geometry.  The entries' split
// rows are then combined by one more launch.  The entries' arguments travel
// in the kernels' parameter space, so the call allocates nothing.
#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace spmm {

static cudaError_t launch_multi(int32_t xtype, const MultiArgs& m, int vmode, int vec, int ch, bool comp,
                                cudaStream_t s) {
    if (xtype == SPMM_F32) return launch_rows_multi_f32(m, vmode, vec, ch, comp, s);
    if (xtype == SPMM_BF16) return launch_rows_multi_bf16(m, vmode, vec, ch, comp, s);
    return launch_rows_multi_f16(m, vmode, vec, ch, comp, s);
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_apply_batched(int32_t n, const spmm_mat_t* A, const void* const* X, void* const* Y,
                                  const int32_t* k, spmm_dtype xtype, int32_t transpose, void* stream) {
    if (n < 1 || !A || !X || !Y || !k) { set_error("spmm_apply_batched: need n >= 1 and non-NULL arrays"); return SPMM_ERR_ARG; }
    if (xtype != SPMM_F32 && xtype != SPMM_BF16 && xtype != SPMM_F16) {
        set_error("spmm_apply_batched: X must be F32, BF16 or F16");
        return SPMM_ERR_ARG;
    }
    NvtxRange range("spmm_apply_batched");
    cudaStream_t s = (cudaStream_t)stream;
    const int esize = xtype == SPMM_F32 ? 4 : 2;
    // ---- validate every entry; group them by kernel instantiation
    struct Entry {
        int i;
        const DevCSR* d;
        int vmode, vec, ch;
        bool comp;
        LaneGeometry gm;
    };
    std::map<std::tuple<int, int, int, int>, std::vector<Entry>> groups;
    std::vector<Entry> all;
    for (int32_t i = 0; i < n; ++i) {
        const std::string who = "spmm_apply_batched: entry " + std::to_string(i);
        const spmm_mat* M = A[i];
        if (!M) { set_error(who + ": handle is NULL"); return SPMM_ERR_ARG; }
        if (k[i] < 1 || k[i] > kMaxK) { set_error(who + ": k must be in 1..64"); return SPMM_ERR_ARG; }
        if (M->streaming) { set_error(who + ": streaming handles are not batched"); return SPMM_ERR_UNSUPPORTED; }
        if (M->relabel) {
            set_error(who + ": handles with SPMM_RELABEL are not batched");
            return SPMM_ERR_UNSUPPORTED;
        }
        if (transpose && !M->has_tr) { set_error(who + ": transpose needs SPMM_WANT_TRANSPOSE"); return SPMM_ERR_ARG; }
        const DevCSR& d = transpose ? M->tr : M->fwd;
        if (d.perm) { set_error(who + ": handles with SPMM_REORDER are not batched"); return SPMM_ERR_UNSUPPORTED; }
        for (int32_t j = 0; j < i; ++j)
            if (A[j] == M) {
                set_error(who + ": the same handle appears twice (its scratch and counter are per handle)");
                return SPMM_ERR_ARG;
            }
        if (d.n_rows == 0 || d.n_tasks == 0) continue;
        if (!X[i] || !Y[i]) { set_error(who + ": X or Y is NULL"); return SPMM_ERR_ARG; }
        const int vmode = value_mode(M, (int32_t)xtype);
        if (vmode < 0) {
            set_error(who + ": 16-bit values need X of the same 16-bit type (or use F32 values)");
            return SPMM_ERR_UNSUPPORTED;
        }
        Entry en;
        en.i = i;
        en.d = &d;
        en.vmode = vmode;
        en.gm = lane_geometry(X[i], k[i], k[i], (int32_t)xtype, static_cast<const float*>(Y[i]), k[i]);
        en.vec = en.gm.vec;
        en.ch = en.gm.ch;
        en.comp = d.partials_comp != nullptr || (M->params.compensated && d.n_slots == 0);
        groups[std::make_tuple(vmode, en.vec, en.ch, (int)en.comp)].push_back(en);
        all.push_back(en);
    }
    // ---- one launch per group (and per kMaxBatch entries of it)
    auto M = std::make_unique<MultiArgs>();
    for (auto& kv : groups) {
        const std::vector<Entry>& es = kv.second;
        for (size_t c0 = 0; c0 < es.size(); c0 += kMaxBatch) {
            const size_t c1 = std::min(es.size(), c0 + (size_t)kMaxBatch);
            *M = MultiArgs{};
            M->n = (int32_t)(c1 - c0);
            int64_t tot = 0;
            bool wide = false;
            for (size_t q = c0; q < c1; ++q) {
                const Entry& en = es[q];
                const spmm_mat* H = A[en.i];
                const DevCSR& d = *en.d;
                FwdArgs& a = M->ent[q - c0];
                a = FwdArgs{};
                a.row_ptr = d.row_ptr;
                a.col_idx = d.col_idx;
                a.val = d.val;
                a.tasks = d.tasks;
                a.n_tasks = d.n_tasks;
                a.partials = d.partials;
                a.n_slots = d.n_slots;
                a.X = X[en.i];
                a.ldx = k[en.i];
                a.Y = static_cast<float*>(Y[en.i]);
                a.ldy = k[en.i];
                a.k = k[en.i];
                a.lanes_log2 = en.gm.lanes_log2;
                a.nvec = en.gm.nvec;
                a.status = H->status;
                a.wait_ns = kWaitNs;
                a.x_evict_last = H->params.x_evict_last;
                a.compensated = en.comp ? 1 : 0;
                a.partials_comp = d.partials_comp;
                M->off[q - c0] = tot;
                tot += d.n_tasks;
                wide = wide || (int64_t)k[en.i] * esize >= kWideRowBytes;
            }
            M->off[M->n] = tot;
            // launch-wide fields: every task, the first entry's counter and status word
            const Entry& first = es[c0];
            M->g.n_tasks = tot;
            M->g.status = A[first.i]->status;
            M->g.wait_ns = kWaitNs;
            M->g.task_chunk = wide ? 1 : kNarrowTaskChunk;
            M->g.task_ctr = first.d->task_ctr;
            cudaError_t e = cudaSuccess;
            if (M->g.task_ctr) e = cudaMemsetAsync(M->g.task_ctr, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = launch_multi((int32_t)xtype, *M, first.vmode, first.vec, first.ch, first.comp, s);
            if (e != cudaSuccess) return cuda_fail(e, "spmm_apply_batched: task kernel");
        }
    }
    // ---- the split rows of every entry
    auto C = std::make_unique<CombineMulti>();
    for (size_t c0 = 0; c0 < all.size(); c0 += kMaxBatch) {
        const size_t c1 = std::min(all.size(), c0 + (size_t)kMaxBatch);
        *C = CombineMulti{};
        for (size_t q = c0; q < c1; ++q) {
            const Entry& en = all[q];
            if (en.d->n_splits == 0) continue;
            CombineEntry& ce = C->ent[C->n++];
            ce.splits = en.d->splits;
            ce.n_splits = en.d->n_splits;
            ce.partials = en.d->partials;
            ce.pcomp = en.d->partials_comp;
            ce.Y = static_cast<float*>(Y[en.i]);
            ce.ldy = k[en.i];
            ce.k = k[en.i];
        }
        if (C->n == 0) continue;
        const cudaError_t e = launch_combine_multi(*C, s);
        if (e != cudaSuccess) return cuda_fail(e, "spmm_apply_batched: combine kernel");
    }
    return SPMM_OK;
}
