// plan.cpp -- host-side warp-task plan for one CSR orientation.
//
// The paper's executor (Section 3.4, Algorithm 1) hands threads batches of
// whole tile rows from a global queue and keeps each output row owned by one
// thread (horizontal partitioning), so no output row is written twice and the
// load stays balanced.  Here the unit is a warp task, and rows are binned by
// degree (the GPU analogue of the paper's tile-row batches and of its COO
// section for single-entry rows, Section 3.2):
//   - short rows (degree <= short_max, including empty and degree-1/2 rows)
//     are packed in runs of consecutive rows, at most task_rows rows and
//     task_nnz nonzeros per task; each lane group of the warp owns whole rows;
//   - a long row (short_max < degree <= long_row) is one task whose nonzeros
//     are shared by all lane groups of the warp;
//   - a hub row (degree > long_row) is split into segments of about task_nnz
//     nonzeros, one task each; every segment writes a partial result and a
//     second pass adds the partials in segment order.
// Tasks keep the natural row order, so a task reads contiguous slices of the
// row pointers and column indices and writes a contiguous block of Y.
#include <algorithm>

#include "internal.h"

namespace spmm {

static int4 desc(int64_t r0, int32_t x, int64_t e0) {
    return make_int4((int)r0, x, (int)(uint32_t)(e0 & 0xffffffffll), (int)(e0 >> 32));
}

// Row-walk efficiency of the short-row runs for G = 2, 4, 8, 16 lane groups:
// in a run, group g takes rows g, g+G, ...; a round (one row per group) lasts
// as long as its longest row, counted in batches of 4 nonzeros (the gathers a
// group keeps in flight) and at least one.  The efficiency is the batches of
// all rounds over G x the longest of each round.
static void walk_efficiency(const int64_t* row_ptr, HostPlan& plan) {
    double done[4] = {0, 0, 0, 0}, taken[4] = {0, 0, 0, 0};
    for (size_t t = 0; t + 1 < plan.tasks.size(); ++t) {
        const int4 d = plan.tasks[t];
        if (d.y < 1) continue;
        for (int gi = 0; gi < 4; ++gi) {
            const int G = 2 << gi;
            for (int j = 0; j < d.y; j += G) {
                int64_t mx = 1;
                for (int q = j; q < std::min(j + G, d.y); ++q) {
                    const int64_t b = (row_ptr[d.x + q + 1] - row_ptr[d.x + q] + 3) / 4;
                    done[gi] += (double)b;
                    mx = std::max(mx, b);
                }
                taken[gi] += (double)G * (double)mx;
            }
        }
    }
    for (int gi = 0; gi < 4; ++gi) plan.walk_eff[gi] = taken[gi] > 0 ? done[gi] / taken[gi] : 1.0;
}

HostPlan build_plan(const int64_t* row_ptr, int64_t n_rows, const Params& p) {
    HostPlan plan;
    const int64_t T = p.task_nnz, R = p.task_rows, LR = p.long_row, SM = p.short_max;
    plan.tasks.reserve((size_t)(row_ptr[n_rows] / T + n_rows / R + 16));
    int64_t r = 0;
    while (r < n_rows) {
        const int64_t d = row_ptr[r + 1] - row_ptr[r];
        if (d > SM) {
            if (d > LR) {
                const int64_t nseg = (d + T - 1) / T;
                const int64_t seglen = (d + nseg - 1) / nseg;
                plan.splits.push_back(make_int4((int)r, (int)nseg, (int)plan.n_slots, 0));
                for (int64_t s = 0; s < nseg; ++s)
                    plan.tasks.push_back(desc(r, (int32_t)(-(plan.n_slots + s) - 1), row_ptr[r] + s * seglen));
                plan.n_slots += nseg;
                plan.n_segments += nseg;
            } else {
                plan.tasks.push_back(desc(r, 0, row_ptr[r]));
                ++plan.n_long;
            }
            ++r;
            continue;
        }
        const int64_t r0 = r;
        int64_t nnz = 0;
        while (r < n_rows && r - r0 < R) {
            const int64_t dr = row_ptr[r + 1] - row_ptr[r];
            if (dr > SM || nnz + dr > T) break;
            nnz += dr;
            ++r;
        }
        plan.tasks.push_back(desc(r0, (int32_t)(r - r0), row_ptr[r0]));
        ++plan.n_short;
    }
    plan.tasks.push_back(desc(n_rows, 0, row_ptr[n_rows]));   // sentinel
    walk_efficiency(row_ptr, plan);
    return plan;
}

// Run j ends at the first task that starts at or after (j + 1) / nb of the
// stored entries and begins a new row (consecutive tasks share a first row
// only as segments of one split row).  The sentinel's row is n_rows.
std::vector<RowBlock> cut_row_blocks(const HostPlan& plan, int nb) {
    std::vector<RowBlock> out;
    const size_t nt = plan.tasks.size() - 1;
    if (nt == 0 || nb < 1) return out;
    auto e0 = [&](size_t t) { return ((int64_t)(uint32_t)plan.tasks[t].z) | ((int64_t)plan.tasks[t].w << 32); };
    auto row = [&](size_t t) { return (int64_t)plan.tasks[t].x; };
    const int64_t total = e0(nt);
    size_t t = 0, sp = 0;
    for (int j = 0; j < nb && t < nt; ++j) {
        RowBlock b;
        b.t0 = (int64_t)t;
        b.r0 = row(t);
        b.s0 = (int64_t)sp;
        size_t u = nt;
        if (j < nb - 1) {
            const int64_t goal = total / nb * (j + 1) + total % nb * (j + 1) / nb;
            u = t + 1;
            while (u < nt && (e0(u) < goal || row(u) == row(u - 1))) ++u;
        }
        b.t1 = (int64_t)u;
        b.r1 = row(u);
        while (sp < plan.splits.size() && (int64_t)plan.splits[sp].x < b.r1) ++sp;
        b.s1 = (int64_t)sp;
        out.push_back(b);
        t = u;
    }
    return out;
}

}  // namespace spmm
