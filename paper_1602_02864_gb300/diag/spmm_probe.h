// spmm_probe.h -- gather-rate diagnostics, built as libspmm_probe.so
// beside libspmm.so (which it links against for the handle and its error
// string).  Not part of the library's interface and not a paper operation:
// they measure the rate of random row gathers, the SpMM's dominant cost, as
// reference rates for the benchmark's reports.  Errors are reported like the library's
// (spmm_last_error).
#pragma once

#include "spmm.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * spmm_probe_gather -- diagnostic: the measured rate of uniformly random row
 * gathers on this GPU, a reference rate for the SpMM's dominant cost
 * (one X row per nonzero).  Gathers rows of row_bytes (a power of two,
 * 4..256) at random row indices from a zero-filled table of table_bytes
 * (4 KiB .. 64 GiB; below the L2 size the rows come from L2, above it from
 * DRAM), eight loads in flight per lane, about 4 GB gathered.
 *   rows_per_s, bytes_per_s   host out
 * Synchronises `stream`; allocates its table.
 */
int spmm_probe_gather(int64_t table_bytes, int32_t row_bytes, double* rows_per_s, double* bytes_per_s,
                      void* stream);

/*
 * spmm_probe_gather_cols -- diagnostic: the gather rate of one matrix's column stream.
 * Replays the handle's own column-index stream (forward, or the transpose if
 * `transpose` != 0) in storage order, gathering for every stored entry one
 * row of row_bytes (a multiple of 4, 4..256; 4*k for an FP32 X of k columns)
 * from a zero table of n_cols rows, and nothing else of the SpMM.  Five runs
 * back to back (the table stays warm, as X does across iterations).
 *   rows_per_s   host out: stored entries per second
 *   bytes_per_s  host out: (row_bytes + 4) per entry per second
 * Synchronises `stream`; allocates its table.  SPMM_ERR_UNSUPPORTED for a
 * streaming handle.
 */
int spmm_probe_gather_cols(spmm_mat_t A, int32_t transpose, int32_t row_bytes, double* rows_per_s,
                           double* bytes_per_s, void* stream);

#ifdef __cplusplus
}
#endif
