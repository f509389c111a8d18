"""SpMM benchmark: in-HBM Y = A X on an R-MAT scale-24 power-law graph.

Workload (one step): Y = A X for every k in the sweep {1, 2, 4, 8, 16, 32, 64}
with float32 X, then 30 PageRank iterations (damping 0.85, one CUDA graph, one
A^T product per iteration), A the pattern-only adjacency matrix of a seeded
R-MAT graph (2^24 vertices, 2^28 generated directed edges, a/b/c/d =
.57/.19/.19/.05, duplicates merged).  The headline value is nonzeros processed
per second over the whole step ((7 + 30) * nnz / step time).  Per k the line also reports
nnz/s, the algorithmic bytes moved per call
    nnz*(4 + value bytes) + 8*(N+1) + N*k*(X element bytes) + N*k*4
as GB/s and as a fraction of the measured HBM copy bandwidth, and the BF16-X
speedup with its error against the FP64 oracle on sampled rows.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

UNIT = "nnz/s"
L2_FLUSH_BYTES = 512 << 20
NOMINAL_HBM_GBS = 8000.0     # nominal HBM3e bandwidth of the part (about 8 TB/s), reported beside the measured peak


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--edge-factor", type=int, default=16)
    ap.add_argument("--ks", default="1,2,4,8,16,32,64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-part-cols", type=int, default=16,
                    help="end-to-end step: X_k and Y_k live in host memory as vertical partitions of at most "
                         "this many columns (Section 3.3), one pass over A each")
    ap.add_argument("--no-ceiling", "--no-gather-probe", dest="no_ceiling", action="store_true",
                    help="skip the gather probes (reference rates of X-row gathers alone)")
    ap.add_argument("--no-stream", action="store_true",
                    help="skip the streaming sub-record (R-MAT scale 26, A in pinned host memory)")
    ap.add_argument("--reorder", action="store_true",
                    help="create the handle with SPMM_REORDER (columns relabelled by degree)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--transpose", action="store_true",
                    help="the k sweep multiplies by A^T (the PageRank product is A^T at k = 1)")
    ap.add_argument("--record-traffic", default=None, metavar="CSV",
                    help="write the traffic record from an ncu raw CSV export of one rows_kernel launch, then exit")
    ap.add_argument("--pagerank-iters", type=int, default=30)
    ap.add_argument("--profile-part", default="steps", choices=["steps", "relabelled"],
                    help="what a profiler started with --profile-from-start off records: the timed steps, "
                         "or one product per k on the relabelled handle")
    ap.add_argument("--no-relabel", action="store_true",
                    help="skip the sub-record of the same sweep on a handle made with SPMM_RELABEL")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the eigensolver (scale 18) and 256-graph batch sub-records of the default line")
    ap.add_argument("--eigs-krylov-full", action="store_true",
                    help="eigs workload: also run the Krylov-Schur solver at full size (300 restarts)")
    ap.add_argument("--workload", default="ksweep",
                    choices=["ksweep", "streaming", "nmf-batched", "eigs", "gather-ceiling", "vpart", "ordering",
                             "file"],
                    help="ksweep: the headline SpMM sweep + PageRank; the others measure the streaming mode, "
                         "the batched launch with NMF and the eigensolver")
    return ap.parse_args()


def metric_name(args):
    pr = f" + PageRank x{args.pagerank_iters}" if args.pagerank_iters else ""
    return f"SpMM nonzeros/s (R-MAT scale {args.scale}, k sweep {args.ks}{pr}, FP32 X)"


# DRAM traffic of the dominant kernel comes from a record that `--record-traffic`
# writes from an ncu capture; the record holds a digest of the library's
# sources and is used only while the sources are unchanged.
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "traffic_rows_kernel_k1.json")


def code_tokens(src: str) -> str:
    """C/C++/CUDA source without its comments, each run of white space one
    blank: what the compiler sees, so an edit to a comment or to the layout
    leaves the digest unchanged."""
    import re
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return re.sub(r"\s+", " ", "".join(out)).strip()


def source_digest() -> str:
    """SHA-256 over the CUDA/C++ sources and the public header (file names
    and their code without comments, in name order)."""
    import hashlib
    h = hashlib.sha256()
    dirs = [os.path.join(ROOT, "paper_1602_02864_gb300", "csrc"), os.path.join(ROOT, "include")]
    for d in dirs:
        for fn in sorted(os.listdir(d)):
            if fn.endswith((".cu", ".cuh", ".h", ".cpp")):
                h.update(fn.encode())
                with open(os.path.join(d, fn), encoding="utf-8", errors="replace") as f:
                    h.update(code_tokens(f.read()).encode())
    return h.hexdigest()


def read_traffic(scale, edge_factor, nnz):
    """DRAM bytes per launch of the k = 1 product (A X, float32) on this
    workload, from the record if it matches the current sources, scaled by
    stored entries when it was taken on a smaller graph; else None."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, "no record"
    if rec.get("source_digest") != source_digest():
        return None, "record taken on other sources"
    if rec.get("edge_factor") != edge_factor or rec.get("transpose"):
        return None, "record taken on another workload"
    return rec["dram_bytes_per_launch"] * nnz / rec["nnz"], f"{TRAFFIC_RECORD[len(ROOT) + 1:]} (R-MAT scale " \
        f"{rec['scale']}, scaled by stored entries)"


def record_traffic(csv_path, args):
    """Write the traffic record from an ncu --csv --page raw export of one
    launch of rows_kernel (dram__bytes_read.sum + dram__bytes_write.sum)."""
    import csv
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f)]
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    names, units, data = rows[hdr], rows[hdr + 1], rows[hdr + 2:]
    scale_of = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    launches = [r for r in data if "rows_kernel" in r[names.index("Kernel Name")]]
    if not launches:
        raise SystemExit("record_traffic: no rows_kernel launch in " + csv_path)
    r = launches[0]
    tot = 0.0
    for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        i = names.index(m)
        tot += float(r[i].replace(",", "")) * scale_of[units[i]]
    A, _ = make_graph(args)
    rec = {"kernel": r[names.index("Kernel Name")], "scale": args.scale, "edge_factor": args.edge_factor,
           "nnz": A.nnz, "dram_bytes_per_launch": tot, "source_digest": source_digest(),
           "workload": f"R-MAT scale {args.scale}, {'A^T' if args.transpose else 'A'} X with k = 1 float32",
           "transpose": bool(args.transpose)}
    os.makedirs(os.path.dirname(TRAFFIC_RECORD), exist_ok=True)
    with open(TRAFFIC_RECORD, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


def vertical_parts(ks, P):
    """The end-to-end step's vertical partitions (Section 3.3): for each k in
    order, (k, c0, c1) for columns c0..c1-1 of X_k, at most P columns each."""
    P = max(1, min(64, int(P)))
    return [(k, c0, min(k, c0 + P)) for k in ks for c0 in range(0, k, P)]


def host_cpu() -> str:
    """The host's CPU as /proc/cpuinfo names it (model name on x86, the
    implementer and part numbers on Arm), with its logical core count."""
    import platform
    name = ""
    try:
        with open("/proc/cpuinfo") as f:
            info = {}
            for line in f:
                if ":" in line:
                    key, val = (t.strip() for t in line.split(":", 1))
                    info.setdefault(key, val)
        name = info.get("model name") or " ".join(
            f"{k} {info[k]}" for k in ("CPU implementer", "CPU part") if k in info)
    except OSError:
        pass
    return f"{platform.machine()} {name}".strip() + f", {os.cpu_count()} logical cores"


def pagerank_iter_bytes(nnz, n):
    """Algorithmic bytes of one PageRank iteration: the A^T product at k = 1
    (column indices, row pointers, z in, y out) plus the update (y, x read and
    written, out-degree, z written)."""
    return alg_bytes(nnz, n, n, 1, 4) + 5 * 4 * n


def alg_bytes(nnz, n_rows, n_cols, k, xbytes, vbytes=0):
    return nnz * (4 + vbytes) + 8 * (n_rows + 1) + n_cols * k * xbytes + n_rows * k * 4


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_graph(args):
    t = time.time()
    A = synth.rmat_csr(args.scale, args.edge_factor << args.scale, seed=0)
    return A, time.time() - t


def cpu_sample_rows(A, target_nnz, seed=7):
    """Seeded sample of rows whose nonzeros add up to about target_nnz."""
    n = A.n_rows
    avg = max(A.nnz / max(n, 1), 1e-9)
    m = int(min(n, max(64, target_nnz / avg)))
    rows = np.unique(synth.sample_rows(n, m, seed=seed))
    nz = int(np.diff(A.row_ptr)[rows].sum())
    return rows, nz


def run_cpu_oracle(A, Xh, ks, rows, threads, pr_iters=0):
    import oracle
    t = time.perf_counter()
    for k in ks:
        oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xh, rows, threads=threads, k=k)
    if pr_iters:
        oracle.pagerank(A.n_rows, A.row_ptr, A.col_idx, 0.85, pr_iters)
    return time.perf_counter() - t


def reference_arm(args, rank, world):
    """The FP64 CPU oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    ks = [int(k) for k in args.ks.split(",")]
    A, _ = make_graph(args)
    kmax = max(ks)
    Xh = synth.dense(A.n_cols, kmax, seed=0)
    threads = oracle.num_threads()
    # size the per-step sample so one step takes about cpu_seconds / 4
    rows, nz = cpu_sample_rows(A, 2_000_000)
    dt = run_cpu_oracle(A, Xh, ks, rows, threads)
    rate = nz * len(ks) / dt
    target = rate * max(args.cpu_seconds / 4, 0.5) / len(ks)
    rows, nz = cpu_sample_rows(A, target, seed=8)
    pr = 1 if args.pagerank_iters else 0
    for _ in range(args.warmup):
        run_cpu_oracle(A, Xh, ks, rows[: max(1, len(rows) // 8)], threads)
    times = [run_cpu_oracle(A, Xh, ks, rows, threads, pr) for _ in range(args.steps)]
    total = sum(times)
    value = (nz * len(ks) + pr * A.nnz) * args.steps / total
    line = {
        "impl": "reference", "metric": metric_name(args), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale}-spmm-ksweep", "scale": args.scale, "n": A.n_rows,
                   "nnz": A.nnz, "ks": ks},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{len(rows)} seeded rows ({nz} nonzeros) of the scale-{args.scale} graph, "
                                   f"all k in the sweep, plus {pr} full PageRank iteration, per step",
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def profiler_range(on: bool):
    """cudaProfilerStart/Stop around the timed steps (no-ops without a profiler)."""
    import torch
    try:
        (torch.cuda.profiler.start if on else torch.cuda.profiler.stop)()
    except Exception:
        pass


def aggregate(units_per_rank, t_local, world):
    """Whole-job throughput of `world` replicas: every rank processed
    units_per_rank units in t_local seconds; the job time is the maximum over
    ranks (an all-reduce over the default process group when world > 1).
    Returns (units per second over all ranks, job seconds)."""
    t = float(t_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        tt = torch.tensor([t], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * units_per_rank / t, t


def event_ms(fn, reps, flush=None):
    """Mean CUDA-event time of fn() on the current stream (L2 flushed first)."""
    import torch
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts)


def base_line(args, metric, value, unit, ms, workload, dtype, extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": {"workload": workload}}
    line.update(extra)
    return line


def link_rates_gbs(nbytes=1 << 30, reps=3):
    """Pinned host <-> device copy rates in GB/s, best of reps: host to
    device alone, device to host alone, and both at once on two streams
    (bytes of both directions over the time of the pair).  Host-timed around
    synchronised copies, so slightly conservative."""
    import torch
    hin = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    hout = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    din = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dout = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(h2d, d2h):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if h2d:
            with torch.cuda.stream(s_in):
                din.copy_(hin, non_blocking=True)
        if d2h:
            with torch.cuda.stream(s_out):
                hout.copy_(dout, non_blocking=True)
        torch.cuda.synchronize()
        return (int(h2d) + int(d2h)) * nbytes / (time.perf_counter() - t0) / 1e9
    rates = {"h2d_GBps": max(timed(True, False) for _ in range(reps)),
             "d2h_GBps": max(timed(False, True) for _ in range(reps)),
             "both_GBps": max(timed(True, True) for _ in range(reps))}
    del hin, hout, din, dout
    return rates


def workload_streaming(args):
    """Streaming mode: A (R-MAT, avg degree 32) in pinned host memory, X and Y
    (k = 4, FP32) in HBM; link bytes per call vs the measured pinned H2D peak."""
    import torch
    import oracle
    from paper_1602_02864_gb300 import spmm
    scale = args.scale if args.scale != 24 else 29
    t = time.time()
    # the GPU generator makes the same graph as rmat_csr without a host-side edge sort
    A = synth.rmat_csr_cuda(scale, 32 << scale, seed=0, pinned=True)
    torch.cuda.empty_cache()
    t_gen = time.time() - t
    N, nnz = A.n_rows, A.nnz
    # pinned host -> device peak: large copies, best of 5
    buf = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    dbuf = torch.empty_like(buf, device="cuda")
    peak = max((1 << 30) / (event_ms(lambda: dbuf.copy_(buf, non_blocking=True), 1) / 1e3) / 1e9 for _ in range(5))
    del buf, dbuf
    t = time.time()
    h = spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None, streaming=True)
    t_create = time.time() - t
    k = 4
    X = torch.from_numpy(synth.dense(N, k, seed=0)).cuda()
    Y = torch.empty((N, k), device="cuda")
    for _ in range(args.warmup):
        h.apply(X, Y=Y)
    # the host link can be shared with other jobs: time the streamed calls
    # interleaved with a copy-only pass over the same host arrays
    ci = torch.from_numpy(A.col_idx).view(torch.uint8)
    rp = torch.from_numpy(A.row_ptr).view(torch.uint8)
    stage = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def copy_only():
        for src in (ci, rp):
            for off in range(0, src.numel(), 256 << 20):
                n = min(256 << 20, src.numel() - off)
                stage[:n].copy_(src[off:off + n], non_blocking=True)
    ms_list, copy_list = [], []
    for _ in range(args.steps):
        ms_list.append(event_ms(lambda: h.apply(X, Y=Y), 1))
        copy_list.append(event_ms(copy_only, 1))
    ms = statistics.median(ms_list)
    copy_ms = statistics.median(copy_list)
    del stage
    peak_after = max((1 << 30) / (event_ms(lambda: dbuf2.copy_(buf2, non_blocking=True), 1) / 1e3) / 1e9
                     for buf2, dbuf2 in [(torch.empty(1 << 30, dtype=torch.uint8).pin_memory(),
                                          torch.empty(1 << 30, dtype=torch.uint8, device="cuda"))] for _ in range(5))
    link_bytes = nnz * 4 + (N + 1) * 8
    # resident mode on the same matrix for context
    hr = spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None)
    Yr = torch.empty_like(Y)
    for _ in range(2):
        hr.apply(X, Y=Yr)
    ms_res = event_ms(lambda: hr.apply(X, Y=Yr), args.steps)
    same = bool(torch.equal(Y, Yr))
    hr.close()
    rows = np.unique(synth.sample_rows(N, 100_000, seed=5))
    Xh = X.cpu().numpy()
    ref = oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xh, rows, threads=oracle.num_threads())
    scale_ = oracle.spmm_rows(A.row_ptr, A.col_idx, None, np.abs(Xh), rows, threads=oracle.num_threads())
    got = Y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    err = float((np.abs(got - ref) / np.maximum(scale_, 1e-300)).max())
    h.sync_status()
    h.close()
    achieved = link_bytes / (ms / 1e3) / 1e9
    return base_line(args, f"streaming SpMM nonzeros/s (R-MAT scale {scale}, avg degree 32, k=4, A in host memory)",
                     nnz / (ms / 1e3), "nnz/s", ms, f"rmat{scale}-streaming-k4", "f32",
                     {"link": {"achieved_GBps": achieved, "peak_pinned_h2d_GBps": peak, "frac": achieved / peak,
                               "peak_pinned_h2d_GBps_after": peak_after,
                               "copy_only_GBps": link_bytes / (copy_ms / 1e3) / 1e9,
                               "frac_of_copy_only": copy_ms / ms,
                               "bytes_per_call": link_bytes,
                               "note": "steps alternate a streamed call and a copy-only pass over the same "
                                       "pinned host arrays (the host link may be shared)"},
                      "resident_ms": ms_res, "bit_identical_to_resident": same,
                      "sampled_rows_max_err_over_absprod": err, "sampled_rows": int(len(rows)),
                      "n": N, "nnz": nnz, "setup_s": {"generate": round(t_gen, 1), "create": round(t_create, 1)}})


def workload_vpart(args):
    """Large dense matrices (Section 5.3): X and Y with p = 32 FP32 columns in
    pinned host memory, multiplied in vertical partitions of c columns
    (c = 1, 2, 4, 8, 16, 32 kept on the device, one pass over A per group),
    against the in-memory SpMM with X and Y resident in HBM."""
    import torch
    import oracle
    from paper_1602_02864_gb300 import spmm
    p = 32
    t = time.time()
    A = synth.rmat_csr(args.scale, args.edge_factor << args.scale, seed=0)
    t_gen = time.time() - t
    N, nnz = A.n_rows, A.nnz
    h = spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None)
    Xh = torch.from_numpy(synth.dense(N, p, seed=0)).pin_memory()
    Yh = torch.empty((N, p), dtype=torch.float32).pin_memory()
    # in-memory reference: X, Y resident, one k = 32 apply
    Xd = Xh.cuda()
    Yd = torch.empty((N, p), device="cuda")
    for _ in range(args.warmup):
        h.apply(Xd, Y=Yd)
    im_ms = event_ms(lambda: h.apply(Xd, Y=Yd), args.steps)
    rows = np.unique(synth.sample_rows(N, 20_000, seed=7))
    Xn = Xh.numpy()
    ref = oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xn, rows, threads=oracle.num_threads())
    scl = oracle.spmm_rows(A.row_ptr, A.col_idx, None, np.abs(Xn), rows, threads=oracle.num_threads())
    per_c = {}
    for c in (1, 2, 4, 8, 16, 32):
        h.apply_host(Xh, Yh, group_cols=c)
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = h.apply_host(Xh, Yh, group_cols=c)
            ts.append((time.perf_counter() - t0) * 1e3)
        ms = statistics.median(ts)
        got = Yh.numpy()[rows].astype(np.float64)
        err = float((np.abs(got - ref) / np.maximum(scl, 1e-300)).max())
        link = 2 * N * p * 4
        per_c[str(c)] = {"groups": g, "ms": round(ms, 3), "nnz_per_s": nnz / (ms / 1e3),
                         "rel_to_in_memory": im_ms / ms, "link_GBps": link / (ms / 1e3) / 1e9,
                         "sampled_max_err_over_absprod": err}
    # Section 3.3's layout: every vertical partition its own contiguous array
    per_c_parts = {}
    for c in (1, 2, 4, 8, 16):
        Xp = [Xh[:, c0:c0 + c].contiguous().pin_memory() for c0 in range(0, p, c)]
        Yp = [torch.empty((N, c), dtype=torch.float32).pin_memory() for _ in Xp]
        h.apply_host_parts(Xp, Yp)
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.apply_host_parts(Xp, Yp)
            ts.append((time.perf_counter() - t0) * 1e3)
        ms = statistics.median(ts)
        got = torch.cat(Yp, dim=1).numpy()[rows].astype(np.float64)
        err = float((np.abs(got - ref) / np.maximum(scl, 1e-300)).max())
        per_c_parts[str(c)] = {"groups": len(Xp), "ms": round(ms, 3), "nnz_per_s": nnz / (ms / 1e3),
                               "rel_to_in_memory": im_ms / ms, "link_GBps": 2 * N * p * 4 / (ms / 1e3) / 1e9,
                               "sampled_max_err_over_absprod": err}
        del Xp, Yp
    per_c_parts["32"] = per_c["32"]
    budget = spmm.spmm_vpart_cols(N, N, p, spmm.SPMM_F32, 8 << 30)
    h.close()
    best = max(list(per_c.values()) + list(per_c_parts.values()), key=lambda d: d["rel_to_in_memory"])
    return base_line(args, f"vertically partitioned SpMM, X and Y ({p} FP32 columns) in host memory "
                           f"(R-MAT scale {args.scale}; nnz/s per call)",
                     best["nnz_per_s"], "nnz/s", best["ms"], f"rmat{args.scale}-vpart-p{p}", "f32",
                     {"in_memory_ms": round(im_ms, 3), "per_columns_in_memory": per_c,
                      "per_columns_in_memory_contiguous_parts": per_c_parts,
                      "cols_for_8GiB_budget": budget, "n": N, "nnz": nnz,
                      "timing": "wall clock per call (host buffers; the call returns with Y complete)",
                      "setup_s": {"generate": round(t_gen, 1)}})


def workload_ordering(args):
    """Vertex-ordering study (Section 5.1, stochastic block model figure): SpMM
    at k = 1 and 8 on graphs of 2^scale vertices and average degree 16 --
    R-MAT in natural and randomly permuted order, and SBM graphs with 16 or
    1024 clusters and 50% or 90% of edges inside clusters, in clustered and
    randomly permuted (unclustered) order.  Each graph runs resident in HBM
    (the paper's in-memory case), streamed from pinned host memory (its
    semi-external analogue) and resident with its vertices renumbered by
    degree (SPMM_RELABEL, vectors in that order); the L2 is flushed before
    each timed call."""
    import torch
    import oracle
    from paper_1602_02864_gb300 import spmm
    N = 1 << args.scale
    deg = args.edge_factor
    specs = [("rmat", None, None, False), ("rmat", None, None, True)]
    for C in (16, 1024):
        for p_in in (0.5, 0.9):
            for perm in (False, True):
                specs.append(("sbm", C, p_in, perm))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    X = {k: torch.from_numpy(synth.dense(N, k, seed=0)).cuda() for k in (1, 8)}
    Y = {k: torch.empty((N, k), device="cuda") for k in (1, 8)}
    rows = np.unique(synth.sample_rows(N, 2000, seed=9))
    Xh8 = X[8].cpu().numpy()
    out = []
    for kind, C, p_in, perm in specs:
        if kind == "rmat":
            A = synth.rmat_permuted_csr(args.scale, deg * N) if perm else synth.rmat_csr(args.scale, deg * N)
            name = "rmat-" + ("permuted" if perm else "natural")
        else:
            A = synth.sbm_csr(N, C, deg, p_in, seed=0, permuted=perm)
            name = f"sbm-C{C}-in{int(p_in * 100)}-" + ("unclustered" if perm else "clustered")
        entry = {"graph": name, "nnz": A.nnz}
        for mode in ("resident", "streaming"):
            h = spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None, streaming=(mode == "streaming"))
            for k in (1, 8):
                for _ in range(2):
                    h.apply(X[k], Y=Y[k])
                ts = []
                for _ in range(args.steps):
                    flush.zero_()
                    ts.append(event_ms(lambda: h.apply(X[k], Y=Y[k]), 1))
                ms = statistics.median(ts)
                entry[f"{mode}_k{k}_ms"] = round(ms, 4)
                entry[f"{mode}_k{k}_nnz_per_s"] = A.nnz / (ms / 1e3)
            if mode == "resident":
                ref = oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xh8, rows, threads=oracle.num_threads())
                scl = oracle.spmm_rows(A.row_ptr, A.col_idx, None, np.abs(Xh8), rows, threads=oracle.num_threads())
                got = Y[8][torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
                entry["sampled_max_err_over_absprod"] = float((np.abs(got - ref) / np.maximum(scl, 1e-300)).max())
            h.sync_status()
            h.close()
        # the same graph renumbered by degree inside the handle (SPMM_RELABEL),
        # vectors in the handle's order: the order the degrees give back to a
        # permuted graph
        hr = spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None, relabel=True)
        for k in (1, 8):
            Xr = hr.to_handle_order(X[k])
            for _ in range(2):
                hr.apply_relabelled(Xr, Y=Y[k])
            ts = []
            for _ in range(args.steps):
                flush.zero_()
                ts.append(event_ms(lambda: hr.apply_relabelled(Xr, Y=Y[k]), 1))
            ms = statistics.median(ts)
            entry[f"relabelled_k{k}_ms"] = round(ms, 4)
            entry[f"relabelled_k{k}_speedup_vs_resident"] = entry[f"resident_k{k}_ms"] / ms
            del Xr
        hr.close()
        for k in (1, 8):
            entry[f"sem_over_im_k{k}"] = entry[f"resident_k{k}_ms"] / entry[f"streaming_k{k}_ms"]
        out.append(entry)
        del A
    nat = out[0]
    return base_line(args, f"vertex-ordering study, SpMM k=1 nonzeros/s on R-MAT and SBM graphs "
                           f"(2^{args.scale} vertices, avg degree {deg})",
                     nat["resident_k1_nnz_per_s"], "nnz/s", nat["resident_k1_ms"],
                     f"ordering-{args.scale}", "f32",
                     {"graphs": out, "l2": "flushed before each timed call",
                      "timing": "median of --steps calls, CUDA events"})


def _fs_type(path):
    """File-system type of the mount holding path (from /proc/mounts)."""
    best, fs = "", "unknown"
    try:
        real = os.path.realpath(path)
        with open("/proc/mounts") as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 3 and real.startswith(parts[1]) and len(parts[1]) > len(best):
                    best, fs = parts[1], parts[2]
    except OSError:
        pass
    return fs


def workload_file(args):
    """Semi-external SpMM (Section 3.1): the matrix in a file on the local file
    system, read on every apply (page cache and O_DIRECT), against the same
    matrix streamed from pinned host memory and resident in HBM; k = 1 and 8."""
    import tempfile
    import torch
    import oracle
    from paper_1602_02864_gb300 import spmm
    N = 1 << args.scale
    A = synth.rmat_csr(args.scale, args.edge_factor * N, seed=0)
    nnz = A.nnz
    d = tempfile.mkdtemp(prefix="spmm_file_")
    path = os.path.join(d, "a.spmm")
    t = time.time()
    spmm.spmm_write_csr_file(path, A)
    t_write = time.time() - t
    file_bytes = os.path.getsize(path)
    X = {k: torch.from_numpy(synth.dense(N, k, seed=0)).cuda() for k in (1, 8)}
    Y = {k: torch.empty((N, k), device="cuda") for k in (1, 8)}
    res = {"fs": _fs_type(d), "file_GB": file_bytes / 1e9, "write_s": round(t_write, 2)}
    handles = [("resident", lambda: spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None)),
               ("host_streaming", lambda: spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None, streaming=True)),
               ("file_buffered", lambda: spmm.SparseMatrix.from_file(path, N, N)),
               ("file_direct", lambda: spmm.SparseMatrix.from_file(path, N, N, direct=True))]
    ref = None
    rows = np.unique(synth.sample_rows(N, 2000, seed=3))
    for name, make in handles:
        try:
            h = make()
        except spmm.SpmmError as e:
            res[name] = {"unavailable": str(e)[:160]}
            continue
        entry = {}
        for k in (1, 8):
            h.apply(X[k], Y=Y[k])
            ts = []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h.apply(X[k], Y=Y[k])
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - t0) * 1e3)
            ms = statistics.median(ts)
            entry[f"k{k}_ms"] = round(ms, 3)
            entry[f"k{k}_nnz_per_s"] = nnz / (ms / 1e3)
            entry[f"k{k}_matrix_GBps"] = (nnz * 4 + (N + 1) * 8) / (ms / 1e3) / 1e9
        got = Y[8][torch.from_numpy(rows).cuda()].cpu().numpy()
        if ref is None:
            ref = got
        entry["identical_to_resident"] = bool(np.array_equal(got, ref))
        h.sync_status()
        h.close()
        res[name] = entry
    Xh = X[8].cpu().numpy()
    o = oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xh, rows, threads=oracle.num_threads())
    scl = oracle.spmm_rows(A.row_ptr, A.col_idx, None, np.abs(Xh), rows, threads=oracle.num_threads())
    res["sampled_max_err_over_absprod"] = float((np.abs(ref - o) / np.maximum(scl, 1e-300)).max())
    os.unlink(path)
    os.rmdir(d)
    best = res.get("file_direct", {}) if "k1_ms" in res.get("file_direct", {}) else res["file_buffered"]
    return base_line(args, f"semi-external SpMM nonzeros/s, R-MAT scale {args.scale} matrix read from a file "
                           f"per apply (k=1)", best["k1_nnz_per_s"], "nnz/s", best["k1_ms"],
                     f"rmat{args.scale}-file", "f32",
                     {"modes": res, "n": N, "nnz": nnz,
                      "timing": "wall clock per apply incl. the file reads (median of --steps)"})


def workload_nmf_batched(args, nmf_ks=(8, 16, 32)):
    """256 Chung-Lu graphs in one block-diagonal handle: batched SpMM vs one
    launch per graph, then NMF (k = 8, 16, 32 by default; 50 steps; FP32 and
    BF16)."""
    import torch
    import oracle
    from paper_1602_02864_gb300 import spmm
    n_graphs = 256
    graphs = [synth.chunglu_csr(g, seed=0) for g in range(n_graphs)]
    nnz = sum(g.nnz for g in graphs)
    nv = sum(g.n_rows for g in graphs)
    h = spmm.SparseMatrix.batched(graphs, transpose=True, weighted=False)
    singles = [spmm.SparseMatrix(g.n_rows, g.n_cols, g.row_ptr, g.col_idx, None) for g in graphs]
    k = 16
    Xs = [torch.from_numpy(synth.dense(g.n_cols, k, seed=i)).cuda() for i, g in enumerate(graphs)]
    Xb = torch.cat(Xs)
    Ys = [torch.empty((g.n_rows, k), device="cuda") for g in graphs]
    Yb = torch.empty((nv, k), device="cuda")
    for _ in range(args.warmup):
        h.apply(Xb, Y=Yb)
        for s_, x, y in zip(singles, Xs, Ys):
            s_.apply(x, Y=y)
    ms_b = event_ms(lambda: h.apply(Xb, Y=Yb), args.steps)

    def per_graph():
        for s_, x, y in zip(singles, Xs, Ys):
            s_.apply(x, Y=y)
    ms_p = event_ms(per_graph, args.steps)
    same = all(torch.equal(Yb[o:o + g.n_rows], y) for o, g, y in
               zip(np.cumsum([0] + [g.n_rows for g in graphs[:-1]]), graphs, Ys))
    # spmm_apply_batched over the 256 separate handles: all k = 16, then k
    # cycling over 1, 8, 33 (three kernel instantiations), against one
    # spmm_apply per graph
    hl = [s_.handle for s_ in singles]
    Yq = [torch.empty_like(y) for y in Ys]
    for _ in range(args.warmup):
        spmm.spmm_apply_batched(hl, Xs, Yq)
    ms_q = event_ms(lambda: spmm.spmm_apply_batched(hl, Xs, Yq), args.steps)
    err_q = max(float(((a - b).abs() / (b.abs() + 1e-6)).max()) for a, b in zip(Yq, Ys))
    kmix = [(1, 8, 33)[i % 3] for i in range(n_graphs)]
    Xm = [torch.from_numpy(synth.dense(g.n_cols, kk, seed=i)).cuda() for i, (g, kk) in enumerate(zip(graphs, kmix))]
    Ym = [torch.empty((g.n_rows, kk), device="cuda") for g, kk in zip(graphs, kmix)]
    Ym1 = [torch.empty_like(y) for y in Ym]

    def per_graph_mixed():
        for s_, x, y in zip(singles, Xm, Ym1):
            s_.apply(x, Y=y)
    for _ in range(args.warmup):
        spmm.spmm_apply_batched(hl, Xm, Ym)
        per_graph_mixed()
    ms_m = event_ms(lambda: spmm.spmm_apply_batched(hl, Xm, Ym), args.steps)
    ms_m1 = event_ms(per_graph_mixed, args.steps)
    nnz_m = sum(g.nnz for g in graphs)
    apply_batched = {"k16_ms": ms_q, "k16_speedup_vs_per_graph": ms_p / ms_q, "k16_max_rel_diff": err_q,
                     "mixed_k_1_8_33_ms": ms_m, "mixed_per_graph_ms": ms_m1,
                     "mixed_speedup_vs_per_graph": ms_m1 / ms_m, "mixed_nnz_per_s": nnz_m / (ms_m / 1e3)}
    # autotuned plans, k = 16: (a) per graph, each graph timed alone on the
    # library's built-in grid (task size, short-row limit, X policy), then the
    # batched call with every entry on its own plan; (b) one plan for the
    # whole batch, chosen by timing the batched call itself
    from paper_1602_02864_gb300 import autotune
    t0 = time.perf_counter()
    chosen = {}
    for s_ in singles:
        best, _, cands = spmm.spmm_autotune(s_.handle, 16, spmm.SPMM_F32, 0, None, reps=2)
        c = cands[best]
        key = f"task_nnz={c['task_nnz']},short_max={c['short_max']},x_l2_policy={c['x_l2_policy']}"
        chosen[key] = chosen.get(key, 0) + 1
    t_tune = time.perf_counter() - t0

    def normwise(Ya, Yb):
        return max(float((a - b).abs().max() / b.abs().max().clamp_min(1e-30)) for a, b in zip(Ya, Yb))
    for _ in range(args.warmup):
        spmm.spmm_apply_batched(hl, Xs, Yq)
    ms_t = event_ms(lambda: spmm.spmm_apply_batched(hl, Xs, Yq), args.steps)
    apply_batched["k16_autotuned_per_graph"] = {
        "ms": ms_t, "speedup_vs_default_plans": ms_q / ms_t, "autotune_s": round(t_tune, 2),
        "max_normwise_diff_vs_default_plans": normwise(Yq, Ys),
        "plans": dict(sorted(chosen.items(), key=lambda kv: -kv[1])[:6])}
    t0 = time.perf_counter()
    tb = autotune.tune_batched(singles, Xs, Yq)
    t_tb = time.perf_counter() - t0
    ms_b2 = event_ms(lambda: spmm.spmm_apply_batched(hl, Xs, Yq), args.steps)
    apply_batched["k16_autotuned_batch"] = {
        "ms": ms_b2, "speedup_vs_default_plans": ms_q / ms_b2, "autotune_s": round(t_tb, 2),
        "plan": {n: tb[n] for n in ("task_nnz", "short_max", "long_row", "x_l2_policy")},
        "candidates": len(tb["candidate_ms"]),
        "candidate_ms_min_median_max": [float(np.min(tb["candidate_ms"])), float(np.median(tb["candidate_ms"])),
                                        float(np.max(tb["candidate_ms"]))],
        "max_normwise_diff_vs_default_plans": normwise(Yq, Ys)}
    for s_ in singles:
        s_.close()
    nmf = {}
    steps = 50
    for kk in nmf_ks:
        for ft, name in ((spmm.SPMM_F32, "f32"), (spmm.SPMM_BF16, "bf16")):
            W0 = torch.from_numpy(np.concatenate([synth.dense(g.n_rows, kk, seed=1000 + i, mode="unit") + 0.01
                                                  for i, g in enumerate(graphs)])).cuda()
            H0 = torch.from_numpy(np.concatenate([synth.dense(g.n_cols, kk, seed=2000 + i, mode="unit") + 0.01
                                                  for i, g in enumerate(graphs)])).cuda()
            W, H = W0.clone(), H0.clone()
            t0 = time.perf_counter()
            obj = h.nmf(kk, steps, W, H, ftype=ft)
            dt = time.perf_counter() - t0
            nmf[f"k{kk}_{name}"] = {"ms_per_call": round(dt * 1e3, 2), "ms_per_step": round(dt * 1e3 / steps, 3),
                                    "spmm_nnz_per_s": 2 * nnz * steps / dt,
                                    "objective_ratio_last_over_first_median":
                                        float(np.median(obj[:, -1] / obj[:, 0])),
                                    "monotone_graphs": int(np.sum(np.all(np.diff(obj, axis=1)
                                                                         <= 1e-5 * obj[:, :-1], axis=1)))}
            if kk == 16:
                # parity on the 4 smallest graphs against the FP64 oracle (FP32
                # factors; BF16 factors: the error of the whole BF16 path)
                offs_r = np.cumsum([0] + [g.n_rows for g in graphs])
                offs_c = np.cumsum([0] + [g.n_cols for g in graphs])
                w0, h0 = W0.cpu().numpy(), H0.cpu().numpy()
                worst = 0.0
                for i in np.argsort([g.n_rows for g in graphs])[:4]:
                    g = graphs[i]
                    _, _, objr = oracle.nmf(g.n_rows, g.n_cols, g.row_ptr, g.col_idx, None,
                                            w0[offs_r[i]:offs_r[i + 1]], h0[offs_c[i]:offs_c[i + 1]], steps)
                    worst = max(worst, float(np.max(np.abs(obj[i] - objr) / objr)))
                nmf[f"k{kk}_{name}"]["oracle_objective_max_rel_err_4_smallest"] = worst
                nmf[f"k{kk}_{name}"]["oracle_objective_final_rel_err_4_smallest"] = float(np.max(
                    [abs(obj[i][-1] - oracle.nmf(graphs[i].n_rows, graphs[i].n_cols, graphs[i].row_ptr,
                                                 graphs[i].col_idx, None, w0[offs_r[i]:offs_r[i + 1]],
                                                 h0[offs_c[i]:offs_c[i + 1]], steps)[2][-1])
                     / obj[i][-1] for i in np.argsort([g.n_rows for g in graphs])[:4]]))
    h.close()
    return base_line(args, "batched SpMM nonzeros/s (256 Chung-Lu graphs, one launch, k=16, FP32)",
                     nnz / (ms_b / 1e3), "nnz/s", ms_b, "chunglu256-batched-k16", "f32",
                     {"per_graph_launches_ms": ms_p, "batched_speedup": ms_p / ms_b, "bit_identical": same,
                      "spmm_apply_batched": apply_batched,
                      "graphs": n_graphs, "vertices": nv, "nnz": nnz, "nmf_50_steps": nmf})


def eigs_reference(S, scale):
    """The FP64 oracle's top-8 eigenvalues of this scale-18 graph from
    tests/golden (written by tests/golden/make_eigs_reference.py, which calls
    only the oracle), if the file describes this very matrix; else None."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", f"eigs_symrmat_lcc{scale}_top8.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for a in (np.ascontiguousarray(S.row_ptr, dtype=np.int64), np.ascontiguousarray(S.col_idx, dtype=np.int32),
              np.ascontiguousarray(S.values, dtype=np.float32)):
        h.update(a.tobytes())
    if rec["graph"]["csr_sha256"] != h.hexdigest():
        return None
    return np.asarray(rec["evals"], dtype=np.float64)


def workload_eigs(args, scales=None):
    """Top 8 eigenpairs of the normalised symmetrised R-MAT graph (largest
    component), block 16: FP32 vs BF16 SpMM inputs; errors vs the FP64 oracle
    at scale 18 (its stored eigenvalues when they match the graph, else a
    fresh oracle run)."""
    import torch
    import oracle
    from paper_1602_02864_gb300 import spmm
    out = {}
    if scales is None:
        scales = (18, args.scale if args.scale != 24 else 25)
    for scale in scales:
        t = time.time()
        S = synth.sym_rmat_lcc(scale, seed=0)
        t_gen = time.time() - t
        n = S.n_rows
        h = spmm.SparseMatrix.from_csr(S)
        V0 = torch.from_numpy(synth.dense(n, 16, seed=1).astype(np.float64)).cuda()
        X = torch.from_numpy(synth.dense(n, 16, seed=2)).cuda()
        Y = torch.empty((n, 16), device="cuda")
        flush = torch.empty(512 << 18, device="cuda")
        ms32 = event_ms(lambda: h.apply(X, Y=Y), args.steps, flush)
        xb = X.to(torch.bfloat16)
        ms16 = event_ms(lambda: h.apply(xb, Y=Y), args.steps, flush)
        res = {"n": n, "nnz": S.nnz, "spmm_k16_ms_f32": ms32, "spmm_k16_ms_bf16": ms16,
               "bf16_spmm_speedup": ms32 / ms16, "generate_s": round(t_gen, 1)}
        ref = None
        if scale == 18:
            ref = eigs_reference(S, scale)
            res["oracle_reference"] = "tests/golden (stored oracle run)" if ref is not None else "oracle run"
            if ref is None:
                Q0 = synth.dense(n, 8, seed=9).astype(np.float64)
                # a plain Lanczos needs a large basis on this clustered spectrum (240 was not enough)
                ref, _, _ = oracle.lanczos(n, S.row_ptr, S.col_idx, S.values, Q0, 8, 1000)
        for xt, name, tol in ((spmm.SPMM_F32, "f32", 1e-6 if scale <= 20 else 1e-5), (spmm.SPMM_BF16, "bf16", 5e-3)):
            # block Krylov-Schur (Section 4.2's method); at scale 25 only with
            # --eigs-krylov-full (it does not converge within 300 restarts there)
            if scale <= 20 or args.eigs_krylov_full:
                t0 = time.perf_counter()
                ev, rs, nrest = h.eigs(8, V0, block=16, max_basis=64, max_restarts=300, tol=tol, xtype=xt)
                dt = time.perf_counter() - t0
                r = {"s": round(dt, 2), "restarts": nrest, "evals": ev.tolist(), "max_residual": float(rs.max())}
                if ref is not None:
                    r["max_rel_err_vs_fp64_oracle"] = float(np.max(np.abs(ev - ref) / np.abs(ref)))
                res[name] = r
            # Chebyshev-filtered subspace iteration (degree 20, block 16); with
            # BF16 filter inputs the true residual stalls near 3e-2 (BF16
            # rounding of every filter step), so that run gets the FP32 target
            # and a fixed budget of 10 iterations, and reports where it stopped
            ftol, fit = (tol, 300) if xt == spmm.SPMM_F32 else (1e-6, 10)
            t0 = time.perf_counter()
            ev, rs, nit = h.eigs_filtered(8, V0, degree=20, lower=-1.0, max_iters=fit, tol=ftol, xtype=xt)
            dt = time.perf_counter() - t0
            r = {"s": round(dt, 2), "iterations": nit, "spmm_calls": nit * 21 + 1, "evals": ev.tolist(),
                 "max_residual": float(rs.max()), "tol": ftol, "converged": bool(rs.max() <= ftol)}
            if ref is not None:
                r["max_rel_err_vs_fp64_oracle"] = float(np.max(np.abs(ev - ref) / np.abs(ref)))
            res[name + "_filtered"] = r
        h.close()
        # the FP32 filtered solve on a handle with the vertices renumbered by
        # degree (SPMM_RELABEL): the start block and the eigenvectors change
        # order once, every product runs in the handle's order
        t0 = time.perf_counter()
        hr = spmm.SparseMatrix.from_csr(S, relabel=True)
        t_create = time.perf_counter() - t0
        Xr = hr.to_handle_order(X)
        ms_rl = event_ms(lambda: hr.apply_relabelled(Xr, Y=Y), args.steps, flush)
        t0 = time.perf_counter()
        ev, rs, nit = hr.eigs_filtered(8, V0, degree=20, lower=-1.0, max_iters=300, tol=res["f32_filtered"]["tol"],
                                       xtype=spmm.SPMM_F32)
        dt = time.perf_counter() - t0
        r = {"s": round(dt, 2), "iterations": nit, "create_s": round(t_create, 2), "spmm_k16_ms_f32": ms_rl,
             "spmm_speedup_vs_input_order": ms32 / ms_rl, "evals": ev.tolist(), "max_residual": float(rs.max()),
             "converged": bool(rs.max() <= res["f32_filtered"]["tol"])}
        if ref is not None:
            r["max_rel_err_vs_fp64_oracle"] = float(np.max(np.abs(ev - ref) / np.abs(ref)))
        res["f32_filtered_relabelled"] = r
        hr.close()
        del Xr
        out[f"scale{scale}"] = res
        del S
    big = out[max(out)]
    return base_line(args, "eigensolver SpMM (k=16) nonzeros/s, BF16 X (R-MAT LCC, normalised)",
                     big["nnz"] / (big["spmm_k16_ms_bf16"] / 1e3), "nnz/s", big["spmm_k16_ms_bf16"],
                     "symrmat-lcc-eigs-top8-block16", "bf16", {"results": out})


def workload_gather_ceiling(args):
    """Random-row gather ceilings: row sizes 4..256 B from tables inside L2
    (64 MB) and in DRAM (8 GB)."""
    from paper_1602_02864_gb300 import probe, spmm  # noqa: F401
    out = {}
    for rb in (4, 8, 16, 32, 64, 128, 256):
        for tb, name in (((64 << 20), "l2_64MB"), ((8 << 30), "dram_8GB")):
            r, b = probe.spmm_probe_gather(tb, rb)
            out[f"{rb}B_{name}"] = {"rows_per_s": r, "GBps": b / 1e9}
    best = max(v["rows_per_s"] for v in out.values())
    return base_line(args, "random row-gather ceiling (rows/s)", best, "rows/s", 0.0, "gather-ceiling", "f32",
                     {"probes": out})


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.record_traffic:
        return record_traffic(args.record_traffic, args)
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload != "ksweep":
        import torch
        torch.cuda.set_device(local)
        fn = {"streaming": workload_streaming, "nmf-batched": workload_nmf_batched, "eigs": workload_eigs,
              "gather-ceiling": workload_gather_ceiling, "vpart": workload_vpart,
              "ordering": workload_ordering, "file": workload_file}
        print(json.dumps(fn[args.workload](args)), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_1602_02864_gb300 import probe, spmm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ks = [int(k) for k in args.ks.split(",")]
    A, t_gen = make_graph(args)
    N, nnz = A.n_rows, A.nnz
    t0 = time.time()
    h = spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None, transpose=args.pagerank_iters > 0 or args.transpose,
                          reorder=args.reorder)
    torch.cuda.synchronize()
    t_create = time.time() - t0
    # autotune the plan of each orientation on a short candidate list
    t0 = time.time()
    from paper_1602_02864_gb300.autotune import POWER_LAW_CANDIDATES
    cands = POWER_LAW_CANDIDATES
    tuned = {}
    kt = 8 if 8 in ks else ks[0]
    best, times, _ = spmm.spmm_autotune(h.handle, kt, spmm.SPMM_F32, int(args.transpose), cands, reps=2)
    tuned["transpose" if args.transpose else "forward"] = dict(cands[best], k=kt, ms=round(float(times[best]), 4))
    if args.pagerank_iters and not args.transpose:
        best, times, _ = spmm.spmm_autotune(h.handle, 1, spmm.SPMM_F32, 1, cands, reps=2)
        tuned["transpose"] = dict(cands[best], k=1, ms=round(float(times[best]), 4))
    t_tune = time.time() - t0
    info = h.info()
    kmax = max(ks)
    Xh = synth.dense(N, kmax, seed=0)
    X64 = torch.from_numpy(Xh).to(dev)
    X = {k: X64[:, :k].contiguous() for k in ks}
    Y = {k: torch.empty((N, k), dtype=torch.float32, device=dev) for k in ks}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    # per product: the task kernel, the combine pass (if rows are split) and,
    # for 4-byte X rows (k = 1 float32), the packing of the hot X rows
    launches_per_apply = 1 + (1 if info["n_split_rows"] > 0 else 0)
    sweep_launches = sum(launches_per_apply + (1 if k == 1 and info["n_hot"] > 0 else 0) for k in ks)
    # per PageRank call: init, scale, reduce, then per iteration the hot-row
    # packing, the task kernel, the combine pass (if rows are split), the
    # update and the reduce
    launches_per_pr_iter = (3 + (1 if info["n_split_rows_t"] > 0 else 0)
                            + (1 if info["n_hot_t"] > 0 else 0))
    xpr = torch.empty(N, dtype=torch.float32, device=dev)
    pr_res = [None]

    def step(xs, ev=None):
        for i, k in enumerate(ks):
            if ev is not None:
                ev[i][0].record(stream)
            h.apply(xs[k], Y=Y[k], transpose=args.transpose)
            if ev is not None:
                ev[i][1].record(stream)
        if args.pagerank_iters:
            if ev is not None:
                ev[-1][0].record(stream)
            _, pr_res[0] = h.pagerank(0.85, args.pagerank_iters, x=xpr)
            if ev is not None:
                ev[-1][1].record(stream)

    # ---- warm-up, then the timed steps (L2 flushed before every step)
    for _ in range(args.warmup):
        flush.zero_()
        step(X)
    barrier()
    per_k = {k: [] for k in ks}
    pr_ms = []
    step_ms = []
    peak_gbs, peak_kind = load_peaks()
    with ClockSampler(local) as clk:
        barrier()
        # a profiler started with --profile-from-start off records only these
        # steps (or, with --profile-part relabelled, only the relabelled products)
        profiler_range(args.profile_part == "steps")
        for _ in range(args.steps):
            flush.zero_()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(len(ks) + 1)]
            step(X, ev)
            torch.cuda.synchronize()
            ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(len(ks))]
            for i, k in enumerate(ks):
                per_k[k].append(ms[i])
            if args.pagerank_iters:
                pr_ms.append(ev[-1][0].elapsed_time(ev[-1][1]))
                ms.append(pr_ms[-1])
            step_ms.append(sum(ms))
        profiler_range(False)
        barrier()
    value, t_total = aggregate(nnz * (len(ks) + args.pagerank_iters) * args.steps, sum(step_ms) / 1e3, world)

    # ---- per-k breakdown; roofline of the dominant launch
    breakdown = {}
    for k in ks:
        ms = statistics.median(per_k[k])
        B = alg_bytes(nnz, N, N, k, 4)
        breakdown[str(k)] = {"ms": round(ms, 4), "nnz_per_s": nnz / (ms / 1e3), "alg_GBps": B / (ms / 1e3) / 1e9,
                             "roofline_frac": B / (ms / 1e3) / 1e9 / peak_gbs,
                             "frac_of_nominal": B / (ms / 1e3) / 1e9 / NOMINAL_HBM_GBS}
    pagerank = None
    if args.pagerank_iters:
        ms = statistics.median(pr_ms)
        it_ms = ms / args.pagerank_iters
        B = pagerank_iter_bytes(nnz, N)
        xh = xpr.double().cpu().numpy()
        pagerank = {"iters": args.pagerank_iters, "ms": round(ms, 3), "ms_per_iter": round(it_ms, 4),
                    "nnz_per_s": nnz / (it_ms / 1e3), "alg_GBps": B / (it_ms / 1e3) / 1e9,
                    "roofline_frac": B / (it_ms / 1e3) / 1e9 / peak_gbs, "sum_x": float(xh.sum()),
                    "min_x": float(xh.min()), "residual_first_last": [float(pr_res[0][0]), float(pr_res[0][-1])]}
    # The dominant kernel: the task kernel's k = 1 instantiation (the k = 1
    # product of the sweep and the A^T product of every PageRank iteration,
    # 1 + iters launches per step), timed by the events around the sweep's
    # k = 1 call (which also holds the hot-row copy and the split-row combine);
    # otherwise the slowest k of the sweep.
    kdom = 1 if (1 in ks and args.pagerank_iters) else max(ks, key=lambda k: statistics.median(per_k[k]))
    dom = breakdown[str(kdom)]
    launches = 1 + (args.pagerank_iters if kdom == 1 and not args.transpose else 0)
    dom_name = (f"rows_kernel k={kdom} f32 ({'A^T' if args.transpose else 'A'} X; {launches} launches per step"
                + (", the A^T product of each PageRank iteration included)" if launches > 1 else ")"))
    traffic, traffic_src = (None, "not recorded for this k")
    if kdom == 1 and not args.transpose:
        traffic, traffic_src = read_traffic(args.scale, args.edge_factor, nnz)

    # ---- gather probes for each k: the rate of the X-row gathers alone (one X
    # row per nonzero), from uniformly random rows of a table of X's size and
    # from this matrix's own column stream replayed with nothing else of the
    # SpMM.  A reference rate, not a bound: from k = 8 on the kernel beats the
    # matrix-stream probe, whose plain gathers keep the hot columns in L2 worse.
    ceilings = {}
    for k in ([] if args.no_ceiling else ks):
        rb = 4
        while rb < 4 * k:
            rb *= 2
        uni, _ = probe.spmm_probe_gather(N * k * 4, rb)
        own, _ = probe.spmm_probe_gather_cols(h.handle, 0, 4 * k)
        ceilings[str(k)] = {"table_MB": round(N * k * 4 / 1e6, 1), "uniform_rows_per_s": uni,
                            "matrix_stream_rows_per_s": own,
                            "frac_of_matrix_stream": breakdown[str(k)]["nnz_per_s"] / own}
    pr_ceiling = None
    if args.pagerank_iters and not args.no_ceiling:
        own, _ = probe.spmm_probe_gather_cols(h.handle, 1, 4)
        pr_ceiling = {"matrix_stream_rows_per_s": own, "frac_of_matrix_stream": pagerank["nnz_per_s"] / own}

    # ---- BF16 X: speedup over FP32 and error on sampled rows vs the oracle
    import oracle
    othreads = oracle.num_threads()
    sample = np.unique(synth.sample_rows(N, 2000, seed=3))
    sample_t = torch.from_numpy(sample).to(dev)
    absX = np.abs(Xh)
    scale = {k: oracle.spmm_rows(A.row_ptr, A.col_idx, None, absX, sample, threads=othreads, k=k) for k in ks}
    del absX
    bf16 = {}
    if not args.no_bf16:
        for k in ks:
            xb = X[k].to(torch.bfloat16)
            yb = torch.empty_like(Y[k])
            for _ in range(3):
                h.apply(xb, Y=yb)
            ts = []
            for _ in range(max(3, args.steps)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.apply(xb, Y=yb)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.mean(ts)
            Xr = xb.float().cpu().numpy()          # bf16 values widen exactly to float32
            ref = oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xr, sample, threads=othreads)
            err = np.abs(yb.index_select(0, sample_t).cpu().numpy().astype(np.float64) - ref)
            del Xr
            B = alg_bytes(nnz, N, N, k, 2)
            bf16[str(k)] = {"ms": round(ms, 4), "speedup_vs_f32": breakdown[str(k)]["ms"] / ms,
                            "nnz_per_s": nnz / (ms / 1e3), "alg_GBps": B / (ms / 1e3) / 1e9,
                            "roofline_frac": B / (ms / 1e3) / 1e9 / peak_gbs,
                            "max_err_over_absprod": float((err / np.maximum(scale[k], 1e-300)).max())}
            del xb, yb

    # ---- parity on sampled rows (FP32 path vs FP64 oracle)
    parity = {}
    for k in ks:
        ref = oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xh, sample, threads=othreads, k=k)
        got = Y[k].index_select(0, sample_t).cpu().numpy().astype(np.float64)
        parity[str(k)] = float((np.abs(got - ref) / np.maximum(scale[k], 1e-300)).max())

    # ---- end to end through the library's host-buffer entry point: every
    # step hands the sweep's X matrices to spmm_apply_host_parts, each X_k in
    # pinned host memory as vertical partitions of at most P columns, each
    # partition a contiguous row-major array (the paper's layout for dense
    # matrices outside memory, Section 3.3; a k wider than P takes one pass
    # over A per partition).  The call copies each part in, multiplies and
    # copies the result out on three streams so the parts overlap, and
    # returns with every Y partition on the host; PageRank runs on the
    # device and its ranks are read back to pinned host memory.  The sweep's
    # A X products and PageRank's A^T products use separate scratch of the
    # handle, so PageRank runs from a second host thread while the sweep's
    # copies hold the link (both calls block their thread; ctypes releases
    # the GIL).  A transposed sweep, or a handle with relabelled columns,
    # shares scratch with PageRank, so there PageRank runs after the sweep.
    e2e = None
    if not args.no_e2e:
        P = max(1, min(64, args.e2e_part_cols))
        cuts = vertical_parts(ks, P)
        Xp = [X[k][:, c0:c1].contiguous().cpu().pin_memory() for k, c0, c1 in cuts]
        Yp = [torch.empty((N, c1 - c0), dtype=torch.float32).pin_memory() for _, c0, c1 in cuts]
        xp_host = torch.empty(N, dtype=torch.float32).pin_memory()
        pr_stream = torch.cuda.Stream()
        pr_err = []

        def pr_part():
            try:
                with torch.cuda.stream(pr_stream):
                    h.pagerank(0.85, args.pagerank_iters, x=xpr, stream=pr_stream)
                    xp_host.copy_(xpr, non_blocking=True)
                pr_stream.synchronize()
            except Exception as ex:            # re-raised by the step
                pr_err.append(ex)

        overlap = bool(args.pagerank_iters) and not args.transpose and not args.reorder

        def e2e_step():
            t = threading.Thread(target=pr_part) if overlap else None
            if t is not None:
                t.start()
            try:
                h.apply_host_parts(Xp, Yp, transpose=args.transpose, stream=stream)
            finally:
                if t is not None:
                    t.join()
            if pr_err:
                raise pr_err[0]
            if args.pagerank_iters and not overlap:
                pr_part()
                if pr_err:
                    raise pr_err[0]
        # one call alone first: it grows the handle's group buffers, which
        # must not overlap other calls on the handle
        h.apply_host_parts(Xp, Yp, transpose=args.transpose, stream=stream)
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_s = []                     # host time of each step (each ends with its results on the host)
        for _ in range(reps):
            ts = time.perf_counter()
            e2e_step()
            step_s.append(time.perf_counter() - ts)
        e1.record(stream)
        torch.cuda.synchronize()
        te = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0)
        # each Y partition against a device product of the same columns (the
        # sweep's own result where the partition is the whole X_k)
        ok = all(torch.equal(Yp[i], (Y[k] if c1 - c0 == k else
                                     h.apply(X[k][:, c0:c1].contiguous(), transpose=args.transpose)).cpu())
                 for i, (k, c0, c1) in enumerate(cuts))
        if args.pagerank_iters:
            ok = ok and torch.equal(xp_host, xpr.cpu())
        hb = sum(N * k * 4 for k in ks)
        db = hb + (N * 4 if args.pagerank_iters else 0)
        e2e = {"value": world * nnz * (len(ks) + args.pagerank_iters) * reps / te, "unit": UNIT,
               "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db, "ms_per_step": 1e3 * te / reps,
               "api": "spmm_apply_host_parts (host X and Y, each X_k and Y_k as vertical partitions of at "
                      f"most {P} columns: {len(cuts)} parts, one pass over A each) + spmm_pagerank + rank read-back"
                      + (" (PageRank on a second host thread during the sweep)" if overlap else ""),
               "part_cols": P, "passes_over_A": len(cuts),
               "step_ms": [round(1e3 * x, 2) for x in step_s],
               "median_step_ms": round(1e3 * statistics.median(step_s), 2),
               "results_match_device": bool(ok)}
        del Xp, Yp
        # the link's floor for the step's bytes: both directions at once, or
        # the slower one-way leg, whichever takes longer
        try:
            lr = link_rates_gbs()
            floor_ms = 1e3 * max((hb + db) / (lr["both_GBps"] * 1e9), hb / (lr["h2d_GBps"] * 1e9),
                                 db / (lr["d2h_GBps"] * 1e9))
            e2e["link"] = dict(lr, floor_ms=floor_ms, frac_of_floor=floor_ms / e2e["ms_per_step"])
        except Exception as ex:                # a report, not a reason to lose the line
            e2e["link"] = {"error": f"{type(ex).__name__}: {ex}"}

    # ---- the same sweep and PageRank on a handle made with SPMM_RELABEL
    # (vertices by decreasing degree): the products with the vectors kept in
    # the handle's order (spmm_apply_relabelled), PageRank through its public
    # call (ranks in and out of the input order once per call), and the first
    # k's result brought back to the input order against this run's Y
    relabelled = None
    if rank == 0 and not args.no_relabel:
        t0 = time.time()
        hr = spmm.SparseMatrix(N, N, A.row_ptr, A.col_idx, None, transpose=args.pagerank_iters > 0,
                               relabel=True)
        torch.cuda.synchronize()
        t_rl = time.time() - t0
        per = {}
        for k in ks:
            Xr = hr.to_handle_order(X[k])
            Yr = torch.empty((N, k), dtype=torch.float32, device=dev)
            hr.apply_relabelled(Xr, Y=Yr)
            flush.zero_()
            profiler_range(args.profile_part == "relabelled")
            hr.apply_relabelled(Xr, Y=Yr)
            profiler_range(False)
            ms = event_ms(lambda: hr.apply_relabelled(Xr, Y=Yr), args.steps, flush)
            B = alg_bytes(nnz, N, N, k, 4)
            d = (hr.to_input_order(Yr) - Y[k]).abs().max().item() / max(Y[k].abs().max().item(), 1e-30)
            per[str(k)] = {"ms": round(ms, 4), "speedup_vs_input_order": breakdown[str(k)]["ms"] / ms,
                           "nnz_per_s": nnz / (ms / 1e3), "roofline_frac": B / (ms / 1e3) / 1e9 / peak_gbs,
                           "max_diff_vs_input_order_result": d}
            del Xr, Yr
        pr_rl = None
        if args.pagerank_iters:
            xrl = torch.empty(N, dtype=torch.float32, device=dev)
            hr.pagerank(0.85, args.pagerank_iters, x=xrl)
            ms = event_ms(lambda: hr.pagerank(0.85, args.pagerank_iters, x=xrl), args.steps)
            pr_rl = {"ms": round(ms, 3), "speedup_vs_input_order": pagerank["ms"] / ms,
                     "max_rel_diff_vs_input_order_ranks":
                         float(((xrl - xpr).abs() / xpr.abs().clamp_min(1e-30)).max().item())}
            del xrl
        rl_ms = sum(v["ms"] for v in per.values()) + (pr_rl["ms"] if pr_rl else 0.0)
        relabelled = {"order": "vertices by decreasing row + column entry count (SPMM_RELABEL)",
                      "create_s": round(t_rl, 2), "per_k": per, "pagerank": pr_rl,
                      "step_ms": round(rl_ms, 3),
                      "nnz_per_s_step": nnz * (len(ks) + args.pagerank_iters) / (rl_ms / 1e3),
                      "note": "products with X and Y kept in the handle's vertex order; not the headline, "
                              "which multiplies in the input order"}
        hr.close()
        torch.cuda.empty_cache()

    # ---- CPU baseline: the oracle on a bounded row sample, all host cores
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = oracle.num_threads()
        rows, nz = cpu_sample_rows(A, 1_000_000)
        dt = run_cpu_oracle(A, Xh, ks, rows, threads)
        target = nz * args.cpu_seconds / max(dt, 1e-3) / 2
        rows, nz = cpu_sample_rows(A, target, seed=9)
        pr = 1 if args.pagerank_iters else 0
        dt = run_cpu_oracle(A, Xh, ks, rows, threads, pr)
        cpu = {"value": (nz * len(ks) + pr * nnz) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{len(rows)} seeded rows ({nz} nonzeros) of the scale-{args.scale} graph, FP64, "
                         f"every k in the sweep, plus {pr} full PageRank iteration (serial) ({dt:.1f} s)",
               "host": host_cpu()}
        # the same oracle on one host thread (a smaller sample, SpMM rows only)
        rows1, nz1 = cpu_sample_rows(A, max(nz // max(threads, 1), 10_000), seed=10)
        dt1 = run_cpu_oracle(A, Xh, ks, rows1, 1)
        cpu["single_thread"] = {"value": nz1 * len(ks) / dt1, "unit": UNIT, "cores": 1,
                                "sample": f"{len(rows1)} seeded rows ({nz1} nonzeros), every k in the sweep, "
                                          f"no PageRank ({dt1:.1f} s)"}
        # per k, on the one-thread sample: all cores and one thread
        cpu["per_k"] = {}
        for k in ks:
            r = {}
            for th in (threads, 1):
                t0 = time.perf_counter()
                oracle.spmm_rows(A.row_ptr, A.col_idx, None, Xh, rows1, threads=th, k=k)
                r["all_cores" if th == threads else "one_thread"] = nz1 / (time.perf_counter() - t0)
            cpu["per_k"][str(k)] = r

    # ---- streaming mode on a smaller graph (R-MAT scale 26, avg degree 32,
    # 8.95 GB of CSR in pinned host memory): link GB/s against the measured
    # pinned host-to-device peak
    streaming = None
    if rank == 0 and not args.no_stream:
        h.close()
        torch.cuda.empty_cache()
        sargs = argparse.Namespace(**vars(args))
        sargs.scale, sargs.steps, sargs.warmup = 26, 5, 2
        sl = workload_streaming(sargs)
        streaming = {"workload": sl["config"]["workload"], "nnz_per_s": sl["value"], "ms_per_call": sl["ms_per_step"],
                     "link": sl["link"], "bit_identical_to_resident": sl["bit_identical_to_resident"],
                     "sampled_rows_max_err_over_absprod": sl["sampled_rows_max_err_over_absprod"]}

    # ---- the other configurations, compact: the eigensolver's errors against
    # the FP64 oracle at scale 18 and the 256-graph batch (one launch, the
    # batched call over separate handles, NMF k = 16)
    configs = None
    if rank == 0 and not args.no_configs:
        if h.handle is not None:
            h.close()
        torch.cuda.empty_cache()
        cargs = argparse.Namespace(**vars(args))
        cargs.steps, cargs.warmup = 5, 2
        t0 = time.time()
        eg = workload_eigs(cargs, scales=(18,))["results"]["scale18"]
        t_eigs = time.time() - t0
        t0 = time.time()
        nb = workload_nmf_batched(cargs, nmf_ks=(16,))
        t_nmf = time.time() - t0
        configs = {
            "eigs_symrmat_lcc18": dict(eg, wall_s=round(t_eigs, 1)),
            "chunglu256_batched": {"nnz_per_s": nb["value"], "ms_per_call": nb["ms_per_step"],
                                   "wall_s": round(t_nmf, 1),
                                   **{key: nb[key] for key in ("per_graph_launches_ms", "batched_speedup",
                                                               "bit_identical", "spmm_apply_batched", "graphs",
                                                               "vertices", "nnz", "nmf_50_steps")}},
        }

    if rank == 0:
        line = {
            "metric": metric_name(args), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}-spmm-ksweep", "scale": args.scale, "n": N, "nnz": nnz,
                       "generated_edges": args.edge_factor << args.scale, "ks": ks, "values": "pattern",
                       "reorder": bool(args.reorder),
                       "l2": "flushed (512 MB write) before every step; inputs > L2",
                       "parallelism": "replicas" if world > 1 else "single"},
            "per_k": breakdown,
            "bf16": bf16,
            "parity_max_err_over_absprod": parity,
            "roofline": {"bound": "hbm", "achieved": dom["alg_GBps"], "peak": peak_gbs, "unit": "GB/s",
                         "frac": dom["roofline_frac"], "traffic": traffic, "traffic_source": traffic_src,
                         "kernel": dom_name, "peak_kind": peak_kind,
                         "alg_bytes_per_launch": alg_bytes(nnz, N, N, kdom, 4),
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": dom["alg_GBps"] / NOMINAL_HBM_GBS},
            "pagerank": pagerank,
            "gather_probe": {"per_k": ceilings, "pagerank": pr_ceiling,
                               "note": "rows/s of gathers alone: uniform = random rows of an X-sized table "
                                       "(spmm_probe_gather); matrix_stream = one row per stored entry of this "
                                       "matrix in storage order (spmm_probe_gather_cols); frac = the SpMM's "
                                       "nnz/s over that; a reference rate, not a bound (frac > 1 from k = 8 on)"},
            "e2e": e2e,
            "streaming": streaming,
            "relabelled": relabelled,
            "configs": configs,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": (sweep_launches + launches_per_pr_iter * args.pagerank_iters
                             + (3 if args.pagerank_iters else 0)) * args.steps,
            "setup_s": {"generate": round(t_gen, 2), "create": round(t_create, 2), "autotune": round(t_tune, 2)},
            "autotuned_plan": tuned,
            "plan": {"tasks": info["n_tasks"], "split_rows": info["n_split_rows"], "segments": info["n_segments"]},
        }
        print(json.dumps(line), flush=True)
    if h.handle is not None:
        h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
