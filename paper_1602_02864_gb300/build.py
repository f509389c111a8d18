"""Build libspmm.so in place: every CUDA/C++ translation unit under csrc/ is
compiled for sm_103a in parallel, then linked into one shared library.  The
gather-ceiling diagnostics under diag/ are linked into libspmm_probe.so,
outside the library's interface."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libspmm.so")
DIAG = os.path.join(HERE, "diag")
PROBE_LIB = os.path.join(HERE, "libspmm_probe.so")
OBJ = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "-I", os.path.join(HERE, "diag"), "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _deps() -> list[str]:
    out = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out += [os.path.join(DIAG, f) for f in os.listdir(DIAG)]
    return out


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(PROBE_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB))
    return all(os.path.getmtime(p) <= t for p in _deps() + [__file__])


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src: str) -> str:
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [cc, *NVCC_FLAGS, "-x", "c++", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or ptxas_info or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {src}")
        return obj

    srcs = sources()
    diag = sorted(os.path.join(DIAG, f) for f in os.listdir(DIAG) if f.endswith(".cu"))
    with ThreadPoolExecutor(max_workers=min(len(srcs) + len(diag), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs + diag))
    lib_objs, diag_objs = objs[:len(srcs)], objs[len(srcs):]
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *lib_objs, "-lcudart"])
    os.replace(tmp, LIB)
    # the diagnostics: a library of their own that uses libspmm.so's handle
    # and error string (found beside it at run time)
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *diag_objs, "-L", HERE, "-lspmm", "-lcudart",
                           "-Xlinker", "-rpath,$ORIGIN"])
    os.replace(tmp, PROBE_LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
