"""Build the CUDA library liblbm.so in-tree (sm_103a only).

Each translation unit under csrc/ is compiled by nvcc in parallel and the
objects are linked into paper_1311_2404_gb300/_lib/liblbm.so.  No
fast-math and no flush-to-zero (the paper reports that FTZ breaks the
entropic model, Sec. 4.4).  Re-running is incremental on file times.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Every translation unit holding a stream-and-collide kernel is compiled
# without multiply-add contraction: the kernels write their fused operations
# explicitly, so the AB and AA instances, the batched kernel, subdomain runs
# and the single-domain kernel apply the same operation sequence and agree
# bitwise.
NO_CONTRACT = ["-fmad=false"]
PER_FILE = {f: NO_CONTRACT for f in ("k_bgk.cu", "k_bgk_q15q27.cu", "k_mrt.cu", "k_elbm.cu",
                                      "k_les.cu", "k_les_q15q27.cu", "k_batch.cu")}
# Sources compiled into several objects, each with its own defines: the ELBM
# kernels, once per lattice code (0 D2Q9, 1 D3Q19, 2 D3Q15, 3 D3Q27) and
# storage group ({F64}, {F32, F32S}, {F16S, BF16S}), so that they build in
# parallel.
VARIANTS = {"k_elbm.cu": [(f"_l{lat}_s{st}", [f"-DELBM_LAT={lat}", f"-DELBM_STORES={st}u"])
                          for lat in (3, 1, 2, 0) for st in (1, 6, 24)]}
# compile the slowest units first
COST = {"k_elbm.cu": 9, "k_les_q15q27.cu": 5, "k_les.cu": 4, "k_bgk_q15q27.cu": 3,
        "k_mrt.cu": 3, "k_bgk.cu": 2, "k_support.cu": 2}
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-fvisibility=hidden", "--ftz=false", "--prec-div=true",
         "--prec-sqrt=true", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = max(_headers_mtime(), os.path.getmtime(os.path.abspath(__file__)))
    objs = []
    todo = []
    for src in srcs:
        base = os.path.basename(src)[:-3]
        for suffix, defs in VARIANTS.get(os.path.basename(src), [("", [])]):
            obj = os.path.join(LIBDIR, "obj", base + suffix + ".o")
            objs.append(obj)
            if not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr):
                todo.append((src, obj, defs))

    def compile_one(item):
        src, obj, defs = item
        t0 = time.time()
        cmd = [nvcc, *ARCH, *FLAGS, *PER_FILE.get(os.path.basename(src), []), *defs, "-c", src,
               "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return obj, time.time() - t0

    if todo:
        todo.sort(key=lambda it: -COST.get(os.path.basename(it[0]), 0))
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for obj, dt in ex.map(compile_one, todo):
                if verbose:
                    print(f"compiled {os.path.basename(obj)} in {dt:.0f} s")
    if todo or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl",
               "-lpthread", "-Xlinker", "--exclude-libs,ALL", "-Xlinker", "-Bsymbolic"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
