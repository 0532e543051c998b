"""Build the in-tree CUDA library libfraclap.so for sm_103a.

Each translation unit is compiled by its own nvcc / g++ process in
parallel, then linked into paper_1802_03770_gb300/libfraclap.so.
Usage: python -m paper_1802_03770_gb300.build [--verbose]
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "libfraclap.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# the persistent batched kernel and its pass bodies are relocatable device
# code, device-linked together (each body function is register-allocated on
# its own; 80 registers keep three 256-thread CTAs per SM)
RDC = ["-rdc=true", "-maxrregcount=80"]
# (source, extra flags, object): ops.cu and batch.cu are compiled in two
# halves each (FP32 and FP64 instantiations) so that their largest parts run
# in parallel
CUDA_SOURCES = [("ops.cu", ["-DFL_OPS_PART=1"], "ops_f32.o"), ("ops.cu", ["-DFL_OPS_PART=2"], "ops_f64.o"),
                ("plan.cu", [], "plan.o"), ("batch.cu", ["-DFL_BATCH_PART=1"], "batch_f32.o"),
                ("batch.cu", ["-DFL_BATCH_PART=2"], "batch_f64.o"), ("unet.cu", [], "unet.o"),
                ("learned.cu", [], "learned.o"), ("domain.cu", [], "domain.o"),
                ("rows_w8.cu", [], "rows_w8.o"),
                ("persist.cu", RDC, "persist.o"), ("persist_body.cu", RDC, "persist_body.o")]
CXX_SOURCES = ["consts.cpp"]


def nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(home, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    if verbose and (res.stdout or res.stderr):
        print(res.stdout + res.stderr, flush=True)
    return res


def build(verbose=False, ptxas_info=False):
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    objs = []
    for src, flags, oname in CUDA_SOURCES:
        obj = os.path.join(BUILD, oname)
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", *flags, *inc, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        jobs.append(cmd)
        objs.append(obj)
    for src in CXX_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", *inc, "-I",
                     os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include"),
                     "-c", os.path.join(CSRC, src), "-o", obj])
        objs.append(obj)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(lambda c: _run(c, verbose), jobs))
    if ptxas_info:
        for r in results:
            sys.stdout.write(r.stderr)
    rdc_objs = [os.path.join(BUILD, o) for _, f, o in CUDA_SOURCES if f is RDC]
    dlink = os.path.join(BUILD, "persist_dlink.o")
    _run([nvcc(), *ARCH, "-dlink", "-Xcompiler", "-fPIC", "-o", dlink, *rdc_objs], verbose)
    _run([nvcc(), *ARCH, "-shared", "-o", OUT, *objs, dlink, "-lcudart"], verbose)
    return OUT


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(OUT)
