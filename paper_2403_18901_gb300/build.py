"""Build libqdec.so (CUDA sm_103a) in-tree: paper_2403_18901_gb300/_build/libqdec.so.

nvcc -gencode arch=compute_103a,code=sm_103a; device code with -fmad=false and
host code with -ffp-contract=off so that no floating-point operation is fused
(the decoder is bit-exact by construction).  No torch dependency.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libqdec.so")
SOURCES = ["gdg_kernel.cu", "learn_kernel.cu", "ranker_kernel.cu", "qdec_api.cu", "dem_host.cpp"]
HEADERS = ["gdg_kernel.cuh", "qdec_internal.h", os.path.join("..", "..", "include", "qdec.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def flags(extra=()):
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "--expt-relaxed-constexpr",
            "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math", *extra]


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(SRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(SRC, h) for h in HEADERS] + [os.path.abspath(__file__)]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in deps):
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = []
    procs = []
    for s in srcs:
        o = os.path.join(OUT_DIR, os.path.basename(s) + ".o")
        extra = ["-Xptxas", "-v"] if (verbose and s.endswith("gdg_kernel.cu")) else []
        cmd = [nvcc(), *flags(extra), "-c", s, "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([nvcc(), ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
