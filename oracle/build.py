"""Compile the CPU oracle (test infrastructure only) into oracle/_build/liboracle.so.

The oracle is plain C, built with -ffp-contract=off so that no floating-point
multiply-add is fused.  Nothing in the product package uses it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["bbcode.c", "dem.c", "gdg.c", "philox.c"]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "qdo.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in deps):
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    compile_lib(HERE, tmp)
    os.replace(tmp, LIB)
    return LIB


def compile_lib(src_dir: str, out: str) -> None:
    """gcc the oracle sources found in src_dir into the shared library out."""
    srcs = [os.path.join(src_dir, s) for s in SOURCES]
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", "-o", out] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)


if __name__ == "__main__":
    print(build(force=True))
