"""Build the FP64 CPU oracle (test infrastructure only) as an in-tree shared library.

gcc, -O2, -ffp-contract=off so that x86-64 and aarch64 hosts round identically,
OpenMP over independent columns only (the per-element arithmetic order is fixed).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cqr_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcqr_oracle.so")


FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc"] + FLAGS + ["-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def build_from_source(text: str, out_dir: str) -> str:
    """Compile another version of the oracle's source (the tests' planted-mistake copies)
    with the same flags into out_dir; returns the library path."""
    src = os.path.join(out_dir, "cqr_oracle_variant.c")
    lib = os.path.join(out_dir, "libcqr_oracle_variant.so")
    with open(src, "w") as fh:
        fh.write(text)
    subprocess.run(["gcc"] + FLAGS + ["-o", lib, src, "-lm"], check=True)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
