"""Compile the FP64 CPU oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain gcc, no fused multiply-add (-ffp-contract=off), no fast-math.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vegas_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def compile_source(src: str, out: str) -> None:
    """Compile an oracle source file into the shared library `out` (the flags
    of the oracle build; the test suite also compiles altered copies of the
    source with it, to check that the pins catch planted mistakes)."""
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter",
           src, "-o", out, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)


def build(force: bool = False) -> str:
    """Build liboracle.so if it is missing or older than its source; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    compile_source(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
