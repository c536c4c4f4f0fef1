"""Compile the plain-C FP64 oracle into a shared library.

Test infrastructure: the oracle is the checker for the CUDA library and is
never linked into it. Built with -ffp-contract=off (no fused multiply-add,
which GCC on aarch64 would otherwise form) and without -ffast-math, so every
product is rounded before it is added, exactly as written in the C source.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def lib_path(mutant: int = 0) -> str:
    name = "liblbm_oracle.so" if mutant == 0 else f"liblbm_oracle_m{mutant}.so"
    return os.path.join(OUT_DIR, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Build the oracle (or a planted-mistake variant) and return its path."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           f"-DOR_MUTANT={mutant}", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(int(sys.argv[1]) if len(sys.argv) > 1 else 0, force=True))
