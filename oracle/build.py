"""Compile the C oracle (``oracle/ryser.c``) into ``oracle/_build``.

Test infrastructure only: the library path never loads what this builds.
Plain gcc, no CUDA; the same flags on x86_64 and aarch64 (no FMA contraction,
so both machines round identically).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ryser.c")
OUT_DIR = os.path.join(HERE, "_build")

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wextra"]


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(OUT_DIR, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Build the oracle (or one planted-mistake variant of it) and return its path."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, f"-DORACLE_MUTANT={int(mutant)}", "-o", tmp, SRC, "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
