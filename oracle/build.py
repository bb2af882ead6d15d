"""Compile the FP64 oracle (plain C, OpenMP) into a shared library for ctypes.

Test infrastructure: the library built here is loaded only by the tests, the
package smoke check and the benchmark's CPU baseline leg.
"""

from __future__ import annotations

import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dlx_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def lib_path() -> str:
    return os.path.join(OUT_DIR, f"libdlx_oracle_{platform.machine()}.so")


def build(force: bool = False, verbose: bool = False) -> str:
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fcx-limited-range", SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=not verbose)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=not verbose)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
