"""Compile the CPU oracle (``qs_oracle.c``) into a shared library with gcc.

Test infrastructure: built by ``__graft_entry__.build()`` and on first use by the tests.
``-ffp-contract=off`` keeps the products and sums exactly as written (no fused
multiply-add), so the oracle rounds the same way on x86-64 and on Arm. OpenMP is used when
the compiler supports it; otherwise the loops run on one thread.
"""
from __future__ import annotations

import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qs_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libqs_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=BUILD_DIR)
    os.close(fd)
    try:
        try:
            subprocess.run(base + ["-fopenmp", SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base + [SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
        os.replace(tmp, LIB_PATH)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True))
