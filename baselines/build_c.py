"""Compiles the C part of the paper-like CPU baseline (baselines/kron_cpu.c) into baselines/_lib.

Plain gcc with OpenMP, portable flags only (the same source builds on x86-64 and aarch64).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_DIR = os.path.join(HERE, "_lib")
KRON_LIB = os.path.join(LIB_DIR, "libkron_cpu.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "kron_cpu.c")
    if not force and os.path.exists(KRON_LIB) and os.path.getmtime(KRON_LIB) >= os.path.getmtime(src):
        return KRON_LIB
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = KRON_LIB + ".tmp"
    subprocess.run(["gcc", "-O3", "-std=c99", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp], check=True)
    os.replace(tmp, KRON_LIB)
    return KRON_LIB


if __name__ == "__main__":
    print(build(force=True))
