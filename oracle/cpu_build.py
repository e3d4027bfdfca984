"""Compile the FP64 C++/OpenMP CPU implementation (cpu_lm.cpp) into oracle/libcpulm.so.

Test and benchmark infrastructure only (the timed CPU comparator); the product path never loads it.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'cpu_lm.cpp')
LIB = os.path.join(HERE, 'libcpulm.so')


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + '.tmp'
    cmd = ['g++', '-O3', '-std=c++17', '-fopenmp', '-fPIC', '-shared', SRC, '-o', tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed for cpu_lm.cpp:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force=True))
