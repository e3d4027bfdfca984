"""FP64 C++/OpenMP CPU calibration (cpu_lm.cpp): StefCal then App. C LM with the whole J^H J of
eq. JHJ:pol, one interval per thread, all host cores.  The benchmark's all-core CPU comparator.

Test and benchmark infrastructure only (see the package header): built by cpu_build.build(),
loaded with ctypes, sharing no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import cpu_build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(cpu_build.build())
        p = C.c_void_p
        _lib.cpu_calibrate_jones_lm.argtypes = [p, p, C.c_int, p, p, p, p, p, p, p, p, p, C.c_double, C.c_int, C.c_int,
                                                C.c_double, C.c_double, p, p, C.c_int]
        _lib.cpu_calibrate_jones_lm.restype = C.c_int
    return _lib


def calibrate_jones_lm(b, gains=None, intervals=None, tol=1e-6, max_iter=2000, lm_after=20, lam0=1e-2, K=10.0,
                       threads=0):
    """Solve the listed (default: all) intervals of a 2x2 synth.Batch.

    Returns (gains [n_gain, 2, 2] complex64 with the listed intervals solved, iters, status, threads used).
    """
    lib = _load()
    idx = np.arange(b.n_int) if intervals is None else np.asarray(intervals, np.int64)
    g = np.ascontiguousarray((b.g0() if gains is None else gains).astype(np.complex64))
    vis = np.ascontiguousarray(b.vis.astype(np.complex64))
    model = np.ascontiguousarray(b.model.astype(np.complex64))
    i64 = lambda a: np.ascontiguousarray(a, np.int64)
    i32 = lambda a: np.ascontiguousarray(a, np.int32)
    row_off, n_samp, n_bl = i64(b.row_off[idx]), i32(b.n_samp[idx]), i32(b.n_bl[idx])
    bl_off, n_ant, gain_off = i32(b.bl_off[idx]), i32(b.n_ant[idx]), i32(b.gain_off[idx])
    a1, a2 = i32(b.ant1), i32(b.ant2)
    iters = np.zeros(len(idx), np.int32)
    status = np.zeros(len(idx), np.int32)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    used = lib.cpu_calibrate_jones_lm(ptr(vis), ptr(model), len(idx), ptr(row_off), ptr(n_samp), ptr(n_bl),
                                      ptr(bl_off), ptr(n_ant), ptr(gain_off), ptr(a1), ptr(a2), ptr(g), float(tol),
                                      int(max_iter), int(lm_after), float(lam0), float(K), ptr(iters), ptr(status),
                                      int(threads))
    return g, iters, status, used
