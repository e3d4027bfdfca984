"""Python binding of the C ABI: argument marshalling only (every step runs in the CUDA library).

Tensors are torch tensors: device tensors for the normal (asynchronous-on-stream) calls, or
pinned CPU tensors with ``host_buffers=True``.  Complex dtypes: torch.complex64 (FP32 path) or
torch.complex128 (FP64 path).  Layout metadata are host NumPy int arrays (see ``Layout``).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N


@dataclass
class Layout:
    """Host description of a batch of solution intervals (fields as in gc_layout)."""
    row_off: np.ndarray
    n_samp: np.ndarray
    n_bl: np.ndarray
    bl_off: np.ndarray
    n_ant: np.ndarray
    gain_off: np.ndarray
    ant1: np.ndarray
    ant2: np.ndarray
    n_rows: int
    n_gain: int
    n_dir: int = 1

    def __post_init__(self):
        self.row_off = np.ascontiguousarray(self.row_off, np.int64)
        for f in ('n_samp', 'n_bl', 'bl_off', 'n_ant', 'gain_off', 'ant1', 'ant2'):
            setattr(self, f, np.ascontiguousarray(getattr(self, f), np.int32))

    @classmethod
    def from_batch(cls, b) -> 'Layout':
        return cls(b.row_off, b.n_samp, b.n_bl, b.bl_off, b.n_ant, b.gain_off, b.ant1, b.ant2, b.n_rows
                   if b.kind != 'dd' else b.vis.shape[0], b.n_gain, b.n_dir)

    @property
    def n_intervals(self) -> int:
        return int(self.row_off.shape[0])

    def c(self) -> N.GcLayout:
        i32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        return N.GcLayout(self.n_intervals, self.row_off.ctypes.data_as(C.POINTER(C.c_int64)), i32(self.n_samp),
                          i32(self.n_bl), i32(self.bl_off), i32(self.n_ant), i32(self.gain_off),
                          int(self.ant1.shape[0]), i32(self.ant1), i32(self.ant2), int(self.n_rows),
                          int(self.n_gain), int(self.n_dir))


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.complex64:
        return N.GC_DTYPE_C64
    if t.dtype == torch.complex128:
        return N.GC_DTYPE_C128
    raise TypeError(f"complex64 or complex128 expected, got {t.dtype}")


def _stream_ptr(dev: torch.device):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_tensor(t, name, host):
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if host and t.is_cuda:
        raise ValueError(f"{name} must be a CPU tensor with host_buffers=True")
    if not host and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def _calibrate(fn_name, vis, model, layout: Layout, gains, tol, max_iter, schedule, compute_chi2, host_buffers,
               want_outputs=True, profile=False, path=N.GC_PATH_AUTO):
    host = bool(host_buffers)
    for t, n in ((vis, 'vis'), (model, 'model'), (gains, 'gains')):
        _check_tensor(t, n, host)
    dt = _dtype_code(vis)
    if model.dtype != vis.dtype or gains.dtype != vis.dtype:
        raise TypeError("vis, model and gains must share one dtype")
    n = layout.n_intervals
    if host:
        iters = torch.zeros(n, dtype=torch.int32).pin_memory() if want_outputs else None
        status = torch.zeros(n, dtype=torch.int32).pin_memory() if want_outputs else None
        chi2 = torch.zeros(n, dtype=torch.float64).pin_memory() if (want_outputs and compute_chi2) else None
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream) if torch.cuda.is_available() else None
    else:
        dev = vis.device
        iters = torch.zeros(n, dtype=torch.int32, device=dev) if want_outputs else None
        status = torch.zeros(n, dtype=torch.int32, device=dev) if want_outputs else None
        chi2 = torch.zeros(n, dtype=torch.float64, device=dev) if (want_outputs and compute_chi2) else None
        stream = _stream_ptr(dev)
    opt = N.GcOptions(float(tol), int(max_iter), int(schedule), dt, 1 if host else 0, 1 if compute_chi2 else 0,
                      1 if profile else 0, int(path))
    lay = layout.c()
    rc = getattr(N.lib(), fn_name)(_ptr(vis), _ptr(model), C.byref(lay), _ptr(gains), C.byref(opt), _ptr(iters),
                                   _ptr(chi2), _ptr(status), stream)
    N.check(rc, fn_name)
    return gains, iters, chi2, status


def calibrate_di_scalar(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                        compute_chi2=False, host_buffers=False, profile=False, path=N.GC_PATH_AUTO):
    """StefCal on scalar DI gains (gc_calibrate_di_scalar); gains are updated in place.

    path: GC_PATH_AUTO (default), GC_PATH_STREAM or GC_PATH_RESIDENT (see include/gaincal.h).
    Returns (gains, iters[n_int] int32, chi2[n_int] float64 or None, status[n_int] int32).
    """
    return _calibrate('gc_calibrate_di_scalar', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile, path=path)


def calibrate_di_jones2x2(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                          compute_chi2=False, host_buffers=False, profile=False, path=N.GC_PATH_AUTO):
    """Polarized StefCal on 2x2 DI gains (gc_calibrate_di_jones2x2); vis/model [rows,2,2], gains [n_gain,2,2]."""
    return _calibrate('gc_calibrate_di_jones2x2', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile, path=path)


def calibrate_dd_cohjones(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                          compute_chi2=False, host_buffers=False, profile=False, path=N.GC_PATH_AUTO):
    """CohJones on DD scalar gains (gc_calibrate_dd_cohjones); model [n_dir, rows], gains [n_gain, n_dir]."""
    return _calibrate('gc_calibrate_dd_cohjones', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile, path=path)


def _jhj_jhr(fn_name, vis, model, layout, gains, jones):
    for t, n in ((vis, 'vis'), (model, 'model'), (gains, 'gains')):
        _check_tensor(t, n, False)
    dt = _dtype_code(vis)
    if jones:
        jhd = torch.empty((layout.n_gain, 2, 2), dtype=vis.dtype, device=vis.device)
        jhj = torch.empty((layout.n_gain, 2, 2), dtype=vis.dtype, device=vis.device)
    else:
        jhd = torch.empty(layout.n_gain, dtype=vis.dtype, device=vis.device)
        jhj = torch.empty(layout.n_gain, dtype=torch.float32 if dt == N.GC_DTYPE_C64 else torch.float64,
                          device=vis.device)
    lay = layout.c()
    rc = getattr(N.lib(), fn_name)(_ptr(vis), _ptr(model), C.byref(lay), _ptr(gains), dt, _ptr(jhd), _ptr(jhj),
                                   _stream_ptr(vis.device))
    N.check(rc, fn_name)
    return jhd, jhj


def jhj_jhr_di_scalar(vis, model, layout, gains):
    """One accumulation pass: (J^H d top half [n_gain] complex, diag J^H J [n_gain] real)."""
    return _jhj_jhr('gc_jhj_jhr_di_scalar', vis, model, layout, gains, False)


def jhj_jhr_di_jones2x2(vis, model, layout, gains):
    """One accumulation pass: (sum D Y^H [n_gain,2,2], sum Y Y^H [n_gain,2,2])."""
    return _jhj_jhr('gc_jhj_jhr_di_jones2x2', vis, model, layout, gains, True)


def autotune_di(vis, model, layout, gains, iters=24):
    """Pick the fastest launch shape for this layout's shape bucket (gc_autotune_di); gains unchanged.

    Returns the fastest iteration-kernel time in ms.
    """
    for t, n in ((vis, 'vis'), (model, 'model'), (gains, 'gains')):
        _check_tensor(t, n, False)
    kind = 1 if vis.dim() == 3 else 0
    best = C.c_double(0.0)
    lay = layout.c()
    rc = N.lib().gc_autotune_di(kind, _ptr(vis), _ptr(model), C.byref(lay), _ptr(gains), _dtype_code(vis),
                                int(iters), C.byref(best), _stream_ptr(vis.device))
    N.check(rc, 'gc_autotune_di')
    return best.value


def profile_last():
    """(iteration-kernel ms, iteration launches, row-iterations) of the last profiled calibrate call."""
    ms = C.c_double(0.0); n = C.c_int64(0); ri = C.c_int64(0)
    N.lib().gc_profile_last(C.byref(ms), C.byref(n), C.byref(ri))
    return ms.value, n.value, ri.value


def profile_detail():
    """(moment-pass ms, baselines x iterations, path) of the last profiled calibrate call."""
    ms = C.c_double(0.0); bi = C.c_int64(0); p = C.c_int32(0)
    N.lib().gc_profile_detail(C.byref(ms), C.byref(bi), C.byref(p))
    return ms.value, bi.value, p.value


def launch_count() -> int:
    return int(N.lib().gc_launch_count())


def release():
    N.check(N.lib().gc_release(), 'gc_release')
