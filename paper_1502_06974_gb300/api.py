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


def _schedule_code(schedule):
    if isinstance(schedule, str):
        return {'stefcal': N.GC_SCHED_STEFCAL, 'gn': N.GC_SCHED_GN, 'lm': N.GC_SCHED_LM}[schedule]
    return int(schedule)


def _check_weights(weights, vis, layout, host):
    """Per-row weights: a contiguous real tensor [n_rows] of vis's precision, where vis is."""
    if weights is None:
        return None
    want = torch.float32 if vis.dtype == torch.complex64 else torch.float64
    if weights.dtype != want or weights.numel() != layout.n_rows:
        raise TypeError(f"weights must be {want} with one value per row ({layout.n_rows})")
    _check_tensor(weights, 'weights', host)
    return weights


def _calibrate(fn_name, vis, model, layout: Layout, gains, tol, max_iter, schedule, compute_chi2, host_buffers,
               want_outputs=True, profile=False, path=N.GC_PATH_AUTO, lm_after=None, lm_lambda0=0.0, lm_K=0.0,
               weights=None):
    host = bool(host_buffers)
    for t, n in ((vis, 'vis'), (model, 'model'), (gains, 'gains')):
        _check_tensor(t, n, host)
    dt = _dtype_code(vis)
    if model.dtype != vis.dtype or gains.dtype != vis.dtype:
        raise TypeError("vis, model and gains must share one dtype")
    weights = _check_weights(weights, vis, layout, host)
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
    opt = N.GcOptions(float(tol), int(max_iter), _schedule_code(schedule), dt, 1 if host else 0,
                      1 if compute_chi2 else 0, int(profile), int(path), 0,
                      N.GC_LM_DEFAULT_AFTER if lm_after is None else int(lm_after), 0, float(lm_lambda0), float(lm_K),
                      None if weights is None else weights.data_ptr())
    lay = layout.c()
    rc = getattr(N.lib(), fn_name)(_ptr(vis), _ptr(model), C.byref(lay), _ptr(gains), C.byref(opt), _ptr(iters),
                                   _ptr(chi2), _ptr(status), stream)
    N.check(rc, fn_name)
    return gains, iters, chi2, status


def calibrate_di_scalar(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                        compute_chi2=False, host_buffers=False, profile=False, path=N.GC_PATH_AUTO, lm_after=None,
                        lm_lambda0=0.0, lm_K=0.0, weights=None):
    """StefCal on scalar DI gains (gc_calibrate_di_scalar); gains are updated in place.

    schedule: GC_SCHED_STEFCAL / GC_SCHED_GN / GC_SCHED_LM, or 'stefcal' / 'gn' / 'lm'; with 'lm',
    lm_after StefCal iterations (None: GC_LM_DEFAULT_AFTER; 0: none) are followed by
    Levenberg-Marquardt with the whole J^H J (lm_lambda0, lm_K: 0 selects the library defaults; see
    include/gaincal.h).
    path: GC_PATH_AUTO (default), GC_PATH_STREAM or GC_PATH_RESIDENT (see include/gaincal.h).
    profile: 0 off, 1 (or True) time the iteration launches, 2 time the accumulate launches alone.
    weights: None or per-row real weights [rows] (float32 for complex64 data, float64 for complex128).
    Returns (gains, iters[n_int] int32, chi2[n_int] float64 or None, status[n_int] int32).
    """
    return _calibrate('gc_calibrate_di_scalar', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile, path=path, lm_after=lm_after, lm_lambda0=lm_lambda0, lm_K=lm_K,
                      weights=weights)


def calibrate_di_jones2x2(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                          compute_chi2=False, host_buffers=False, profile=False, path=N.GC_PATH_AUTO, lm_after=None,
                          lm_lambda0=0.0, lm_K=0.0, weights=None):
    """Polarized StefCal (or, with schedule 'lm', StefCal then Levenberg-Marquardt with the whole
    J^H J) on 2x2 DI gains (gc_calibrate_di_jones2x2); vis/model [rows,2,2], gains [n_gain,2,2];
    weights as for calibrate_di_scalar (one per 2x2 row)."""
    return _calibrate('gc_calibrate_di_jones2x2', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile, path=path, lm_after=lm_after, lm_lambda0=lm_lambda0, lm_K=lm_K,
                      weights=weights)


def profile_lm():
    """(ms, launches, flop) of the Levenberg-Marquardt phase of the last profiled DI calibration."""
    ms, n, fl = C.c_double(0.0), C.c_int64(0), C.c_double(0.0)
    N.check(N.lib().gc_profile_lm(C.byref(ms), C.byref(n), C.byref(fl)), 'gc_profile_lm')
    return ms.value, n.value, fl.value


LM_PHASES = ('blocks_and_gradient', 'matrix', 'factor_forward', 'back_substitution', 'trial_chi2_decision',
             'factor.panel_load', 'factor.panel_solve', 'factor.trailing_update')


def profile_lm_phases():
    """{phase: SM cycles} of the same LM phase (see gc_profile_lm_phases)."""
    buf = (C.c_double * len(LM_PHASES))()
    N.check(N.lib().gc_profile_lm_phases(buf, len(LM_PHASES)), 'gc_profile_lm_phases')
    return dict(zip(LM_PHASES, list(buf)))


def calibrate_dd_cohjones(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                          compute_chi2=False, host_buffers=False, profile=False, path=N.GC_PATH_AUTO):
    """CohJones on DD scalar gains (gc_calibrate_dd_cohjones); model [n_dir, rows], gains [n_gain, n_dir]."""
    return _calibrate('gc_calibrate_dd_cohjones', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile, path=path)


def calibrate_dd_alljones(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                          compute_chi2=False, host_buffers=False, profile=False, path=N.GC_PATH_AUTO):
    """AllJones on DD scalar gains (gc_calibrate_dd_alljones); same layout as calibrate_dd_cohjones."""
    return _calibrate('gc_calibrate_dd_alljones', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile, path=path)


def calibrate_dd_cohjones2x2(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                             compute_chi2=False, host_buffers=False, profile=False):
    """Polarized CohJones (gc_calibrate_dd_cohjones2x2); vis [rows, 2, 2], model [n_dir, rows, 2, 2],
    gains [n_gain, n_dir, 2, 2], all complex64."""
    return _calibrate('gc_calibrate_dd_cohjones2x2', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile)


def calibrate_dd_alljones2x2(vis, model, layout, gains, tol=1e-6, max_iter=1000, schedule=N.GC_SCHED_STEFCAL,
                             compute_chi2=False, host_buffers=False, profile=False):
    """Polarized AllJones (gc_calibrate_dd_alljones2x2); same layout as calibrate_dd_cohjones2x2."""
    return _calibrate('gc_calibrate_dd_alljones2x2', vis, model, layout, gains, tol, max_iter, schedule, compute_chi2,
                      host_buffers, profile=profile)


def calibrate_di_smooth(vis, model, n_t, n_f, ant1, ant2, n_ant, gains, sigma_t, sigma_f, tol=1e-6, max_iter=1000,
                        schedule=N.GC_SCHED_STEFCAL, compute_chi2=False):
    """Per-sample gains smoothed in time and frequency (gc_calibrate_di_smooth_scalar / _jones2x2,
    Sect. 3.4).  vis/model [n_t * n_f * n_bl] complex64 (2x2: [.., 2, 2]), time-major then channel
    then baseline; gains [n_t * n_f * n_ant] (2x2: [.., 2, 2]) updated in place; sigma_t / sigma_f
    the Gaussian kernel widths in samples.  Returns (gains, iters[1], chi2[n_t * n_f] or None, status[1])."""
    jones = vis.dim() == 3
    for t, n in ((vis, 'vis'), (model, 'model'), (gains, 'gains')):
        _check_tensor(t, n, False)
        if t.dtype != torch.complex64:
            raise TypeError(f"{n} must be complex64")
    a1 = np.ascontiguousarray(ant1, np.int32)
    a2 = np.ascontiguousarray(ant2, np.int32)
    sm = N.GcSmooth(int(n_t), int(n_f), int(a1.shape[0]), int(n_ant), a1.ctypes.data_as(C.POINTER(C.c_int32)),
                    a2.ctypes.data_as(C.POINTER(C.c_int32)), float(sigma_t), float(sigma_f))
    dev = vis.device
    iters = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    chi2 = torch.zeros(int(n_t) * int(n_f), dtype=torch.float64, device=dev) if compute_chi2 else None
    opt = N.GcOptions(float(tol), int(max_iter), _schedule_code(schedule), N.GC_DTYPE_C64, 0, 1 if compute_chi2 else 0)
    fn = 'gc_calibrate_di_smooth_jones2x2' if jones else 'gc_calibrate_di_smooth_scalar'
    rc = getattr(N.lib(), fn)(_ptr(vis), _ptr(model), C.byref(sm), _ptr(gains), C.byref(opt), _ptr(iters), _ptr(chi2),
                              _ptr(status), _stream_ptr(dev))
    N.check(rc, fn)
    return gains, iters, chi2, status


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


# ----------------------------------------------------------------------------- learned warm start

MLP_DIMS = (48, 256, 256, 8)


class Mlp:
    """Device buffers of the warm-start network (gc_mlp): FP32 params, gradients, Adam moments and
    the BF16 copy used by inference.  ``params`` is a flat float32 vector (layout in gaincal.h)."""

    def __init__(self, params, device, dims=MLP_DIMS):
        params = np.ascontiguousarray(params, np.float32)
        self.dims = tuple(int(d) for d in dims)
        self.params = torch.from_numpy(params).to(device)
        self.grads = torch.zeros_like(self.params)
        self.adam_m = torch.zeros_like(self.params)
        self.adam_v = torch.zeros_like(self.params)
        self.params_bf16 = torch.zeros(self.params.numel(), dtype=torch.bfloat16, device=device)
        self.step = 0
        i, h1, h2, o = self.dims
        self._c = N.GcMlp(i, h1, h2, o, self.params.data_ptr(), self.grads.data_ptr(), self.adam_m.data_ptr(),
                          self.adam_v.data_ptr(), self.params_bf16.data_ptr())

    def c(self):
        return C.byref(self._c)

    def work(self, n):
        return torch.empty(int(N.lib().gc_mlp_work_floats(self.c(), int(n))), dtype=torch.float32,
                           device=self.params.device)


def _f32(t, name):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")


def mlp_forward_f32(net: Mlp, x):
    _f32(x, 'x')
    n = x.shape[0]
    y = torch.empty((n, net.dims[3]), dtype=torch.float32, device=x.device)
    N.check(N.lib().gc_mlp_forward_f32(net.c(), _ptr(x), n, _ptr(y), _ptr(net.work(n)), _stream_ptr(x.device)),
            'gc_mlp_forward_f32')
    return y


def mlp_grad_f32(net: Mlp, x, t):
    """(gradient like params, loss) of mean((y - t)^2)."""
    _f32(x, 'x'); _f32(t, 't')
    n = x.shape[0]
    g = torch.empty_like(net.params)
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    N.check(N.lib().gc_mlp_grad_f32(net.c(), _ptr(x), _ptr(t), n, _ptr(g), _ptr(loss), _ptr(net.work(n)),
                                    _stream_ptr(x.device)), 'gc_mlp_grad_f32')
    return g, loss


def mlp_train_step(net: Mlp, x, t, lr, work=None, loss=None):
    """One Adam step; returns the device loss tensor (before the step)."""
    _f32(x, 'x'); _f32(t, 't')
    n = x.shape[0]
    net.step += 1
    loss = torch.zeros(1, dtype=torch.float32, device=x.device) if loss is None else loss
    work = net.work(n) if work is None else work
    N.check(N.lib().gc_mlp_train_step(net.c(), _ptr(x), _ptr(t), n, float(lr), net.step, _ptr(loss), _ptr(work),
                                      _stream_ptr(x.device)), 'gc_mlp_train_step')
    return loss


def mlp_infer_bf16(net: Mlp, x):
    _f32(x, 'x')
    n = x.shape[0]
    y = torch.empty((n, net.dims[3]), dtype=torch.float32, device=x.device)
    N.check(N.lib().gc_mlp_infer_bf16(net.c(), _ptr(x), n, _ptr(y), _stream_ptr(x.device)), 'gc_mlp_infer_bf16')
    return y


def _i64_dev(index, device):
    if isinstance(index, torch.Tensor):
        if index.dtype != torch.int64 or index.device != device or not index.is_contiguous():
            raise ValueError("index must be a contiguous int64 tensor on the data's device")
        return index
    return torch.from_numpy(np.ascontiguousarray(index, np.int64)).to(device)


def rows_gather_f32(src, index):
    """dst[r] = src[index[r]] for a float32 [m, w] CUDA tensor (gc_rows_gather_f32); index: host or device int64."""
    src2 = src.reshape(src.shape[0], -1)
    _f32(src2, 'src')
    idx = _i64_dev(index, src.device)
    n, w = int(idx.numel()), int(src2.shape[1])
    dst = torch.empty((n, w), dtype=torch.float32, device=src.device)
    N.check(N.lib().gc_rows_gather_f32(_ptr(src2), w, _ptr(idx), n, _ptr(dst), _stream_ptr(src.device)),
            'gc_rows_gather_f32')
    return dst


def col_stats_f32(x, index=None, zero_const_mean=True):
    """(mean, sd) float64 [w] device tensors of the columns of x over the rows `index` (all rows if None)."""
    _f32(x, 'x')
    w = int(x.shape[1])
    idx = None if index is None else _i64_dev(index, x.device)
    n = int(x.shape[0] if idx is None else idx.numel())
    mean = torch.empty(w, dtype=torch.float64, device=x.device)
    sd = torch.empty(w, dtype=torch.float64, device=x.device)
    N.check(N.lib().gc_col_stats_f32(_ptr(x), w, None if idx is None else _ptr(idx), n, int(bool(zero_const_mean)),
                                     _ptr(mean), _ptr(sd), _stream_ptr(x.device)), 'gc_col_stats_f32')
    return mean, sd


def standardize_f32(x, mean, sd):
    """(x - mean) / sd per column (mean None: x / sd), float32 out (gc_standardize_f32)."""
    _f32(x, 'x')
    out = torch.empty_like(x)
    N.check(N.lib().gc_standardize_f32(_ptr(x), int(x.shape[1]), int(x.shape[0]), None if mean is None else _ptr(mean),
                                       _ptr(sd), _ptr(out), _stream_ptr(x.device)), 'gc_standardize_f32')
    return out


def mlp_fold_standardization(net: Mlp, mean, sd, tsd):
    """Fold input standardisation and output scaling into the network in place."""
    for t, nm in ((mean, 'mean'), (sd, 'sd'), (tsd, 'tsd')):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous float64 CUDA tensor")
    N.check(N.lib().gc_mlp_fold_standardization(net.c(), _ptr(mean), _ptr(sd), _ptr(tsd),
                                                _stream_ptr(net.params.device)), 'gc_mlp_fold_standardization')


def _as_f32_view(g):
    """complex64 [n, 2, 2] -> float32 [n, 8] view (no copy)."""
    if g.dtype == torch.complex64:
        return torch.view_as_real(g).reshape(g.shape[0], -1)
    return g


def ws_features_jones(hist, jhd, jhj, lead, in_width=48):
    """Features (x [n, in_width], rot [n, 2]) from hist [n, 4, 2, 2] c64, jhd/jhj [n, 2, 2] c64, lead [n] f32."""
    h = torch.view_as_real(hist.contiguous()).reshape(hist.shape[0], 32)
    n = h.shape[0]
    x = torch.empty((n, in_width), dtype=torch.float32, device=h.device)
    rot = torch.empty((n, 2), dtype=torch.float32, device=h.device)
    N.check(N.lib().gc_ws_features_jones(_ptr(h), 32, _ptr(jhd.contiguous()), _ptr(jhj.contiguous()),
                                         _ptr(lead.contiguous()), n, in_width, _ptr(x), _ptr(rot),
                                         _stream_ptr(h.device)), 'gc_ws_features_jones')
    return x, rot


def ws_target_jones(g1, g_next, rot):
    """Training targets [n, 8] = e^{-i phi} (g_next - g1) from c64 [n, 2, 2] gains and rot [n, 2]."""
    n = g1.shape[0]
    t = torch.empty((n, 8), dtype=torch.float32, device=g1.device)
    N.check(N.lib().gc_ws_target_jones(_ptr(g1.contiguous()), _ptr(g_next.contiguous()), _ptr(rot), n, _ptr(t),
                                       _stream_ptr(g1.device)), 'gc_ws_target_jones')
    return t


def calibrate_di_jones2x2_warm(vis, model, layout: Layout, solutions, hist_off, lead, net, gains, tol=1e-6,
                               max_iter=1000, schedule=N.GC_SCHED_STEFCAL, compute_chi2=False, profile=False,
                               want_start=False, lm_after=None, lm_lambda0=0.0, lm_K=0.0):
    """gc_calibrate_di_jones2x2_warm: solve from the learned start (net=None: previous solution).
    schedule / lm_*: as calibrate_di_jones2x2 (with 'lm' the StefCal and LM iterations start from
    the chosen start).

    solutions: complex64 device [n_sol, 2, 2]; hist_off: host int32 [n_int, 4]; lead: host float32 [n_int].
    Returns (gains, iters, chi2 or None, status, used, dchi2, start or None).
    """
    for t, nm in ((vis, 'vis'), (model, 'model'), (gains, 'gains'), (solutions, 'solutions')):
        _check_tensor(t, nm, False)
        if t.dtype != torch.complex64:
            raise TypeError(f"{nm} must be complex64")
    hist_off = np.ascontiguousarray(hist_off, np.int32)
    lead = np.ascontiguousarray(lead, np.float32)
    n = layout.n_intervals
    if hist_off.shape != (n, 4) or lead.shape != (n,):
        raise ValueError("hist_off must be [n_intervals, 4] and lead [n_intervals]")
    dev = vis.device
    iters = torch.zeros(n, dtype=torch.int32, device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    used = torch.zeros(n, dtype=torch.int32, device=dev)
    dchi2 = torch.zeros(n, dtype=torch.float64, device=dev)
    chi2 = torch.zeros(n, dtype=torch.float64, device=dev) if compute_chi2 else None
    start = torch.empty_like(gains) if want_start else None
    w = N.GcWarm(solutions.data_ptr(), int(solutions.shape[0]), hist_off.ctypes.data_as(C.POINTER(C.c_int32)),
                 lead.ctypes.data_as(C.POINTER(C.c_float)), C.pointer(net._c) if net is not None else None,
                 used.data_ptr(), dchi2.data_ptr(), start.data_ptr() if start is not None else None)
    opt = N.GcOptions(float(tol), int(max_iter), _schedule_code(schedule), N.GC_DTYPE_C64, 0,
                      1 if compute_chi2 else 0, 1 if profile else 0, N.GC_PATH_AUTO, 0,
                      N.GC_LM_DEFAULT_AFTER if lm_after is None else int(lm_after), 0, float(lm_lambda0), float(lm_K))
    lay = layout.c()
    rc = N.lib().gc_calibrate_di_jones2x2_warm(_ptr(vis), _ptr(model), C.byref(lay), C.byref(w), _ptr(gains),
                                               C.byref(opt), _ptr(iters), _ptr(chi2), _ptr(status), _stream_ptr(dev))
    N.check(rc, 'gc_calibrate_di_jones2x2_warm')
    return gains, iters, chi2, status, used, dchi2, start


def calibrate_di_jones2x2_wavefront(vis, model, layout: Layout, n_t, n_fb, lag, net, gains, tol=1e-6, max_iter=1000,
                                    gate_tol=0.0, lead_scale=32.0, max_lead=1, schedule=N.GC_SCHED_STEFCAL,
                                    compute_chi2=False):
    """gc_calibrate_di_jones2x2_wavefront: the whole time-major grid in one iteration loop, waves of
    `lag` times joining with learned starts (net=None: previous solution).  gains: the first wave's
    start on input, the canonical-gauge solutions on return.

    Returns (gains, iters, chi2 or None, status, used, wave_k [n_waves] host int32).
    """
    for t, nm in ((vis, 'vis'), (model, 'model'), (gains, 'gains')):
        _check_tensor(t, nm, False)
        if t.dtype != torch.complex64:
            raise TypeError(f"{nm} must be complex64")
    n = layout.n_intervals
    dev = vis.device
    iters = torch.zeros(n, dtype=torch.int32, device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    used = torch.zeros(n, dtype=torch.int32, device=dev)
    chi2 = torch.zeros(n, dtype=torch.float64, device=dev) if compute_chi2 else None
    n_waves = (int(n_t) + int(lag) - 1) // int(lag)
    wave_k = np.zeros(max(n_waves, 1), np.int32)
    wf = N.GcWavefront(int(n_t), int(n_fb), int(lag), int(max_lead), float(lead_scale), float(gate_tol),
                       C.pointer(net._c) if net is not None else None, used.data_ptr(),
                       wave_k.ctypes.data_as(C.POINTER(C.c_int32)))
    opt = N.GcOptions(float(tol), int(max_iter), int(schedule), N.GC_DTYPE_C64, 0, 1 if compute_chi2 else 0, 0,
                      N.GC_PATH_AUTO)
    lay = layout.c()
    rc = N.lib().gc_calibrate_di_jones2x2_wavefront(_ptr(vis), _ptr(model), C.byref(lay), C.byref(wf), _ptr(gains),
                                                    C.byref(opt), _ptr(iters), _ptr(chi2), _ptr(status),
                                                    _stream_ptr(dev))
    N.check(rc, 'gc_calibrate_di_jones2x2_wavefront')
    return gains, iters, chi2, status, used, wave_k[:n_waves]


def gauge_fix_di(gains, layout: Layout):
    """Canonical gauge in place (gc_gauge_fix_di); gains [n_gain] (scalar) or [n_gain, 2, 2]."""
    _check_tensor(gains, 'gains', False)
    kind = 1 if gains.dim() == 3 else 0
    lay = layout.c()
    N.check(N.lib().gc_gauge_fix_di(kind, _ptr(gains), C.byref(lay), _dtype_code(gains), _stream_ptr(gains.device)),
            'gc_gauge_fix_di')
    return gains


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


def set_wait_limit(tries: int):
    """Polls of the 2x2 accumulate kernel's bounded copy wait on the current device (< 0: default)."""
    N.check(N.lib().gc_set_wait_limit(int(tries)), 'gc_set_wait_limit')
