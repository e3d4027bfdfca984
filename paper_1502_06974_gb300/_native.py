"""ctypes view of ``libgaincal.so`` (the C ABI declared in include/gaincal.h).

Loading fails loudly: there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'libgaincal.so')

GC_OK = 0
GC_ERR = {-1: 'GC_ERR_ARG', -2: 'GC_ERR_LAYOUT', -3: 'GC_ERR_ANTENNA', -4: 'GC_ERR_DTYPE', -5: 'GC_ERR_CUDA',
          -6: 'GC_ERR_LIMIT'}
GC_ERR_ARG, GC_ERR_LIMIT = -1, -6
GC_ST_OK, GC_ST_NOT_CONVERGED, GC_ST_NONFINITE, GC_ST_NODATA, GC_ST_SINGULAR_FLAG = 0, 1, 2, 3, 16
GC_DTYPE_C64, GC_DTYPE_C128 = 0, 1
GC_SCHED_STEFCAL, GC_SCHED_GN, GC_SCHED_LM = 0, 1, 2
GC_LM_MAX_UNKNOWNS, GC_LM_DEFAULT_AFTER, GC_LM_DEFAULT_LAMBDA0, GC_LM_DEFAULT_K = 512, 20, 1e-2, 10.0
GC_PATH_AUTO, GC_PATH_STREAM, GC_PATH_RESIDENT, GC_PATH_MOMENTS = 0, 1, 2, 3
GC_MAX_ANT, GC_MAX_DIR = 1024, 10

# Every symbol include/gaincal.h declares (checked by the CPU test suite).
EXPORTS = [
    'gc_calibrate_di_scalar', 'gc_calibrate_di_jones2x2', 'gc_calibrate_dd_cohjones', 'gc_calibrate_dd_alljones',
    'gc_calibrate_dd_cohjones2x2', 'gc_calibrate_dd_alljones2x2', 'gc_calibrate_di_smooth_scalar',
    'gc_calibrate_di_smooth_jones2x2',
    'gc_jhj_jhr_di_scalar', 'gc_jhj_jhr_di_jones2x2', 'gc_jhj_jhr_di_jones2x2_noalloc',
    'gc_chi2_di_jones2x2', 'gc_mlp_work_floats', 'gc_mlp_forward_f32', 'gc_mlp_grad_f32', 'gc_mlp_train_step',
    'gc_mlp_infer_bf16', 'gc_ws_features_jones', 'gc_ws_target_jones', 'gc_calibrate_di_jones2x2_warm',
    'gc_calibrate_di_jones2x2_wavefront', 'gc_gauge_fix_di',
    'gc_autotune_di', 'gc_profile_last', 'gc_profile_detail', 'gc_profile_lm', 'gc_profile_lm_phases', 'gc_error_string', 'gc_status_string', 'gc_last_cuda_error', 'gc_set_wait_limit', 'gc_rows_gather_f32', 'gc_col_stats_f32',
    'gc_standardize_f32', 'gc_mlp_fold_standardization', 'gc_launch_count', 'gc_release',
]

_p = C.c_void_p
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)


class GcLayout(C.Structure):
    _fields_ = [('n_intervals', C.c_int32), ('row_off', _i64p), ('n_samp', _i32p), ('n_bl', _i32p),
                ('bl_off', _i32p), ('n_ant', _i32p), ('gain_off', _i32p), ('n_bl_table', C.c_int32),
                ('ant1', _i32p), ('ant2', _i32p), ('n_rows', C.c_int64), ('n_gain', C.c_int32),
                ('n_dir', C.c_int32)]


class GcOptions(C.Structure):
    _fields_ = [('tol', C.c_double), ('max_iter', C.c_int32), ('schedule', C.c_int32), ('dtype', C.c_int32),
                ('host_buffers', C.c_int32), ('compute_chi2', C.c_int32), ('profile', C.c_int32),
                ('path', C.c_int32), ('reserved', C.c_int32), ('lm_after', C.c_int32), ('lm_reserved', C.c_int32),
                ('lm_lambda0', C.c_double), ('lm_K', C.c_double), ('weights', C.c_void_p)]


class GcSmooth(C.Structure):
    _fields_ = [('n_t', C.c_int32), ('n_f', C.c_int32), ('n_bl', C.c_int32), ('n_ant', C.c_int32),
                ('ant1', _i32p), ('ant2', _i32p), ('sigma_t', C.c_double), ('sigma_f', C.c_double)]


class GcMlp(C.Structure):
    _fields_ = [('in_', C.c_int32), ('h1', C.c_int32), ('h2', C.c_int32), ('out', C.c_int32),
                ('params', C.c_void_p), ('grads', C.c_void_p), ('adam_m', C.c_void_p), ('adam_v', C.c_void_p),
                ('params_bf16', C.c_void_p)]


class GcWarm(C.Structure):
    _fields_ = [('solutions', C.c_void_p), ('n_solutions', C.c_int64), ('hist_off', _i32p),
                ('lead', C.POINTER(C.c_float)), ('net', C.POINTER(GcMlp)), ('used_out', C.c_void_p),
                ('dchi2_out', C.c_void_p), ('start_out', C.c_void_p)]


class GcWavefront(C.Structure):
    _fields_ = [('n_t', C.c_int32), ('n_fb', C.c_int32), ('lag', C.c_int32), ('max_lead', C.c_int32),
                ('lead_scale', C.c_float),
                ('gate_tol', C.c_double), ('net', C.POINTER(GcMlp)), ('used_out', C.c_void_p),
                ('wave_k_out', _i32p)]


_lib = None


def lib() -> C.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgaincal.so not found at {LIB_PATH}: run paper_1502_06974_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        cal = [_p, _p, C.POINTER(GcLayout), _p, C.POINTER(GcOptions), _p, _p, _p, _p]
        for name in ('gc_calibrate_di_scalar', 'gc_calibrate_di_jones2x2', 'gc_calibrate_dd_cohjones',
                     'gc_calibrate_dd_alljones', 'gc_calibrate_dd_cohjones2x2', 'gc_calibrate_dd_alljones2x2'):
            f = getattr(L, name)
            f.argtypes = cal
            f.restype = C.c_int
        for name in ('gc_jhj_jhr_di_scalar', 'gc_jhj_jhr_di_jones2x2', 'gc_jhj_jhr_di_jones2x2_noalloc'):
            f = getattr(L, name)
            f.argtypes = [_p, _p, C.POINTER(GcLayout), _p, C.c_int32, _p, _p, _p]
            f.restype = C.c_int
        for name in ('gc_calibrate_di_smooth_scalar', 'gc_calibrate_di_smooth_jones2x2'):
            f = getattr(L, name)
            f.argtypes = [_p, _p, C.POINTER(GcSmooth), _p, C.POINTER(GcOptions), _p, _p, _p, _p]
            f.restype = C.c_int
        L.gc_error_string.argtypes = [C.c_int]
        L.gc_error_string.restype = C.c_char_p
        L.gc_status_string.argtypes = [C.c_int]
        L.gc_status_string.restype = C.c_char_p
        L.gc_last_cuda_error.argtypes = []
        L.gc_last_cuda_error.restype = C.c_char_p
        L.gc_rows_gather_f32.argtypes = [_p, C.c_int32, _p, C.c_int64, _p, _p]
        L.gc_rows_gather_f32.restype = C.c_int
        L.gc_col_stats_f32.argtypes = [_p, C.c_int32, _p, C.c_int64, C.c_int32, _p, _p, _p]
        L.gc_col_stats_f32.restype = C.c_int
        L.gc_standardize_f32.argtypes = [_p, C.c_int32, C.c_int64, _p, _p, _p, _p]
        L.gc_standardize_f32.restype = C.c_int
        L.gc_mlp_fold_standardization.argtypes = [C.POINTER(GcMlp), _p, _p, _p, _p]
        L.gc_mlp_fold_standardization.restype = C.c_int
        L.gc_set_wait_limit.argtypes = [C.c_int32]
        L.gc_set_wait_limit.restype = C.c_int
        L.gc_launch_count.argtypes = []
        L.gc_launch_count.restype = C.c_int64
        L.gc_profile_last.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.gc_profile_last.restype = C.c_int
        L.gc_chi2_di_jones2x2.argtypes = [_p, _p, C.POINTER(GcLayout), _p, C.c_int32, _p, _p]
        L.gc_chi2_di_jones2x2.restype = C.c_int
        mlpp = C.POINTER(GcMlp)
        L.gc_mlp_work_floats.argtypes = [mlpp, C.c_int32]
        L.gc_mlp_work_floats.restype = C.c_size_t
        L.gc_mlp_forward_f32.argtypes = [mlpp, _p, C.c_int32, _p, _p, _p]
        L.gc_mlp_forward_f32.restype = C.c_int
        L.gc_mlp_grad_f32.argtypes = [mlpp, _p, _p, C.c_int32, _p, _p, _p, _p]
        L.gc_mlp_grad_f32.restype = C.c_int
        L.gc_mlp_train_step.argtypes = [mlpp, _p, _p, C.c_int32, C.c_float, C.c_int32, _p, _p, _p]
        L.gc_mlp_train_step.restype = C.c_int
        L.gc_mlp_infer_bf16.argtypes = [mlpp, _p, C.c_int32, _p, _p]
        L.gc_mlp_infer_bf16.restype = C.c_int
        L.gc_ws_features_jones.argtypes = [_p, C.c_int32, _p, _p, _p, C.c_int32, C.c_int32, _p, _p, _p]
        L.gc_ws_features_jones.restype = C.c_int
        L.gc_ws_target_jones.argtypes = [_p, _p, _p, C.c_int32, _p, _p]
        L.gc_ws_target_jones.restype = C.c_int
        L.gc_calibrate_di_jones2x2_warm.argtypes = [_p, _p, C.POINTER(GcLayout), C.POINTER(GcWarm), _p,
                                                    C.POINTER(GcOptions), _p, _p, _p, _p]
        L.gc_calibrate_di_jones2x2_warm.restype = C.c_int
        L.gc_calibrate_di_jones2x2_wavefront.argtypes = [_p, _p, C.POINTER(GcLayout), C.POINTER(GcWavefront), _p,
                                                         C.POINTER(GcOptions), _p, _p, _p, _p]
        L.gc_calibrate_di_jones2x2_wavefront.restype = C.c_int
        L.gc_gauge_fix_di.argtypes = [C.c_int32, _p, C.POINTER(GcLayout), C.c_int32, _p]
        L.gc_gauge_fix_di.restype = C.c_int
        L.gc_autotune_di.argtypes = [C.c_int32, _p, _p, C.POINTER(GcLayout), _p, C.c_int32, C.c_int32,
                                     C.POINTER(C.c_double), _p]
        L.gc_autotune_di.restype = C.c_int
        L.gc_profile_detail.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        L.gc_profile_detail.restype = C.c_int
        L.gc_profile_lm.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L.gc_profile_lm.restype = C.c_int
        L.gc_profile_lm_phases.argtypes = [C.POINTER(C.c_double), C.c_int32]
        L.gc_profile_lm_phases.restype = C.c_int
        L.gc_release.argtypes = []
        L.gc_release.restype = C.c_int
        _lib = L
    return _lib


def check(rc: int, what: str) -> int:
    """Raise on a negative return code; return the count of non-converged intervals otherwise."""
    if rc < 0:
        L = lib()
        msg = L.gc_error_string(rc).decode()
        if rc == -5:
            msg += ': ' + L.gc_last_cuda_error().decode()
        raise RuntimeError(f"{what} failed ({GC_ERR.get(rc, rc)}): {msg}")
    return rc
