"""The C ABI library builds, loads and exports what include/gaincal.h declares (CPU only).

No compute call is made here: only argument validation, which runs on the host before any
CUDA call, and a call that must report a CUDA error code (not crash) when no GPU is visible.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest
import torch

from paper_1502_06974_gb300 import _native as N
from paper_1502_06974_gb300 import build
from paper_1502_06974_gb300 import synth
from paper_1502_06974_gb300.api import Layout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, 'include', 'gaincal.h')


@pytest.fixture(scope='module')
def lib():
    build.build()
    return N.lib()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r'/\*.*?\*/', '', txt, flags=re.S)
    return sorted(set(re.findall(r'\b(gc_[a-z0-9_]+)\s*\(', txt)))


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no declarations parsed"
    out = subprocess.run(['nm', '-D', '--defined-only', N.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r' T (gc_[a-z0-9_]+)', out))
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    assert sorted(N.EXPORTS) == declared


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / 'sz.c'
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gaincal.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gc_layout), sizeof(gc_options),'
                   ' offsetof(gc_layout, n_rows), offsetof(gc_options, reserved), offsetof(gc_layout, n_dir),'
                   ' offsetof(gc_options, lm_after), offsetof(gc_options, lm_lambda0), offsetof(gc_options, lm_K),'
                   ' offsetof(gc_options, weights));'
                   'return 0;}\n')
    exe = tmp_path / 'sz'
    subprocess.run(['gcc', '-I', os.path.join(ROOT, 'include'), str(src), '-o', str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [C.sizeof(N.GcLayout), C.sizeof(N.GcOptions), N.GcLayout.n_rows.offset,
                    N.GcOptions.reserved.offset, N.GcLayout.n_dir.offset, N.GcOptions.lm_after.offset,
                    N.GcOptions.lm_lambda0.offset, N.GcOptions.lm_K.offset, N.GcOptions.weights.offset]


def _call(lib, fn, lay, opt, vis=1, model=1, gains=1):
    p = lambda v: C.c_void_p(v) if v else None
    return getattr(lib, fn)(p(vis), p(model), C.byref(lay), p(gains), C.byref(opt), None, None, None, None)


def _layout():
    b = synth.make_di_scalar(n_ant=5, n_t=2, n_chan=2, t_per=1, f_per=2, dtype=np.complex64)
    return Layout.from_batch(b)


def _opt(**kw):
    o = N.GcOptions(1e-6, 10, 0, 0, 0, 0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("fn", ['gc_calibrate_di_scalar', 'gc_calibrate_di_jones2x2'])
def test_validation_errors_are_return_codes(lib, fn):
    lay = _layout()
    bad = Layout(**lay.__dict__); bad.ant2 = bad.ant2.copy(); bad.ant2[0] = bad.ant1[0]
    keep = [bad]
    assert _call(lib, fn, bad.c(), _opt()) == -3                         # p == q
    bad2 = Layout(**lay.__dict__); bad2.ant1 = bad2.ant1.copy(); bad2.ant1[1] = 9
    keep.append(bad2)
    assert _call(lib, fn, bad2.c(), _opt()) == -3                        # antenna beyond n_ant
    bad3 = Layout(**lay.__dict__); bad3.n_rows = lay.n_rows - 1
    assert _call(lib, fn, bad3.c(), _opt()) == -2                        # rows beyond the buffer
    bad4 = Layout(**lay.__dict__); bad4.gain_off = bad4.gain_off + 1
    assert _call(lib, fn, bad4.c(), _opt()) == -2                        # gains beyond n_gain
    bad5 = Layout(**lay.__dict__); bad5.n_ant = np.full_like(bad5.n_ant, 2000); bad5.n_gain = 4000
    bad5.gain_off = np.array([0, 2000], np.int32)
    assert _call(lib, fn, bad5.c(), _opt()) == -6                        # above GC_MAX_ANT
    good = lay.c()
    assert _call(lib, fn, good, _opt(max_iter=0)) == -1
    assert _call(lib, fn, good, _opt(schedule=5)) == -1
    assert _call(lib, fn, good, _opt(dtype=7)) == -4
    assert _call(lib, fn, good, _opt(), vis=0) == -1
    # Levenberg-Marquardt schedule: options checked, complex64 moment path only, size limit
    assert _call(lib, fn, good, _opt(schedule=2, lm_K=0.5)) == -1
    assert _call(lib, fn, good, _opt(schedule=2, lm_lambda0=-1.0)) == -1
    assert _call(lib, fn, good, _opt(schedule=2, lm_reserved=1)) == -1
    assert _call(lib, fn, good, _opt(schedule=2, dtype=1)) == -4
    assert _call(lib, fn, good, _opt(schedule=2, path=1)) == -1
    big = Layout(**lay.__dict__); big.n_ant = np.full_like(big.n_ant, 300); big.n_gain = 600
    big.gain_off = np.array([0, 300], np.int32)
    assert _call(lib, fn, big.c(), _opt(schedule=2)) == -6               # above GC_LM_MAX_UNKNOWNS
    keep.clear()


def test_no_gpu_reports_cuda_error(lib):
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    lay = _layout()
    vis = np.zeros(lay.n_rows, np.complex64)
    g = np.ones(lay.n_gain, np.complex64)
    rc = lib.gc_calibrate_di_scalar(vis.ctypes.data_as(C.c_void_p), vis.ctypes.data_as(C.c_void_p),
                                    C.byref(lay.c()), g.ctypes.data_as(C.c_void_p), C.byref(_opt()), None, None,
                                    None, None)
    assert rc == -5
    assert lib.gc_last_cuda_error().decode()


def test_empty_batch_is_ok(lib):
    lay = Layout(np.zeros(0, np.int64), *[np.zeros(0, np.int32)] * 5, np.zeros(0, np.int32), np.zeros(0, np.int32),
                 0, 0)
    assert _call(lib, 'gc_calibrate_di_scalar', lay.c(), _opt(), vis=0, model=0, gains=0) == 0


def test_strings(lib):
    assert lib.gc_error_string(-3).decode().startswith('antenna')
    assert lib.gc_status_string(16).decode().startswith('converged')
    assert lib.gc_status_string(3).decode() == 'no data'
    assert lib.gc_launch_count() >= 0
