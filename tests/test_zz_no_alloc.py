"""The allocation-free accumulation pass (gc_jhj_jhr_di_jones2x2_noalloc).

Some callers cannot let a library allocate device memory -- a pipeline that reserved its device
memory at start-up, or an application whose allocator owns the GPU.  For them the library offers
one entry point whose scratch lives in a static device array instead of cudaMalloc'd memory.  These
tests call it through the C ABI and check that it returns what the allocating entry point returns
and what the FP64 oracle's closed-form blocks give (eq. JHJ:pol's diagonal blocks and J^H D, within
the accumulation tolerance of the other GPU tests: 2e-5 relative per antenna for complex64, 1e-12
for complex128), on two calls in a row, with intervals split into several work items so the
scratch partial sums are used, and on a large layout followed by a smaller one of another dtype
on the same stream (the static array's tables, items and scratch re-laid out between calls).

This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from helpers import device_batch, per_slot_relerr
from oracle import blocks
from paper_1502_06974_gb300 import _native as N
from paper_1502_06974_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _noalloc(vis, model, lay, g):
    jhd = torch.full((lay.n_gain, 2, 2), float('nan'), dtype=vis.dtype, device=vis.device)
    jhj = torch.full((lay.n_gain, 2, 2), float('nan'), dtype=vis.dtype, device=vis.device)
    dt = N.GC_DTYPE_C64 if vis.dtype == torch.complex64 else N.GC_DTYPE_C128
    cl = lay.c()
    rc = N.lib().gc_jhj_jhr_di_jones2x2_noalloc(C.c_void_p(vis.data_ptr()), C.c_void_p(model.data_ptr()),
                                                 C.byref(cl), C.c_void_p(g.data_ptr()), dt,
                                                 C.c_void_p(jhd.data_ptr()), C.c_void_p(jhj.data_ptr()),
                                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, jhd, jhj


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_noalloc_matches_allocating_pass(gpu_lib, monkeypatch, dtype):
    monkeypatch.setenv("GAINCAL_TARGET_ROWS_JONES", "500")     # several items per interval: scratch in use
    b = synth.make_di_jones(n_ant=30, n_t=2, n_chan=8, t_per=1, f_per=4, dtype=dtype)
    vis, model, _, lay = device_batch(b)
    r = synth.rng_for(17, 3)
    g = torch.from_numpy(synth.jones_gains(r, b.n_gain, 0.1, 0.05).astype(dtype)).cuda()
    ref_d, ref_j = api.jhj_jhr_di_jones2x2(vis, model, lay, g)
    for _ in range(2):
        rc, jhd, jhj = _noalloc(vis, model, lay, g)
        assert rc == 0, N.lib().gc_last_cuda_error()
        torch.cuda.synchronize()
        assert per_slot_relerr(jhd.cpu().numpy(), ref_d.cpu().numpy()) < 2e-5
        assert per_slot_relerr(jhj.cpu().numpy(), ref_j.cpu().numpy()) < 2e-5


def _oracle(b, g):
    g = np.asarray(g, np.complex128)
    ref = [blocks.jones_blocks(g[iv['gain_slice']], iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
           for iv in (b.interval(i) for i in range(b.n_int))]
    return np.concatenate([r['CD'] for r in ref]), np.concatenate([r['H'] for r in ref])


def test_noalloc_large_then_small_layout_against_oracle(gpu_lib, monkeypatch):
    """A 48-antenna complex64 layout of 8 intervals split into several items, then a 7-antenna
    complex128 layout of 3 intervals in one item each, on one stream: each against the oracle."""
    monkeypatch.setenv("GAINCAL_TARGET_ROWS_JONES", "2000")
    cases = [(synth.make_di_jones(n_ant=48, n_t=4, n_chan=8, t_per=2, f_per=4, dtype=np.complex64), 2e-5),
             (synth.make_di_jones(n_ant=7, n_t=3, n_chan=2, t_per=1, f_per=2, dtype=np.complex128), 1e-12)]
    for n, (b, tol) in enumerate(cases):
        vis, model, _, lay = device_batch(b)
        gh = synth.jones_gains(synth.rng_for(23, n), b.n_gain, 0.1, 0.05).astype(b.vis.dtype)
        rc, jhd, jhj = _noalloc(vis, model, lay, torch.from_numpy(gh).cuda())
        assert rc == 0, N.lib().gc_last_cuda_error()
        torch.cuda.synchronize()
        CD, H = _oracle(b, gh)
        assert per_slot_relerr(jhd.cpu().numpy(), CD) < tol, n
        assert per_slot_relerr(jhj.cpu().numpy(), H) < tol, n


def test_noalloc_rejects_beyond_its_limit(gpu_lib):
    """More distinct baseline tables than the static array is laid out for: a clear error, no launch."""
    n = 65
    a1 = np.zeros(n, np.int32); a2 = np.ones(n, np.int32)
    lay = api.Layout(np.zeros(n, np.int64), np.ones(n, np.int32), np.ones(n, np.int32), np.arange(n),
                     np.full(n, 2, np.int32), np.zeros(n, np.int32), a1, a2, 1, 2)
    vis = torch.zeros((1, 2, 2), dtype=torch.complex64, device='cuda')
    g = torch.zeros((2, 2, 2), dtype=torch.complex64, device='cuda')
    rc, _, _ = _noalloc(vis, vis, lay, g)
    assert rc == N.GC_ERR_LIMIT
