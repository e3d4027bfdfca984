"""Per-row weights on the GPU (Sect. 2.4, eqs. JHJ:DI:tfw, JHR:DI:tfw) against the weighted FP64
oracle.

Weights are drawn uniform in [0.5, 2] with 10% of the rows flagged (weight 0), the usual use of
W.  Every path that takes them is compared with the oracle's weighted iteration on the same
inputs (iterates after k steps within 1e-5, FP32; 1e-11, FP64), weighted chi^2 within 1e-4, and
the LM schedule with the oracle's weighted least-squares gains; unit weights give bitwise the
unweighted result; the paths that do not take weights refuse them.
"""
import numpy as np
import pytest
import torch

from helpers import device_batch, per_slot_relerr
from oracle import diagonal, gauge, wirtinger
from paper_1502_06974_gb300 import _native as N
from paper_1502_06974_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _weights(b, seed=12, flag=0.1):
    r = synth.rng_for(seed, 31)
    w = r.uniform(0.5, 2.0, b.n_rows)
    w[r.uniform(size=b.n_rows) < flag] = 0.0
    b.weights = w
    return torch.from_numpy(w.astype(np.float32 if b.vis.dtype == np.complex64 else np.float64))


def _fn(b):
    return api.calibrate_di_jones2x2 if b.kind == 'jones' else api.calibrate_di_scalar


CASES = [pytest.param('scalar', N.GC_PATH_MOMENTS, id='scalar-moments'),
         pytest.param('scalar', N.GC_PATH_STREAM, id='scalar-stream'),
         pytest.param('jones', N.GC_PATH_MOMENTS, id='jones-moments'),
         pytest.param('jones', N.GC_PATH_STREAM, id='jones-stream')]


def _batch(kind):
    if kind == 'scalar':
        return synth.make_di_scalar(n_ant=24, n_t=4, n_chan=8, t_per=2, f_per=4, dtype=np.complex64)
    return synth.make_config(2, small=True)


@pytest.mark.parametrize("kind,path", CASES)
@pytest.mark.parametrize("k", [1, 2, 5])
def test_weighted_iterates_match(gpu_lib, kind, path, k):
    b = _batch(kind)
    w = _weights(b).cuda()
    vis, model, g0, lay = device_batch(b)
    g, iters, chi2, st = _fn(b)(vis, model, lay, g0, tol=0.0, max_iter=k, path=path, weights=w, compute_chi2=True)
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=k)
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5
    gg = g.cpu().numpy()
    for i in range(b.n_int):
        iv = b.interval(i)
        ref = diagonal.chi2_interval(b.kind, gg[iv['gain_slice']], iv['vis'], iv['model'], iv['ant1'], iv['ant2'],
                                     iv['weights'])
        assert abs(float(chi2[i]) - ref) <= 1e-4 * ref


def test_weighted_fp64_scalar(gpu_lib):
    b = synth.make_config(1)
    w = _weights(b).cuda()
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_scalar(vis, model, lay, g0, tol=1e-10, max_iter=500, weights=w)
    gr, its, conv = diagonal.solve_batch(b, tol=1e-10, max_iter=500)
    assert conv.all()
    assert gauge.rel_error('scalar', g.cpu().numpy(), gr) < 1e-10


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_weighted_lm_reaches_weighted_least_squares(gpu_lib, kind):
    """StefCal x20 then LM with J^H W J: every interval within 1e-5 of the oracle's weighted
    least-squares gains (App. C LM on the closed-form J^H W J, from the oracle's own start)."""
    b = _batch(kind)
    w = _weights(b).cuda()
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = _fn(b)(vis, model, lay, g0, tol=1e-6, max_iter=400, schedule='lm', weights=w)
    assert ((st.cpu().numpy() & 15) == 0).all()
    gg = g.cpu().numpy()
    for i in range(b.n_int):
        iv = b.interval(i)
        start = b.g0()[iv['gain_slice']].astype(np.complex128)
        r = diagonal.iterate(kind, start, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'], tol=0.0,
                             max_iter=20, weights=iv['weights'])
        prob = wirtinger.ClosedFormProblem(kind, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'],
                                           weights=iv['weights'])
        ref, _, _ = wirtinger.levenberg_marquardt(prob, r['g'], tol=1e-12, max_iter=400, lam0=1e-2, K=10.0, gauge=True)
        assert gauge.rel_error(kind, gg[iv['gain_slice']], ref) < 1e-5, i


@pytest.mark.parametrize("kind,path", CASES)
def test_unit_weights_are_bitwise_unweighted(gpu_lib, kind, path):
    b = _batch(kind)
    vis, model, g0, lay = device_batch(b)
    ones = torch.ones(b.n_rows, dtype=torch.float32, device='cuda')
    g1, it1, _, _ = _fn(b)(vis, model, lay, g0.clone(), tol=1e-6, max_iter=50, path=path)
    g2, it2, _, _ = _fn(b)(vis, model, lay, g0.clone(), tol=1e-6, max_iter=50, path=path, weights=ones)
    assert torch.equal(g1, g2) and torch.equal(it1, it2)


def test_weights_from_host_buffers(gpu_lib):
    b = _batch('jones')
    w = _weights(b)
    vis, model, g0, lay = device_batch(b)
    gd, itd, _, _ = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=60, weights=w.cuda())
    gh = torch.from_numpy(b.g0()).pin_memory()
    gh, ith, _, _ = api.calibrate_di_jones2x2(vis.cpu().pin_memory(), model.cpu().pin_memory(), lay, gh, tol=1e-6,
                                              max_iter=60, host_buffers=True, weights=w.pin_memory())
    assert torch.equal(gd.cpu(), gh) and torch.equal(itd.cpu(), ith)


def test_paths_without_weights_refuse_them(gpu_lib):
    b = _batch('jones')
    w = _weights(b).cuda()
    vis, model, g0, lay = device_batch(b)
    with pytest.raises(RuntimeError, match='GC_ERR_ARG'):
        api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), max_iter=5, path=N.GC_PATH_RESIDENT, weights=w)
    bd = synth.make_config(3, small=True)
    wd = _weights(bd).cuda()
    vd, md, gd0, ld = device_batch(bd)
    opt = N.GcOptions(1e-6, 5, 0, N.GC_DTYPE_C64, 0, 0, 0, 0, 0, 20, 0, 0.0, 0.0, wd.data_ptr())
    import ctypes as C
    lay = ld.c()
    rc = N.lib().gc_calibrate_dd_cohjones(C.c_void_p(vd.data_ptr()), C.c_void_p(md.data_ptr()), C.byref(lay),
                                          C.c_void_p(gd0.data_ptr()), C.byref(opt), None, None, None, None)
    assert rc == N.GC_ERR_ARG
