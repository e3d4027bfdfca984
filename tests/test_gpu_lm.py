"""Levenberg-Marquardt with the whole J^H J (GC_SCHED_LM) against the FP64 oracle.

One LM step (App. C, eq. LM with the gauge-fixed damped matrix) is compared with the oracle's
lm_step on the closed-form normal equations of eq. JHJ:pol / eq. JHJ:DI; converged gains are
compared with the oracle's own least-squares solution (App. C LM in FP64 from the oracle's own
start, run to a relative step of 1e-12), never with an oracle run seeded by the GPU's answer.
Tolerance: max ||dG_p|| / ||G_p|| <= 1e-5 after phase alignment (the FP32 path's bar).
"""
import numpy as np
import pytest
import torch

from oracle import diagonal, gauge, wirtinger
from paper_1502_06974_gb300 import api, synth
from paper_1502_06974_gb300 import _native as N
from tests.helpers import device_batch

pytestmark = pytest.mark.gpu
TOL_GAIN = 1e-5


def _oracle_ls(kind, b, i, n_stefcal=20, tol=1e-12):
    """FP64 least-squares gains of interval i: StefCal from the unit start, then App. C LM."""
    iv = b.interval(i)
    g0 = b.g0()[iv['gain_slice']]
    r = diagonal.iterate(kind, g0, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'], tol=0.0,
                         max_iter=n_stefcal)
    prob = wirtinger.ClosedFormProblem(kind, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
    g, it, hist = wirtinger.levenberg_marquardt(prob, r['g'], tol=tol, max_iter=400, lam0=1e-2, K=10.0, gauge=True)
    return g, prob


def _gpu_lm(b, gains0=None, **kw):
    vis, model, g0, lay = device_batch(b)
    g = g0.clone() if gains0 is None else torch.from_numpy(np.ascontiguousarray(gains0)).to(g0.device)
    fn = api.calibrate_di_jones2x2 if b.kind == 'jones' else api.calibrate_di_scalar
    g, it, _, st = fn(vis, model, lay, g, schedule='lm', **kw)
    torch.cuda.synchronize()
    return g.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("lam", [1e-1, 1e-2])
def test_jones_single_lm_step_matches_oracle(gpu_lib, lam):
    """lm_after = 0, max_iter = 1: the GPU takes exactly one LM step from the given gains; the
    oracle takes eq. LM with the same lambda and gauge direction on the closed-form J^H J."""
    b = synth.make_config(2, small=True)
    start = diagonal.solve_batch(b, tol=0.0, max_iter=12)[0].astype(np.complex64)
    g, it, st = _gpu_lm(b, start, tol=0.0, max_iter=1, lm_after=0, lm_lambda0=lam)
    assert np.all(it == 1)
    for i in range(b.n_int):
        iv = b.interval(i)
        s = start[iv['gain_slice']].astype(np.complex128)
        prob = wirtinger.ClosedFormProblem('jones', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
        H, rhs = prob.normal_equations(s)
        z = prob.to_z(s)
        dz = wirtinger.lm_step(H, rhs, lam, wirtinger.gauge_direction(z))[: z.shape[0]]
        trial = prob.from_z(z + dz)
        c0, c1 = prob.chi2(s), prob.chi2(trial)
        assert abs(c1 - c0) > 1e-6 * c0           # the decision is not a close call
        ref = trial if c1 < c0 else s
        err = np.max(np.linalg.norm((g[iv['gain_slice']] - ref).reshape(iv['n_ant'], -1), axis=1)
                     / np.linalg.norm(ref.reshape(iv['n_ant'], -1), axis=1))
        assert err < TOL_GAIN, (i, err)


def test_scalar_single_lm_step_matches_oracle(gpu_lib):
    b = synth.make_di_scalar(n_ant=24, n_t=2, n_chan=4, t_per=1, f_per=4, dtype=np.complex64)
    start = diagonal.solve_batch(b, tol=0.0, max_iter=3)[0].astype(np.complex64)
    lam = 1e-2
    g, it, st = _gpu_lm(b, start, tol=0.0, max_iter=1, lm_after=0, lm_lambda0=lam)
    for i in range(b.n_int):
        iv = b.interval(i)
        s = start[iv['gain_slice']].astype(np.complex128)
        prob = wirtinger.ClosedFormProblem('scalar', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
        H, rhs = prob.normal_equations(s)
        dz = wirtinger.lm_step(H, rhs, lam, wirtinger.gauge_direction(s))[: s.shape[0]]
        c0, c1 = prob.chi2(s), prob.chi2(s + dz)
        ref = s + dz if c1 < c0 else s
        err = np.max(np.abs(g[iv['gain_slice']] - ref) / np.abs(ref))
        assert err < TOL_GAIN, (i, err)


def test_jones_lm_converges_to_oracle_least_squares(gpu_lib):
    """Small 2x2 workload (16 antennas, 4 intervals): every interval converges (status OK) to the
    oracle's FP64 least-squares gains within 1e-5."""
    b = synth.make_config(2, small=True)
    g, it, st = _gpu_lm(b, tol=1e-6, max_iter=400)
    assert np.all((st & 15) == N.GC_ST_OK), st
    for i in range(b.n_int):
        ref, prob = _oracle_ls('jones', b, i)
        iv = b.interval(i)
        err = gauge.rel_error('jones', g[iv['gain_slice']], ref)
        assert err < TOL_GAIN, (i, err, int(it[i]))


def test_scalar_lm_converges_to_oracle_least_squares(gpu_lib):
    b = synth.make_di_scalar(n_ant=32, n_t=4, n_chan=8, t_per=2, f_per=4, dtype=np.complex64)
    g, it, st = _gpu_lm(b, tol=1e-6, max_iter=200)
    assert np.all((st & 15) == N.GC_ST_OK), st
    for i in range(b.n_int):
        ref, _ = _oracle_ls('scalar', b, i)
        iv = b.interval(i)
        assert gauge.rel_error('scalar', g[iv['gain_slice']], ref) < TOL_GAIN


def test_jones_lm_full_size_sampled(gpu_lib):
    """The 64-antenna, 960-interval 2x2 workload at full size, one call: every interval converges;
    three sampled intervals match the oracle's least-squares gains within 1e-5."""
    b = synth.make_config(2)
    g, it, st = _gpu_lm(b, tol=1e-6, max_iter=2000)
    assert np.all((st & 15) == N.GC_ST_OK), np.unique(st, return_counts=True)
    for i in (0, 417, 959):
        iv = b.interval(i)
        ref, _ = _oracle_ls('jones', b, i)
        err = gauge.rel_error('jones', g[iv['gain_slice']], ref)
        assert err < TOL_GAIN, (i, err, int(it[i]))
