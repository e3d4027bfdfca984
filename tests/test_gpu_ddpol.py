"""GPU parity of polarized CohJones and polarized AllJones (2x2 direction-dependent gains,
Sect. 4.4) against the FP64 oracle.

The GPU reduces each interval's samples once to the Hermitian Gram matrix of every baseline's
stacked row [D, M^(1) .. M^(Nd)] and forms the per-antenna H (2Nd x 2Nd) and CD from it in FP32
with compensated sums; CohJones solves H X^H = CD^H (FP32 Cholesky, one float-float refinement
step), AllJones takes G^(d) += C^(d) H[d, d]^-1 with C = CD - X H in float-float.  The oracle
builds the same blocks from the raw rows (and, in its pins, from the explicit Jacobian).
Tolerance: max ||dG|| / ||G|| over antenna slots <= 1e-5 (iterates and converged solutions, the
FP32 target); chi^2 within 1e-4 relative.

These methods contract slowly on 2x2 problems (like polarized StefCal, they ignore the
off-diagonal antenna blocks): about 1,000-2,000 iterations to a relative step of 1e-6 on the
small workload, so converged results are compared with the oracle run from the same start to the
same tolerance, whose stopping point the FP32 iterates follow within 1e-5.
"""
import numpy as np
import pytest
import torch

from helpers import device_batch, per_slot_relerr
from oracle import diagonal, gauge
from paper_1502_06974_gb300 import api, synth

pytestmark = pytest.mark.gpu
FN = {'cohjones': api.calibrate_dd_cohjones2x2, 'alljones': api.calibrate_dd_alljones2x2}


def _small(n_dir=4, n_ant=12):
    return synth.make_dd_jones(n_ant=n_ant, n_dir=n_dir, n_t=4, n_chan=8, t_per=2, f_per=8)


@pytest.mark.parametrize("method", ['cohjones', 'alljones'])
@pytest.mark.parametrize("k", [1, 2, 5])
def test_iterates_match(gpu_lib, method, k):
    b = _small()
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = FN[method](vis, model, lay, g0, tol=0.0, max_iter=k)
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=k, method=method)
    assert (iters.cpu().numpy() == k).all()
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


@pytest.mark.parametrize("method,n_dir", [('cohjones', 1), ('cohjones', 3), ('cohjones', 9), ('cohjones', 10),
                                          ('alljones', 2), ('alljones', 9)])
def test_direction_counts_ragged_tile(gpu_lib, method, n_dir):
    """Direction counts from 1 to the maximum 10, on 66 baselines (a ragged last moment tile)."""
    b = _small(n_dir)
    assert b.n_bl[0] % 4 != 0
    vis, model, g0, lay = device_batch(b)
    g, _, _, _ = FN[method](vis, model, lay, g0, tol=0.0, max_iter=3)
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=3, method=method)
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


@pytest.mark.parametrize("method", ['cohjones', 'alljones'])
def test_converged_small_and_chi2(gpu_lib, method):
    b = _small()
    vis, model, g0, lay = device_batch(b)
    g, iters, chi2, st = FN[method](vis, model, lay, g0, tol=1e-6, max_iter=6000, compute_chi2=True)
    st = st.cpu().numpy()
    assert ((st & 15) == 0).all(), st
    gr, its, conv = diagonal.solve_batch(b, tol=1e-6, max_iter=6000, method=method)
    assert conv.all()
    gg = g.cpu().numpy()
    assert gauge.rel_error('dd_jones', gg, gr, b.n_ant, b.gain_off) < 1e-5
    for i in range(b.n_int):
        iv = b.interval(i)
        ref = diagonal.chi2_interval('dd_jones', gg[iv['gain_slice']], iv['vis'], iv['model'], iv['ant1'], iv['ant2'])
        assert abs(float(chi2[i]) - ref) <= 1e-4 * ref


def test_gn_schedule(gpu_lib):
    b = _small()
    vis, model, g0, lay = device_batch(b)
    g, _, _, _ = api.calibrate_dd_cohjones2x2(vis, model, lay, g0, tol=0.0, max_iter=4, schedule='gn')
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=4, schedule='gn')
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


@pytest.mark.parametrize("method", ['cohjones', 'alljones'])
def test_single_direction_matches_di_jones_on_gpu(gpu_lib, method):
    """N_d = 1: both methods are polarized StefCal; the GPU's DD path and its DI path agree."""
    b = synth.make_di_jones(n_ant=20, n_t=2, n_chan=8, t_per=1, f_per=4, n_src=6)
    vis, model, g0, lay = device_batch(b)
    gs, _, _, _ = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=0.0, max_iter=7)
    lay_dd = api.Layout(**{**lay.__dict__, 'n_dir': 1})
    gd, _, _, _ = FN[method](vis, model.reshape(1, -1, 2, 2).contiguous(), lay_dd,
                             g0.clone().reshape(-1, 1, 2, 2).contiguous(), tol=0.0, max_iter=7)
    assert per_slot_relerr(gd.cpu().numpy().reshape(-1, 2, 2), gs.cpu().numpy()) < 1e-5


def test_full_size_sampled_iterates(gpu_lib):
    """The 62-antenna, 9-direction, 12 x 160-sample workload in one call per method: the iterates
    after two steps of a sampled interval match the oracle's."""
    b = synth.make_dd_jones()
    vis, model, g0, lay = device_batch(b)
    iv = b.interval(5)
    for method in ('cohjones', 'alljones'):
        g, iters, _, st = FN[method](vis, model, lay, g0.clone(), tol=0.0, max_iter=2)
        r = diagonal.iterate('dd_jones', b.g0()[iv['gain_slice']], iv['vis'], iv['model'], iv['ant1'], iv['ant2'],
                             iv['n_ant'], tol=0.0, max_iter=2, method=method)
        assert per_slot_relerr(g.cpu().numpy()[iv['gain_slice']], r['g']) < 1e-5


def test_host_buffers(gpu_lib):
    b = _small()
    vis, model, g0, lay = device_batch(b)
    gd, itd, _, _ = api.calibrate_dd_cohjones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=300)
    gh = torch.from_numpy(b.g0()).pin_memory()
    gh, ith, _, _ = api.calibrate_dd_cohjones2x2(vis.cpu().pin_memory(), model.cpu().pin_memory(), lay, gh, tol=1e-6,
                                                 max_iter=300, host_buffers=True)
    assert torch.equal(gd.cpu(), gh) and torch.equal(itd.cpu(), ith)
