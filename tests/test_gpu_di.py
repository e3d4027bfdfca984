"""GPU parity of the direction-independent path (scalar and 2x2 StefCal) against the FP64 oracle.

Tolerances.  FP32 path: a per-antenna sum has terms carrying a few roundings each
(eps = 6e-8), summed in chains of <= 16 samples and slot lists of <= ~16 baselines per tile,
then compensated across tiles and items; with no cancellation in J^H J (positive terms) and little
in J^H d, 2e-5 relative per antenna bounds it with margin.  Gains are compared after the global
phase alignment of the gauge (Sect. 2.1), max over antennas of ||dg|| / ||g||, against 1e-5.
FP64 path: 1e-11.
"""
import os

import numpy as np
import pytest
import torch

from helpers import device_batch, oracle_ls, per_slot_relerr
from oracle import blocks, diagonal, gauge, wirtinger
from paper_1502_06974_gb300 import _native as N
from paper_1502_06974_gb300 import api, synth

pytestmark = pytest.mark.gpu
PATHS = [pytest.param(N.GC_PATH_STREAM, id='stream'), pytest.param(N.GC_PATH_MOMENTS, id='moments'),
         pytest.param(N.GC_PATH_RESIDENT, id='resident')]


def _oracle_blocks(b, g):
    outs = []
    for i in range(b.n_int):
        iv = b.interval(i)
        gi = g[iv['gain_slice']]
        if b.kind == 'scalar':
            outs.append(blocks.scalar_blocks(gi, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant']))
        else:
            outs.append(blocks.jones_blocks(gi, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant']))
    return outs


def _random_gains(b, seed=7):
    r = synth.rng_for(seed, 99)
    if b.kind == 'jones':
        return synth.jones_gains(r, b.n_gain, 0.1, 0.05)
    return synth.scalar_gains(r, b.n_gain, 0.1)


@pytest.mark.parametrize("target", [None, 300])
def test_jhj_jhr_scalar_fp64_cfg1(gpu_lib, monkeypatch, target):
    """Accumulation pass, 16 antennas x 40 samples in FP64, single- and multi-item intervals."""
    if target:
        monkeypatch.setenv("GAINCAL_TARGET_ROWS_SCALAR", str(target))
    b = synth.make_config(1)
    vis, model, _, lay = device_batch(b)
    g = _random_gains(b)
    jhd, jhj = api.jhj_jhr_di_scalar(vis, model, lay, torch.from_numpy(g).cuda())
    ref = _oracle_blocks(b, g)[0]
    assert per_slot_relerr(jhd.cpu().numpy(), ref['cd']) < 1e-12
    assert per_slot_relerr(jhj.cpu().numpy(), ref['A']) < 1e-12


@pytest.mark.parametrize("n_ant,n_samp,target", [(40, 20, None), (40, 20, 1000), (5, 3, None), (70, 6, 3000)])
def test_jhj_jhr_scalar_fp32_tiles(gpu_lib, monkeypatch, n_ant, n_samp, target):
    """Several 256-baseline tiles with a ragged tail, and intervals split into several items."""
    if target:
        monkeypatch.setenv("GAINCAL_TARGET_ROWS_SCALAR", str(target))
    b = synth.make_di_scalar(n_ant=n_ant, n_t=n_samp, n_chan=2, t_per=n_samp // 2 or 1, f_per=2,
                             dtype=np.complex64)
    vis, model, _, lay = device_batch(b)
    g = _random_gains(b).astype(np.complex64)
    jhd, jhj = api.jhj_jhr_di_scalar(vis, model, lay, torch.from_numpy(g).cuda())
    ref = _oracle_blocks(b, g.astype(np.complex128))
    cd = np.concatenate([r['cd'] for r in ref]); A = np.concatenate([r['A'] for r in ref])
    assert per_slot_relerr(jhd.cpu().numpy(), cd) < 2e-5
    assert per_slot_relerr(jhj.cpu().numpy(), A) < 2e-5


@pytest.mark.parametrize("target", [None, 500])
def test_jhj_jhr_jones_fp32(gpu_lib, monkeypatch, target):
    if target:
        monkeypatch.setenv("GAINCAL_TARGET_ROWS_JONES", str(target))
    b = synth.make_di_jones(n_ant=30, n_t=2, n_chan=8, t_per=1, f_per=4)   # 435 baselines: 2 tiles, ragged
    vis, model, _, lay = device_batch(b)
    g = _random_gains(b).astype(np.complex64)
    jhd, jhj = api.jhj_jhr_di_jones2x2(vis, model, lay, torch.from_numpy(g).cuda())
    ref = _oracle_blocks(b, g.astype(np.complex128))
    CD = np.concatenate([r['CD'] for r in ref]); H = np.concatenate([r['H'] for r in ref])
    assert per_slot_relerr(jhd.cpu().numpy(), CD) < 2e-5
    assert per_slot_relerr(jhj.cpu().numpy(), H) < 2e-5


def test_jhj_jhr_jones_fp64(gpu_lib):
    b = synth.make_di_jones(n_ant=20, n_t=1, n_chan=4, t_per=1, f_per=4, dtype=np.complex128)
    vis, model, _, lay = device_batch(b)
    g = _random_gains(b)
    jhd, jhj = api.jhj_jhr_di_jones2x2(vis, model, lay, torch.from_numpy(g).cuda())
    ref = _oracle_blocks(b, g)
    assert per_slot_relerr(jhd.cpu().numpy(), ref[0]['CD']) < 1e-12
    assert per_slot_relerr(jhj.cpu().numpy(), ref[0]['H']) < 1e-12


def test_calibrate_scalar_cfg1_fp64(gpu_lib):
    """The FP64 workload (16 antennas, one interval): StefCal to 1e-12 vs oracle GN and the iteration."""
    b = synth.make_config(1)
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_scalar(vis, model, lay, g0, tol=1e-12, max_iter=500)
    torch.cuda.synchronize()
    iv = b.interval(0)
    ref = diagonal.iterate('scalar', b.g0(), iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'], tol=1e-12)
    assert int(st[0]) == 0
    assert abs(int(iters[0]) - ref['iters']) <= 1
    assert gauge.rel_error('scalar', g.cpu().numpy(), ref['g']) < 1e-11
    prob = wirtinger.Problem('scalar', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
    g_gn, _, _ = wirtinger.gauss_newton(prob, b.g0(), tol=1e-14)
    assert gauge.rel_error('scalar', g.cpu().numpy(), g_gn) < 1e-10


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_jones_iterates_match(gpu_lib, k, path):
    """Iterate-level parity: after exactly k steps (GN, average, GN, ...) the gains agree."""
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0, tol=0.0, max_iter=k, path=path)
    gr, its, _ = diagonal.solve_batch(b, tol=0.0, max_iter=k)
    assert (iters.cpu().numpy() == k).all()
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


@pytest.mark.parametrize("path", PATHS)
def test_scalar_iterates_match_fp32(gpu_lib, path):
    b = synth.make_di_scalar(n_ant=24, n_t=6, n_chan=4, t_per=3, f_per=2, dtype=np.complex64)
    vis, model, g0, lay = device_batch(b)
    for k in (1, 2, 5):
        g, iters, _, _ = api.calibrate_di_scalar(vis, model, lay, g0.clone(), tol=0.0, max_iter=k, path=path)
        gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=k)
        assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


@pytest.mark.parametrize("path", PATHS)
def test_jones_converged_small(gpu_lib, path):
    """Run to tol = 1e-6 (the tolerance the throughput measurement uses) and compare."""
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    g, iters, chi2, st = api.calibrate_di_jones2x2(vis, model, lay, g0, tol=1e-6, max_iter=20000, compute_chi2=True,
                                                   path=path)
    gr, its, conv = diagonal.solve_batch(b, tol=1e-6, max_iter=20000)
    assert conv.all() and (st.cpu().numpy() == 0).all()
    e = gauge.rel_error('jones', g.cpu().numpy(), gr, b.n_ant, b.gain_off)
    assert e < 1e-5, e
    it = iters.cpu().numpy()
    assert np.all(np.abs(it - its) <= np.maximum(5, 0.02 * its)), (it, its)
    ch = chi2.cpu().numpy()
    for i in range(b.n_int):
        iv = b.interval(i)
        ref = diagonal.chi2_interval('jones', g.cpu().numpy()[iv['gain_slice']], iv['vis'], iv['model'],
                                     iv['ant1'], iv['ant2'])
        assert abs(ch[i] - ref) <= 1e-4 * ref


@pytest.mark.parametrize("path", PATHS)
def test_scalar_multi_interval_fp32(gpu_lib, monkeypatch, path):
    """Several uneven intervals (different antenna counts and lengths) in one batch, split items."""
    monkeypatch.setenv("GAINCAL_TARGET_ROWS_SCALAR", "700")
    out = synth.make_uneven(n_intervals=12, ant_choices=(4, 9, 23), t_max=5, f_max=6, only='scalar')
    b = out['scalar']
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_scalar(vis, model, lay, g0, tol=1e-7, max_iter=2000, path=path)
    gr, its, conv = diagonal.solve_batch(b, tol=1e-7, max_iter=2000)
    assert (st.cpu().numpy() == 0).all()
    assert gauge.rel_error('scalar', g.cpu().numpy(), gr, b.n_ant, b.gain_off) < 1e-5


@pytest.mark.parametrize("path", PATHS)
def test_host_buffers_match_device(gpu_lib, path):
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    gd, itd, _, _ = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=5000, path=path)
    gh = torch.from_numpy(b.g0()).pin_memory()
    gh, ith, _, _ = api.calibrate_di_jones2x2(vis.cpu().pin_memory(), model.cpu().pin_memory(), lay, gh, tol=1e-6,
                                              max_iter=5000, host_buffers=True, path=path)
    assert torch.equal(gd.cpu(), gh)
    assert torch.equal(itd.cpu(), ith)


@pytest.mark.parametrize("path", PATHS)
def test_bitwise_reproducible(gpu_lib, path):
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    g1, i1, _, _ = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=500, path=path)
    g2, i2, _, _ = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=500, path=path)
    assert torch.equal(g1, g2) and torch.equal(i1, i2)


def test_errors_are_codes(gpu_lib):
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    bad = api.Layout(**{**lay.__dict__})
    bad.ant2 = bad.ant2.copy(); bad.ant2[3] = bad.ant1[3]
    with pytest.raises(RuntimeError, match="GC_ERR_ANTENNA"):
        api.calibrate_di_jones2x2(vis, model, bad, g0, tol=1e-6, max_iter=5)
    bad = api.Layout(**{**lay.__dict__})
    bad.n_rows = lay.n_rows - 1
    with pytest.raises(RuntimeError, match="GC_ERR_LAYOUT"):
        api.calibrate_di_jones2x2(vis, model, bad, g0, tol=1e-6, max_iter=5)


@pytest.mark.parametrize("path", PATHS)
def test_nodata_and_singular(gpu_lib, path):
    """An empty interval reports NODATA; an antenna with no baselines is flagged singular."""
    b = synth.make_di_scalar(n_ant=8, n_t=2, n_chan=2, t_per=1, f_per=2, dtype=np.complex64)
    vis, model, g0, lay = device_batch(b)
    lay.n_samp = lay.n_samp.copy(); lay.n_samp[1] = 0
    lay.n_ant = lay.n_ant.copy(); lay.n_ant[0] = 9           # antenna 8 has no baselines
    lay.gain_off = np.array([0, 9], np.int32); lay.n_gain = 17
    g0 = torch.ones(17, dtype=torch.complex64, device='cuda')
    g, iters, _, st = api.calibrate_di_scalar(vis, model, lay, g0, tol=1e-6, max_iter=200, path=path)
    st = st.cpu().numpy()
    assert st[1] == 3 and int(iters[1]) == 0
    assert st[0] == 0 | 16
    assert complex(g[8].cpu()) == 1.0


@pytest.mark.parametrize("path", PATHS)
def test_jones_full_size_sampled_iterates(gpu_lib, path):
    """The full 64-antenna, 960-interval workload in the bench's launch configuration: 40 iterations on
    the GPU, sampled intervals against the oracle's 40 iterations."""
    b = synth.make_config(2)
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0, tol=0.0, max_iter=40, path=path)
    gg = g.cpu().numpy()
    assert (iters.cpu().numpy() == 40).all()
    for i in (0, 517, 959):
        gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=40, intervals=[i])
        iv = b.interval(i)
        assert per_slot_relerr(gg[iv['gain_slice']], gr) < 1e-5


@pytest.mark.parametrize("cluster", ["1", "2", "8"])
def test_resident_cluster_sizes_agree(gpu_lib, monkeypatch, cluster):
    """The resident kernel split over 1, 2 or 8 CTAs per interval gives the oracle's iterates."""
    monkeypatch.setenv("GAINCAL_CLUSTER", cluster)
    b = synth.make_di_jones(n_ant=24, n_t=3, n_chan=8, t_per=1, f_per=8)
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0, tol=0.0, max_iter=9, path=N.GC_PATH_RESIDENT)
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=9)
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


def test_resident_uneven_jones_batch(gpu_lib):
    """Uneven 2x2 intervals (antenna counts 6..30, 1..12 samples) in one persistent launch."""
    out = synth.make_uneven(n_intervals=24, ant_choices=(6, 13, 30), t_max=3, f_max=4, only='jones')
    b = out['jones']
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0, tol=0.0, max_iter=25, path=N.GC_PATH_RESIDENT)
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=25)
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


@pytest.mark.parametrize("chunks", ["1", "4"])
def test_moments_multi_tile_intervals(gpu_lib, monkeypatch, chunks):
    """Moment path with intervals spanning several 256-baseline tiles (1128 baselines: 5 tiles), with
    the per-antenna slot lists summed in 1 or 4 chunks."""
    monkeypatch.setenv("GAINCAL_RED_CHUNKS", chunks)
    b = synth.make_di_jones(n_ant=48, n_t=2, n_chan=4, t_per=1, f_per=2)
    vis, model, g0, lay = device_batch(b)
    g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0, tol=0.0, max_iter=7, path=N.GC_PATH_MOMENTS)
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=7)
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


@pytest.mark.parametrize("path", [N.GC_PATH_STREAM, N.GC_PATH_MOMENTS])
def test_graph_and_plain_loops_agree(gpu_lib, monkeypatch, path):
    """Graph-captured iteration segments, one launch per iteration, the persistent loop kernel, the
    single-launch iteration and the accumulate variants give bitwise identical results, including a
    max_iter that is not a multiple of the segment length."""
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    out = []
    # (graph, persistent loop): one launch per iteration, graph segments, and (moment path) the
    # persistent cooperative loop kernel with grid barriers between the two phases
    # and (moment path) the accumulate kernel with register prefetch, shared-memory staging or bulk
    # copies into a two-stage ring, and one cooperative launch per iteration (update of k - 1, then
    # accumulate of k) vs two launches
    modes = [("0", "0", "0", "0"), ("1", "0", "0", "0")]
    if path == N.GC_PATH_MOMENTS:
        modes += [("0", "1", "0", "0"), ("1", "0", "1", "0"), ("1", "0", "2", "0"), ("0", "0", "2", "0"),
                  ("1", "0", "3", "0"), ("0", "0", "3", "0"),
                  ("1", "0", "1", "1"), ("0", "0", "1", "1"), ("1", "0", "0", "1")]
    for graph, loop, pf, step1 in modes:
        monkeypatch.setenv("GAINCAL_GRAPH", graph)
        monkeypatch.setenv("GAINCAL_LOOP", loop)
        monkeypatch.setenv("GAINCAL_ACC_PREFETCH", pf)
        monkeypatch.setenv("GAINCAL_STEP1", step1)
        g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=37, path=path)
        out.append((g.cpu(), iters.cpu(), st.cpu()))
    if path == N.GC_PATH_MOMENTS:   # accumulate launches timed alone (profile 2): same results
        for v in ("GAINCAL_GRAPH", "GAINCAL_LOOP", "GAINCAL_ACC_PREFETCH", "GAINCAL_STEP1"):
            monkeypatch.delenv(v)
        g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=37, path=path,
                                                    profile=2)
        out.append((g.cpu(), iters.cpu(), st.cpu()))
        ms, n, _ = api.profile_last()
        assert ms > 0 and n == int(iters.max())
    for o in out[1:]:
        assert torch.equal(out[0][0], o[0]) and torch.equal(out[0][1], o[1]) and torch.equal(out[0][2], o[2])
    assert (out[0][1].numpy() <= 37).all()


def test_bulk_accumulate_with_unaligned_gains(gpu_lib, monkeypatch):
    """The bulk-copy accumulate copies the gains with the tile only when they start on a 16-byte
    boundary; gains 8 bytes off it are read from global memory instead, with identical results."""
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    monkeypatch.setenv("GAINCAL_ACC_PREFETCH", "3")
    ga, ia, _, sa = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=40)
    flat = torch.zeros(g0.numel() + 1, dtype=g0.dtype, device=g0.device)
    gu = flat[1:].view(g0.shape)
    gu.copy_(g0)
    assert gu.data_ptr() % 16 == 8
    gu, iu, _, su = api.calibrate_di_jones2x2(vis, model, lay, gu, tol=1e-6, max_iter=40)
    assert torch.equal(ga, gu) and torch.equal(ia, iu) and torch.equal(sa, su)
    monkeypatch.setenv("GAINCAL_ACC_PREFETCH", "1")
    g1, i1, _, s1 = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=1e-6, max_iter=40)
    assert torch.equal(ga, g1) and torch.equal(ia, i1)


def test_autotune_then_parity(gpu_lib):
    """The autotuner picks a launch shape; gains are restored and the tuned solve keeps parity."""
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    g = g0.clone()
    best = api.autotune_di(vis, model, lay, g, iters=8)
    assert best > 0 and torch.equal(g, g0)
    g, iters, _, st = api.calibrate_di_jones2x2(vis, model, lay, g, tol=0.0, max_iter=6)
    gr, _, _ = diagonal.solve_batch(b, tol=0.0, max_iter=6)
    assert per_slot_relerr(g.cpu().numpy(), gr) < 1e-5


def test_uneven_mixed_batch_autotuned_sampled(gpu_lib):
    """The uneven workload's distribution (antenna counts 16..64, 1-32 times x 1-16 channels, scalar
    and 2x2 mixed) on 512 intervals, autotuned, one batched call per kind, each solved by StefCal
    then Levenberg-Marquardt with the whole J^H J: every interval converges, and the three smallest
    and two median-size intervals of each kind match the oracle's FP64 least-squares gains (from its
    own start) within 1e-5."""
    d = synth.make_uneven(n_intervals=512)
    for kind, fn in (('scalar', api.calibrate_di_scalar), ('jones', api.calibrate_di_jones2x2)):
        b = d[kind]
        vis, model, g0, lay = device_batch(b)
        api.autotune_di(vis, model, lay, g0.clone())
        g, it, _, st = fn(vis, model, lay, g0.clone(), tol=1e-6, max_iter=2000, schedule='lm', lm_K=2.0)
        assert (st.cpu().numpy() == 0).all(), kind
        g = g.cpu().numpy()
        order = np.argsort(b.n_samp.astype(np.int64) * b.n_bl)
        for i in list(order[:3]) + list(order[len(order) // 2:len(order) // 2 + 2]):
            iv = b.interval(int(i))
            ls = oracle_ls(kind, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
            assert gauge.rel_error(kind, g[iv['gain_slice']], ls) < 1e-5, (kind, int(i))
