"""GPU parity of the learned warm start (network kernels, features, start selection, gauge) against
the FP64 oracle, and what the trained network gains over starting without it.

Tolerances.  FP32 network kernels: each output is a sum of <= 256 products per layer (or, for
weight gradients, of n rows) in FP32, so 1e-5 of the largest magnitude bounds the rounding with
margin.  BF16 inference: weights and activations carry a relative rounding of 2^-9 each, three
layers deep, so outputs agree with the FP64 forward to a few parts in 1e3 of their scale: 2e-2
of the RMS output is asserted.  chi^2 differences from the moments: sums of FP32 terms whose size
is set by sum |d|^2, hence an absolute bound of 1e-5 * sum |d|^2.
"""
import numpy as np
import pytest
import torch

from helpers import device_batch, oracle_ls, per_slot_relerr
from oracle import diagonal, gauge, mlp, warm
from paper_1502_06974_gb300 import api, synth, warmstart

pytestmark = pytest.mark.gpu
DIMS = api.MLP_DIMS


def _params(seed=0, out_scale=1.0):
    p = mlp.init_params(DIMS, np.random.default_rng(seed))
    i, h1, h2, o = DIMS
    o3 = i * h1 + h1 + h1 * h2 + h2
    p[o3:] *= out_scale
    p[i * h1:i * h1 + h1] = 0.05                 # small positive biases keep most units active
    return p.astype(np.float32)


def _xt(n=300, seed=1):
    r = np.random.default_rng(seed)
    return r.normal(size=(n, DIMS[0])).astype(np.float32), r.normal(size=(n, DIMS[3])).astype(np.float32)


# ------------------------------------------------------------------------------------ network kernels

def test_mlp_forward_and_gradient_match_oracle(gpu_lib):
    p = _params()
    x, t = _xt()
    net = api.Mlp(p, 'cuda')
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = api.mlp_forward_f32(net, xd).cpu().numpy()
    _, _, yr = mlp.forward(p, DIMS, x)
    assert np.max(np.abs(y - yr)) <= 1e-5 * np.max(np.abs(yr))
    g, loss = api.mlp_grad_f32(net, xd, td)
    lr_, gr = mlp.loss_and_grad(p, DIMS, x, t)
    assert abs(float(loss.item()) - lr_) <= 1e-5 * lr_
    g = g.cpu().numpy()
    # per parameter block, relative to the block's largest entry
    i, h1, h2, o = DIMS
    bounds = np.cumsum([0, i * h1, h1, h1 * h2, h2, h2 * o, o])
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert np.max(np.abs(g[a:b] - gr[a:b])) <= 1e-5 * max(np.max(np.abs(gr[a:b])), 1e-30), (a, b)


def test_adam_steps_match_oracle(gpu_lib):
    p = _params(2)
    x, t = _xt(256, 3)
    net = api.Mlp(p, 'cuda')
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    pr, m, v = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    g_first = None
    for step in range(1, 4):
        api.mlp_train_step(net, xd, td, 1e-3)
        _, gr = mlp.loss_and_grad(pr, DIMS, x, t)
        g_first = gr if g_first is None else g_first
        pr, m, v = mlp.adam_step(pr, gr, m, v, step, 1e-3)
    # three steps of about lr each (|m_hat| / sqrt(v_hat) stays near 1 while gradients keep their
    # sign): compare the displacement, not the parameters.  Adam divides by |g|, so entries whose
    # gradient is at FP32 rounding level may move either way: those are only held to the step size.
    d_gpu = net.params.cpu().numpy().astype(np.float64) - p
    d_ref = pr - p
    assert np.max(np.abs(d_gpu)) <= 3e-3 * 1.05
    big = np.abs(g_first) >= 1e-3 * np.max(np.abs(g_first))
    assert big.mean() > 0.5
    assert np.max(np.abs(d_gpu - d_ref)[big]) <= 1e-2 * 3e-3


def test_training_reduces_the_loss(gpu_lib):
    """A learnable target (a fixed random linear map of the input): 300 Adam steps cut the MSE 10x."""
    r = np.random.default_rng(4)
    x = r.normal(size=(4096, DIMS[0])).astype(np.float32)
    A = r.normal(size=(DIMS[0], DIMS[3])) / np.sqrt(DIMS[0])
    t = (x @ A).astype(np.float32)
    net = api.Mlp(_params(5, 0.1), 'cuda')
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = float(api.mlp_grad_f32(net, xd, td)[1].item())
    for _ in range(300):
        idx = torch.from_numpy(r.integers(0, 4096, 512)).cuda()
        api.mlp_train_step(net, xd[idx].contiguous(), td[idx].contiguous(), 1e-3)
    last = float(api.mlp_grad_f32(net, xd, td)[1].item())
    assert last < 0.1 * first, (first, last)


def test_bf16_inference_matches_oracle(gpu_lib):
    """Against the oracle's bfloat16 forward pass (same roundings; the kernel's FP32 sums can move a
    hidden activation across a bfloat16 rounding boundary now and then): 1e-3 of the RMS output.
    Against FP64: the bfloat16 rounding itself, 2e-2 of the RMS output."""
    p = _params(6)
    x, _ = _xt(1000, 7)                      # several row tiles and a ragged tail (1000 = 62 * 16 + 8)
    net = api.Mlp(p, 'cuda')
    y16 = api.mlp_infer_bf16(net, torch.from_numpy(x).cuda()).cpu().numpy()
    _, _, yr = mlp.forward(p, DIMS, x)
    ye = mlp.forward_bf16(p, DIMS, x)
    rms = np.sqrt(np.mean(yr ** 2))
    assert np.sqrt(np.mean((y16 - ye) ** 2)) <= 1e-3 * rms, np.sqrt(np.mean((y16 - ye) ** 2)) / rms
    assert np.max(np.abs(y16 - ye)) <= 1e-2 * rms
    assert np.sqrt(np.mean((y16 - yr) ** 2)) <= 2e-2 * rms


def test_mlp_rejects_other_shapes_and_empty_is_noop(gpu_lib):
    from paper_1502_06974_gb300 import _native as N
    net = api.Mlp(_params(), 'cuda')
    net._c.h1 = 128
    with pytest.raises(RuntimeError, match='GC_ERR_LIMIT'):
        api.mlp_infer_bf16(net, torch.zeros((4, 48), device='cuda'))
    net._c.h1 = 256
    assert api.mlp_infer_bf16(net, torch.zeros((0, 48), device='cuda')).shape == (0, 8)


# ------------------------------------------------------------------------------------ features, targets, gauge

def _solved_grid(seed=synth.SEED, tol=1e-6):
    b = synth.make_config(5, seed=seed, small=True)
    vis, model, _, lay = device_batch(b)
    grid = warmstart.Grid.from_batch(b)
    g, it, st = warmstart.solve_plain(vis, model, grid, tol, 20000, gauge=False)
    assert (st.cpu().numpy() == 0).all()
    return b, vis, model, lay, grid, g


def test_gauge_fix_matches_oracle(gpu_lib):
    b, vis, model, lay, grid, g = _solved_grid()
    raw = g.cpu().numpy()
    api.gauge_fix_di(g, lay)
    fixed = g.cpu().numpy()
    for i in range(b.n_int):
        sl = b.interval(i)['gain_slice']
        ref = warm.canonical_gauge(raw[sl])
        assert np.max(np.abs(fixed[sl] - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_features_and_targets_match_oracle(gpu_lib):
    b, vis, model, lay, grid, g = _solved_grid()
    api.gauge_fix_di(g, lay)
    sol = g.cpu().numpy().astype(np.complex128)
    na = grid.n_ant
    # history for interval (t, f) from times t-2 .. t-5 (lead 2); interval rows as the library lays them out
    t_all = np.repeat(np.arange(grid.n_t), grid.n_fb)
    f_all = np.tile(np.arange(grid.n_fb), grid.n_t)
    hidx = np.maximum(t_all[:, None] - 2 - np.arange(4), 0) * grid.n_fb + f_all[:, None]
    hist = np.stack([sol.reshape(b.n_int, na, 2, 2)[hidx[:, j]] for j in range(4)], axis=2).reshape(-1, 4, 2, 2)
    g1 = np.ascontiguousarray(hist[:, 0])
    lead = np.full(b.n_gain, 2.0 / 32, np.float32)
    hd = torch.from_numpy(hist.astype(np.complex64)).cuda()
    g1d = torch.from_numpy(g1.astype(np.complex64)).cuda()
    jhd, jhj = api.jhj_jhr_di_jones2x2(vis, model, lay, g1d)
    x, rot = api.ws_features_jones(hd, jhd, jhj, torch.from_numpy(lead).cuda())
    tgt = api.ws_target_jones(g1d, g, rot)
    x, rot, tgt = x.cpu().numpy(), rot.cpu().numpy(), tgt.cpu().numpy()
    for i in range(0, b.n_int, 7):
        iv = b.interval(i)
        sl = iv['gain_slice']
        gn, ok = warm.gn_gains(g1[sl], iv['vis'], iv['model'], iv['ant1'], iv['ant2'], na)
        xr, rr = warm.features(hist[sl], gn, ok, lead[sl])
        assert np.max(np.abs(x[sl] - xr)) <= 2e-5 * max(1.0, np.max(np.abs(xr))), i
        np.testing.assert_allclose(rot[sl, 0] + 1j * rot[sl, 1], rr, atol=1e-6)
        tr = warm.target(g1[sl], sol[sl], rr)
        assert np.max(np.abs(tgt[sl] - tr)) <= 1e-6


# ------------------------------------------------------------------------------------ warm-started solve

@pytest.mark.parametrize("with_net", [False, True])
def test_warm_solve_matches_oracle(gpu_lib, with_net):
    b, vis, model, lay, grid, g = _solved_grid()
    api.gauge_fix_di(g, lay)
    sol = g.cpu().numpy().astype(np.complex128)
    na = grid.n_ant
    t0, nt = 8, 8
    nb = nt * grid.n_fb
    i0 = t0 * grid.n_fb
    sub = b.subset(np.arange(i0, i0 + nb))
    v, m, _, slay = device_batch(sub)
    tp = t0 - 1
    f_all = np.tile(np.arange(grid.n_fb), nt)
    t_all = np.repeat(np.arange(t0, t0 + nt), grid.n_fb)
    hoff = ((np.maximum(tp - np.arange(4), 0)[None, :] * grid.n_fb + f_all[:, None]) * na).astype(np.int32)
    lead = ((t_all - tp) / 32.0).astype(np.float32)
    p = _params(9, 0.02)
    net = api.Mlp(p, 'cuda') if with_net else None
    gw = torch.zeros((sub.n_gain, 2, 2), dtype=torch.complex64, device='cuda')
    gw, it, _, st, used, dchi2, start = api.calibrate_di_jones2x2_warm(v, m, slay, g, hoff, lead, net, gw, tol=1e-6,
                                                                       max_iter=20000, want_start=True)
    st, used, dchi2, start = st.cpu().numpy(), used.cpu().numpy(), dchi2.cpu().numpy(), start.cpu().numpy()
    assert (st == 0).all()
    decided = 0
    for j in range(nb):
        iv = sub.interval(j)
        sl = iv['gain_slice']
        g1 = sol[(hoff[j, 0] // na) * na:(hoff[j, 0] // na) * na + na]
        if not with_net:
            assert used[j] == 0 and dchi2[j] == 0
            assert np.array_equal(start[sl], g1.astype(np.complex64))
            continue
        hist = np.stack([sol[hoff[j, k]:hoff[j, k] + na] for k in range(4)], axis=1)
        gn, ok = warm.gn_gains(g1, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], na)
        x, rot = warm.features(hist, gn, ok, np.full(na, lead[j]))
        delta = mlp.forward_bf16(p, DIMS, x)
        prop = warm.propose(g1, delta, rot)
        _, used_ref, dc_ref = warm.select(iv, g1, prop)
        d2 = float(np.sum(np.abs(iv['vis']) ** 2))
        if used[j]:
            assert np.max(np.abs(start[sl] - prop)) <= 1e-2 * np.max(np.abs(delta)) + 2e-6, \
                (j, np.max(np.abs(start[sl] - prop)), np.max(np.abs(delta)))
            dc_at = diagonal.chi2_interval('jones', start[sl], iv['vis'], iv['model'], iv['ant1'], iv['ant2']) - \
                diagonal.chi2_interval('jones', g1, iv['vis'], iv['model'], iv['ant1'], iv['ant2'])
            assert abs(dchi2[j] - dc_at) <= 1e-5 * d2, (j, dchi2[j], dc_at)
        else:
            assert np.array_equal(start[sl], g1.astype(np.complex64))
            assert dchi2[j] >= 0
        if abs(dc_ref) > 2e-5 * d2:                  # clear cases (beyond FP32 chi^2 error) decide the same way
            assert bool(used[j]) == used_ref, (j, dc_ref, dchi2[j])
            decided += 1
    if with_net:
        assert decided >= 1
    # the iteration from the chosen start converges to the oracle's solution from the same start
    gw = gw.cpu().numpy()
    for j in (0, nb // 2, nb - 1):
        iv = sub.interval(j)
        sl = iv['gain_slice']
        ref = diagonal.iterate('jones', start[sl].astype(np.complex128), iv['vis'], iv['model'], iv['ant1'],
                               iv['ant2'], na, tol=1e-6, max_iter=20000)
        assert ref['converged']
        assert gauge.rel_error('jones', gw[sl], ref['g']) < 1e-5
        assert abs(int(it[j].item()) - ref['iters']) <= max(5, 0.02 * ref['iters'])


def test_warm_rejects_bad_history(gpu_lib):
    b, vis, model, lay, grid, g = _solved_grid()
    sub = b.subset(np.arange(0, 2))
    v, m, _, slay = device_batch(sub)
    gw = torch.zeros((sub.n_gain, 2, 2), dtype=torch.complex64, device='cuda')
    hoff = np.zeros((2, 4), np.int32)
    hoff[1, 2] = g.shape[0] - 1                      # runs past the end of `solutions`
    with pytest.raises(RuntimeError, match='GC_ERR_ARG'):
        api.calibrate_di_jones2x2_warm(v, m, slay, g, hoff, np.zeros(2, np.float32), None, gw)


# ------------------------------------------------------------------------------------ what the network gains

def test_trained_network_beats_previous_solution(gpu_lib):
    """Trained on one seed's solver output, evaluated on another: lower prediction error than the
    previous-solution start, and fewer iterations than the unit start; every solve (Levenberg-
    Marquardt with the whole J^H J, the benchmark's method) reaches the same least-squares gains
    as the oracle's FP64 solution from its own start, within 1e-5 on sampled intervals."""
    kw = dict(n_ant=32, n_t=192, n_chan=32)
    lag, tol = 16, 1e-6
    cold = dict(schedule='lm', lm_after=20, lm_K=2.0)
    warm = dict(schedule='lm', lm_after=0, lm_K=2.0, lm_lambda0=1e-6)
    bt = synth.make_warm(seed=101, **kw)
    vt, mt, _, _ = device_batch(bt)
    grid = warmstart.Grid.from_batch(bt)
    st_sol, _, st = warmstart.solve_plain(vt, mt, grid, tol, 2000, **cold)
    assert (st.cpu().numpy() == 0).all()
    x, t = warmstart.training_set(vt, mt, grid, st_sol, lag, np.random.default_rng(0))
    res = warmstart.train(x, t, epochs=30, batch=512, lr=1e-3)
    assert res.val_mse < 0.5 * res.val_mse_zero, (res.val_mse, res.val_mse_zero)
    be = synth.make_warm(seed=202, **kw)
    ve, me, _, _ = device_batch(be)
    g_plain, it_plain, st_plain = warmstart.solve_plain(ve, me, grid, tol, 2000, **cold)
    prev = warmstart.solve_wavefront(ve, me, grid, lag, None, tol, 2000, first=cold, **warm)
    lrn = warmstart.solve_wavefront(ve, me, grid, lag, res.net, tol, 2000, first=cold, **warm)
    assert (st_plain.cpu().numpy() == 0).all()
    for r in (prev, lrn):
        assert (r.status == 0).all()
    it_plain = it_plain.cpu().numpy()
    later = np.repeat(np.arange(grid.n_t), grid.n_fb) >= lag    # the first block has no history
    assert lrn.iters[later].mean() < 0.5 * it_plain[later].mean()
    assert lrn.used[later].mean() > 0.5
    gp, gl, gv = g_plain.cpu().numpy(), lrn.gains.cpu().numpy(), prev.gains.cpu().numpy()
    for i in (0, be.n_int // 2 + 5, be.n_int - 1):
        iv = be.interval(i)
        ref = oracle_ls('jones', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
        for g in (gp, gl, gv):
            assert gauge.rel_error('jones', g[iv['gain_slice']], ref) < 1e-5, i


# ------------------------------------------------------------------------------------ wavefront solve

@pytest.mark.parametrize("gate_tol,max_lead", [(1e-4, 1), (0.0, 12)])
def test_wavefront_solutions_are_converged_fixed_points(gpu_lib, gate_tol, max_lead):
    """Every interval of the pipelined wavefront (StefCal only) meets StefCal's stopping rule -- the
    FP64 iteration restarted at its solution stops again within a few steps -- and lies within
    StefCal's reach of the FP64 least-squares gains computed by the oracle from its own start: the
    weakly constrained common-unitary direction contracts at ~0.9975 per iteration, so a 1e-6 step
    stops up to ~1e-6 / 0.0025 = 4e-4 from the fixed point (the LM schedule closes that gap; the
    pipelined wavefront runs StefCal only).  Output in the canonical gauge; waves join in order.
    Early starts on unfinished histories (gate_tol) and histories further back (max_lead)."""
    b = synth.make_config(5, small=True)
    vis, model, _, lay = device_batch(b)
    grid = warmstart.Grid.from_batch(b)
    net = api.Mlp(_params(9, 0.02), 'cuda')
    r = warmstart.solve_pipelined(vis, model, grid, 8, net, 1e-6, 20000, gate_tol=gate_tol, max_lead=max_lead)
    assert (r.status == 0).all()
    assert np.all(np.diff(r.wave_k) >= 0) and r.wave_k[0] == 0 and len(r.wave_k) == 6
    g = r.gains.cpu().numpy()
    for i in range(0, b.n_int, 11):
        iv = b.interval(i)
        sl = iv['gain_slice']
        s = np.sum(g[sl, 0, 0] + g[sl, 1, 1])
        assert abs(s.imag) <= 1e-5 * abs(s) and s.real > 0
        # stopping rule: the FP64 iteration restarted at the GPU's solution stops again within a few steps
        step = diagonal.iterate('jones', g[sl].astype(np.complex128), iv['vis'], iv['model'], iv['ant1'],
                                iv['ant2'], iv['n_ant'], tol=1e-6, max_iter=50)
        assert step['converged'], i
        ls = oracle_ls('jones', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
        assert gauge.rel_error('jones', g[sl], ls) < 2e-3, i


def test_wavefront_with_finished_histories_matches_sequential_waves(gpu_lib):
    """gate_tol = 0 waits for finished histories: the same starts (up to the rounding of the gauge
    rotation) as solving wave after wave, so the same iteration counts and solutions."""
    b = synth.make_config(5, small=True)
    vis, model, _, lay = device_batch(b)
    grid = warmstart.Grid.from_batch(b)
    pipe = warmstart.solve_pipelined(vis, model, grid, 8, None, 1e-6, 20000, gate_tol=0.0)
    seq = warmstart.solve_wavefront(vis, model, grid, 8, None, 1e-6, 20000)
    assert (pipe.status == 0).all() and (seq.status == 0).all()
    assert np.all(np.abs(pipe.iters - seq.iters) <= np.maximum(5, 0.02 * seq.iters))
    e = gauge.rel_error('jones', pipe.gains.cpu().numpy(), seq.gains.cpu().numpy(), b.n_ant, b.gain_off)
    assert e < 1e-4, e


def test_full_size_learned_wavefront_sampled(gpu_lib):
    """The 5760-interval GP-gain workload at full size in the configuration the benchmark times
    (waves of 32 times, BF16 network trained on another seed's solutions, Levenberg-Marquardt from
    each start): every interval converges, and sampled intervals match the oracle's FP64
    least-squares gains (from its own start) within 1e-5."""
    cold = dict(schedule='lm', lm_after=20, lm_K=2.0)
    warm = dict(schedule='lm', lm_after=0, lm_K=2.0, lm_lambda0=1e-6)
    bt = synth.make_warm(seed=synth.SEED + 1000, n_t=64)
    vt, mt, _, _ = device_batch(bt)
    gt = warmstart.Grid.from_batch(bt)
    sol_t, _, st_t = warmstart.solve_plain(vt, mt, gt, 1e-6, 2000, **cold)
    assert (st_t.cpu().numpy() == 0).all()
    x, t = warmstart.training_set(vt, mt, gt, sol_t, 32, np.random.default_rng(0), n_samples=20000)
    res = warmstart.train(x, t, epochs=20, batch=1024)
    del vt, mt, sol_t, x, t
    b = synth.make_config(5)
    vis, model, _, lay = device_batch(b)
    grid = warmstart.Grid.from_batch(b)
    r = warmstart.solve_wavefront(vis, model, grid, 32, res.net, 1e-6, 2000, first=cold, **warm)
    assert (r.status == 0).all()
    later = np.repeat(np.arange(grid.n_t), grid.n_fb) >= 32
    assert r.used[later].mean() > 0.5
    g = r.gains.cpu().numpy()
    for i in (0, 1000, 2901, b.n_int - 1):
        iv = b.interval(i)
        ls = oracle_ls('jones', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
        assert gauge.rel_error('jones', g[iv['gain_slice']], ls) < 1e-5, i
