"""Learned warm start: training data from the solver's own solutions, training with the library's
FP32 kernels, and the lag-L wavefront solve with the BF16 network.

Host logic only: index bookkeeping, minibatch order, feature standardisation folded into the
network's first and last layers, and the loop over wavefront blocks.  Every calibration step, the
features, the network's forward/backward/Adam and the inference run in the CUDA library.

Workload shape: a time-major grid of intervals (interval i = t * n_fb + f, n_t times, n_fb
frequency blocks), every interval with the same antennas, baselines and samples.  The network
for interval (t, f) sees the antenna's four most recent solutions of block f that are already
known.  Solving time steps one by one would leave only n_fb intervals per launch, so the solve
runs as a lag-L wavefront: the times [wL, (w+1)L) form one batched launch, all predicted from the
solutions at times wL-1 .. wL-4 with lead t - (wL-1) in 1..L.  The first block starts from unit
gains.  Solutions are put in the canonical gauge (sum_p tr(G_p) real, non-negative) as they are
produced, so that a sequence of them is smooth in time.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native as N
from . import api

LEAD_SCALE = 32.0        # lead (in intervals) is divided by this before it enters the network


@dataclass
class Grid:
    """A time-major grid of identical intervals (see the module docstring)."""
    n_t: int
    n_fb: int
    n_ant: int
    n_samp: int
    ant1: np.ndarray
    ant2: np.ndarray

    @classmethod
    def from_batch(cls, b):
        return cls(int(b.meta['n_t']), int(b.meta['n_fb']), int(b.n_ant[0]), int(b.n_samp[0]), b.ant1, b.ant2)

    @property
    def n_bl(self):
        return int(len(self.ant1))

    @property
    def rows(self):
        return self.n_samp * self.n_bl

    def layout(self, n_int):
        """Layout of n_int consecutive intervals (rows and gains from 0)."""
        return api.Layout(np.arange(n_int, dtype=np.int64) * self.rows, np.full(n_int, self.n_samp),
                          np.full(n_int, self.n_bl), np.zeros(n_int), np.full(n_int, self.n_ant),
                          np.arange(n_int) * self.n_ant, self.ant1, self.ant2, n_int * self.rows,
                          n_int * self.n_ant)


def _identity(n, device):
    g = torch.zeros((n, 2, 2), dtype=torch.complex64, device=device)
    g[:, 0, 0] = 1
    g[:, 1, 1] = 1
    return g


def solve_plain(vis, model, grid: Grid, tol, max_iter, gauge=True, **sched):
    """All intervals in one batched launch from unit gains; returns (gains, iters, status).
    sched: schedule / lm_after / lm_lambda0 / lm_K of calibrate_di_jones2x2."""
    n_int = grid.n_t * grid.n_fb
    lay = grid.layout(n_int)
    g = _identity(n_int * grid.n_ant, vis.device)
    g, it, _, st = api.calibrate_di_jones2x2(vis, model, lay, g, tol=tol, max_iter=max_iter, **sched)
    if gauge:
        api.gauge_fix_di(g, lay)
    return g, it, st


def _hist_index(t_new, f, n_fb):
    """Interval indices [..., 4] of the 4 solutions ending at time t_new (clamped at time 0)."""
    tt = np.maximum(t_new[..., None] - np.arange(4), 0)
    return tt * n_fb + f[..., None]


def training_set(vis, model, grid: Grid, sols, lag, rng, n_samples=None):
    """(x [m, 48], target [m, 8]) float32 device tensors from solved, gauge-fixed intervals.

    For every interval (t, f) with t >= 4 a lead l in 1..min(lag, t-3) is drawn (lag: the largest
    lead the solve will ask for); its history is the solutions at t-l .. t-l-3 and its target the
    solution at t.  The features need C and H at g1 = solution(t-l) on interval t's data: one
    accumulation pass over all intervals.
    """
    n_int = grid.n_t * grid.n_fb
    na = grid.n_ant
    t_all = np.repeat(np.arange(grid.n_t), grid.n_fb)
    f_all = np.tile(np.arange(grid.n_fb), grid.n_t)
    ok = t_all >= 4
    lead = np.ones(n_int, np.int64)
    lead[ok] = rng.integers(1, np.minimum(lag, t_all[ok] - 3) + 1)
    hidx = _hist_index(np.maximum(t_all - lead, 0), f_all, grid.n_fb)          # [n_int, 4]
    dev = vis.device
    rows = (hidx[:, :, None] * na + np.arange(na)[None, None, :])                # [n_int, 4, na]
    rows = np.transpose(rows, (0, 2, 1))                                         # [n_int, na, 4]
    sol8 = torch.view_as_real(sols).reshape(sols.shape[0], 8)
    hist = torch.view_as_complex(api.rows_gather_f32(sol8, rows.reshape(-1)).reshape(n_int * na, 4, 2, 2, 2))
    g1 = torch.view_as_complex(api.rows_gather_f32(sol8, rows[:, :, 0].reshape(-1)).reshape(n_int * na, 2, 2, 2))
    lay = grid.layout(n_int)
    jhd, jhj = api.jhj_jhr_di_jones2x2(vis, model, lay, g1)
    lead_rows = torch.from_numpy(np.repeat(lead.astype(np.float32) / LEAD_SCALE, na)).to(dev)
    x, rot = api.ws_features_jones(hist, jhd, jhj, lead_rows)
    tgt = api.ws_target_jones(g1, sols, rot)
    keep = np.nonzero(np.repeat(ok, na))[0]
    if n_samples is not None and n_samples < keep.size:
        keep = np.sort(rng.choice(keep, n_samples, replace=False))
    return api.rows_gather_f32(x, keep), api.rows_gather_f32(tgt, keep)


def he_init(dims, rng):
    i, h1, h2, o = dims
    return np.concatenate([rng.normal(0.0, np.sqrt(2.0 / i), i * h1), np.zeros(h1),
                           rng.normal(0.0, np.sqrt(2.0 / h1), h1 * h2), np.zeros(h2),
                           rng.normal(0.0, np.sqrt(2.0 / h2), h2 * o), np.zeros(o)]).astype(np.float32)


@dataclass
class TrainResult:
    net: api.Mlp
    losses: list = field(default_factory=list)
    val_mse: float = float('nan')        # held-out MSE of the network's delta
    val_mse_zero: float = float('nan')   # held-out MSE of delta = 0 (the previous-solution start)
    seconds: float = 0.0
    steps: int = 0


def train(x, t, epochs=40, batch=1024, lr=1e-3, seed=0, val_frac=0.1, dims=api.MLP_DIMS):
    """Adam on mean((y - t)^2) with standardised inputs and targets; returns a TrainResult whose
    network takes raw features and predicts raw deltas (the standardisation is folded in)."""
    rng = np.random.default_rng(seed)
    m = x.shape[0]
    perm = rng.permutation(m)
    n_val = max(1, int(m * val_frac))
    dev = x.device
    x, t = x.contiguous(), t.contiguous()
    tr = perm[n_val:]
    tr_t = torch.from_numpy(np.ascontiguousarray(tr, np.int64)).to(dev)
    mu, sd = api.col_stats_f32(x, tr_t, zero_const_mean=True)
    _, tsd = api.col_stats_f32(t, tr_t, zero_const_mean=False)
    xs = api.standardize_f32(x, mu, sd)
    ts = api.standardize_f32(t, None, tsd)
    net = api.Mlp(he_init(dims, rng), dev, dims)
    res = TrainResult(net)
    work = net.work(batch)
    n_tr = tr.size
    nb = max(0, (n_tr - batch) // batch + 1)
    losses = torch.zeros((epochs, max(nb, 1)), dtype=torch.float32, device=dev)   # one slot per step
    xb = torch.empty((batch, x.shape[1]), dtype=torch.float32, device=dev)
    tb = torch.empty((batch, t.shape[1]), dtype=torch.float32, device=dev)
    L = N.lib()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = torch.from_numpy(np.ascontiguousarray(tr[rng.permutation(n_tr)], np.int64)).to(dev)
        st = api._stream_ptr(dev)
        for j in range(nb):
            idx = order[j * batch:(j + 1) * batch]
            N.check(L.gc_rows_gather_f32(api._ptr(xs), xs.shape[1], api._ptr(idx), batch, api._ptr(xb), st),
                    'gc_rows_gather_f32')
            N.check(L.gc_rows_gather_f32(api._ptr(ts), ts.shape[1], api._ptr(idx), batch, api._ptr(tb), st),
                    'gc_rows_gather_f32')
            api.mlp_train_step(net, xb, tb, lr, work=work, loss=losses[ep, j:j + 1])
        res.steps += nb
    torch.cuda.synchronize(dev)
    res.seconds = time.perf_counter() - t0
    lh = losses.cpu().numpy().astype(np.float64)
    res.losses = [float(lh[ep, :nb].mean()) if nb else 0.0 for ep in range(epochs)]
    api.mlp_fold_standardization(net, mu, sd, tsd)
    vidx = perm[:n_val]
    yv = api.mlp_forward_f32(net, api.rows_gather_f32(x, vidx)).cpu().numpy().astype(np.float64)
    tv = api.rows_gather_f32(t, vidx).cpu().numpy().astype(np.float64)
    res.val_mse = float(np.mean((yv - tv) ** 2))
    res.val_mse_zero = float(np.mean(tv ** 2))
    return res


@dataclass
class WavefrontResult:
    gains: torch.Tensor
    iters: np.ndarray
    status: np.ndarray
    used: np.ndarray
    seconds: float
    launches: int


def solve_pipelined(vis, model, grid: Grid, lag, net, tol, max_iter, gate_tol=0.0, max_lead=1):
    """The whole grid in one library call: waves of `lag` times join the running iteration as soon
    as a history of 4 finished times lies within `max_lead` steps before them
    (gc_calibrate_di_jones2x2_wavefront)."""
    n_int = grid.n_t * grid.n_fb
    dev = vis.device
    g = _identity(n_int * grid.n_ant, dev)
    launches0 = api.launch_count()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    g, it, _, st, used, wave_k = api.calibrate_di_jones2x2_wavefront(vis, model, grid.layout(n_int), grid.n_t,
                                                                     grid.n_fb, lag, net, g, tol=tol,
                                                                     max_iter=max_iter, gate_tol=gate_tol,
                                                                     lead_scale=LEAD_SCALE, max_lead=max_lead)
    torch.cuda.synchronize(dev)
    sec = time.perf_counter() - t0
    r = WavefrontResult(g, it.cpu().numpy(), st.cpu().numpy(), used.cpu().numpy(), sec,
                        api.launch_count() - launches0)
    r.wave_k = wave_k
    return r


def solve_wavefront(vis, model, grid: Grid, lag, net, tol, max_iter, first=None, **sched):
    """Solve the grid block by block (lag-L wavefront, one library call per wave, each wave waiting
    for the previous one to finish); net=None starts from the previous solution.  sched: schedule /
    lm_after / lm_lambda0 / lm_K of the warm-started waves; first: the same for the first wave (which
    starts from unit gains; default: sched)."""
    first = sched if first is None else first
    n_int = grid.n_t * grid.n_fb
    na = grid.n_ant
    dev = vis.device
    sols = torch.empty((n_int * na, 2, 2), dtype=torch.complex64, device=dev)
    iters = np.zeros(n_int, np.int32)
    status = np.zeros(n_int, np.int32)
    used = np.zeros(n_int, np.int32)
    blk = lag * grid.n_fb
    gbuf = _identity(blk * na, dev)
    lay_full = grid.layout(blk)
    launches0 = api.launch_count()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for t0_blk in range(0, grid.n_t, lag):
        nt = min(lag, grid.n_t - t0_blk)
        nb = nt * grid.n_fb
        i0 = t0_blk * grid.n_fb
        lay = lay_full if nb == blk else grid.layout(nb)
        r0, r1 = i0 * grid.rows, (i0 + nb) * grid.rows
        g = gbuf[:nb * na]
        v, m = vis[r0:r1], model[r0:r1]
        if t0_blk == 0:
            g.copy_(_identity(nb * na, dev))
            _, it, _, st = api.calibrate_di_jones2x2(v, m, lay, g, tol=tol, max_iter=max_iter, **first)
            us = None
        else:
            tp = t0_blk - 1
            t_all = np.repeat(np.arange(t0_blk, t0_blk + nt), grid.n_fb)
            f_all = np.tile(np.arange(grid.n_fb), nt)
            hoff = (_hist_index(np.full(nb, tp), f_all, grid.n_fb) * na).astype(np.int32)
            lead = ((t_all - tp) / LEAD_SCALE).astype(np.float32)
            _, it, _, st, us, _, _ = api.calibrate_di_jones2x2_warm(v, m, lay, sols, hoff, lead, net, g, tol=tol,
                                                                     max_iter=max_iter, **sched)
        api.gauge_fix_di(g, lay)
        sols[i0 * na:(i0 + nb) * na].copy_(g)
        iters[i0:i0 + nb] = it.cpu().numpy()
        status[i0:i0 + nb] = st.cpu().numpy()
        if us is not None:
            used[i0:i0 + nb] = us.cpu().numpy()
    torch.cuda.synchronize(dev)
    return WavefrontResult(sols, iters, status, used, time.perf_counter() - t0, api.launch_count() - launches0)
