#!/usr/bin/env python
"""Throughput of gain calibration to convergence: visibilities calibrated per second.

Workload (the full-Jones direction-independent problem): 64 antennas (2016 baselines), 2x2 Jones,
60 times x 64 channels at 1.0-1.4 GHz, solution intervals of 1 time x 4 channels (960 intervals,
7,741,440 rows of 2x2 complex64), 20 polarized point sources, true Jones = diagonal gains
(amplitude 1 + N(0, 0.1), phase U(-pi, pi)) plus leakage CN(0, 0.02), noise sigma = 0.01,
seed 150206974 (+ rank).  Every interval is solved from identity gains by 20 StefCal iterations
followed by Levenberg-Marquardt with the whole J^H J (App. C, eq. LM), to a relative LM step of
1e-6, which puts every interval within 1e-5 of the FP64 least-squares gains (checked on sampled
intervals against the FP64 oracle run from its own start; reported as max_err_vs_oracle).

One step = reset the gains to identity + one gc_calibrate_di_jones2x2 call over all 960 intervals
(iterations run until every interval has converged).  value = rows calibrated / device time, inputs
resident in HBM (495 MB of vis + model, larger than L2, so no flush is needed).  e2e = the same
call with pinned host buffers, host<->device copies inside the timed region.

Under torchrun each rank solves its own copy of the workload on its own GPU (independent
intervals, no collective on the data path: weak scaling); rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle (the same method in NumPy) on one interval per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOL = 1e-6                  # relative LM step at which an interval stops
LM_K = 2.0                  # App. C damping factor (K = 2, 3, 5, 10 measured; 2 the fastest)
LM_AFTER = 20               # StefCal iterations before the first LM step
TOL_STEFCAL = 1e-6          # the StefCal-only comparison stops at this relative step
MAX_ITER = 20000
SAMPLE_INTERVALS = (0, 480, 959)   # checked against the FP64 oracle's least-squares gains
BYTES_PER_ROW = 64          # vis + model, one 2x2 complex64 each (algorithmic bytes per row)
MOMENT_BYTES = 192          # per baseline: P (4x4 complex64) + R (4x4 float32), written once by the moment pass
N_PATH_STREAM, N_PATH_RESIDENT, N_PATH_MOMENTS = 1, 2, 3
METRIC = "visibilities calibrated/s to convergence at <=1e-5 gain err; learned+batched vs plain"
UNIT = "visibilities/s"
WORKLOAD = ("di_jones2x2: 64 ant (2016 bl), 60 t x 64 ch, intervals 1 t x 4 ch (960), 20 polarized sources; "
            "20 StefCal iterations + Levenberg-Marquardt (whole J^H J) to a relative step of 1e-6")
SCHED = dict(schedule='lm', lm_after=LM_AFTER, lm_K=LM_K)


def _env_rank():
    return int(os.environ.get('RANK', 0)), int(os.environ.get('WORLD_SIZE', 1)), int(os.environ.get('LOCAL_RANK', 0))


def rank_seed(rank: int) -> int:
    """Each rank solves its own copy of the workload, drawn with its own seed."""
    from paper_1502_06974_gb300 import synth
    return synth.SEED + rank


def make_workload(rank: int):
    from paper_1502_06974_gb300 import synth
    return synth.make_di_jones(seed=rank_seed(rank))


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value over all ranks (the slowest rank's time); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix='.csv')
            os.close(fd)
            self.f = open(self.path, 'w')
            self.proc = subprocess.Popen(['nvidia-smi', f'--query-gpu={self.FIELDS}', '--format=csv,noheader,nounits',
                                          '-lms', '200'], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for line in open(self.path):
            p = [x.strip() for x in line.split(',')]
            if len(p) < 9:
                continue
            if gpu_index is not None and p[0] != str(gpu_index):
                continue
            try:
                sm.append(float(p[1])); mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith('active'):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------ CPU oracle
def oracle_solve(b, i, tol=TOL, n_stefcal=LM_AFTER, K=LM_K):
    """The FP64 oracle's solution of interval i from its own unit start: the same schedule (StefCal,
    then App. C LM on the closed-form whole J^H J) in NumPy.  Returns (gains, seconds, cpu/wall)."""
    from oracle import diagonal, wirtinger
    iv = b.interval(i)
    g0 = b.g0()[iv['gain_slice']]
    t0 = time.perf_counter(); c0 = time.process_time()
    r = diagonal.iterate('jones', g0, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'], tol=0.0,
                         max_iter=n_stefcal)
    prob = wirtinger.ClosedFormProblem('jones', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
    g, _, _ = wirtinger.levenberg_marquardt(prob, r['g'], tol=tol, max_iter=400, lam0=1e-2, K=K, gauge=True)
    wall = time.perf_counter() - t0
    return g, wall, (time.process_time() - c0) / max(wall, 1e-9)


def oracle_errors(b, gains, intervals=SAMPLE_INTERVALS, refs=None):
    """max over antennas of ||G_p - G_ref,p|| / ||G_ref,p|| after phase alignment, per sampled
    interval, G_ref the oracle's least-squares gains (tol 1e-12, its own start)."""
    from oracle import gauge
    refs = refs if refs is not None else {i: oracle_solve(b, i, tol=1e-12)[0] for i in intervals}
    out = {}
    for i in intervals:
        iv = b.interval(i)
        out[int(i)] = gauge.rel_error('jones', gains[iv['gain_slice']], refs[i])
    return out, refs


def cpu_openmp_block(seed, n_t=4):
    """The FP64 C++/OpenMP implementation of the same method (oracle/cpu_lm.cpp) on all host cores:
    the workload's first n_t x 16 intervals (drawn identically), one interval per thread."""
    from oracle import cpu
    from paper_1502_06974_gb300 import synth
    b = synth.make_di_jones(seed=seed, n_t=n_t)
    cpu.calibrate_jones_lm(b, intervals=[0], tol=TOL, K=LM_K, lm_after=LM_AFTER)     # load / warm the library
    t0 = time.perf_counter()
    _, iters, status, used = cpu.calibrate_jones_lm(b, tol=TOL, K=LM_K, lm_after=LM_AFTER)
    wall = time.perf_counter() - t0
    return {"value": b.n_rows / wall, "unit": UNIT, "cores": int(used), "kind": "cpp_openmp_fp64",
            "converged": int(np.sum(status == 0)),
            "sample": (f"FP64 C++/OpenMP, the same method (StefCal x{LM_AFTER}, then LM on the whole J^H J, "
                       f"K={LM_K:g}, relative step {TOL:g}), the workload's first {b.n_int} intervals "
                       f"({b.n_rows} rows) on {used} threads: {wall:.2f} s")}


def cpu_baseline_block(b, interval=0):
    g, wall, threads = oracle_solve(b, interval)
    rows = int(b.n_samp[interval]) * int(b.n_bl[interval])
    return {"value": rows / wall, "unit": UNIT, "cores": max(1, int(round(threads))), "kind": "oracle",
            "sample": (f"FP64 NumPy oracle, the same method (StefCal x{LM_AFTER}, then App. C LM on the whole "
                       f"J^H J to a relative step of {TOL:g}) on 1 interval of {rows} rows: {wall:.2f} s")}


# ------------------------------------------------------------------------------------ helpers
def kernel_source_hash(files=('di_kernels.cu', 'resident.cu', 'kinds.cuh', 'common.cuh', 'internal.h')):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, 'paper_1502_06974_gb300', 'csrc', f), 'rb') as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


LM_SOURCES = ('lm.cu', 'kinds.cuh', 'common.cuh', 'internal.h')


def ncu_summary(name, files):
    """A committed ncu summary (json) when it was taken on the current kernel sources; None otherwise."""
    p = os.path.join(ROOT, 'profiles', name)
    try:
        d = json.load(open(p))
    except Exception:
        return None
    return d if d.get('kernel_hash') == kernel_source_hash(files) else None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json'))), "of measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "of fallback"


# ------------------------------------------------------------------------------------ arms
def run_reference(args):
    """The FP64 oracle, as it stands, on the host cores: each step solves one interval of the
    workload with the same method (StefCal, then App. C LM on the whole J^H J, same tolerance).
    The intervals are alike, so visibilities/s of one interval is the rate of the whole job."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from paper_1502_06974_gb300 import synth
    b = synth.make_di_jones(seed=rank_seed(0), n_t=1)   # the workload's first 16 intervals, drawn identically
    samples = []
    rows = threads = None
    for k in range(args.warmup + args.steps):
        i = k % b.n_int
        _, wall, threads = oracle_solve(b, i)
        rows = int(b.n_samp[i]) * int(b.n_bl[i])
        if k >= args.warmup:
            samples.append(wall)
    wall = statistics.median(samples)
    value = rows / wall
    cores = max(1, int(round(threads)))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "rows": 7741440, "intervals": 960, "tol": TOL},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": (f"each step: the FP64 NumPy oracle solves 1 interval ({rows} rows) of the "
                                       f"workload with the same method and tolerance; ms_per_step is that solve")},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


WARM_LAG = 32           # wave length (time steps) of the learned wavefront
WARM_LAMBDA0 = 1e-6     # initial LM damping of the warm-started waves (their start is already close: a
                        # larger value damps the weakly constrained directions for several iterations)
WARM_WORKLOAD = ("di_jones2x2 warm start: 64 ant (2016 bl), 720 t x 64 ch, intervals 1 t x 8 ch (5760), GP gains "
                 "(30 min / 50 MHz correlation, amplitude 0.1, phase 1 rad); Levenberg-Marquardt to a relative "
                 "step of 1e-6 from every start")


def be_interval(be, ve, me, ge, i):
    """Rows of interval i of the GP-gain workload (moved back from the device: the host copy was freed)."""
    r0, r1 = i * ge.rows, (i + 1) * ge.rows
    vis = ve[r0:r1].cpu().numpy().reshape(ge.n_samp, ge.n_bl, 2, 2)
    model = me[r0:r1].cpu().numpy().reshape(ge.n_samp, ge.n_bl, 2, 2)
    return {'vis': vis, 'model': model}


def warm_start_block(dev, args):
    """Learned warm start + batched path vs the plain batched solver on the GP-gain workload, every
    solve to the same tolerance with the same method (LM with the whole J^H J).

    The network is trained first (its own observation, another seed), then the same 5760 intervals
    are solved with the data resident: plain (all intervals from unit gains in one call: StefCal x20,
    then LM); the previous-solution and learned starts in waves of 32 times, one call per wave (the
    first wave as plain, the others LM straight from the start)."""
    import torch
    from paper_1502_06974_gb300 import api, synth, warmstart
    t0 = time.perf_counter()
    bt = synth.make_warm(seed=synth.SEED + 1000, n_t=160)
    vt, mt = torch.from_numpy(bt.vis).to(dev), torch.from_numpy(bt.model).to(dev)
    gt = warmstart.Grid.from_batch(bt)
    sol_t, _, st_t = warmstart.solve_plain(vt, mt, gt, TOL, MAX_ITER, **SCHED)
    x, t = warmstart.training_set(vt, mt, gt, sol_t, WARM_LAG, np.random.default_rng(0), n_samples=50000)
    res = warmstart.train(x, t, epochs=40, batch=1024, lr=1e-3)
    del vt, mt, sol_t, x, t
    prep_s = time.perf_counter() - t0
    be = synth.make_config(5)
    ve, me = torch.from_numpy(be.vis).to(dev), torch.from_numpy(be.model).to(dev)
    del be.vis, be.model
    ge = warmstart.Grid.from_batch(be)
    n_int = ge.n_t * ge.n_fb
    lay = ge.layout(n_int)
    if not args.no_autotune:
        api.autotune_di(ve, me, lay, warmstart._identity(n_int * ge.n_ant, dev), iters=24)
    stream = torch.cuda.current_stream(dev)
    warm_sched = dict(schedule='lm', lm_after=0, lm_K=LM_K, lm_lambda0=WARM_LAMBDA0)

    def timed(fn, reps=3):
        fn()                                   # warm-up (plan, graph capture)
        times = []
        for _ in range(reps):                  # the median of reps calls
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        return out, float(np.median(times))

    (gp, itp, stp), ms_plain = timed(lambda: warmstart.solve_plain(ve, me, ge, TOL, MAX_ITER, **SCHED))
    prev, ms_prev = timed(lambda: warmstart.solve_wavefront(ve, me, ge, WARM_LAG, None, TOL, MAX_ITER, first=SCHED,
                                                            **warm_sched))
    lrn, ms_lrn = timed(lambda: warmstart.solve_wavefront(ve, me, ge, WARM_LAG, res.net, TOL, MAX_ITER, first=SCHED,
                                                          **warm_sched))
    itp = itp.cpu().numpy()
    rows = ge.rows * n_int
    g_true = be.g_true
    # every start must reach the FP64 least-squares gains: sampled intervals against the oracle
    samp = (0, n_int // 2 + 3, n_int - 1)
    refs = {}
    for i in samp:
        from oracle import diagonal, wirtinger
        iv = be_interval(be, ve, me, ge, i)
        r0 = diagonal.iterate('jones', np.tile(np.eye(2, dtype=np.complex128), (ge.n_ant, 1, 1)), iv['vis'],
                              iv['model'], ge.ant1, ge.ant2, ge.n_ant, tol=0.0, max_iter=LM_AFTER)
        prob = wirtinger.ClosedFormProblem('jones', iv['vis'], iv['model'], ge.ant1, ge.ant2, ge.n_ant)
        refs[i] = wirtinger.levenberg_marquardt(prob, r0['g'], tol=1e-12, max_iter=400, lam0=1e-2, K=LM_K,
                                                gauge=True)[0]

    def err_oracle(g):
        from oracle import gauge
        gg = g.cpu().numpy()
        return max(gauge.rel_error('jones', gg[i * ge.n_ant:(i + 1) * ge.n_ant], refs[i]) for i in samp)

    def err_truth(g):
        # max over antennas of ||G e^{i phi} - G_true|| / ||G_true||, phi the least-squares global
        # phase of each interval (solutions are defined up to that phase)
        est = g.cpu().numpy().astype(np.complex128).reshape(n_int, ge.n_ant, 4)
        ref = g_true.reshape(n_int, ge.n_ant, 4)
        ph = np.exp(1j * np.angle(np.sum(ref * np.conj(est), axis=(1, 2))))
        d = np.linalg.norm(est * ph[:, None, None] - ref, axis=2) / np.linalg.norm(ref, axis=2)
        return float(d.max())

    def agree(g, ref):
        # the solutions of two starts must be the same least-squares point: max relative difference
        a = g.cpu().numpy().astype(np.complex128).reshape(n_int, ge.n_ant, 4)
        r = ref.cpu().numpy().astype(np.complex128).reshape(n_int, ge.n_ant, 4)
        ph = np.exp(1j * np.angle(np.sum(r * np.conj(a), axis=(1, 2))))
        return float((np.linalg.norm(a * ph[:, None, None] - r, axis=2) / np.linalg.norm(r, axis=2)).max())

    def entry(ms, iters, status, extra=None):
        d = {"ms": ms, "value": rows / (ms / 1e3), "iters_mean": float(np.mean(iters)),
             "iters_max": int(np.max(iters)), "interval_iterations": int(np.sum(iters)),
             "converged": int(np.sum((status & 15) == 0))}
        d.update(extra or {})
        return d

    return {"workload": WARM_WORKLOAD, "metric": METRIC, "unit": UNIT, "lag": WARM_LAG,
            "schedule": ("plain: one call from unit gains (StefCal x20 then LM); waves: lag x 8 intervals per "
                         "gc_calibrate_di_jones2x2_warm call, predicted from the 4 solutions before the wave, LM "
                         "from the start; every solve to a relative LM step of 1e-6; each time the median of 3 "
                         "calls after a warm-up call"),
            "plain": entry(ms_plain, itp, stp.cpu().numpy(), {"max_err_vs_truth": err_truth(gp),
                                                              "max_err_vs_oracle": err_oracle(gp)}),
            "previous_solution": entry(ms_prev, prev.iters, prev.status, {"max_err_vs_truth": err_truth(prev.gains),
                                                                          "max_err_vs_oracle": err_oracle(prev.gains),
                                                                          "max_diff_vs_plain": agree(prev.gains, gp)}),
            "learned": entry(ms_lrn, lrn.iters, lrn.status,
                             {"proposals_taken": float(np.mean(lrn.used[np.repeat(np.arange(ge.n_t), ge.n_fb)
                                                                       >= WARM_LAG])),
                              "max_err_vs_truth": err_truth(lrn.gains), "max_err_vs_oracle": err_oracle(lrn.gains),
                              "max_diff_vs_plain": agree(lrn.gains, gp)}),
            "oracle_sampled_intervals": list(samp),
            "warm_lambda0": WARM_LAMBDA0,
            "speedup_learned_vs_plain": ms_plain / ms_lrn,
            "speedup_learned_vs_previous_solution": ms_prev / ms_lrn,
            "training": {"trajectories": 50000, "observation": "160 t x 64 ch of the same array, another seed",
                         "adam_steps": res.steps, "train_s": res.seconds, "prep_s": prep_s,
                         "val_mse": res.val_mse, "val_mse_previous_solution": res.val_mse_zero}}


UNEVEN_WORKLOAD = ("uneven: independent intervals, N_ant U{16,24,32,48,64}, 1-32 t x 1-16 ch, scalar or 2x2 "
                   "(Bernoulli 1/2), 5 sources each, sigma 0.01; StefCal x20 then LM to a relative step of 1e-6; "
                   "one call per kind, back to back on one stream")


def oracle_ls_interval(kind, iv, tol=1e-12):
    """The oracle's FP64 least-squares gains of one interval from its own unit start."""
    from oracle import diagonal, wirtinger
    na = iv['n_ant']
    g0 = np.tile(np.eye(2, dtype=np.complex128), (na, 1, 1)) if kind == 'jones' else np.ones(na, np.complex128)
    r = diagonal.iterate(kind, g0, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], na, tol=0.0, max_iter=LM_AFTER)
    prob = wirtinger.ClosedFormProblem(kind, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], na)
    return wirtinger.levenberg_marquardt(prob, r['g'], tol=tol, max_iter=400, lam0=1e-2, K=LM_K, gauge=True)[0]


def uneven_block(dev, args):
    """The uneven batched workload at full size (4096 intervals, ~0.46 G rows, ~18.5 GB of vis + model):
    both kinds to convergence with the LM schedule, sampled intervals against the oracle."""
    import torch
    from oracle import gauge
    from paper_1502_06974_gb300 import api, synth
    t0 = time.perf_counter()
    d = synth.make_uneven(n_intervals=args.uneven_intervals, workers=min(32, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    out = {"workload": UNEVEN_WORKLOAD, "intervals": int(args.uneven_intervals), "metric": METRIC, "unit": UNIT,
           "generation_s": gen_s}
    tot_ms = 0.0
    tot_rows = 0
    errs = []
    for kind, fn in (('scalar', api.calibrate_di_scalar), ('jones', api.calibrate_di_jones2x2)):
        b = d[kind]
        vis = torch.from_numpy(b.vis).to(dev)
        model = torch.from_numpy(b.model).to(dev)
        g0 = torch.from_numpy(b.g0()).to(dev)
        lay = api.Layout.from_batch(b)
        if not args.no_autotune:
            api.autotune_di(vis, model, lay, g0.clone(), iters=24)
        fn(vis, model, lay, g0.clone(), tol=TOL, max_iter=2000, **SCHED)           # warm-up (plans)
        g = g0.clone()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        g, it, _, st = fn(vis, model, lay, g, tol=TOL, max_iter=2000, **SCHED)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        it = it.cpu().numpy(); st = st.cpu().numpy(); gh = g.cpu().numpy()
        order = np.argsort(b.n_samp.astype(np.int64) * b.n_bl)
        samp = [int(order[0]), int(order[len(order) // 2])]
        e = [gauge.rel_error(kind, gh[b.interval(i)['gain_slice']], oracle_ls_interval(kind, b.interval(i)))
             for i in samp]
        errs += e
        out[kind] = {"intervals": b.n_int, "rows": b.n_rows, "ms": ms, "value": b.n_rows / (ms / 1e3),
                     "iters_mean": float(it.mean()), "iters_max": int(it.max()),
                     "converged": int(np.sum((st & 15) == 0)), "oracle_sampled_intervals": samp,
                     "max_err_vs_oracle": max(e)}
        tot_ms += ms
        tot_rows += b.n_rows
        del vis, model, g0, g
        torch.cuda.empty_cache()
    out.update({"rows": tot_rows, "ms": tot_ms, "value": tot_rows / (tot_ms / 1e3), "max_err_vs_oracle": max(errs)})
    return out


DD_WORKLOAD = ("dd_cohjones: 62 ant (1891 bl), 9 directions x 3 sources, 120 t x 16 ch, intervals 10 t x 16 ch "
               "(12), direction gains 1+N(0,0.2) x U(-pi,pi), sigma 0.02, tol 1e-6")


def dd_block(dev, args, peaks, which):
    """The direction-dependent CohJones workload: full calibration time, and the moment pass (vis +
    9 model planes read once per call, 80 B per row; HBM-bound) against the HBM roofline."""
    import torch
    from paper_1502_06974_gb300 import api, synth
    b = synth.make_config(3)
    vis, model = torch.from_numpy(b.vis).to(dev), torch.from_numpy(b.model).to(dev)
    g0 = torch.from_numpy(b.g0()).to(dev)
    lay = api.Layout.from_batch(b)
    stream = torch.cuda.current_stream(dev)
    api.calibrate_dd_cohjones(vis, model, lay, g0.clone(), tol=TOL, max_iter=MAX_ITER)     # warm-up (plan)
    times = []
    for _ in range(5):  # median of five full calibrations
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        g = g0.clone()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        _, it, _, st = api.calibrate_dd_cohjones(vis, model, lay, g, tol=TOL, max_iter=MAX_ITER)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    api.calibrate_dd_cohjones(vis, model, lay, g0.clone(), tol=TOL, max_iter=MAX_ITER, profile=True)
    it_ms, it_n, _ = api.profile_last()
    mom_ms, bl_it, _ = api.profile_detail()
    nd = b.n_dir
    mom_bytes = b.n_rows * (8 + 8 * nd) + int(np.sum(b.n_bl)) * (nd * (nd + 1) // 2 + nd) * 8
    it = it.cpu().numpy()
    return {"workload": DD_WORKLOAD, "metric": METRIC, "unit": UNIT, "rows": b.n_rows,
            "ms": ms, "value": b.n_rows / (ms / 1e3),
            "iters_median": int(np.median(it)), "iters_max": int(it.max()),
            "converged": int(np.sum((st.cpu().numpy() & 15) == 0)),
            "roofline_moment_pass": {"bound": "hbm", "achieved": mom_bytes / (mom_ms / 1e3) / 1e9,
                                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                     "frac": mom_bytes / (mom_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                                     "kernel": "dd_moment_kernel<9>", "ms": mom_ms, "bytes": mom_bytes,
                                     "peak_source": which},
            "iterations": {"launches": it_n, "avg_launch_us": it_ms * 1e3 / max(it_n, 1),
                           "kernel": "dd_iter_kernel<9> (per (interval, antenna): 9x9 block from the moments, "
                                     "FP32 Cholesky in registers + one float-float refinement step; the stop "
                                     "decision deferred to the next launch)",
                           "moments_bytes": int(np.sum(b.n_bl)) * (nd * (nd + 1) // 2 + nd) * 8}}


def fp32_peak(dev, peaks):
    """(TFLOP/s, source): the FP32 FMA issue rate, 128 lanes per SM at the maximum SM clock."""
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12, f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop (FMA) x {mhz:.0f} MHz"


def _median_ms(dev, fn, reps=3):
    """Median over reps of fn() bracketed by CUDA events on the current stream (after one warm-up)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = fn()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    return float(np.median(times)), out


ALLJONES_WORKLOAD = ("dd_alljones: the CohJones geometry (62 ant, 9 directions x 3 sources, 120 t x 16 ch, intervals "
                     "10 t x 16 ch) with source fluxes within 10:1 (log10 S in [-0.5, 0.5]), tol 1e-6")


def alljones_block(dev, args, peaks, which):
    """Scalar AllJones (Sect. 3.2.3) against CohJones on one workload where both converge."""
    import torch
    from paper_1502_06974_gb300 import api, synth
    b = synth.make_dd(log_flux=(-0.5, 0.5))
    vis, model = torch.from_numpy(b.vis).to(dev), torch.from_numpy(b.model).to(dev)
    g0 = torch.from_numpy(b.g0()).to(dev)
    lay = api.Layout.from_batch(b)
    out = {"workload": ALLJONES_WORKLOAD, "metric": METRIC, "unit": UNIT, "rows": b.n_rows}
    for name, fn in (("alljones", api.calibrate_dd_alljones), ("cohjones", api.calibrate_dd_cohjones)):
        ms, (_, it, _, st) = _median_ms(dev, lambda: fn(vis, model, lay, g0.clone(), tol=TOL, max_iter=MAX_ITER))
        it = it.cpu().numpy()
        out[name] = {"ms": ms, "value": b.n_rows / (ms / 1e3), "iters_median": int(np.median(it)),
                     "iters_max": int(it.max()), "converged": int(np.sum((st.cpu().numpy() & 15) == 0))}
    fn = api.calibrate_dd_alljones
    fn(vis, model, lay, g0.clone(), tol=TOL, max_iter=MAX_ITER, profile=True)
    it_ms, it_n, _ = api.profile_last()
    out["alljones"]["avg_iteration_launch_us"] = it_ms * 1e3 / max(it_n, 1)
    return out


DDPOL_WORKLOAD = ("dd_jones2x2: 62 ant (1891 bl), 9 directions x 3 polarized sources (fractional polarization "
                  "0.3-0.7), 120 t x 16 ch, intervals 10 t x 16 ch (12), 2x2 gains per direction, sigma 0.02")
DDPOL_MAX_ITER = 3000


def ddpol_block(dev, args, peaks, which):
    """Polarized CohJones / AllJones (Sect. 4.4): calibration to tol 1e-6 (or the iteration cap: these
    methods contract slowly on 2x2 problems), and the Gram moment pass (vis + 9 model planes, 320 B
    per row read once; 16 complex products per Gram tile and sample: ALU-bound) against both roofs."""
    import torch
    from paper_1502_06974_gb300 import api, synth
    b = synth.make_dd_jones()
    vis, model = torch.from_numpy(b.vis).to(dev), torch.from_numpy(b.model).to(dev)
    g0 = torch.from_numpy(b.g0()).to(dev)
    lay = api.Layout.from_batch(b)
    nd = b.n_dir
    T = nd + 1
    NT = T * (T + 1) // 2
    out = {"workload": DDPOL_WORKLOAD, "metric": METRIC, "unit": UNIT, "rows": b.n_rows, "max_iter": DDPOL_MAX_ITER}
    for name, fn in (("cohjones", api.calibrate_dd_cohjones2x2), ("alljones", api.calibrate_dd_alljones2x2)):
        ms, (_, it, _, st) = _median_ms(dev, lambda: fn(vis, model, lay, g0.clone(), tol=TOL, max_iter=DDPOL_MAX_ITER),
                                        reps=1)
        it = it.cpu().numpy()
        fn(vis, model, lay, g0.clone(), tol=TOL, max_iter=DDPOL_MAX_ITER, profile=True)
        it_ms, it_n, _ = api.profile_last()
        mom_ms, _, _ = api.profile_detail()
        out[name] = {"ms": ms, "value": b.n_rows / (ms / 1e3), "iters_median": int(np.median(it)),
                     "iters_max": int(it.max()), "converged": int(np.sum((st.cpu().numpy() & 15) == 0)),
                     "avg_iteration_launch_us": it_ms * 1e3 / max(it_n, 1), "moment_pass_ms": mom_ms}
    mom_ms = out["cohjones"]["moment_pass_ms"]
    rd = b.n_rows * 32 * (1 + nd)
    wr = int(np.sum(b.n_bl)) * NT * 16 * 8
    flops = b.n_rows * NT * 16 * 8
    peak_tf, src = fp32_peak(dev, peaks)
    out["roofline_moment_pass"] = {
        "bound": "alu", "kernel": f"ddpol_moment_kernel<{nd}> (Hermitian Gram of [D, M^(1)..M^(9)] per baseline)",
        "achieved": flops / (mom_ms / 1e3) / 1e12, "unit": "TFLOP/s", "peak": peak_tf,
        "frac": flops / (mom_ms / 1e3) / 1e12 / peak_tf, "flop": flops, "peak_source": src,
        "hbm": {"bytes": rd + wr, "achieved": (rd + wr) / (mom_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                "frac": (rd + wr) / (mom_ms / 1e3) / 1e9 / peaks["hbm_gbs"], "peak_source": which}}
    return out


WEIGHTS_WORKLOAD = ("the headline 2x2 workload with per-row weights U(0.5, 2) and 10% of the rows flagged (weight 0); "
                    "StefCal x20 then LM on J^H W J to a relative step of 1e-6")


def weights_block(dev, args, b, vis, model, lay, g0):
    """Per-row weights (Sect. 2.4) on the headline workload: time, and the error against the oracle's
    weighted least-squares gains on a sampled interval."""
    import torch
    from oracle import diagonal, gauge, wirtinger
    from paper_1502_06974_gb300 import api, synth
    r = synth.rng_for(12, 31)
    w = r.uniform(0.5, 2.0, b.n_rows)
    w[r.uniform(size=b.n_rows) < 0.1] = 0.0
    wd = torch.from_numpy(w.astype(np.float32)).to(dev)
    ms, (g, it, _, st) = _median_ms(dev, lambda: api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), tol=TOL,
                                                                           max_iter=MAX_ITER, weights=wd, **SCHED))
    it = it.cpu().numpy()
    iv = b.interval(0)
    wi = w[int(b.row_off[0]):int(b.row_off[0]) + int(b.n_samp[0]) * int(b.n_bl[0])].reshape(int(b.n_samp[0]), -1)
    st0 = diagonal.iterate('jones', b.g0()[iv['gain_slice']].astype(np.complex128), iv['vis'], iv['model'],
                           iv['ant1'], iv['ant2'], iv['n_ant'], tol=0.0, max_iter=LM_AFTER, weights=wi)
    prob = wirtinger.ClosedFormProblem('jones', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'], weights=wi)
    ref, _, _ = wirtinger.levenberg_marquardt(prob, st0['g'], tol=1e-12, max_iter=400, lam0=1e-2, K=10.0, gauge=True)
    err = gauge.rel_error('jones', g.cpu().numpy()[iv['gain_slice']], ref)
    return {"workload": WEIGHTS_WORKLOAD, "metric": METRIC, "unit": UNIT, "ms": ms, "value": b.n_rows / (ms / 1e3),
            "iters_median": int(np.median(it)), "iters_max": int(it.max()),
            "converged": int(np.sum((st.cpu().numpy() & 15) == 0)), "max_err_vs_oracle_interval0": err}


SMOOTH_WORKLOAD = ("smooth: per-sample gains (Gaussian process, 30 min / 1 GHz), 64 ant (2016 bl), {nt} t x 64 ch, "
                   "one solution per sample, sigma {sig}; Gaussian kernel sigma_t 4 samples, sigma_f 0")


def smooth_block(dev, args, peaks, which):
    """Smoothing in time and frequency (Sect. 3.4), scalar and 2x2: wall time, iterations, and the
    per-iteration accumulation pass (the rows read once per iteration, HBM-bound) against HBM."""
    import torch
    from paper_1502_06974_gb300 import api, synth
    out = {}
    for kind, nt, sig, max_iter in (("scalar", 240, 2.0, 2000), ("jones", 120, 2.0, 100)):
        b = synth.make_smooth(kind, n_ant=64, n_t=nt, n_chan=64, sigma=sig, f_corr_hz=1e9)
        vis, model = torch.from_numpy(b.vis).to(dev), torch.from_numpy(b.model).to(dev)
        g0 = torch.from_numpy(b.g0()).to(dev)
        call = lambda: api.calibrate_di_smooth(vis, model, nt, 64, b.ant1, b.ant2, 64, g0.clone(), 4.0, 0.0,
                                               tol=TOL, max_iter=max_iter)
        ms, (_, it, _, st) = _median_ms(dev, call, reps=1)
        iters = int(it.cpu().numpy()[0])
        row_b = 16 if kind == "scalar" else 64
        out[kind] = {"workload": SMOOTH_WORKLOAD.format(nt=nt, sig=sig) + (" (2x2: a fixed iteration cap; the "
                     "polarized update contracts slowly)" if kind == "jones" else ""),
                     "rows": b.n_rows, "ms": ms, "iters": iters, "status": int(st.cpu().numpy()[0]),
                     "ms_per_iteration": ms / max(iters, 1),
                     "rows_read_per_iteration_gbs": b.n_rows * row_b / (ms / max(iters, 1) / 1e3) / 1e9,
                     "hbm_frac_rows_only": b.n_rows * row_b / (ms / max(iters, 1) / 1e3) / 1e9 / peaks["hbm_gbs"],
                     "peak_source": which}
        del vis, model
        torch.cuda.empty_cache()
    return out


def run_gpu(args):
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=dev)
    from paper_1502_06974_gb300 import api, build
    build.build()
    if args.dd_only:  # the direction-dependent workload alone (one JSON line)
        if rank == 0:
            peaks, which = measured_peaks()
            print(json.dumps(dd_block(dev, args, peaks, which)))
        return 0
    if args.ddpol_only:  # the polarized direction-dependent workload alone (one JSON line)
        if rank == 0:
            peaks, which = measured_peaks()
            print(json.dumps(ddpol_block(dev, args, peaks, which)))
        return 0
    b = make_workload(rank)
    lay = api.Layout.from_batch(b)
    vis = torch.from_numpy(b.vis).to(dev)
    model = torch.from_numpy(b.model).to(dev)
    g0 = torch.from_numpy(b.g0()).to(dev)
    gains = g0.clone()
    stream = torch.cuda.current_stream(dev)

    lm = args.schedule == 'lm'
    sched = SCHED if lm else dict(schedule='stefcal', path=args.path)
    tol, max_iter = (0.0, args.iters) if args.iters else (TOL if lm else TOL_STEFCAL, MAX_ITER)

    def step(profile=False):
        gains.copy_(g0)
        return api.calibrate_di_jones2x2(vis, model, lay, gains, tol=tol, max_iter=max_iter, profile=profile, **sched)

    tuned_ms = None
    if not args.no_autotune:   # launch shapes picked on this data, before any timing
        tuned_ms = api.autotune_di(vis, model, lay, gains, iters=24)
    for _ in range(args.warmup):
        _, iters, _, status = step()
    torch.cuda.synchronize(dev)
    its = iters.cpu().numpy()
    st = status.cpu().numpy()

    # timed region
    sampler = ClockSampler()
    if rank == 0:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    n0 = api.launch_count()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    kms = 0.0; kl = 0; kri = 0; kmom = 0.0; kbi = 0; path_used = None
    lms = 0.0; lml = 0; lmf = 0.0
    e0.record(stream)
    for _ in range(args.steps):
        step(profile=True)
        ms_k, n_k, ri_k = api.profile_last()
        mom_k, bi_k, path_used = api.profile_detail()
        kms += ms_k; kl += n_k; kri += ri_k; kmom += mom_k; kbi += bi_k
        if lm:
            a, n, f = api.profile_lm()
            lms += a; lml += n; lmf += f
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = api.launch_count() - n0
    clocks = sampler.stop(gpu_index=None) if rank == 0 else None
    ms = max_over_ranks(ms, dist, dev)
    rows_total = b.n_rows * args.steps * world
    value = rows_total / (ms / 1e3)
    g_sol = gains.cpu().numpy()

    # the accumulate kernel of the diagonal iterations timed alone (outside the timed region): one
    # more full solve in which every accumulate launch is bracketed by CUDA events on the call's stream
    acc = None
    if path_used == N_PATH_MOMENTS:
        step(profile=2)
        acc_ms, acc_n, _ = api.profile_last()
        _, acc_bi, _ = api.profile_detail()
        acc = (acc_ms, acc_n, acc_bi)

    # end to end through the public API with pinned host buffers
    g0H = torch.from_numpy(b.g0()).pin_memory()
    e2e_s = float('nan')
    if not args.no_e2e:
        visH = torch.from_numpy(b.vis).pin_memory()
        modelH = torch.from_numpy(b.model).pin_memory()
        gH = g0H.clone().pin_memory()
        api.calibrate_di_jones2x2(visH, modelH, lay, gH, tol=tol, max_iter=max_iter, host_buffers=True, **sched)
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            gH.copy_(g0H)
            api.calibrate_di_jones2x2(visH, modelH, lay, gH, tol=tol, max_iter=max_iter, host_buffers=True, **sched)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, dist, dev)

    # StefCal alone to a relative step of 1e-6 (the diagonal method without LM), for comparison
    stefcal_only = None
    if lm and rank == 0 and not args.no_stefcal_compare and not args.iters:
        gains.copy_(g0)
        api.calibrate_di_jones2x2(vis, model, lay, gains, tol=TOL_STEFCAL, max_iter=MAX_ITER)
        gains.copy_(g0)
        torch.cuda.synchronize(dev)
        f0 = torch.cuda.Event(enable_timing=True); f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        _, it_sc, _, st_sc = api.calibrate_di_jones2x2(vis, model, lay, gains, tol=TOL_STEFCAL, max_iter=MAX_ITER)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        stefcal_only = {"ms": f0.elapsed_time(f1), "tol": TOL_STEFCAL, "g": gains.cpu().numpy(),
                        "iters_median": int(np.median(it_sc.cpu().numpy())), "iters_max": int(it_sc.max().item())}

    if rank == 0:
        peaks, which = measured_peaks()
        props = torch.cuda.get_device_properties(dev)
        n_sm = props.multi_processor_count
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        extra = {}
        if lm and not args.iters:
            errs, refs = oracle_errors(b, g_sol)
            extra["max_err_vs_oracle"] = max(errs.values())
            extra["err_vs_oracle_sampled"] = errs
            if stefcal_only is not None:
                e_sc, _ = oracle_errors(b, stefcal_only.pop("g"), refs=refs)
                stefcal_only["max_err_vs_oracle"] = max(e_sc.values())
                stefcal_only["value"] = b.n_rows / (stefcal_only["ms"] / 1e3)
        roof_acc = None
        if acc is not None:
            acc_ms, acc_n, acc_bi = acc
            avg_launch_s = (acc_ms / 1e3) / max(acc_n, 1)
            bytes_per_launch = acc_bi * MOMENT_BYTES / max(acc_n, 1)
            roof_acc = {"bound": "hbm", "achieved": bytes_per_launch / avg_launch_s / 1e9, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": bytes_per_launch / avg_launch_s / 1e9 / peaks["hbm_gbs"],
                        "kernel": "di_macc_bulk_kernel<JonesMom> (moment-space J^H D / diag J^H J per 256-baseline "
                                  "tile, bulk copies into a two-stage shared-memory ring)",
                        "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_s * 1e6, "launches": acc_n,
                        "timed": "every accumulate launch of one full solve, CUDA events on the call's stream",
                        "peak_source": which}
        mom_bytes = (b.n_rows * BYTES_PER_ROW + b.n_int * int(b.n_bl[0]) * MOMENT_BYTES) * args.steps
        roof_mom = {"bound": "hbm", "achieved": mom_bytes / (kmom / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": mom_bytes / (kmom / 1e3) / 1e9 / peaks["hbm_gbs"],
                    "kernel": ("di_moment_direct_kernel<JonesMom>" if int(np.max(b.n_samp)) <= 16
                               else "di_moment_kernel<JonesMom>"), "ms_per_step": kmom / args.steps,
                    "peak_source": which} if kmom > 0 else None
        if lm:
            # dominant kernel: the LM iteration kernel, bound by FP32 FMA issue (no tensor cores):
            # achieved = algorithmic flops of its Cholesky factorisations and triangular solves /
            # the summed CUDA-event time of its launches in the timed steps
            peak_tf = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
            n_unk = 8 * int(b.n_ant[0])
            flop_per_ii = n_unk ** 3 / 3.0 + 2.0 * n_unk ** 2
            ii_per_launch = lmf / flop_per_ii / max(lml, 1)
            summ = ncu_summary('lm_iter_jones_cfg2.json', LM_SOURCES)
            roof = {"bound": "alu", "achieved": lmf / (lms / 1e3) / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": lmf / (lms / 1e3) / 1e12 / peak_tf,
                    "traffic": (summ["dram_bytes_per_interval_iteration"] * ii_per_launch) if summ else None,
                    "kernel": ("lm_iter_kernel<LMJones> (per interval: whole J^H J from the moments, FP32 blocked "
                               "Cholesky + triangular solves, FP64 chi^2 and damping decision)"),
                    "flop_per_launch": lmf / max(lml, 1), "interval_iterations_per_launch": ii_per_launch,
                    "avg_launch_us": lms * 1e3 / max(lml, 1), "launches": lml,
                    "timed": "every LM iteration launch of the timed steps, CUDA events on the call's stream",
                    "peak_source": (f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop (FMA) x {sm_mhz:.0f} MHz")}
        else:
            roof = roof_acc
        med_it = int(np.median(its))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD if lm else WORKLOAD.split(';')[0] + f"; StefCal to {TOL_STEFCAL:g}",
                          "rows_per_gpu": b.n_rows, "intervals": b.n_int, "tol": tol,
                          "schedule": (f"StefCal x{LM_AFTER} then LM (K={LM_K:g}, lambda0 1e-2)" if lm else "StefCal"),
                          "l2": "inputs (495 MB vis+model) larger than L2; no flush",
                          "iters_median": med_it, "iters_max": int(its.max()),
                          "converged": int(np.sum((st & 15) == 0)),
                          "parallelism": f"replicas x{world} (independent intervals per GPU)",
                          "autotuned": tuned_ms is not None, **extra},
               "roofline": roof,
               "roofline_accumulate": roof_acc if lm else None,
               "roofline_moment_pass": roof_mom,
               "time_split_ms_per_step": {"moment_pass": kmom / args.steps, "stefcal_iterations": kms / args.steps,
                                          "lm_iterations": lms / args.steps} if lm else None,
               "stefcal_only": stefcal_only,
               "path": {N_PATH_RESIDENT: "resident", N_PATH_MOMENTS: "moments"}.get(path_used, "stream"),
               "e2e": {"value": b.n_rows * world / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": int(b.vis.nbytes + b.model.nbytes + g0H.numel() * 8),
                       "d2h_bytes_per_step": int(g0H.numel() * 8 + 2 * 4 * b.n_int)},
               "gpu_launches": int(launches),
               "clocks": clocks}
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_block(b, 0)
            out["cpu_baseline_openmp"] = cpu_openmp_block(rank_seed(0))
        if not args.no_weights and world == 1:
            out["weights"] = weights_block(dev, args, b, vis, model, lay, g0)
        if not args.no_warm and world == 1:
            del vis, model
            torch.cuda.empty_cache()
            out["warm_start"] = warm_start_block(dev, args)
        if not args.no_dd and world == 1:
            out["dd_cohjones"] = dd_block(dev, args, peaks, which)
        if not args.no_uneven and world == 1:
            out["uneven"] = uneven_block(dev, args)
        if not args.no_dd and world == 1:
            out["dd_alljones"] = alljones_block(dev, args, peaks, which)
            out["dd_jones2x2"] = ddpol_block(dev, args, peaks, which)
        if not args.no_smooth and world == 1:
            out["smooth"] = smooth_block(dev, args, peaks, which)
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='gaincal', choices=['gaincal', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-autotune', action='store_true')
    ap.add_argument('--no-warm', action='store_true', help='skip the learned warm start comparison')
    ap.add_argument('--no-dd', action='store_true', help='skip the direction-dependent (CohJones) workload')
    ap.add_argument('--dd-only', action='store_true', help='run only the direction-dependent workload')
    ap.add_argument('--ddpol-only', action='store_true', help='run only the polarized direction-dependent workload')
    ap.add_argument('--no-uneven', action='store_true', help='skip the uneven batched workload')
    ap.add_argument('--no-weights', action='store_true', help='skip the weighted headline solve')
    ap.add_argument('--no-smooth', action='store_true', help='skip the smoothing workloads')
    ap.add_argument('--uneven-intervals', type=int, default=4096, help='intervals of the uneven workload')
    ap.add_argument('--path', type=int, default=0,
                    help='StefCal schedule only: 0 auto (moments), 1 raw-row streaming, 2 resident, 3 moments')
    ap.add_argument('--schedule', default='lm', choices=['lm', 'stefcal'],
                    help='lm (default): StefCal x20 then LM with the whole J^H J; stefcal: StefCal alone to 1e-6')
    ap.add_argument('--no-stefcal-compare', action='store_true', help='skip the StefCal-only comparison solve')
    ap.add_argument('--iters', type=int, default=0,
                    help='run exactly this many iterations per step (tol 0) instead of converging; for profiling')
    args = ap.parse_args()
    if args.impl == 'reference':
        return run_reference(args)
    return run_gpu(args)


if __name__ == '__main__':
    sys.exit(main())
