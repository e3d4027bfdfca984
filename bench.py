#!/usr/bin/env python
"""Throughput of gain calibration to convergence: visibilities calibrated per second.

Workload (the full-Jones direction-independent problem): 64 antennas (2016 baselines), 2x2 Jones,
60 times x 64 channels at 1.0-1.4 GHz, solution intervals of 1 time x 4 channels (960 intervals,
7,741,440 rows of 2x2 complex64), 20 polarized point sources, true Jones = diagonal gains
(amplitude 1 + N(0, 0.1), phase U(-pi, pi)) plus leakage CN(0, 0.02), noise sigma = 0.01,
seed 150206974 (+ rank).  Every interval is solved by polarized StefCal from identity gains to a
relative step tolerance of 1e-6.

One step = reset the gains to identity + one gc_calibrate_di_jones2x2 call over all 960 intervals
(iterations run until every interval has converged).  value = rows calibrated / device time, inputs
resident in HBM (495 MB of vis + model, larger than L2, so no flush is needed).  e2e = the same
call with pinned host buffers, host<->device copies inside the timed region.

Under torchrun each rank solves its own copy of the workload on its own GPU (independent
intervals, no collective on the data path: weak scaling); rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle (the paper's iteration in NumPy) on a bounded sample.
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

TOL = 1e-6
MAX_ITER = 20000
BYTES_PER_ROW = 64          # vis + model, one 2x2 complex64 each (algorithmic bytes per row per iteration)
MOMENT_BYTES = 192          # per baseline: P (4x4 complex64) + R (4x4 float32), written once by the moment pass
FLOP_PER_BASELINE_ITER = 320  # per baseline per iteration: 2 x (4x4 complex mat-vec + 4x4 real mat-vec)
N_PATH_STREAM, N_PATH_RESIDENT, N_PATH_MOMENTS = 1, 2, 3
METRIC = "visibilities calibrated/s to convergence at <=1e-5 gain err; learned+batched vs plain"
UNIT = "visibilities/s"
WORKLOAD = "di_jones2x2: 64 ant (2016 bl), 60 t x 64 ch, intervals 1 t x 4 ch (960), 20 polarized sources, tol 1e-6"


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
def oracle_sample(b, n_iter=120, interval=0):
    """Time the FP64 oracle iteration (NumPy, the paper's steps) on one interval for n_iter steps.

    Returns (seconds per iteration, rows of the interval, cpu-seconds / wall-seconds).
    """
    from oracle import diagonal
    iv = b.interval(interval)
    g0 = b.g0()[iv['gain_slice']]
    t0 = time.perf_counter(); c0 = time.process_time()
    diagonal.iterate('jones', g0, iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'], tol=0.0,
                     max_iter=n_iter)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return wall / n_iter, int(iv['vis'].shape[0] * iv['vis'].shape[1]), cpu / max(wall, 1e-9)


def cpu_baseline_block(b, iters_to_converge, n_iter=120):
    per_it, rows, threads = oracle_sample(b, n_iter)
    value = rows / (per_it * iters_to_converge)
    return {"value": value, "unit": UNIT, "cores": max(1, int(round(threads))), "kind": "oracle",
            "sample": (f"FP64 NumPy oracle (diagonal iteration), 1 interval of {rows} rows x {n_iter} iterations "
                       f"({per_it * 1e3:.2f} ms/iteration), extrapolated to {iters_to_converge} iterations "
                       f"(median iteration count to tol {TOL:g} on the GPU run)")}


# ------------------------------------------------------------------------------------ helpers
def kernel_source_hash():
    h = hashlib.sha256()
    for f in ('di_kernels.cu', 'resident.cu', 'kinds.cuh', 'common.cuh', 'internal.h'):
        with open(os.path.join(ROOT, 'paper_1502_06974_gb300', 'csrc', f), 'rb') as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(name, unit):
    """DRAM bytes per launch of a kernel from a committed ncu summary (json) when it was taken on the
    current kernel sources; None otherwise."""
    p = os.path.join(ROOT, 'profiles', name)
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get('kernel_hash') != kernel_source_hash():
        return None
    if unit == 'moments':
        return d['dram_bytes_per_launch'] / d['baselines_per_launch']
    return d.get('dram_bytes_per_launch')


def ncu_traffic_per_row():
    """DRAM bytes per processed row of the iteration kernel from the committed ncu summary, if it was
    taken on the current kernel source; None otherwise."""
    p = os.path.join(ROOT, 'profiles', 'di_iter_jones_cfg2.json')
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get('kernel_hash') != kernel_source_hash():
        return None
    return d['dram_bytes_per_launch'] / d['rows_per_launch']


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json'))), "of measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "of fallback"


# ------------------------------------------------------------------------------------ arms
def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    b = make_workload(0)
    iters = args.ref_iters
    samples = []
    per_it = rows = threads = None
    for k in range(args.warmup + args.steps):
        per_it, rows, threads = oracle_sample(b, n_iter=args.ref_sample_iters, interval=k % b.n_int)
        if k >= args.warmup:
            samples.append(per_it)
    per_it = statistics.median(samples)
    value = rows / (per_it * iters)
    cores = max(1, int(round(threads)))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_it * iters * 1e3 * b.n_int,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "rows": b.n_rows, "intervals": b.n_int, "tol": TOL},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": (f"each step: FP64 NumPy oracle, 1 interval ({rows} rows) x "
                                       f"{args.ref_sample_iters} iterations, extrapolated to {iters} iterations")},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


WARM_LAG = 32           # wave length (time steps) of the learned wavefront
WARM_GATE = 1e-5        # pipelined wavefront: a wave joins once its history's relative steps fall below this
WARM_WORKLOAD = ("di_jones2x2 warm start: 64 ant (2016 bl), 720 t x 64 ch, intervals 1 t x 8 ch (5760), GP gains "
                 "(30 min / 50 MHz correlation, amplitude 0.1, phase 1 rad), tol 1e-6")


def warm_start_block(dev, args):
    """Learned warm start + batched path vs the plain batched solver on the GP-gain workload.

    The network is trained first (its own observation, another seed), then the same 5760 intervals
    are solved with the data resident: plain (all intervals from unit gains in one call); the
    previous-solution and learned starts in waves of 32 times, one call per wave; and the same two
    starts pipelined in one call (a wave joins once its history has settled to WARM_GATE)."""
    import torch
    from paper_1502_06974_gb300 import api, synth, warmstart
    t0 = time.perf_counter()
    bt = synth.make_warm(seed=synth.SEED + 1000, n_t=160)
    vt, mt = torch.from_numpy(bt.vis).to(dev), torch.from_numpy(bt.model).to(dev)
    gt = warmstart.Grid.from_batch(bt)
    sol_t, _, st_t = warmstart.solve_plain(vt, mt, gt, TOL, MAX_ITER)
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

    def timed(fn):
        fn()                                   # warm-up (plan, graph capture)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return out, e0.elapsed_time(e1)

    (gp, itp, stp), ms_plain = timed(lambda: warmstart.solve_plain(ve, me, ge, TOL, MAX_ITER))
    prev, ms_prev = timed(lambda: warmstart.solve_wavefront(ve, me, ge, WARM_LAG, None, TOL, MAX_ITER))
    lrn, ms_lrn = timed(lambda: warmstart.solve_wavefront(ve, me, ge, WARM_LAG, res.net, TOL, MAX_ITER))
    # the same two starts in one library call, waves joining the running iteration (pipelined)
    pprev, ms_pprev = timed(lambda: warmstart.solve_pipelined(ve, me, ge, WARM_LAG, None, TOL, MAX_ITER,
                                                              gate_tol=WARM_GATE))
    plrn, ms_plrn = timed(lambda: warmstart.solve_pipelined(ve, me, ge, WARM_LAG, res.net, TOL, MAX_ITER,
                                                            gate_tol=WARM_GATE))
    itp = itp.cpu().numpy()
    rows = ge.rows * n_int
    g_true = be.g_true

    def err_truth(g):
        # max over antennas of ||G e^{i phi} - G_true|| / ||G_true||, phi the least-squares global
        # phase of each interval (solutions are defined up to that phase)
        est = g.cpu().numpy().astype(np.complex128).reshape(n_int, ge.n_ant, 4)
        ref = g_true.reshape(n_int, ge.n_ant, 4)
        ph = np.exp(1j * np.angle(np.sum(ref * np.conj(est), axis=(1, 2))))
        d = np.linalg.norm(est * ph[:, None, None] - ref, axis=2) / np.linalg.norm(ref, axis=2)
        return float(d.max())

    def entry(ms, iters, status, extra=None):
        d = {"ms": ms, "value": rows / (ms / 1e3), "iters_mean": float(np.mean(iters)),
             "iters_max": int(np.max(iters)), "interval_iterations": int(np.sum(iters)),
             "converged": int(np.sum((status & 15) == 0))}
        d.update(extra or {})
        return d

    return {"workload": WARM_WORKLOAD, "metric": METRIC, "unit": UNIT, "lag": WARM_LAG,
            "schedule": "waves of lag x 8 intervals, one gc_calibrate_di_jones2x2_warm call each, predicted from "
                        "the 4 solutions before the wave",
            "plain": entry(ms_plain, itp, stp.cpu().numpy(), {"max_err_vs_truth": err_truth(gp)}),
            "previous_solution": entry(ms_prev, prev.iters, prev.status, {"max_err_vs_truth": err_truth(prev.gains)}),
            "learned": entry(ms_lrn, lrn.iters, lrn.status,
                             {"proposals_taken": float(np.mean(lrn.used[np.repeat(np.arange(ge.n_t), ge.n_fb)
                                                                       >= WARM_LAG])),
                              "max_err_vs_truth": err_truth(lrn.gains)}),
            "pipelined": {
                "schedule": f"one gc_calibrate_di_jones2x2_wavefront call: a wave of lag x 8 intervals joins the "
                            f"running iteration once the 4 times before it have finished or taken a relative step "
                            f"below {WARM_GATE:g}",
                "previous_solution": entry(ms_pprev, pprev.iters, pprev.status,
                                           {"max_err_vs_truth": err_truth(pprev.gains)}),
                "learned": entry(ms_plrn, plrn.iters, plrn.status, {"max_err_vs_truth": err_truth(plrn.gains)}),
                "speedup_learned_vs_plain": ms_plain / ms_plrn,
                "speedup_learned_vs_previous_solution": ms_pprev / ms_plrn},
            "speedup_learned_vs_plain": ms_plain / ms_lrn,
            "speedup_learned_vs_previous_solution": ms_prev / ms_lrn,
            "speedup_best_learned_vs_plain": ms_plain / min(ms_lrn, ms_plrn),
            "training": {"trajectories": 50000, "observation": "160 t x 64 ch of the same array, another seed",
                         "adam_steps": res.steps, "train_s": res.seconds, "prep_s": prep_s,
                         "val_mse": res.val_mse, "val_mse_previous_solution": res.val_mse_zero}}


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
                                     "FP32 Cholesky in registers + one float-float refinement step)", "moments_bytes": int(np.sum(b.n_bl)) * (nd * (nd + 1) // 2 + nd) * 8}}


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
    b = make_workload(rank)
    lay = api.Layout.from_batch(b)
    vis = torch.from_numpy(b.vis).to(dev)
    model = torch.from_numpy(b.model).to(dev)
    g0 = torch.from_numpy(b.g0()).to(dev)
    gains = g0.clone()
    stream = torch.cuda.current_stream(dev)

    tol, max_iter = (0.0, args.iters) if args.iters else (TOL, MAX_ITER)

    def step(profile=False):
        gains.copy_(g0)
        return api.calibrate_di_jones2x2(vis, model, lay, gains, tol=tol, max_iter=max_iter, profile=profile,
                                         path=args.path)

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
    e0.record(stream)
    for _ in range(args.steps):
        step(profile=True)
        ms_k, n_k, ri_k = api.profile_last()
        mom_k, bi_k, path_used = api.profile_detail()
        kms += ms_k; kl += n_k; kri += ri_k; kmom += mom_k; kbi += bi_k
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

    # the accumulate kernel timed alone (outside the timed region): one more full solve in which
    # every accumulate launch is bracketed by CUDA events on the call's stream
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
        api.calibrate_di_jones2x2(visH, modelH, lay, gH, tol=tol, max_iter=max_iter, host_buffers=True, path=args.path)
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            gH.copy_(g0H)
            api.calibrate_di_jones2x2(visH, modelH, lay, gH, tol=tol, max_iter=max_iter, host_buffers=True,
                                      path=args.path)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, dist, dev)

    if rank == 0:
        peaks, which = measured_peaks()
        roof_iter = None
        if path_used == N_PATH_RESIDENT:
            # dominant kernel: the cluster-resident iteration kernel (one launch per step); the
            # moment pass (HBM-bound) is reported beside it
            n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
            sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
            peak_tf = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12        # FP32 FMA lanes x 2 flop x clock
            flops = kbi * FLOP_PER_BASELINE_ITER
            achieved = flops / (kms / 1e3) / 1e12
            tpl = ncu_traffic('di_resident_jones_cfg2.json', 'resident')
            roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved / peak_tf, "traffic": (tpl * kl / max(kl, 1)) if tpl is not None else None,
                    "kernel": "di_resident_kernel<JonesMom> (moment-space J^H D / J^H J + 2x2 update, on chip)",
                    "flop_per_launch": flops / max(kl, 1), "avg_launch_us": kms * 1e3 / max(kl, 1),
                    "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz"}
            mom_bytes = (b.n_rows * BYTES_PER_ROW + b.n_int * int(b.n_bl[0]) * MOMENT_BYTES) * args.steps
            roof_mom = {"bound": "hbm", "achieved": mom_bytes / (kmom / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": mom_bytes / (kmom / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "kernel": "di_moment_kernel<JonesMom>", "ms_per_step": kmom / args.steps,
                        "peak_source": which}
        elif path_used == N_PATH_MOMENTS:
            # dominant kernel: the moment-space accumulate kernel, 192 B of moments per active
            # baseline per iteration (HBM-bound), each launch timed alone in one full solve; the
            # whole iteration (accumulate + solve launches, graph segments) over the timed steps
            # and the one-off moment pass are reported beside it
            acc_ms, acc_n, acc_bi = acc
            avg_launch_s = (acc_ms / 1e3) / max(acc_n, 1)
            bytes_per_launch = acc_bi * MOMENT_BYTES / max(acc_n, 1)
            achieved = bytes_per_launch / avg_launch_s / 1e9
            tpb = ncu_traffic('di_macc_jones_cfg2.json', 'moments')   # DRAM bytes per active baseline
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"],
                    "traffic": (tpb * acc_bi / max(acc_n, 1)) if tpb is not None else None,
                    "kernel": "di_macc_bulk_kernel<JonesMom> (moment-space J^H D / diag J^H J per 256-baseline tile, bulk copies into a two-stage shared-memory ring)",
                    "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_s * 1e6, "launches": acc_n,
                    "timed": "every accumulate launch of one full solve, CUDA events on the call's stream",
                    "peak_source": which}
            it_bytes = kbi * MOMENT_BYTES
            roof_iter = {"achieved": it_bytes / (kms / 1e3) / 1e9, "unit": "GB/s",
                         "frac": it_bytes / (kms / 1e3) / 1e9 / peaks["hbm_gbs"],
                         "timed": "accumulate + solve launches of every iteration in the timed steps (graph "
                                  "segments bracketed by CUDA events)", "iterations": kl,
                         "avg_iteration_us": kms * 1e3 / max(kl, 1)}
            mom_bytes = (b.n_rows * BYTES_PER_ROW + b.n_int * int(b.n_bl[0]) * MOMENT_BYTES) * args.steps
            roof_mom = {"bound": "hbm", "achieved": mom_bytes / (kmom / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": mom_bytes / (kmom / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "kernel": ("di_moment_direct_kernel<JonesMom>" if int(np.max(b.n_samp)) <= 16
                                   else "di_moment_kernel<JonesMom>"), "ms_per_step": kmom / args.steps,
                        "peak_source": which}
        else:
            avg_launch_s = (kms / 1e3) / max(kl, 1)
            bytes_per_launch = kri * BYTES_PER_ROW / max(kl, 1)
            achieved = bytes_per_launch / avg_launch_s / 1e9
            tpr = ncu_traffic_per_row()
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"],
                    "traffic": (tpr * kri / max(kl, 1)) if tpr is not None else None,
                    "kernel": "di_iter_kernel<float, JonesKind> (accumulate J^H D, diag J^H J + StefCal update)",
                    "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_s * 1e6,
                    "peak_source": which}
            roof_mom = None
        med_it = int(np.median(its))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD, "rows_per_gpu": b.n_rows, "intervals": b.n_int, "tol": TOL,
                          "l2": "inputs (495 MB vis+model) larger than L2; no flush",
                          "iters_median": med_it, "iters_max": int(its.max()),
                          "converged": int(np.sum((st & 15) == 0)),
                          "parallelism": f"replicas x{world} (independent intervals per GPU)",
                          "autotuned": tuned_ms is not None},
               "roofline": roof,
               "roofline_moment_pass": roof_mom,
               "roofline_iteration": roof_iter,
               "path": {N_PATH_RESIDENT: "resident", N_PATH_MOMENTS: "moments"}.get(path_used, "stream"),
               "e2e": {"value": b.n_rows * world / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": int(b.vis.nbytes + b.model.nbytes + g0H.numel() * 8),
                       "d2h_bytes_per_step": int(g0H.numel() * 8 + 2 * 4 * b.n_int)},
               "gpu_launches": int(launches),
               "clocks": clocks}
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_block(b, med_it)
        if not args.no_warm and world == 1:
            del vis, model
            torch.cuda.empty_cache()
            out["warm_start"] = warm_start_block(dev, args)
        if not args.no_dd and world == 1:
            out["dd_cohjones"] = dd_block(dev, args, peaks, which)
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
    ap.add_argument('--path', type=int, default=0, help='0 auto (moments), 1 raw-row streaming, 2 resident, 3 moments')
    ap.add_argument('--iters', type=int, default=0,
                    help='run exactly this many iterations per step (tol 0) instead of converging; for profiling')
    ap.add_argument('--ref-iters', type=int, default=3200, help='iterations the reference arm extrapolates to')
    ap.add_argument('--ref-sample-iters', type=int, default=40)
    args = ap.parse_args()
    if args.impl == 'reference':
        return run_reference(args)
    return run_gpu(args)


if __name__ == '__main__':
    sys.exit(main())
