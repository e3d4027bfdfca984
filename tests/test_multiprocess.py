"""The multi-GPU bench path on CPU: two gloo ranks (127.0.0.1) run the host logic bench.py uses when
it is launched with torchrun (one rank per GPU, replicas of the workload, no collective on the data
path): each rank draws its own workload seed, the timed region is closed by a barrier, the reported
time is the maximum over ranks, and the reference arm runs on rank 0 only."""
import argparse
import json
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import bench
    dist.init_process_group('gloo', init_method=f'tcp://127.0.0.1:{port}', rank=rank, world_size=world)
    try:
        seed = bench.rank_seed(rank)
        t = bench.max_over_ranks(10.0 * (rank + 1), dist, 'cpu')   # rank r "took" 10 (r + 1) ms
        dist.barrier()
        os.environ['RANK'], os.environ['WORLD_SIZE'] = str(rank), str(world)
        args = argparse.Namespace(gpus=world, steps=1, warmup=0)
        ref_rc = bench.run_reference(args) if rank != 0 else 0    # non-zero ranks return at once
        with open(os.path.join(outdir, f'r{rank}.json'), 'w') as f:
            json.dump({'seed': seed, 'time': t, 'ref_rc': ref_rc}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f'r{i}.json')) for i in range(world)]
    assert r[0]['seed'] != r[1]['seed']                      # independent replicas
    assert r[0]['time'] == r[1]['time'] == 20.0               # every rank reports the slowest rank's time
    assert r[1]['ref_rc'] == 0


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, 'cpu') == 3.5
