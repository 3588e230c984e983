"""The N > 1 path of the bench, on CPU: two gloo ranks decode disjoint shot
ranges (the oracle stands in for the GPU decoder; nothing here touches a
GPU) and reduce their failure counts and times; the result equals one
process decoding all shards."""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2403_18901_gb300 import replicas  # noqa: E402

N_BATCHES, B = 2, 12


def _decode(rank):
    from conftest import oracle_dem
    from paper_2403_18901_gb300.workloads import preset
    o = oracle_dem("72", 0.004, 6)
    params = preset("paper", k_guess=2, p=0.004)
    fails = 0
    for b in range(N_BATCHES):
        det, obs = o.sample(99, replicas.shot_offset(rank, N_BATCHES, B, b), B)
        f, _, _ = o.run_shots(params, det, obs, threads=1)
        fails += int((f > 0).sum())
    return fails


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f = _decode(rank)
        total = replicas.sum_over_ranks(f)
        t = replicas.max_over_ranks(float(rank + 1))
        ranges = [replicas.shot_offset(rank, N_BATCHES, B, b) for b in range(N_BATCHES)]
        gathered = [None] * world
        dist.all_gather_object(gathered, ranges)
        if rank == 0:
            np.save(out, np.array([total, t] + [x for r in gathered for x in r], np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_process():
    port = 29500 + os.getpid() % 1000
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r.npy")
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = np.load(out)
    total, t, offs = int(res[0]), res[1], res[2:].astype(np.int64)
    assert t == 2.0  # max over ranks
    # disjoint, contiguous shot ranges
    starts = sorted(offs)
    assert len(set(starts)) == len(starts) and all(b - a == B for a, b in zip(starts, starts[1:]))
    assert total == _decode(0) + _decode(1)
