"""The multi-GPU form of the benchmark is N independent replicas (one problem per
rank, no data exchange): its host logic -- per-rank instances, the slowest rank's
time, the whole-job value -- checked with two gloo ranks on the CPU."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank_main(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.replica_workload(rank)
        inst = bench.cs_inputs.workload_instance(dict(w, N=60, M=40, nnz=6))
        local_time = 1.0 + 0.5 * rank  # the slower rank sets the job's time
        t = bench.max_over_ranks(local_time, dist, "cpu")
        v = bench.job_value(world, 3, t)
        dist.barrier()
        out[rank] = (w["seed"], float(inst.A[0, 0]), t, v)
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    (s0, a0, t0, v0), (s1, a1, t1, v1) = out[0], out[1]
    assert s1 == s0 + 1 and a0 != a1          # independent problems per rank
    assert t0 == t1 == pytest.approx(1.5)     # both ranks report the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 3 / 1.5)


def test_single_process_value():
    import bench

    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_value(1, 5, 2.0) == pytest.approx(2.5)
    np.testing.assert_equal(bench.replica_workload(0)["seed"], 0)
