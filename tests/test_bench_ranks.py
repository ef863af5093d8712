"""Host logic of the multi-GPU benchmark path on CPU: two gloo ranks.

Directions are independent, so `bench.py --gpus N` runs one replica per rank
with no data exchange; the only cross-rank steps are the timing barrier and
the max over ranks.  Checked here without a GPU: each rank gets its own
seeded batch (rank 0 the workload's), the job time is the slowest rank's on
every rank, and the whole-job value counts every rank's work.
"""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads
        w = workloads.workload("dirs16")
        th, ph, al = bench.rank_directions(w, rank, 16)
        ms = 100.0 + 25.0 * rank                     # rank 1 is the slow one
        dist.barrier()
        job_ms = bench.max_over_ranks(ms, world, "cpu")
        value = bench.job_value(1000, 5, world, job_ms)
        np.savez(os.path.join(out, "r%d.npz" % rank), th=th, ph=ph, al=al, job_ms=job_ms,
                 value=value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(os.path.join(tmp_path, "r%d.npz" % k)) for k in range(world)]
    sys.path.insert(0, ROOT)
    import workloads
    w = workloads.workload("dirs16")
    assert np.array_equal(r[0]["th"], w["theta"]) and np.array_equal(r[0]["ph"], w["phi"])
    assert not np.allclose(r[0]["th"], r[1]["th"])
    for k in range(world):
        assert len(r[k]["th"]) == 16
        assert np.all((r[k]["th"] >= 0) & (r[k]["th"] <= np.pi / 3))
        assert float(r[k]["job_ms"]) == 125.0
        assert float(r[k]["value"]) == pytest.approx(1000 * 5 * world / 0.125)
