"""The multi-GPU form of the bench is replicas only (independent problems,
one per rank, no data-path collective): two gloo ranks on the CPU check the
whole-job aggregation (slowest rank's time, summed work) and that the ranks
build distinct replicas."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, pairs, simt = bench.combine_ranks(10.0 + rank, 1000 * (rank + 1), 0.5 * (rank + 1), dist, "cpu")
    cases = bench.make_cases("dam_gate", seed=rank)
    out[rank] = (ms, pairs, simt, float(np.asarray(cases[0].f_r).sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_and_summed_work():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        ms, pairs, simt, _ = out[r]
        assert ms == 11.0                       # the slowest rank
        assert pairs == 3000.0 and simt == 1.5  # summed over the ranks
    assert out[0][3] != out[1][3]               # seeds differ: distinct replicas
