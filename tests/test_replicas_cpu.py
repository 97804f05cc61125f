"""The multi-GPU mode is replicas only: every rank runs its own circuit and the job's
rate is (units summed over ranks) / (slowest rank's time).  The reduction runs here
with two gloo ranks on the CPU (127.0.0.1 rendezvous); no GPU is touched."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    elapsed, units = b.replica_reduce(10.0 + 5 * rank, 49.0 + rank, dist, "cpu")
    out[rank] = (elapsed, units, b.replica_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_sum_of_units():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        elapsed, units, seed = out[r]
        assert elapsed == 15.0 and units == 99.0       # max(10, 15), 49 + 50
    assert out[0][2] != out[1][2]                        # distinct replica circuits


def test_single_rank_is_the_identity():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod1", os.path.join(root, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert b.replica_reduce(3.5, 49, None) == (3.5, 49)
