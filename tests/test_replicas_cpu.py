"""The multi-GPU path is replicas only (one independent solve per rank, no data-path
collective): the benchmark's rank aggregation, run as two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    w, r, local = bench.dist_setup()
    # rank r timed 5 steps in (100 + 50 r) ms and 3 end-to-end steps in (60 + 10 r) ms
    total, e2e = bench.replica_max(dist, [100.0 + 50.0 * r, 60.0 + 10.0 * r], "cpu")
    out[rank] = (w, r, local, total, e2e, bench.replica_throughput(w, 5, total))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replica_aggregation():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        w, r, local, total, e2e, value = out[rank]
        assert (w, r, local) == (world, rank, rank)
        assert total == 150.0 and e2e == 70.0          # the slowest rank bounds the job
        assert value == pytest.approx(2 * 5 / 0.150)   # whole-job steps per second


def test_single_process_aggregation():
    bench = _bench()
    assert bench.replica_max(None, [3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.replica_throughput(1, 4, 2000.0) == 2.0
