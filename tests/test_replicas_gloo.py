"""The multi-GPU form is replicas only (independent problems, no collective in the data
path); its one cross-rank step is the timing reduction of bench.py: the job's step
time is the slowest rank's and the throughput counts every rank's points.  Checked
here with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [10.0 + rank, 20.0 - rank]  # rank 1 is slower in the first, faster in the second
    ms, val = bench.replica_throughput(ms_local, 1000, world, torch.device("cpu"))
    out.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, val in res:
        assert ms == [11.0, 20.0]                       # max over ranks, per entry
        assert val == pytest.approx([2 * 1000 / 11e-3 / 1e6, 2 * 1000 / 20e-3 / 1e6])


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms, val = bench.replica_throughput([4.0], 2_000_000, 1)
    assert ms == [4.0] and val == pytest.approx([500.0])
