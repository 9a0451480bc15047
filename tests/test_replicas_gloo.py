"""The multi-GPU path of bench.py (independent replicas, one per rank): the
timed region's duration is the maximum over ranks and the value is the units
of all ranks over that time.  Exercised with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, outdir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    t = bench.max_over_ranks(times[rank], device="cpu")
    v = bench.replicas_value(1000.0, t, dist.get_world_size())
    dist.barrier()
    with open(os.path.join(outdir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{t!r} {v!r}")
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank(tmp_path):
    port = _free_port()
    times = [12.5, 20.0]
    mp.spawn(_rank, args=(2, port, times, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        t, v = (float(x) for x in (tmp_path / f"rank{r}.txt").read_text().split())
        assert t == 20.0
        assert v == pytest.approx(2 * 1000.0 / 0.020)


def test_single_process_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.replicas_value(500.0, 10.0, 1) == pytest.approx(50000.0)
