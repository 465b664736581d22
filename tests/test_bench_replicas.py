"""The bench's multi-GPU path is replicas only (one independent solve per rank, no data-path
collective): the host-side aggregation (max of the ranks' device times, whole-job value =
ranks x per-rank DOF x V-cycles / that time) checked with two gloo ranks on the CPU."""
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


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    times = [10.0, 25.0]  # ms of device time per rank
    dofv = 1.0e6          # DOF x V-cycles of one replica
    dist.barrier()
    tmax, value = bench.aggregate(times[rank], dofv, ws, dist, "cpu")
    out[rank] = (tmax, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        tmax, value = res[r]
        assert tmax == 25.0
        assert value == pytest.approx(ws * 1.0e6 / 25.0e-3)
