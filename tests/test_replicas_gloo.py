"""The multi-GPU form of the benchmark is replicas (the sort does not shard
without an exchange step): each rank sorts its own copy and the job's step
time is the maximum over ranks.  The host-side aggregation is checked here
with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import importlib.util
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    ms, value = bench.aggregate_replicas(10.0 + 5.0 * rank, 1_000_000, 2, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, value = res[rank]
        assert ms == 15.0                                  # the slower rank's step time
        assert value == pytest.approx(2_000_000 / 0.015 / 1e9)   # both ranks' keys
