"""The benchmark's multi-rank path on CPU: two gloo ranks (torchrun-style
environment, 127.0.0.1 rendezvous) time different local durations; the
reported time is the slowest rank's and the whole-job throughput counts every
rank's units (weak scaling, independent replicas)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_init("gloo")
    bench.barrier(w)
    local_ms = 10.0 * (r + 1)  # rank 1 is the slow one
    ms, value = bench.weak_scaling_value(local_ms, w, units_per_rank=1000, steps=4)
    out.put((r, w, ms, value))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_two_gloo_ranks(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms, value in res:
        assert w == ws
        assert ms == 20.0                                  # max over ranks
        assert value == pytest.approx(ws * 1000 * 4 / 0.020)  # all ranks' units / slowest time
