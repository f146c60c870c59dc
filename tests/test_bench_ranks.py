"""The bench's multi-rank host logic (one flow replica per GPU, no data-path collective) with
two gloo ranks on the CPU: the barrier, the max-over-ranks time and the whole-job throughput."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    b = _bench()
    assert b._dist() == (ws, rank, rank)
    b._sync_all(torch, ws, cuda=False)
    t = b._max_over_ranks(torch, times[rank], ws, device="cpu")
    b._sync_all(torch, ws, cuda=False)
    out[rank] = (t, b._job_throughput(1000.0, ws, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    times = [12.5, 17.0]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, times, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(ws):
        t, thr = out[r]
        assert t == max(times)
        assert thr == pytest.approx(1000.0 * ws / (max(times) * 1e-3))


def test_single_rank_is_a_no_op():
    b = _bench()
    assert b._max_over_ranks(torch, 3.0, 1) == 3.0
    assert b._job_throughput(10.0, 1, 2.0) == pytest.approx(5000.0)
