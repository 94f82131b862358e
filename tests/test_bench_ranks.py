"""The replicas path of bench.py with two gloo ranks on the CPU: whole-job
time is the slowest rank's, work is the sum over ranks; the reference arm
prints from rank 0 only."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        res = b.aggregate_ranks(10.0 + rank, 20.0 - rank, 1000.0 * (rank + 1), 7.0, world, torch.device("cpu"))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_aggregate_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert got[r] == (11.0, 20.0, 3000.0, 14.0)


def test_single_rank_passes_through():
    b = _bench()
    assert b.aggregate_ranks(1.0, 2.0, 3.0, 4.0, 1, None) == (1.0, 2.0, 3.0, 4.0)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    assert b.run_reference(None, None) is None
    assert capsys.readouterr().out == ""
