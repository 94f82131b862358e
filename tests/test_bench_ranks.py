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


def test_reference_arm_line_carries_the_contract_keys(monkeypatch, capsys):
    """The reference arm (the FP64 oracle on all host cores) prints one JSON
    line with the same metric and unit as the GPU arm, its own cpu_baseline
    and an e2e object without host-device traffic."""
    import json
    import types
    from paper_2405_02914_gb300 import inputs as I
    b = _bench()
    monkeypatch.setenv("RANK", "0")
    args = types.SimpleNamespace(gpus=1, steps=2, warmup=3)
    b.run_reference(args, I.scene_small(cx=8, cy=8, cz=4, n_press=10))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == b.METRIC and d["unit"] == b.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2
    import oracle as O
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == O.threads()
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_phases_of_the_press_slip_rotate_trajectory():
    """The bench splits its timed frames by the trajectory's phases, read
    from the keyframes (press 5000, slip 7500, rotate 7500 substeps)."""
    from paper_2405_02914_gb300 import inputs as I
    b = _bench()
    ph = b._phases(I.scene_pad4m().keyframes)
    assert ph[:3] == [("press", 0, 5000), ("slip", 5000, 12500), ("rotate", 12500, 20000)]
    assert ph[3][0] == "hold" and ph[3][1] == 20000
