"""Multi-process host logic of the benchmark's replica mode, on CPU with the
gloo backend (world size 2): every rank times its own independent replica,
the job's step time is the slowest rank's, and the whole-job throughput
counts the units of all ranks.  No GPU and no data-path collective: the
product is not sharded; the one all-reduce is of the timing."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [3.0, 5.0, 4.0, 1.0][rank]
        ms, value = bench.replicas_value(local_ms, 1000, world, "cpu")
        q.put((rank, ms, value, bench.dist_env()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_take_the_slowest_rank(world):
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([3.0, 5.0, 4.0, 1.0][:world])
    for rank, ms, value, env in res:
        assert ms == slowest
        assert value == pytest.approx(world * 1000 / (slowest / 1e3))
        assert env == (rank, world, 0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replicas_value(2.0, 500, 1, "cpu")
    assert ms == 2.0 and value == pytest.approx(500 / 2e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    a = argparse.Namespace(n=1 << 20, d=32, k=16, steps=1, warmup=0, gpus=2)
    assert bench.run_reference(a) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    # rank 0 times the oracle and prints one JSON line with the keys the
    # benchmark contract asks of the reference arm (small n: seconds)
    sys.path.insert(0, ROOT)
    import argparse
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    a = argparse.Namespace(n=4096, d=8, k=4, steps=2, warmup=1, gpus=1, engine="auto")
    bench.run_reference(a)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["steps"] == 2
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
    assert rec["e2e"]["value"] == rec["value"] and rec["cpu_baseline"]["kind"] == "oracle"
    assert {"value", "unit", "cores", "kind", "sample"} <= set(rec["cpu_baseline"])
