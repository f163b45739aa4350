"""The multi-GPU bench path runs independent replicas (a single problem does
not shard): each rank times its own cycles, rank 0 reports the slowest rank's
time and the DoFs of all replicas.  The host logic runs here as 2 gloo ranks
on CPU; the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out.put((rank, ms, bench.replicas_value(ws, 1000, 10, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank_and_all_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [12.5, 20.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 20.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.020)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    assert bench.replicas_value(1, 2364419, 100, 180.0) == pytest.approx(2364419 * 100 / 0.18)


def test_reference_arm_works_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    W = dict(bench.WORKLOADS["2d512"])

    class A:
        steps, warmup, gpus = 1, 1, 2
    assert bench.run_reference(A(), W) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the contract's keys, on a 64^2 3-level size override so
    that it finishes in seconds here."""
    import json
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3", "--warmup", "3",
           "--N", "64", "--levels", "3"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "V-cycle DoFs/s" and d["unit"] == "DoF/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 3 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["vs_baseline"] is None
    assert d["config"]["levels"] == 3 and "size override" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
