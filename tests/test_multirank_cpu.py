"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).

Each rank fits its own replica (weak scaling); the only collectives are the
barrier and the max over ranks of the step times.  These tests run the
cross-rank reduction and the whole-job rate on two processes, and check that
the reference arm prints only on rank 0.
"""
import io
import os
import socket
import sys
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [0.5 + rank, 0.1 * (world - rank)]  # rank 1 has the slower fit, rank 0 the slower evaluate
    got = bench.reduce_max(local, dist, device="cpu")
    value = bench.job_throughput(world, 1_000_000, got[0])
    dist.barrier()
    q.put((rank, got, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    for rank, got, value in res:
        assert got == [1.5, 0.2]
        assert value == pytest.approx(2 * 1_000_000 / 1.5)


def test_reduce_max_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 1.0]) == [3.0, 1.0]
    assert bench.job_throughput(1, 10, 2.0) == 5.0


def test_reference_arm_prints_only_on_rank_zero():
    sys.path.insert(0, ROOT)
    import bench
    args = bench.argparse.Namespace(ref_points=2000, workload="scale", warmup=0, steps=1)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, rank=1, world=2)
    assert buf.getvalue() == ""
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, rank=0, world=2)
    line = buf.getvalue().strip()
    import json
    d = json.loads(line)
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_command_line_contract():
    # the reference arm as the benchmark is launched: one JSON line with every
    # key of the contract, the oracle's own CPU timing in cpu_baseline
    import json
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--ref-points", "3000"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
