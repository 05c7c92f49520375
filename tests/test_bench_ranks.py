"""The multi-rank path of bench.py on CPU: two gloo ranks time different
amounts of work; the job's numbers must be the slowest rank's time and the
bytes of all ranks (weak scaling, no collective on the data path)."""
import multiprocessing as mp
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
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r spends (r + 1) ms on (r + 1) GB
        q.put((rank, bench.aggregate_ranks(float(rank + 1), (rank + 1) * 1e9, dist)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_bytes():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, total, gbps = out[r]
        assert ms == 2.0
        assert total == 3e9
        assert abs(gbps - 3e9 / 2e-3 / 1e9) < 1e-9


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(4.0, 8e9) == (4.0, 8e9, 2000.0)


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the CPU oracle on the host cores) prints one JSON line with
    the keys the benchmark contract names, on the headline workload's metric and config."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GB/s"
    assert d["config"]["workload"] == bench.WORKLOAD and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
