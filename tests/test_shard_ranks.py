"""Bin-range sharding on CPU ranks (gloo, world size 2 and 3): each rank takes its
bins from ``shard.shard_bins``, computes what those bins select with the oracle
(``oracle.binned_range``), and ``shard.gather_indices`` concatenates the ranks'
lists in rank order; the result must be the oracle's whole-series output.  x has
gaps and runs of equal values, so the cuts between ranks also fall where bins
are empty."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    from paper_2307_05389_gb300 import inputs
    rng = np.random.default_rng(90)
    n = 40_003
    y = inputs.random_walk(n, "float32", seed=91)
    y[rng.choice(n, 30, replace=False)] = np.nan
    gaps = rng.choice([0, 0, 1, 3, 500], size=n - 1)
    x = np.concatenate([[0], np.cumsum(gaps)]).astype(np.int64)
    out = []
    for algo in ("minmax", "m4"):
        for xx in (None, x):
            for n_out in (4, 400, 4000):
                out.append((algo, xx, y, n_out, "propagate" if n_out != 400 else "ignore"))
    return out


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2307_05389_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        results = []
        for algo, x, y, n_out, nan in _cases():
            nb = n_out // shard.PER_BIN[algo]
            b0, b1 = shard.shard_bins(nb, rank, world)
            local = torch.from_numpy(oracle.binned_range(algo, x, y, n_out, b0, b1, nan))
            results.append(shard.gather_indices(local).numpy())
        # an empty contribution from some ranks and a longer one from others
        local = torch.arange(rank * 3, dtype=torch.int64)
        results.append(shard.gather_indices(local).numpy())
        q.put((rank, results))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_bins_concatenate_to_the_whole_output(world):
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cases = _cases()
    for r in range(world):
        for (algo, x, y, n_out, nan), res in zip(cases, got[r]):
            np.testing.assert_array_equal(res, oracle.downsample(algo, x, y, n_out, nan), err_msg=f"{algo} {n_out}")
        np.testing.assert_array_equal(got[r][-1], np.concatenate([np.arange(k * 3) for k in range(world)]))


def test_shard_bins_partition():
    sys.path.insert(0, ROOT)
    from paper_2307_05389_gb300 import shard
    for nb in (0, 1, 5, 1000, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_bins(nb, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == nb
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
    with pytest.raises(ValueError):
        shard.shard_bins(10, 2, 2)
