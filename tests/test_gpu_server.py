"""Served form: viewport queries over resident series, continuous batching.

Each query's result must equal the oracle on the range it selects (indices
shifted to the whole series), and a query must return the same indices when
it runs alone as when it runs inside a mix of concurrently submitted queries
(the served analogue of the paper's consistency across threading
configurations, Section 2.2)."""
import threading

import numpy as np
import pytest

import oracle
from paper_2307_05389_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

N = 300_000


@pytest.fixture(scope="module")
def world():
    import torch
    ys = [inputs.random_walk(N, "float32", seed=60 + i) for i in range(3)]
    xs = [inputs.exponential_x(N, seed=70 + i) for i in range(3)]
    ys[2][::1013] = np.nan
    dys = [torch.from_numpy(y).cuda() for y in ys]
    dxs = [torch.from_numpy(x).cuda() for x in xs]
    srv = binding.Server("float32", "float64", streams=3, max_batch=64)
    ids = [srv.add_series(dy, dx) for dy, dx in zip(dys, dxs)]
    yield dict(ys=ys, xs=xs, srv=srv, ids=ids, keep=(dys, dxs))
    srv.close()


def expected(w, sid, algo, n_out, x_range=None, index_range=None, nan="propagate", ratio=4):
    y, x = w["ys"][sid], w["xs"][sid]
    if x_range is not None:
        lo = int(np.searchsorted(x, x_range[0], "left"))
        hi = int(np.searchsorted(x, x_range[1], "right"))
    else:
        lo, hi = max(0, index_range[0]), min(len(y), index_range[1])
        hi = max(hi, lo)
    r = oracle.downsample(algo, x[lo:hi], y[lo:hi], n_out, nan=nan, minmax_ratio=ratio)
    return r + lo


def random_queries(w, seed, count):
    rng = np.random.default_rng(seed)
    qs = []
    for _ in range(count):
        sid = int(rng.integers(0, 3))
        algo = ["minmax", "m4", "minmaxlttb"][int(rng.integers(0, 3))]
        n_out = int([500, 1000, 2000, 4000][int(rng.integers(0, 4))])
        nan = ["propagate", "ignore"][int(rng.integers(0, 2))]
        x = w["xs"][sid]
        span = int(10 ** rng.uniform(1, np.log10(N)))
        start = int(rng.integers(0, N - span + 1))
        if rng.random() < 0.7:
            q = dict(sid=sid, algo=algo, n_out=n_out, nan=nan, x_range=(x[start], x[start + span - 1]))
        else:
            q = dict(sid=sid, algo=algo, n_out=n_out, nan=nan, index_range=(start, start + span))
        qs.append(q)
    return qs


def submit(w, q):
    return w["srv"].submit(w["ids"][q["sid"]], q["algo"], q["n_out"], x_range=q.get("x_range"),
                           index_range=q.get("index_range"), nan=q["nan"])


def test_each_query_matches_the_oracle_on_its_range(world):
    qs = random_queries(world, 1, 120)
    tickets = [submit(world, q) for q in qs]
    for q, t in zip(qs, tickets):
        got, lat = world["srv"].result(t)
        exp = expected(world, q["sid"], q["algo"], q["n_out"], q.get("x_range"), q.get("index_range"), q["nan"])
        np.testing.assert_array_equal(got, exp, err_msg=str(q))
        assert lat > 0


def test_same_result_alone_and_in_a_mix(world):
    probe = dict(sid=1, algo="minmaxlttb", n_out=1000, nan="propagate", x_range=(world["xs"][1][1000], world["xs"][1][250_000]))
    alone, _ = world["srv"].result(submit(world, probe))
    mix = random_queries(world, 2, 300)
    results = {}

    def producer(part, tag):
        for i, q in enumerate(part):
            results[(tag, i)] = submit(world, q)
    # several threads submit concurrently; the probe goes in the middle
    threads = [threading.Thread(target=producer, args=(mix[k::3], k)) for k in range(3)]
    for t in threads:
        t.start()
    probe_ticket = submit(world, probe)
    for t in threads:
        t.join()
    in_mix, _ = world["srv"].result(probe_ticket)
    np.testing.assert_array_equal(in_mix, alone)
    np.testing.assert_array_equal(alone, expected(world, 1, "minmaxlttb", 1000, probe["x_range"]))
    for key, t in results.items():
        world["srv"].result(t)
    st = world["srv"].stats()
    assert st["completed"] >= 300 and st["batches"] >= 2 and st["p99_us"] >= st["p50_us"] > 0


def test_edge_ranges(world):
    srv = world["srv"]
    x = world["xs"][0]
    cases = [dict(index_range=(5, 5)), dict(index_range=(10, 11)), dict(index_range=(10, 12)),
             dict(index_range=(-50, 100)), dict(index_range=(N - 3, N + 100)),
             dict(x_range=(x[-1] + 1.0, x[-1] + 2.0)), dict(x_range=(x[100], x[100])),
             dict(x_range=(-1e30, 1e30))]
    for algo in ("minmax", "m4", "minmaxlttb"):
        for c in cases:
            t = srv.submit(world["ids"][0], algo, 8, **c)
            got, _ = srv.result(t)
            np.testing.assert_array_equal(got, expected(world, 0, algo, 8, c.get("x_range"), c.get("index_range")),
                                          err_msg=f"{algo} {c}")


def test_invalid_queries_rejected(world):
    srv = world["srv"]
    with pytest.raises(binding.TsdsError):
        srv.submit(world["ids"][0], "minmax", 5)
    with pytest.raises(binding.TsdsError):
        srv.submit(world["ids"][0], "m4", 6)
    with pytest.raises(binding.TsdsError):
        srv.submit(99, "minmax", 8)
    with pytest.raises(binding.TsdsError):
        srv.submit(world["ids"][0], "minmaxlttb", 2)


def test_tight_memory_budget_still_serves_everything():
    import torch
    y = inputs.random_walk(100_000, "float32", seed=80)
    srv = binding.Server("float32", streams=2, max_batch=8, memory_budget=200_000)
    dy = torch.from_numpy(y).cuda()
    sid = srv.add_series(dy)
    ts = [srv.submit(sid, "minmax", 100, index_range=(i * 1000, i * 1000 + 50_000)) for i in range(20)]
    for i, t in enumerate(ts):
        got, _ = srv.result(t)
        lo = i * 1000
        np.testing.assert_array_equal(got, oracle.minmax(None, y[lo:lo + 50_000], 100) + lo)
    srv.close()
