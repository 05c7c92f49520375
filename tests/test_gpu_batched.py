"""Batched form (one launch sequence for many series) vs the CPU oracle and vs
the single-series calls, index for index.  Batches mix sizes from empty to
several windows, n_out >= n series, and both algorithms; plans are executed
more than once, with graphs and autotuning, and re-executed after the data
changed in place (Section 2.2's consistency across threading configurations,
here across launch shapes)."""
import os
import numpy as np
import pytest

import oracle
from paper_2307_05389_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def make_batch(seed, count, dtype="float32", with_x=False, max_len=600_000):
    rng = np.random.default_rng(seed)
    lens = np.concatenate([[0, 1, 3, 17], rng.integers(1, max_len, count - 4)])
    lens[5] = max_len * 2 + 12345           # one series spanning many windows
    n_outs = (rng.integers(4, 4001, count) // 4) * 4
    n_outs[6] = 4
    ys = [inputs.random_walk(int(n), dtype, seed=seed * 1000 + i) if n else np.zeros(0, dtype) for i, n in enumerate(lens)]
    xs = [inputs.geometric_x(int(n), seed=seed * 1000 + i) for i, n in enumerate(lens)] if with_x else None
    return ys, xs, n_outs


def to_dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() if len(a) else torch.zeros(0, dtype=getattr(torch, a.dtype.name), device="cuda")
            for a in arrs]


def results(outs, counts):
    import torch
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    return [o[:int(k)].cpu().numpy() for o, k in zip(outs, c)]


@pytest.mark.parametrize("algo", ["minmax", "m4"])
@pytest.mark.parametrize("with_x", [False, True])
def test_batched_matches_oracle(algo, with_x):
    ys, xs, n_outs = make_batch(1 + with_x, 40, with_x=with_x)
    outs, counts = binding.downsample_batched(algo, to_dev(ys), n_outs, xs=to_dev(xs) if xs else None)
    got = results(outs, counts)
    for i, y in enumerate(ys):
        exp = oracle.downsample(algo, xs[i] if xs else None, y, int(n_outs[i]))
        np.testing.assert_array_equal(got[i], exp, err_msg=f"series {i} n={len(y)} n_out={n_outs[i]}")


@pytest.mark.parametrize("dtype", ["int8", "uint16", "float64", "float16"])
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
def test_batched_dtypes_and_nan(dtype, nan):
    rng = np.random.default_rng(7)
    ys = []
    for i in range(12):
        n = int(rng.integers(1000, 200_000))
        y = inputs.ties_and_specials(n, dtype, seed=i)
        ys.append(y)
    n_outs = np.full(len(ys), 200)
    outs, counts = binding.downsample_batched("minmax", to_dev(ys), n_outs, nan=nan, y_dtype=dtype)
    got = results(outs, counts)
    for i, y in enumerate(ys):
        np.testing.assert_array_equal(got[i], oracle.minmax(None, y, 200, nan))


@pytest.mark.parametrize("graph,autotune", [(False, False), (True, False), (True, True)])
def test_plan_executes_repeatedly_and_sees_new_data(graph, autotune):
    import torch
    ys, _, n_outs = make_batch(3, 30)
    dys = to_dev(ys)
    plan = binding.Plan("m4", dys, n_outs, graph=graph, autotune=autotune)
    for _ in range(2):
        got = results(*plan.execute())
        for i, y in enumerate(ys):
            np.testing.assert_array_equal(got[i], oracle.m4(None, y, int(n_outs[i])))
    # overwrite every series in place and execute again
    new = [inputs.random_walk(len(y), "float32", seed=99 + i) if len(y) else y for i, y in enumerate(ys)]
    for d, h in zip(dys, new):
        if len(h):
            d.copy_(torch.from_numpy(h))
    got = results(*plan.execute())
    for i, y in enumerate(new):
        np.testing.assert_array_equal(got[i], oracle.m4(None, y, int(n_outs[i])))
    info = plan.info()
    assert info["window_bytes"] % 16 == 0 and info["windows"] > 0
    plan.close()


def test_batched_equals_single_series_calls():
    ys, xs, n_outs = make_batch(4, 25, with_x=True)
    dys, dxs = to_dev(ys), to_dev(xs)
    outs, counts = binding.downsample_batched("minmax", dys, n_outs, xs=dxs)
    got = results(outs, counts)
    for i in range(len(ys)):
        if len(ys[i]) == 0:
            assert len(got[i]) == 0
            continue
        single = binding.downsample("minmax", dys[i], int(n_outs[i]), x=dxs[i])
        np.testing.assert_array_equal(got[i], single.cpu().numpy())


def test_batched_rejects_mixed_x_and_bad_n_out():
    import torch
    ys = to_dev([inputs.random_walk(100, "float32", 1), inputs.random_walk(100, "float32", 2)])
    xs = to_dev([inputs.geometric_x(100, 1), inputs.geometric_x(100, 2)])
    outs, counts = binding.batch_buffers(ys, [8, 8], ys[0].device)
    arr = binding._series_array(ys, [8, 8], xs, outs, counts)
    arr[1, 0] = 0                                      # series 1 without x
    assert binding.tsds_batched(0, binding._array_ptr(arr), 2, binding.DTYPES["int64"],
                                binding.DTYPES["float32"], 0, None) == 1
    assert "x" in binding.last_error()
    arr = binding._series_array(ys, [8, 6], None, outs, counts)
    assert binding.tsds_batched(1, binding._array_ptr(arr), 2, 0, binding.DTYPES["float32"], 0, None) == 1
    torch.cuda.synchronize()


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("algo", ["minmax", "m4"])
def test_split_pass_small_and_large_bins(graph, algo):
    """A batch with series in all three groups of the automatic variant (bins
    of tens of bytes: segmented windows; a few KB: a warp per bin; hundreds
    of KB: register-streaming windows) runs a launch per group; every series
    must still match the oracle, bins cut by windows included."""
    rng = np.random.default_rng(21)
    ys, n_outs = [], []
    for i in range(24):
        if i % 3 == 1:
            n = int(rng.integers(20_000, 90_000)); n_out = 4000    # bins of tens of bytes
        elif i % 3 == 2:
            n = int(rng.integers(100_000, 400_000)); n_out = 400   # bins of a few KB
        else:
            n = int(rng.integers(2_000_000, 3_000_000)); n_out = 40    # bins of hundreds of KB
        ys.append(inputs.ties_and_specials(n, "float32", seed=100 + i) if i % 4 == 0 else
                  inputs.random_walk(n, "float32", seed=100 + i))
        n_outs.append(n_out)
    n_outs = np.array(n_outs)
    dys = to_dev(ys)
    plan = binding.Plan(algo, dys, n_outs, graph=graph, autotune=False)
    assert plan.info()["variant"] == "auto"
    for _ in range(2):
        got = results(*plan.execute())
        for i, y in enumerate(ys):
            np.testing.assert_array_equal(got[i], oracle.downsample(algo, None, y, int(n_outs[i])),
                                          err_msg=f"series {i}")
    plan.close()
    outs, counts = binding.downsample_batched(algo, dys, n_outs)
    got = results(outs, counts)
    for i, y in enumerate(ys):
        np.testing.assert_array_equal(got[i], oracle.downsample(algo, None, y, int(n_outs[i])))


@pytest.mark.parametrize("algo", ["minmax", "m4"])
def test_batched_with_x_and_many_bins(algo):
    """A batch mixing series with thousands of x-space bins and series with a handful."""
    ys, xs, _ = make_batch(9, 24, with_x=True, max_len=300_000)
    rng = np.random.default_rng(10)
    per = 2 if algo == "minmax" else 4
    n_outs = rng.choice([4, 8, 60, 400, 4000, 20_000, 60_000], len(ys)).astype(np.int64)
    n_outs[5] = 32_768 * per // 2         # the long series: >= 4096 bins either way
    n_outs = (n_outs // per) * per
    outs, counts = binding.downsample_batched(algo, to_dev(ys), n_outs, xs=to_dev(xs))
    got = results(outs, counts)
    for i, y in enumerate(ys):
        exp = oracle.downsample(algo, xs[i], y, int(n_outs[i]))
        np.testing.assert_array_equal(got[i], exp, err_msg=f"series {i} n={len(y)} n_out={n_outs[i]}")


def test_graph_plan_created_first_in_a_fresh_process(tmp_path):
    """A graph plan made before any kernel of its sequence has run in the process (no autotune,
    so nothing runs before the capture): the capture must not fail, and the replay must give
    the one-shot batched call's output."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import torch\n"
        "from paper_2307_05389_gb300 import binding, inputs\n"
        "ys = [torch.from_numpy(inputs.random_walk(n, 'float32', seed=s)).cuda() for s, n in ((1, 200_000), (2, 5_000), (3, 2_000_000))]\n"
        "n_outs = [4000, 400, 1000]\n"
        "for algo in ('minmax', 'm4'):\n"
        "    plan = binding.Plan(algo, ys, n_outs, graph=True, autotune=False)\n"
        "    plan.execute(); torch.cuda.synchronize()\n"
        "    outs, counts = binding.downsample_batched(algo, ys, n_outs); torch.cuda.synchronize()\n"
        "    for i in range(3):\n"
        "        k = int(counts[i]); assert int(plan.counts[i]) == k\n"
        "        assert torch.equal(plan.outs[i][:k], outs[i][:k])\n"
        "    plan.close()\n"
        "print('ok')\n" % root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]
