"""Checked mode: with tsds_checked on, every entry point that takes x verifies
on the device that x is sorted non-decreasing with no NaN before it launches
anything else.  An x out of order is rejected with TSDS_EINVAL naming the first
bad position, leaves the outputs untouched and launches only the check; an x in
order gives the same indices as the unchecked call.  (Unsorted x is only ever
passed with the mode on: the check runs and answers before any other kernel.)"""
import numpy as np
import pytest

import paper_2307_05389_gb300 as pkg
from paper_2307_05389_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

N = 100_003
ALGOS = ("minmax", "m4", "everynth", "lttb", "minmaxlttb")


@pytest.fixture
def checked():
    prev = pkg.tsds_checked(1)
    yield
    pkg.tsds_checked(prev)


def _series(x_dtype="int64"):
    y = inputs.random_walk(N, "float32", seed=91)
    if x_dtype == "int64":
        x = inputs.geometric_x(N, seed=92)
    else:
        x = inputs.exponential_x(N, seed=92).astype(x_dtype)
    return y, x


def _call(algo, y, x, n_out=1000):
    import torch
    out = torch.full((n_out + 8,), -3, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    binding.downsample(algo, y, n_out, x=x, out=out, out_count=cnt, sync=False)
    torch.cuda.synchronize()
    return out, cnt


@pytest.mark.parametrize("algo", ALGOS)
def test_sorted_x_gives_the_unchecked_result(algo, checked):
    import torch
    y, x = _series()
    x[10:20] = x[10]                               # repeats are in order
    dy, dx = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    out_c, cnt_c = _call(algo, dy, dx)
    pkg.tsds_checked(0)
    out_u, cnt_u = _call(algo, dy, dx)
    assert int(cnt_c.item()) == int(cnt_u.item()) > 0
    k = int(cnt_c.item())
    assert torch.equal(out_c[:k], out_u[:k])


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("x_dtype,bad", [("int64", 777), ("float64", 0), ("float32", N - 2)])
def test_unsorted_x_is_rejected_before_any_other_launch(algo, x_dtype, bad, checked):
    import torch
    y, x = _series(x_dtype)
    x[bad], x[bad + 1] = x[bad + 1], x[bad]        # x[bad] > x[bad+1]
    assert x[bad] > x[bad + 1]
    dy, dx = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    before = pkg.tsds_kernel_launches()
    with pytest.raises(binding.TsdsError) as e:
        _call(algo, dy, dx)
    assert e.value.status == 1
    assert f"i = {bad}" in str(e.value) and "checked mode" in str(e.value)
    assert pkg.tsds_kernel_launches() - before == 1


@pytest.mark.parametrize("pos", [0, 4321, N - 1])
def test_nan_in_x_is_rejected_at_its_position(pos, checked):
    import torch
    y, x = _series("float64")
    x[pos] = np.nan
    dy, dx = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    out = torch.full((1008,), -3, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    with pytest.raises(binding.TsdsError) as e:
        binding.downsample("minmax", dy, 1000, x=dx, out=out, out_count=cnt, sync=False)
    assert f"i = {pos}" in str(e.value)
    torch.cuda.synchronize()
    assert int(cnt.item()) == -7 and bool((out == -3).all())


def test_values_form_is_checked(checked):
    import torch
    y, x = _series()
    x[5000] = x[5001] + 3
    dy, dx = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    with pytest.raises(binding.TsdsError) as e:
        binding.downsample_values("m4", dy, 1000, x=dx)
    assert "i = 5000" in str(e.value)


def test_batched_names_the_series(checked):
    import torch
    ys, xs = [], []
    for i in range(5):
        y = inputs.random_walk(20_000 + 1000 * i, "float32", seed=100 + i)
        x = inputs.geometric_x(len(y), seed=200 + i)
        if i == 3:
            x[12_345] = x[12_346] + 1
        ys.append(torch.from_numpy(y).cuda())
        xs.append(torch.from_numpy(x).cuda())
    with pytest.raises(binding.TsdsError) as e:
        binding.downsample_batched("minmax", ys, [400] * 5, xs=xs)
    assert "series 3" in str(e.value) and "i = 12345" in str(e.value)
    with pytest.raises(binding.TsdsError):
        binding.Plan("m4", ys, [400] * 5, xs=xs)
    xs[3] = torch.from_numpy(inputs.geometric_x(len(ys[3]), seed=203)).cuda()
    outs, counts = binding.downsample_batched("minmax", ys, [400] * 5, xs=xs)
    torch.cuda.synchronize()
    assert all(int(c) > 0 for c in counts.cpu().numpy())


def test_server_rejects_an_unsorted_series(checked):
    import torch
    y = inputs.random_walk(50_000, "float32", seed=300)
    x = inputs.exponential_x(50_000, seed=301)
    srv = binding.Server("float32", "float64", streams=1, max_batch=8)
    try:
        good = srv.add_series(torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda())
        assert good == 0
        xb = x.copy()
        xb[100] = np.nan
        with pytest.raises(binding.TsdsError) as e:
            srv.add_series(torch.from_numpy(y).cuda(), torch.from_numpy(xb).cuda())
        assert "i = 100" in str(e.value)
    finally:
        srv.close()
