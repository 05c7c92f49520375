"""Failure detection without a GPU fault: device allocations made to fail on
the host (tsds_inject_alloc_failures) surface as TSDS_ENOMEM with a message,
and the next call on the same context returns the oracle's result.  (The
bounded-wait path is covered by the wait-timeout test in the parity suite.)"""
import numpy as np
import pytest

import oracle
import paper_2307_05389_gb300 as pkg
from paper_2307_05389_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

ENOMEM = 2


@pytest.fixture
def series():
    import torch
    y = inputs.random_walk(300_003, "float32", seed=31)
    x = inputs.geometric_x(len(y), seed=32)
    return y, x, torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()


@pytest.mark.parametrize("algo", ["minmax", "m4", "lttb", "minmaxlttb", "everynth"])
@pytest.mark.parametrize("with_x", [False, True])
def test_single_series_allocation_failure(series, algo, with_x):
    y, x, dy, dx = series
    xs, dxs = (x, dx) if with_x else (None, None)
    pkg.tsds_inject_alloc_failures(1)
    try:
        with pytest.raises(binding.TsdsError) as e:
            binding.downsample(algo, dy, 1000, x=dxs)
        assert e.value.status == ENOMEM
        assert "memory" in str(e.value).lower()
    finally:
        pkg.tsds_inject_alloc_failures(0)
    got = binding.downsample(algo, dy, 1000, x=dxs).cpu().numpy()
    assert np.array_equal(got, oracle.downsample(algo, xs, y, 1000))


def test_batched_and_plan_allocation_failure():
    import torch
    ys = [inputs.random_walk(n, "float32", seed=40 + i) for i, n in enumerate((1000, 50_000, 250_000))]
    dys = [torch.from_numpy(y).cuda() for y in ys]
    n_outs = [100, 400, 2000]
    for make in (lambda: binding.downsample_batched("minmax", dys, n_outs),
                 lambda: binding.Plan("m4", dys, n_outs),
                 lambda: binding.downsample_batched("minmaxlttb", dys, n_outs)):
        pkg.tsds_inject_alloc_failures(1)
        try:
            with pytest.raises(binding.TsdsError) as e:
                make()
            assert e.value.status == ENOMEM
        finally:
            pkg.tsds_inject_alloc_failures(0)
    outs, counts = binding.downsample_batched("minmaxlttb", dys, n_outs)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    for i, y in enumerate(ys):
        assert np.array_equal(outs[i][:int(c[i])].cpu().numpy(), oracle.minmaxlttb(None, y, n_outs[i]))


def test_injection_counts_down_and_clears():
    import torch
    dy = torch.from_numpy(inputs.random_walk(10_000, "float32", seed=50)).cuda()
    pkg.tsds_inject_alloc_failures(2)
    try:
        for _ in range(2):
            with pytest.raises(binding.TsdsError):
                binding.downsample("minmax", dy, 100)
        assert len(binding.downsample("minmax", dy, 100)) > 0
        pkg.tsds_inject_alloc_failures(5)
        pkg.tsds_inject_alloc_failures(0)
        assert len(binding.downsample("minmax", dy, 100)) > 0
    finally:
        pkg.tsds_inject_alloc_failures(0)
