"""Batched MinMaxLTTB (tsds_batched_minmaxlttb): many series of uneven length
in one launch sequence give, series by series, exactly the oracle's MinMaxLTTB
(the preselection of Section 1 followed by LTTB), for both NaN modes, several
ratios, with and without x, including the degenerate series (empty, one or
two points, n_out >= n, a preselection that keeps every interior point)."""
import numpy as np
import pytest

import oracle
from paper_2307_05389_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

LENGTHS = [0, 1, 2, 3, 5, 17, 100, 999, 4000, 4003, 10_000, 65_537, 123_457, 400_000]
N_OUTS = [3, 4, 7, 100, 1000, 4000]


def _batch(dtype, seed, with_x):
    rng = np.random.default_rng(seed)
    ys, xs, n_outs = [], [], []
    for i, n in enumerate(LENGTHS):
        if dtype == "float64":
            y = inputs.quantised_nan(n, seed=seed + i) if n else np.zeros(0)
        else:
            y = inputs.random_walk(n, dtype, seed=seed + i)
        ys.append(y)
        xs.append(inputs.exponential_x(n, seed=seed + 100 + i) if with_x else None)
        n_outs.append(int(rng.choice(N_OUTS)))
    return ys, (xs if with_x else None), n_outs


@pytest.mark.parametrize("dtype,with_x", [("float64", False), ("float32", False), ("float64", True),
                                          ("float32", True)])
@pytest.mark.parametrize("nan", ["propagate", "ignore"])
@pytest.mark.parametrize("ratio", [1, 4, 30])
def test_batched_minmaxlttb_matches_the_oracle(dtype, with_x, nan, ratio):
    import torch
    ys, xs, n_outs = _batch(dtype, seed=500 + ratio, with_x=with_x)
    dys = [torch.from_numpy(np.ascontiguousarray(y)).cuda() for y in ys]
    dxs = [torch.from_numpy(x).cuda() for x in xs] if xs is not None else None
    outs, counts = binding.downsample_batched("minmaxlttb", dys, n_outs, xs=dxs, nan=nan, minmax_ratio=ratio,
                                              y_dtype=dtype, x_dtype="float64" if with_x else None)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    for i, y in enumerate(ys):
        want = oracle.minmaxlttb(xs[i] if xs is not None else None, y, n_outs[i], ratio, nan)
        got = outs[i][:int(c[i])].cpu().numpy()
        assert np.array_equal(got, want), f"series {i}: n={len(y)}, n_out={n_outs[i]}"


def test_batched_minmaxlttb_equals_single_calls_on_many_series():
    """300 series of log-uniform length in [10, 2e5]: the batched outputs equal the
    single-series calls one by one (the single-series path is itself oracle-checked)."""
    import torch
    rng = np.random.default_rng(77)
    lens = np.round(10 ** rng.uniform(1, 5.3, 300)).astype(np.int64)
    n_outs = [int(v) for v in rng.integers(3, 3000, 300)]
    walk = inputs.random_walk(int(lens.sum()), "float32", seed=78)
    offs = np.concatenate([[0], np.cumsum(lens)])
    dwalk = torch.from_numpy(walk).cuda()
    ys = [dwalk[int(offs[i]):int(offs[i + 1])] for i in range(len(lens))]
    outs, counts = binding.downsample_batched("minmaxlttb", ys, n_outs, minmax_ratio=4)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    for i, y in enumerate(ys):
        single = binding.downsample("minmaxlttb", y, n_outs[i], minmax_ratio=4).cpu().numpy()
        assert np.array_equal(outs[i][:int(c[i])].cpu().numpy(), single), f"series {i}"
