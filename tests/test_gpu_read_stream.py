"""The read-only streaming probe reads every byte once: the XOR of all 8-byte
words it folds into the sink equals the XOR numpy computes on the host, for
sizes that end inside the unrolled body, in the remainder loop, and at one
vector."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nbytes", [16, 48, 4096 + 16, (1 << 20) + 16 * 37, 64 << 20, (200 << 20) + 16])
def test_read_stream_folds_every_word(nbytes):
    import torch

    import paper_2307_05389_gb300 as pkg
    rng = np.random.default_rng(nbytes)
    host = rng.integers(0, 2 ** 63, size=nbytes // 8, dtype=np.int64)
    buf = torch.from_numpy(host).cuda()
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    launches = pkg.tsds_kernel_launches()
    pkg.read_stream(buf, sink)
    torch.cuda.synchronize()
    assert pkg.tsds_kernel_launches() == launches + 1
    want = np.bitwise_xor.reduce(host.view(np.uint64))
    assert np.uint64(sink.cpu().numpy().view(np.uint64)[0]) == want


def test_read_stream_accumulates_into_the_sink():
    import torch

    import paper_2307_05389_gb300 as pkg
    host = np.arange(1, 1 + 4096, dtype=np.int64)
    buf = torch.from_numpy(host).cuda()
    sink = torch.full((1,), 0x5A5A, dtype=torch.int64, device="cuda")
    pkg.read_stream(buf, sink)
    pkg.read_stream(buf, sink)                       # twice: the fold cancels
    torch.cuda.synchronize()
    assert int(sink.item()) == 0x5A5A
