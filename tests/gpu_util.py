"""Helpers for the GPU tests: move seeded numpy inputs to the device as raw
bytes (any of the eleven dtypes) and call the C ABI through the binding."""
import numpy as np

from paper_2307_05389_gb300 import binding

ALGOS = ("minmax", "m4", "lttb", "minmaxlttb", "everynth")


class DevArray:
    """A numpy array's bytes on the GPU, optionally starting `offset_elems`
    elements past a 256-byte boundary (to exercise unaligned starts)."""

    def __init__(self, a, offset_elems=0):
        import torch
        a = np.ascontiguousarray(a)
        self.dtype = a.dtype.name
        self.n = a.shape[0]
        off = offset_elems * a.dtype.itemsize
        self.buf = torch.zeros(a.nbytes + off + 16, dtype=torch.uint8, device="cuda")
        if a.nbytes:
            self.buf[off:off + a.nbytes].copy_(torch.from_numpy(a.view(np.uint8).reshape(-1)))
        self.ptr = self.buf.data_ptr() + off


def call(algo, x, y, n_out, nan="propagate", ratio=4, stream=None, out_cap=None, offset=0):
    """Run one C ABI call; returns (status, indices or None)."""
    import torch
    yd = DevArray(y, offset)
    xd = DevArray(x, offset) if x is not None else None
    n = len(y)
    cap = out_cap if out_cap is not None else max(n, n_out, 1)
    out = torch.full((cap,), -7, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    import ctypes
    sp = ctypes.c_void_p(st.cuda_stream)
    xa = (xd.ptr if xd else None, binding.DTYPES[xd.dtype] if xd else 0)
    common = (*xa, yd.ptr, binding.DTYPES[yd.dtype], n, n_out)
    nm = binding.NAN_MODES[nan]
    if algo == "minmaxlttb":
        r = binding.tsds_minmaxlttb(*common, ratio, nm, out.data_ptr(), cnt.data_ptr(), sp)
    else:
        fn = {"minmax": binding.tsds_minmax, "m4": binding.tsds_m4, "lttb": binding.tsds_lttb,
              "everynth": binding.tsds_everynth}[algo]
        r = fn(*common, nm, out.data_ptr(), cnt.data_ptr(), sp)
    if r != 0:
        return r, None
    st.synchronize()
    k = int(cnt.item())
    res = out.cpu().numpy()
    assert k >= 0, "count not written"
    assert np.all(res[k:] == -7), "wrote past the count"
    return 0, res[:k]


def run(algo, x, y, n_out, nan="propagate", ratio=4, **kw):
    r, idx = call(algo, x, y, n_out, nan, ratio, **kw)
    assert r == 0, f"status {r}: {binding.last_error()}"
    return idx
