"""gridspt_power_noalloc: the shell power estimator for callers that cannot
allocate device memory (a host framework whose allocator owns the GPU memory,
or a plugin handed only its input and output buffers). Its per-block scratch is
a static array inside the library, so the caller passes inputs and outputs
only. Checked through the C ABI against gridspt_power (caller scratch) on two
calls in a row with different inputs, so that state left by the first call
cannot leak into the second. Both entry points run the same kernels with the
same fixed-order reductions, so the results must agree bit for bit. Collected
last on purpose."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1807_04215_gb300 import _lib  # noqa: E402
from paper_1807_04215_gb300 import gridspt as g  # noqa: E402

pytestmark = pytest.mark.gpu


def _call_noalloc(plan, a, b, edges):
    lib = _lib.load()
    e = (ctypes.c_double * len(edges))(*edges)
    nb = len(edges) - 1
    out = torch.full((nb,), -1.0, dtype=torch.float64, device="cuda")
    nk = torch.full((nb,), -1, dtype=torch.int64, device="cuda")
    st = lib.gridspt_power_noalloc(plan.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                   nb, e, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(nk.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check("gridspt_power_noalloc", st)
    return out, nk


def test_power_noalloc_matches_power_on_two_calls():
    N, L = 64, 500.0
    plan = g.Plan(N, 3, L, batch=2)
    d1 = g.make_linear_field(plan, [21, 22])
    spectra = g.run_orders(plan, d1)
    kF = 2 * math.pi / L
    edges1 = [kF * (b + 0.5) for b in range(17)]
    edges2 = [0.02 * (0.4 / 0.02) ** (i / 24) for i in range(25)]
    cases = [(d1[0], d1[0], edges1), (d1[1], spectra[1, 1, 0], edges2)]
    for a, b, edges in cases:
        got, nk = _call_noalloc(plan, a, b, edges)
        ref, nkr = g.power(plan, a, b, edges)
        torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(nk.cpu().numpy(), nkr.cpu().numpy())
        assert np.array_equal(got, ref)
        assert np.all(got[nkr.cpu().numpy() == 0] == 0)


def test_power_noalloc_rejects_too_many_bins():
    N, L = 32, 250.0
    plan = g.Plan(N, 3, L)
    d1 = g.make_linear_field(plan, [1])
    kF = 2 * math.pi / L
    edges = [kF * (0.5 + 15.0 * i / 65) for i in range(66)]   # 65 bins > 64
    with pytest.raises(_lib.GridsptError) as ei:
        _call_noalloc(plan, d1[0], d1[0], edges)
    assert ei.value.status == 1
    assert "nbins=65" in str(ei.value)
