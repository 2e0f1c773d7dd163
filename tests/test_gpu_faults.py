"""Failure handling without faulting a GPU: injected host-side failures
(GRIDSPT_FAULT_INJECT) must surface as status codes with no leak, leave the
context usable, and later calls must give correct results."""
import os

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1807_04215_gb300 import _lib  # noqa: E402
from paper_1807_04215_gb300 import gridspt as g  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture
def inject(monkeypatch):
    def set_(v):
        monkeypatch.setenv("GRIDSPT_FAULT_INJECT", v)
    yield set_
    monkeypatch.delenv("GRIDSPT_FAULT_INJECT", raising=False)


def test_plan_allocation_failure_reports_nomem_without_leak(inject):
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    inject("plan_alloc")
    for _ in range(200):
        with pytest.raises(_lib.GridsptError) as ei:
            g.Plan(64, 3, 500.0)
        assert ei.value.status == 3          # GRIDSPT_E_NOMEM
    os.environ.pop("GRIDSPT_FAULT_INJECT")
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 2 << 20            # the first allocation was released each time


def test_launch_failure_is_reported_and_recoverable(inject):
    plan = g.Plan(32, 3, 250.0)
    d1 = g.make_linear_field(plan, [3])
    ref = g.run_orders(plan, d1).clone()
    inject("launch")
    with pytest.raises(_lib.GridsptError) as ei:
        g.run_orders(plan, d1)
    assert ei.value.status == 4              # GRIDSPT_E_CUDA
    assert "launch" in str(ei.value)
    os.environ.pop("GRIDSPT_FAULT_INJECT")
    assert torch.equal(g.run_orders(plan, d1), ref)


def test_invalid_arguments_are_rejected_before_any_launch():
    plan = g.Plan(32, 3, 250.0)
    d1 = g.make_linear_field(plan, [3])
    spectra = torch.empty(plan.half_shape(1, 2, 2), dtype=torch.complex64, device="cuda")
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    lib = _lib.load()
    import ctypes
    st = lib.gridspt_run_orders(plan.handle, ctypes.c_void_p(d1.data_ptr()), 2, ctypes.c_void_p(spectra.data_ptr()),
                                ctypes.c_void_p(small.data_ptr()), 16, None)
    assert st == 1 and b"workspace" in lib.gridspt_last_error()
    st = lib.gridspt_run_orders(plan.handle, ctypes.c_void_p(d1.data_ptr() + 4), 2,
                                ctypes.c_void_p(spectra.data_ptr()), ctypes.c_void_p(small.data_ptr()), 16, None)
    assert st == 1 and b"aligned" in lib.gridspt_last_error()
    kF = 6.283185307179586 / 250.0
    with pytest.raises(_lib.GridsptError):
        g.power(plan, d1[0], d1[0], [kF * i for i in range(40)])     # above the Nyquist wavenumber
    with pytest.raises(_lib.GridsptError):
        g.bispectrum(plan, d1[0], d1[0], [kF * i for i in range(20)])  # shells beyond 2 k_Ny / 3


def test_bounded_device_wait_reports_timeout_and_context_stays_usable():
    """A device wait that nothing completes gives up after its limit, the status
    word reports it (GRIDSPT_E_TIMEOUT), and the next calls work."""
    import ctypes
    plan = g.Plan(32, 3, 250.0)
    g.check(plan)
    lib = _lib.load()
    assert lib.gridspt_selftest_bounded_wait(plan.handle, None) == 0
    with pytest.raises(_lib.GridsptError) as ei:
        g.check(plan)
    assert ei.value.status == 5
    g.check(plan)                       # status was reset
    d1 = g.make_linear_field(plan, [3])
    a = g.run_orders(plan, d1).clone()
    assert torch.equal(g.run_orders(plan, d1), a)
    g.check(plan)
    del ctypes


def test_non_finite_estimator_result_is_reported_as_numeric():
    """A NaN planted in an input spectrum (inside a bin) makes that bin's power
    NaN; gridspt_check reports GRIDSPT_E_NUMERIC once and resets, and the next
    call on finite inputs is correct and clean. Same for the bispectrum."""
    import math
    N, L = 32, 250.0
    plan = g.Plan(N, 3, L)
    d1 = g.make_linear_field(plan, [5])
    kF = 2 * math.pi / L
    edges = [kF * (b + 0.5) for b in range(9)]
    ref, _ = g.power(plan, d1[0], d1[0], edges)
    ref = ref.clone()
    g.check(plan)
    bad = d1[0].clone()
    bad[3, 0, 0] = complex(float("nan"), 0.0)          # |s| = 3: bin 2
    p, _ = g.power(plan, bad, bad, edges)
    assert math.isnan(float(p[2])) and torch.isfinite(p[:2]).all()
    with pytest.raises(_lib.GridsptError) as ei:
        g.check(plan)
    assert ei.value.status == 6                       # GRIDSPT_E_NUMERIC
    g.check(plan)                                     # reset by the previous check
    again, _ = g.power(plan, d1[0], d1[0], edges)
    assert torch.equal(again, ref)
    g.check(plan)
    kc = kF * N / 4
    bed = [kc * i / 4 for i in range(5)]
    E, _ = g.bispectrum(plan, bad, d1[0], bed)
    with pytest.raises(_lib.GridsptError) as ei:
        g.check(plan)
    assert ei.value.status == 6
    E, _ = g.bispectrum(plan, d1[0], d1[0], bed)
    g.check(plan)
    assert torch.isfinite(E).all()
