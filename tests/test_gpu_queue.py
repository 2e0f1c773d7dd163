"""Persistent work queue (gridspt_multi_create / gridspt_run_orders_multi): the
recursion of plans of different grid sizes in one launch of one persistent
kernel, bit for bit equal to gridspt_run_orders of each plan; the bounded waits
report a stalled stage as GRIDSPT_E_TIMEOUT (the stall is planted on the host:
one stage never counts its tiles done); unsupported requests are refused."""
import math
import os

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1807_04215_gb300 import _lib  # noqa: E402
from paper_1807_04215_gb300 import gridspt as g  # noqa: E402

pytestmark = pytest.mark.gpu


def _eager(plans, d1s):
    out = []
    for p, d in zip(plans, d1s):
        out.append(g.run_orders(p, d).clone())
    return out


def _queue(plans, d1s):
    m = g.Multi(plans, d1s)
    sp = m.launch()
    torch.cuda.synchronize()
    for p in plans:
        g.check(p)
    res = [x.clone() for x in sp]
    m.close()
    return res


@pytest.mark.parametrize("tuning", [None, (0, 0, 0, 0, 0)])
def test_mixed_sizes_in_one_launch_equal_separate_runs(tuning):
    """128^3, 192^3 and 256^3 at the same cell size (L = 500, 750, 1000 Mpc/h),
    two realisations each, n_max = 5: one launch, bitwise equal to separate runs
    (each with its own tile choices: autotuned, or the default tiles)."""
    sizes = [(128, 500.0), (192, 750.0), (256, 1000.0)]
    plans = [g.Plan(n, 5, L, batch=2) for n, L in sizes]
    for p in plans:
        if tuning is None:
            g.autotune(p)
        else:
            g.set_tuning(p, list(tuning))
    d1s = [g.make_linear_field(p, [2000 + 10 * i, 2001 + 10 * i]) for i, p in enumerate(plans)]
    ref = _eager(plans, d1s)
    got = _queue(plans, d1s)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


@pytest.mark.parametrize("kw", [dict(n_max=3), dict(n_max=8), dict(n_max=5, truncate=True),
                                dict(n_max=4, kcut_nl=0.3), dict(n_max=5, kcut_lin=0.12)])
def test_queue_options_equal_separate_runs(kw):
    """Other orders and cuts (band-limited orders, higher-order cut, truncated
    orders, the 8th order's split pair launches) on 64^3 and 96^3 grids."""
    n_max = kw.pop("n_max")
    plans = [g.Plan(64, n_max, 250.0, **kw), g.Plan(96, n_max, 375.0, **kw)]
    d1s = [g.make_linear_field(p, [7 + i]) for i, p in enumerate(plans)]
    ref = _eager(plans, d1s)
    got = _queue(plans, d1s)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_resume_through_the_queue():
    """start_order > 2: the queue resumes from stored lower orders like run_orders."""
    plan = g.Plan(64, 5, 250.0)
    d1 = g.make_linear_field(plan, [3])
    full = g.run_orders(plan, d1).clone()
    part = full.clone()
    part[:, 2:] = 0
    m = g.Multi([plan], [d1], spectra=[part], start_orders=[4])
    m.launch()
    torch.cuda.synchronize()
    m.close()
    assert torch.equal(part, full)


def test_stalled_stage_times_out_and_is_reported(monkeypatch):
    """A stage that never counts its tiles done (planted on the host): the tiles
    waiting for it give up after their limit, the status word of plans[0]
    reports GRIDSPT_E_TIMEOUT, every block returns, and the next queue runs
    normally."""
    plans = [g.Plan(64, 3, 250.0), g.Plan(96, 3, 375.0)]
    d1s = [g.make_linear_field(p, [1 + i]) for i, p in enumerate(plans)]
    monkeypatch.setenv("GRIDSPT_FAULT_INJECT", "queue_stall")
    m = g.Multi(plans, d1s)
    monkeypatch.delenv("GRIDSPT_FAULT_INJECT")
    m.launch()
    with pytest.raises(_lib.GridsptError) as ei:
        g.check(plans[0])
    assert ei.value.status == 5
    m.close()
    g.check(plans[0])                          # reset by the previous check
    ref = _eager(plans, d1s)
    got = _queue(plans, d1s)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_unsupported_requests_are_refused():
    """A size the queue kernel has no tile bodies for, and the divergence form:
    GRIDSPT_E_UNSUPPORTED before anything is read or launched."""
    import ctypes
    lib = _lib.load()
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    for plan in (g.Plan(512, 3, 2000.0), g.Plan(64, 3, 250.0, form="divergence")):
        one = lambda T, x: (T * 1)(x)  # noqa: E731
        h = ctypes.c_void_p()
        st = lib.gridspt_multi_create(one(ctypes.c_void_p, plan.handle.value), 1, one(ctypes.c_void_p, ptr.value),
                                      None, one(ctypes.c_void_p, ptr.value), one(ctypes.c_void_p, ptr.value),
                                      one(ctypes.c_size_t, 64), ctypes.byref(h))
        assert st == 2 and not h.value
