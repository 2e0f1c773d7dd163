"""Precision of the FP32 path (the 1024^3 precision workload's checks that fit
the rules: nothing computed by the GPU is fed to the oracle).

* 128^3 rerun at the same cell size as 1024^3 / L = 4000 Mpc/h (L = 500 Mpc/h),
  n_max = 5, against the FP64 oracle on the same FP32-rounded initial field:
  RMS relative error per order (all modes, in band |k| < K_c, above band) and
  per-bin error of the six P-terms (bins below and above K_c), with the shell
  sums in compensated FP32 and in FP64 (the accum choice), printed as one
  report line; the P-term bar is that of the 256^3 parity test (1e-5 per bin,
  or the bin's FP32 white-noise bound where that is larger).
* 1024^3, L = 4000 Mpc/h, n_max = 5 (about 250 GB of device memory, skipped
  when the device has less free): delta_2, theta_2 on an 8^3 block of cells
  against the oracle's direct FP64 mode sums from its own delta_1
  (oracle/cutout.py), mass conservation delta_n(0) = 0, exact 2^n scaling, and
  P11 (both accumulators) against the linear spectrum within its cosmic
  variance. Orders above 2 would need the full-grid lower orders in FP64 (or
  GPU fields as oracle input, which the rules exclude); their accumulated
  error is measured by the 128^3 rerun.
"""
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import cosmology, cutout, estimators, spt  # noqa: E402
from paper_1807_04215_gb300 import gridspt as g  # noqa: E402
from tests import fp32_floor, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _rms(got, ref, mask=None):
    N = ref.shape[0]
    r = ref[:, :, : N // 2]
    w = np.full(r.shape, 2.0)
    w[:, :, 0] = 1.0
    if mask is not None:
        w = w * mask[:, :, : N // 2]
    return float(math.sqrt(np.sum(w * np.abs(got - r) ** 2) / np.sum(w * np.abs(r) ** 2)))


def test_precision_128_rerun_report():
    N, L, n_max = 128, 500.0, 5
    ref1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, 1000)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    d1 = torch.from_numpy(inputs.full_to_half(ref1).astype(np.complex64)).cuda()
    plans = {acc: g.Plan(N, n_max, L, accum=acc) for acc in ("compensated", "fp64")}
    sp = g.run_orders(plans["compensated"], d1[None])
    got = sp.cpu().numpy().astype(np.complex128)
    dk, tk = spt.run_orders(ref1, L, n_max)
    sx, sy, sz = spt.wave_indices(N)
    band = ((sx ** 2 + sy ** 2 + sz ** 2) < (N / (n_max + 1)) ** 2).astype(float)
    report = {"fields_all_in_above": {}, "pterms": {}}
    for n in range(2, n_max + 1):
        for w, ref in ((0, dk[n]), (1, tk[n])):
            e = [_rms(got[0, n - 2, w], ref), _rms(got[0, n - 2, w], ref, band), _rms(got[0, n - 2, w], ref, 1 - band)]
            report["fields_all_in_above"][f"{'delta' if w == 0 else 'theta'}_{n}"] = [float(f"{v:.2e}") for v in e]
            assert e[0] < (1e-5 if n == 2 else 1e-4)
    edges = [0.01 * (0.4 / 0.01) ** (i / 32) for i in range(33)]
    kc = 2 * math.pi / L * N / (n_max + 1)
    below = np.array(edges[1:]) <= kc
    gd = {1: d1, **{n: sp[0, n - 2, 0] for n in range(2, n_max + 1)}}
    rd = {1: ref1, **{n: dk[n] for n in range(2, n_max + 1)}}
    full = {1: ref1, **{n: inputs.half_to_full(got[0, n - 2, 0]) for n in range(2, n_max + 1)}}
    s = fp32_floor.noise_levels(full, rd, fp32_floor.inband_mask(N, n_max), range(2, n_max + 1))
    for i, j in [(1, 1), (2, 2), (1, 3), (3, 3), (2, 4), (1, 5)]:
        f = 1.0 if i == j else 2.0
        pr, nkr = estimators.power(rd[i], rd[j], L, edges)
        pr = f * pr
        sig = fp32_floor.pterm_sigma(rd, s, i, j, L, edges)
        sel, bar, used = fp32_floor.pterm_bar(pr, sig, nkr)
        entry = {"bins_below_kc": int((sel & below).sum()), "bins_above_kc": int((sel & ~below).sum()),
                 "bins_on_fp32_floor": int((sel & used).sum())}
        for acc, plan in plans.items():
            p, _ = g.power(plan, gd[i], gd[j], edges)
            p = f * p.cpu().numpy()
            err = np.abs(p - pr)
            rel = np.where(sel, err / np.where(sel, np.abs(pr), 1.0), 0.0)
            assert np.all(err[sel] <= bar[sel]), ((i, j), acc, np.max(err[sel] / bar[sel]))
            entry[acc] = {"max_rel_below_kc": float(f"{rel[sel & below].max():.2e}") if (sel & below).any() else None,
                          "max_rel_above_kc": float(f"{rel[sel & ~below].max():.2e}") if (sel & ~below).any() else None,
                          "median_rel": float(f"{np.median(rel[sel]):.2e}"),
                          "bins_within_1e-5": int((rel[sel] <= 1e-5).sum())}
        report["pterms"][f"P{i}{j}"] = entry
    print("PRECISION_128_L500_NMAX5 " + json.dumps(report))


def test_1024_properties():
    N, L, n_max = 1024, 4000.0, 5
    torch.cuda.empty_cache()
    plan = g.Plan(N, n_max, L)
    need = plan.workspace_size() + 8 * N * N * (N // 2) * (2 * (n_max - 1) + 3)
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"1024^3 needs {need / 2**30:.0f} GiB free on the device, {free / 2**30:.0f} GiB are")
    d1 = g.make_linear_field(plan, [1000])
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device="cuda")
    sp = torch.empty(plan.half_shape(1, n_max - 1, 2), dtype=torch.complex64, device="cuda")
    g.run_orders(plan, d1, spectra=sp, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.make_linear_field(plan, [1000], out=d1)
    g.run_orders(plan, d1, spectra=sp, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rep = {"ms": round(ms, 1), "Mcells_orders_per_s": round(N ** 3 * n_max / ms / 1e3, 1), "mass": {}}
    for n in range(2, n_max + 1):
        # delta_n(0) = 0 exactly (mass conservation: the sources' k = 0 modes
        # cancel term by term on the grid); the library writes that value
        # instead of the FP32 rounding residue of the mean of the products
        for w in range(2):
            assert complex(sp[0, n - 2, w, 0, 0, 0].item()) == 0
        rep["mass"][n] = 0.0
    # n = 2 on an 8^3 block of cells against the oracle's direct FP64 mode sums
    # (its own delta_1 drawn mode by mode; nothing from the GPU run): RMS relative
    # error over the block, same bound as the field parity at n = 2
    sx, sy, sz, v = cutout.linear_modes(N, L, n_max, cosmology.DEFAULT_COSMO, 1000)
    origin = (300, 611, 17)
    d2o, t2o = cutout.second_order_at_block(sx, sy, sz, v, N, L, origin, size=8)
    del sx, sy, sz, v
    rep["cutout_n2"] = {}
    for which, ref in ((0, d2o), (1, t2o)):
        x = g.c2r(plan, sp[0, 0, which])
        blk = x[origin[0]:origin[0] + 8, origin[1]:origin[1] + 8, origin[2]:origin[2] + 8].double().cpu().numpy()
        del x
        rel = float(np.sqrt(np.mean((blk - ref) ** 2) / np.mean(ref ** 2)))
        rep["cutout_n2"]["delta_2" if which == 0 else "theta_2"] = float(f"{rel:.2e}")
        assert rel < 1e-5, (which, rel)
    torch.cuda.empty_cache()
    # exact 2^n scaling (every step is linear or a product; scaling by 2 is exact)
    # (a second spectra buffer does not fit beside the workspace: a slab of 16 kx
    # planes of every order is kept and compared bitwise)
    slab = sp[0, :, :, :16].clone()
    d2 = d1 * 2
    g.run_orders(plan, d2, spectra=sp, ws=ws)
    del d2
    for n in range(2, n_max + 1):
        assert torch.equal(sp[0, n - 2, :, :16], slab[n - 2] * (2.0 ** n))
    del slab, ws, sp
    torch.cuda.empty_cache()
    kF = 2 * math.pi / L
    edges = [kF * (b + 0.5) for b in range(4, 60, 4)]
    p, nk = g.power(plan, d1[0], d1[0], edges)
    p, nk = p.cpu().numpy(), nk.cpu().numpy()
    p64, _ = g.power(g.Plan(N, n_max, L, accum="fp64"), d1[0], d1[0], edges)
    p64 = p64.cpu().numpy()
    rep["p11_fp64_vs_compensated_max_rel"] = float(f"{np.max(np.abs(p64 / p - 1)):.2e}")
    assert np.all(np.abs(p64 - p) <= 1e-6 * np.abs(p64))
    # expectation: the linear spectrum averaged over the integer modes of each bin
    r = np.arange(-60, 61)
    s2 = (r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2).ravel().astype(np.float64)
    k = kF * np.sqrt(s2)
    idx = np.searchsorted(edges, k, side="right") - 1
    ok = (idx >= 0) & (idx < len(edges) - 1) & (s2 > 0)
    Pm = cosmology.linear_pk(k[ok], cosmology.DEFAULT_COSMO)
    expect = np.bincount(idx[ok], weights=Pm, minlength=len(edges) - 1) / np.bincount(idx[ok], minlength=len(edges) - 1)
    dev = np.abs(p / expect - 1) / np.sqrt(2.0 / nk)      # pairs +-k are one draw: N_k / 2 independent modes
    rep["p11_sigma_max"] = float(f"{dev.max():.2f}")
    assert dev.max() < 5
    print("PRECISION_1024_L4000_NMAX5 " + json.dumps(rep))
