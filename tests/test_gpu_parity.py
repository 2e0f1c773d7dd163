"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 fields and transforms against FP64):
* fields: RMS relative error over all modes (= over all cells, Parseval)
  <= 1e-5 at n = 2 and <= 1e-4 at every n <= 5;
* initial field: FP64 arithmetic rounded to FP32 on the GPU, so each mode within
  2^-23 relative of the oracle (a few ulp of headroom);
* shell power estimator on identical inputs: <= 1e-5 relative per bin; N_k
  bit-exact (integer counting); P-terms from GPU fields: <= 1e-5 relative per
  bin for P11 and P22, and per bin within max(1e-5 |P|, 6 sigma_b) for the
  loop terms P13, P33, P24, P15, sigma_b the bin's white-noise bound at the GPU's own field
  noise level (tests/fp32_floor.py), that level within 1.5 times an
  independent FP32 implementation's;
* bispectrum: N_tri within FP32 rounding of the cubes, E within 1e-4 of its
  scale (FP32 shell fields, Kahan/FP64 sums);
* transforms alone: RMS relative error <= 2e-6.
Inputs to the recursion are the oracle's FP64 initial field rounded to FP32, so
that both sides start from the same numbers; nothing computed by the GPU is
ever fed to the oracle.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import cosmology, estimators, spt  # noqa: E402
from paper_1807_04215_gb300 import gridspt as g  # noqa: E402
from tests import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
COSMO = cosmology.DEFAULT_COSMO


def to_dev(full):
    half = inputs.full_to_half(full).astype(np.complex64)
    return torch.from_numpy(half).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def rms_rel(got_half, ref_full):
    """Parseval-weighted RMS relative error of a half spectrum vs a full grid."""
    N = ref_full.shape[0]
    ref = ref_full[:, :, : N // 2]
    w = np.full(ref.shape, 2.0)
    w[:, :, 0] = 1.0
    num = np.sum(w * np.abs(got_half - ref) ** 2)
    den = np.sum(w * np.abs(ref) ** 2)
    return math.sqrt(num / den)


# ------------------------------------------------------------- initial field
@pytest.mark.parametrize("N,L,n_max,seed", [(64, 500.0, 3, 1000), (48, 300.0, 5, 7), (12, 100.0, 2, 3)])
def test_linear_field_matches_oracle(N, L, n_max, seed):
    plan = g.Plan(N, n_max, L)
    d1 = host(g.make_linear_field(plan, [seed])[0])
    ref = spt.linear_field(N, L, n_max, COSMO, seed)[:, :, : N // 2]
    assert np.array_equal(d1 != 0, ref != 0)          # identical cut / Nyquist decisions
    assert np.abs(d1 - ref).max() <= 2.0 ** -23 * 4 * np.abs(ref).max()
    nz = ref != 0
    assert np.max(np.abs(d1[nz] - ref[nz]) / np.abs(ref[nz])) < 4e-7


def test_linear_field_batch_uses_each_seed():
    N, L = 32, 200.0
    plan = g.Plan(N, 3, L, batch=3)
    d = g.make_linear_field(plan, [5, 6, 7])
    for b, s in enumerate([5, 6, 7]):
        ref = spt.linear_field(N, L, 3, COSMO, s)[:, :, : N // 2]
        assert np.abs(host(d[b]) - ref).max() <= 1e-6 * np.abs(ref).max()


# ------------------------------------------------------------- transforms
@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256])
def test_c2r_matches_oracle(N):
    plan = g.Plan(N, 2, 100.0)
    full = spt.forward(inputs.random_real((N, N, N), N))
    full[spt.nyquist_mask(N)] = 0
    got = g.c2r(plan, to_dev(full)).cpu().numpy().astype(np.float64)
    ref = spt.backward(full).real
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-6


@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256])
def test_r2c_matches_oracle(N):
    plan = g.Plan(N, 2, 100.0)
    x = inputs.random_real((2, N, N, N), 100 + N)
    got = g.r2c(plan, torch.from_numpy(x.astype(np.float32)).cuda())
    for f in range(2):
        ref = spt.forward(x[f].astype(np.float32).astype(np.float64))
        ref[spt.nyquist_mask(N)] = 0
        assert rms_rel(host(got[f]), ref) < 2e-6


def test_c2r_in_place_equals_out_of_place():
    N = 64
    plan = g.Plan(N, 2, 100.0)
    full = spt.forward(inputs.random_real((N, N, N), 9))
    full[spt.nyquist_mask(N)] = 0
    a = to_dev(full)
    out = g.c2r(plan, a)
    b = a.clone()
    g.c2r(plan, b, out=b.view(torch.float32).view(N, N, N))
    assert torch.equal(out, b.view(torch.float32).view(N, N, N))


# ------------------------------------------------------------- recursion
def _parity_case(N, L, n_max, seed, kcut_nl=0.0, kcut_lin=0.0):
    plan = g.Plan(N, n_max, L, kcut_lin=kcut_lin, kcut_nl=kcut_nl)
    ref1 = spt.linear_field(N, L, n_max, COSMO, seed, kcut_lin=kcut_lin or None)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))  # FP32-rounded input
    spectra = g.run_orders(plan, to_dev(ref1)[None])
    dk, tk = spt.run_orders(ref1, L, n_max, kcut_nl=kcut_nl or None)
    errs = {}
    for n in range(2, n_max + 1):
        for which, ref in ((0, dk[n]), (1, tk[n])):
            errs[(n, which)] = rms_rel(host(spectra[0, n - 2, which]), ref)
    return errs


@pytest.mark.parametrize("N,L,n_max,seed", [
    (64, 500.0, 3, 1000),    # 64^3, L = 500, n_max = 3 workload
    (32, 250.0, 4, 11),
    (48, 300.0, 5, 12),      # radix-3 path, ragged tiles
    (24, 150.0, 5, 13),
    (96, 400.0, 3, 14),
])
def test_recursion_matches_oracle(N, L, n_max, seed):
    errs = _parity_case(N, L, n_max, seed)
    for (n, which), e in errs.items():
        tol = 1e-5 if n == 2 else 1e-4
        assert e < tol, (n, which, e)


@pytest.mark.parametrize("N,L,n_max,form", [(8, 60.0, 2, "nine_term"), (16, 100.0, 2, "nine_term"),
                                              (12, 80.0, 3, "nine_term"), (8, 60.0, 3, "divergence"),
                                              (12, 80.0, 2, "divergence")])
def test_smallest_grids_and_lowest_orders(N, L, n_max, form):
    """Degenerate ends: the smallest grids (N = 8, and N = 12 with its 6-point
    row transform) and n_max = 2 (only the diagonal pair, no fused z-pass
    pairs), in both source forms, against the oracle."""
    plan = g.Plan(N, n_max, L, form=form)
    ref1 = spt.linear_field(N, L, n_max, COSMO, 5)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    sp = g.run_orders(plan, to_dev(ref1)[None])
    oracle = spt.run_orders if form == "nine_term" else spt.run_orders_divergence
    dk, tk = oracle(ref1, L, n_max)
    for n in range(2, n_max + 1):
        for which, ref in ((0, dk[n]), (1, tk[n])):
            assert rms_rel(host(sp[0, n - 2, which]), ref) < (1e-5 if n == 2 else 1e-4), (n, which)


def test_first_order_only_is_a_no_op():
    """n_max = 1: there is nothing to form beyond delta_1; run_orders accepts an
    empty spectra array and a zero-byte workspace."""
    plan = g.Plan(16, 1, 100.0)
    assert plan.workspace_size() == 0
    d1 = g.make_linear_field(plan, [3])
    sp = g.run_orders(plan, d1)
    assert sp.numel() == 0


@pytest.mark.slow
def test_recursion_matches_oracle_128_fifth_order():
    errs = _parity_case(128, 500.0, 5, 21)
    for (n, which), e in errs.items():
        assert e < (1e-5 if n == 2 else 1e-4), (n, which, e)


def test_recursion_with_a_cut_above_nyquist_matches_oracle():
    """A linear cut past every grid mode (0.99 sqrt(3) k_Ny): order 1 moves every
    column (the band covers the grid) and the initial field's amplitude table
    stops at the largest |s|^2 on the grid; products fold, identically on both
    sides."""
    N, L = 24, 150.0
    kny = math.pi * N / L
    errs = _parity_case(N, L, 3, 61, kcut_lin=0.99 * math.sqrt(3.0) * kny)
    for (n, which), e in errs.items():
        assert e < (1e-5 if n == 2 else 1e-4), (n, which, e)


def test_recursion_with_nonlinear_cut_matches_oracle():
    kF = 2 * math.pi / 300.0
    errs = _parity_case(48, 300.0, 4, 31, kcut_nl=kF * 14.5, kcut_lin=kF * 9.0)
    for (n, which), e in errs.items():
        assert e < 1e-4, (n, which, e)


def test_single_plane_wave_closed_form_on_gpu():
    """Zel'dovich closed form of a 1D wave at every order (FP32 tolerance)."""
    N, L, A = 32, 100.0, 0.1
    plan = g.Plan(N, 5, L)
    d1 = to_dev(inputs.plane_waves(N, [((1, 0, 0), A)]))[None]
    spectra = g.run_orders(plan, d1)
    for n in range(2, 6):
        exp = np.zeros((N, N, N // 2), complex)
        for m in range(n % 2, n + 1, 2):
            j = (n - m) // 2
            v = (-1) ** j * m ** n * (A / 2) ** n / (math.factorial(j) * math.factorial(m + j))
            exp[m % N, 0, 0] = v
            exp[-m % N, 0, 0] = v
        for which in (0, 1):
            got = host(spectra[0, n - 2, which])
            assert np.abs(got - exp).max() < 1e-5 * (A / 2) ** n * 2 ** n, (n, which)


@pytest.mark.parametrize("N,n_max,s", [(768, 5, (12, 24, 36)), (1024, 3, (16, -8, 8))])
def test_oblique_plane_wave_closed_form_large_grid(N, n_max, s):
    """Zel'dovich closed form of one oblique wave on the largest grids, where the
    fused z pass runs with its reduced row tile. The spectrum is built and
    checked on the device (a dense host copy would take gigabytes): harmonic m
    of order n sits at m s (kz > 0 for every stored harmonic), every other mode
    must vanish.

    The wave number scales with N: FP32 rounding leaves a noise floor at all
    wave numbers, and every order's gradients raise it by up to k_Ny / |k_s|
    relative to the wave, so a long wave on a large grid (k_Ny / |k_s| ~ 100)
    shows 1e-4 off-harmonic residuals at n = 5 that are rounding, not error.
    With |s| ~ N / 20 the ratio is ~ 9, as for fields filled up to the cut."""
    A = 0.1
    free, _ = torch.cuda.mem_get_info()
    plan = g.Plan(N, n_max, 1000.0 * N / 256)
    need = plan.workspace_size() + 8 * N * N * (N // 2) * (2 * (n_max - 1) + 1)
    if free < need + (1 << 30):
        pytest.skip(f"needs {need / 2**30:.0f} GiB on the device")
    d1 = torch.zeros(plan.half_shape(1), dtype=torch.complex64, device="cuda")
    d1[0, s[0] % N, s[1] % N, s[2]] = A / 2
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device="cuda")
    sp = torch.empty(plan.half_shape(1, n_max - 1, 2), dtype=torch.complex64, device="cuda")
    g.run_orders(plan, d1, spectra=sp, ws=ws)
    del ws
    for n in range(2, n_max + 1):
        tol = 1e-5 * (A / 2) ** n * 2 ** n
        for which in (0, 1):
            got = sp[0, n - 2, which]
            for m in range(n % 2, n + 1, 2):
                if m == 0:                                  # carries 0 (mass conservation)
                    continue
                j = (n - m) // 2
                v = (-1) ** j * m ** n * (A / 2) ** n / (math.factorial(j) * math.factorial(m + j))
                idx = (m * s[0] % N, m * s[1] % N, m * s[2])
                assert abs(complex(got[idx].item()) - v) < tol, (n, which, m)
                got[idx] = 0
            assert float(got.abs().max()) < tol, (n, which)
    del sp, d1
    torch.cuda.empty_cache()


def test_modes_of_delta1_above_the_cut_are_ignored():
    """run_orders applies delta_1's cut: a mode added above it (inside and
    outside the band of columns the order-1 passes move) changes nothing."""
    N, L, n_max = 48, 300.0, 4
    plan = g.Plan(N, n_max, L)
    d1 = g.make_linear_field(plan, [91])
    ref = g.run_orders(plan, d1)
    r = N / (n_max + 1)                          # cut radius in units of k_F
    dirty = d1.clone()
    dirty[0, 9, 3, 2] = 0.5 + 0.25j              # |s|^2 = 94 > r^2, every component inside the band
    dirty[0, 2, 1, 15] = 0.25                    # kz beyond the band
    assert 9 * 9 + 3 * 3 + 2 * 2 > r * r and 15 > r
    assert torch.equal(g.run_orders(plan, dirty), ref)


def test_order_two_spectra_vanish_outside_their_band():
    """delta_2, theta_2 are products of two order-1 fields whose components are
    at most c1 = floor(sqrt(s2_lin)); with 4 c1 < N no product wraps, so every
    mode with |s_y| or s_z above 2 c1 is zero. The oracle's full computation is
    zero there to FP64 rounding; the GPU forms only the band columns (|ky|,
    kz < B, B = 2 c1 + 2 rounded to even) and writes exact zeros elsewhere."""
    N, L, n_max = 64, 500.0, 5
    plan = g.Plan(N, n_max, L)
    ref1 = spt.linear_field(N, L, n_max, COSMO, 5)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    sp = g.run_orders(plan, to_dev(ref1)[None])
    r = N / (n_max + 1)
    c1 = math.isqrt(math.floor(r * r))
    B = 2 * c1 + 1
    B += B & 1
    assert 4 * c1 < N and B < N // 2
    sy = np.fft.fftfreq(N, 1.0 / N).astype(int)[None, :, None]
    kz = np.arange(N // 2)[None, None, :]
    out = (np.abs(sy) >= B) | (kz >= B)
    out = np.broadcast_to(out, (N, N, N // 2))
    dk, tk = spt.run_orders(ref1, L, 2)
    for which, ref in ((0, dk[2]), (1, tk[2])):
        half = ref[:, :, : N // 2]
        assert np.abs(half[out]).max() <= 1e-12 * np.abs(half).max()       # the exact values
        got = host(sp[0, 0, which])
        assert np.all(got[out] == 0)
        assert rms_rel(got, ref) < 1e-5


def test_every_order_band_limited_by_a_low_linear_cut():
    """A linear cut at 6.5 k_F (c1 = 6) on 64^3 keeps 4 c1 < N/2, so orders 2, 3
    and 4 each move only their band columns (B = 14, 20, 26) with no cut on the
    higher orders: all orders against the oracle, and exact zeros where a mode
    has |s_y| or s_z >= B."""
    N, L, n_max = 64, 500.0, 5
    kF = 2 * math.pi / L
    errs = _parity_case(N, L, n_max, 61, kcut_lin=kF * 6.5)
    for (n, which), e in errs.items():
        assert e < (1e-5 if n == 2 else 1e-4), (n, which, e)
    plan = g.Plan(N, n_max, L, kcut_lin=kF * 6.5)
    ref1 = spt.linear_field(N, L, n_max, COSMO, 61, kcut_lin=kF * 6.5)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    sp = g.run_orders(plan, to_dev(ref1)[None])
    sy = np.abs(np.fft.fftfreq(N, 1.0 / N).astype(int))[None, :, None]
    kz = np.arange(N // 2)[None, None, :]
    for m, B in ((2, 14), (3, 20), (4, 26)):
        out = np.broadcast_to((sy >= B) | (kz >= B), (N, N, N // 2))
        for w in range(2):
            assert np.all(host(sp[0, m - 2, w])[out] == 0), (m, w)


@pytest.mark.parametrize("N,L,n_max,seed", [(64, 500.0, 5, 71), (48, 300.0, 4, 72)])
def test_truncated_orders_match_the_oracle_below_the_cut(N, L, n_max, seed):
    """truncate=1 cuts every order j >= 2 at min(j, n_max + 1 - j) K_c, all that
    the orders above it use for their modes below K_c: delta_n, theta_n on the
    modes |k| <= K_c against the full FP64 oracle recursion (the field bars of
    the default path, over those modes), and exact zeros above each order's
    cut."""
    plan = g.Plan(N, n_max, L, truncate=True)
    ref1 = spt.linear_field(N, L, n_max, COSMO, seed)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    sp = g.run_orders(plan, to_dev(ref1)[None])
    dk, tk = spt.run_orders(ref1, L, n_max)
    r = N / (n_max + 1)
    s = np.fft.fftfreq(N, 1.0 / N).astype(np.int64)
    s2 = s[:, None, None] ** 2 + s[None, :, None] ** 2 + np.arange(N // 2)[None, None, :] ** 2
    w = np.full(s2.shape, 2.0)
    w[:, :, 0] = 1.0
    inb = s2 <= math.floor(r * r)
    for n in range(2, n_max + 1):
        cut = math.floor((min(n, n_max + 1 - n) * r) ** 2)
        for which, ref in ((0, dk[n]), (1, tk[n])):
            got = host(sp[0, n - 2, which])
            half = ref[:, :, : N // 2]
            err = math.sqrt(np.sum((w * np.abs(got - half) ** 2)[inb]) / np.sum((w * np.abs(half) ** 2)[inb]))
            assert err < (1e-5 if n == 2 else 1e-4), (n, which, err)
            assert np.all(got[s2 > cut] == 0), (n, which)


def test_resume_equals_full_run_bitwise():
    N, L, n_max = 64, 400.0, 5
    plan = g.Plan(N, n_max, L)
    d1 = g.make_linear_field(plan, [77])
    full = g.run_orders(plan, d1)
    part = full.clone()
    part[:, 2:] = 0           # forget orders 4 and 5
    g.run_orders(plan, d1, start_order=4, spectra=part)
    assert torch.equal(full, part)


def test_eighth_order_matches_oracle():
    """Highest supported order (n_max = 8): orders 5..8 run pair launches whose
    targets are split so that no output has more than three partner fields."""
    errs = _parity_case(48, 300.0, 8, 41)
    for (n, which), e in errs.items():
        assert e < (1e-5 if n == 2 else 1e-4), (n, which, e)


@pytest.mark.parametrize("start", [5, 7])
def test_resume_at_high_order_equals_full_run_bitwise(start):
    """Resuming at order 7 of n_max = 8 leaves only targets fed by two higher
    orders (j >= 2) in the first pair launches of order 5: they must be split
    over two launches."""
    N, L, n_max = 32, 200.0, 8
    plan = g.Plan(N, n_max, L)
    d1 = g.make_linear_field(plan, [78])
    full = g.run_orders(plan, d1)
    part = full.clone()
    part[:, start - 2:] = 0
    g.run_orders(plan, d1, start_order=start, spectra=part)
    assert torch.equal(full, part)


def test_run_is_bitwise_repeatable_and_batched_equals_single():
    N, L, n_max = 48, 300.0, 4
    plan2 = g.Plan(N, n_max, L, batch=2)
    d = g.make_linear_field(plan2, [1, 2])
    a = g.run_orders(plan2, d)
    b = g.run_orders(plan2, d)
    assert torch.equal(a, b)
    plan1 = g.Plan(N, n_max, L)
    s = g.run_orders(plan1, d[1:2].contiguous())
    assert torch.equal(a[1:2], s)


def test_power_of_two_scaling_bitwise():
    """delta_1 -> 2 delta_1 gives delta_n -> 2^n delta_n exactly (every step is
    linear or a product, and scaling by 2 is exact in FP32)."""
    N, L, n_max = 64, 500.0, 5
    plan = g.Plan(N, n_max, L)
    d1 = g.make_linear_field(plan, [3])
    a = g.run_orders(plan, d1)
    b = g.run_orders(plan, d1 * 2)
    for n in range(2, n_max + 1):
        assert torch.equal(b[:, n - 2], a[:, n - 2] * (2.0 ** n))


# ------------------------------------------------------------- estimators
def _bins_linear(L, nb):
    kF = 2 * math.pi / L
    return [kF * (b + 0.5) for b in range(nb + 1)]


def _bins_log(lo, hi, nb):
    return [lo * (hi / lo) ** (i / nb) for i in range(nb + 1)]


@pytest.mark.parametrize("N,L,edges", [
    (64, 500.0, _bins_linear(500.0, 16)),
    (64, 1000.0, _bins_log(0.01, 0.19, 12)),
    (48, 300.0, _bins_linear(300.0, 20)),
])
def test_power_estimator_matches_oracle(N, L, edges):
    """The estimator alone: GPU and oracle estimators on the same FP32 spectra
    (the oracle's initial field and its third-order field, rounded to FP32)."""
    n_max = 3
    plan = g.Plan(N, n_max, L)
    ref1 = spt.linear_field(N, L, n_max, COSMO, 5)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    dk, _ = spt.run_orders(ref1, L, n_max)
    d3 = inputs.half_to_full(inputs.full_to_half(dk[3]).astype(np.complex64))
    d1g, d3g = to_dev(ref1), to_dev(d3)
    for a, b, ra, rb in [(d1g, d1g, ref1, ref1), (d3g, d3g, d3, d3), (d1g, d3g, ref1, d3)]:
        p, nk = g.power(plan, a, b, edges)
        pr, nkr = estimators.power(ra, rb, L, edges)
        assert np.array_equal(nk.cpu().numpy(), nkr)
        p = p.cpu().numpy()
        sel = nkr > 0
        assert np.all(np.abs(p[sel] - pr[sel]) <= 1e-5 * np.abs(pr[sel])), np.abs(p[sel] / pr[sel] - 1).max()


@pytest.mark.parametrize("N,L,n_max,edges", [
    (64, 500.0, 3, _bins_linear(500.0, 16)),
    (64, 250.0, 5, _bins_log(0.03, 0.7, 16)),
])
def test_power_terms_end_to_end(N, L, n_max, edges):
    """P-terms from GPU fields vs oracle fields on the same FP32 initial field,
    per bin with N_k > 0 and |P| > 1e-3 max |P|: P11 and P22 within 1e-5; the
    loop terms P13, P33, P24, P15 within max(1e-5 |P|, 6 sigma_b), sigma_b the
    white-noise bound of the bin for the noise level s_n that the GPU's delta_n
    carries (tests/fp32_floor.py). FP32 rounding of the real-space orders alone
    moves the lowest-k bins of the loop terms by more than 1e-5
    (tests/test_fp32_floor.py). s_n itself must stay within 1.5 times the level
    of an independent FP32 implementation of the recursion."""
    from tests import fp32_floor
    plan = g.Plan(N, n_max, L)
    ref1 = spt.linear_field(N, L, n_max, COSMO, 5)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    d1 = to_dev(ref1)
    spectra = g.run_orders(plan, d1[None])
    dk, _ = spt.run_orders(ref1, L, n_max)
    gd = {1: d1, **{n: spectra[0, n - 2, 0] for n in range(2, n_max + 1)}}
    rd = {1: ref1, **{n: dk[n] for n in range(2, n_max + 1)}}
    full = {1: ref1, **{n: inputs.half_to_full(spectra[0, n - 2, 0].cpu().numpy()) for n in range(2, n_max + 1)}}
    mask = fp32_floor.inband_mask(N, n_max)
    s = fp32_floor.noise_levels(full, rd, mask, range(2, n_max + 1))
    s32 = fp32_floor.noise_levels(fp32_floor.recursion_fp32(ref1, L, n_max), rd, mask, range(2, n_max + 1))
    for n in range(2, n_max + 1):
        assert s[n] <= 1.5 * s32[n], (n, s[n], s32[n])
    terms = [(1, 1), (2, 2), (1, 3)] + ([(3, 3), (2, 4), (1, 5)] if n_max >= 5 else [])
    for i, j in terms:
        f = 1.0 if i == j else 2.0
        p, nk = g.power(plan, gd[i], gd[j], edges)
        pr, nkr = estimators.power(rd[i], rd[j], L, edges)
        assert np.array_equal(nk.cpu().numpy(), nkr)
        p, pr = f * p.cpu().numpy(), f * pr
        sig = fp32_floor.pterm_sigma(rd, s, i, j, L, edges)
        sel, bar, _ = fp32_floor.pterm_bar(pr, sig, nkr)
        err = np.abs(p - pr)
        assert np.all(err[sel] <= bar[sel]), ((i, j), np.max(err[sel] / bar[sel]))
        if j <= 2:
            assert np.all(err[sel] <= 1e-5 * np.abs(pr[sel])), ((i, j), np.max(err[sel] / np.abs(pr[sel])))


def test_power_is_bitwise_repeatable():
    N, L = 64, 500.0
    plan = g.Plan(N, 3, L)
    d1 = g.make_linear_field(plan, [9])[0]
    e = _bins_linear(L, 16)
    a, _ = g.power(plan, d1, d1, e)
    b, _ = g.power(plan, d1, d1, e)
    assert torch.equal(a, b)


@pytest.mark.parametrize("N,L,nb", [(32, 250.0, 6), (48, 300.0, 8)])
def test_bispectrum_matches_oracle(N, L, nb):
    n_max = 3
    plan = g.Plan(N, n_max, L)
    ref1 = spt.linear_field(N, L, n_max, COSMO, 19)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    dk, _ = spt.run_orders(ref1, L, 2)
    kc = 2 * math.pi / L * N / (n_max + 1)
    edges = [kc * i / nb for i in range(nb + 1)]
    d1 = to_dev(ref1)
    d2 = to_dev(dk[2])
    E, nt = g.bispectrum(plan, d1, d2, edges)
    Er, ntr = estimators.bispectrum_equilateral(ref1, dk[2].astype(np.complex64).astype(np.complex128), L, edges)
    nt = nt.cpu().numpy()
    assert np.allclose(nt, ntr, rtol=1e-6, atol=1e-3)
    E = E.cpu().numpy()
    sel = ntr > 0.5
    assert np.all(np.abs(E[sel] - Er[sel]) <= 1e-4 * np.abs(Er[sel]).max())


def test_bispectrum_on_smaller_grids_matches_full_grid_oracle():
    """Shells whose components stay below B are evaluated on the smallest
    supported grid S > 3 (B - 1) (inputs copied onto it); at 128^3 with twelve
    shells up to |s| = 42.4 < N/3 the shells run on grids 12 ... 96 and the last
    ones on the full grid. E and N_tri against the oracle's full-grid FFT
    estimator on the same FP32-rounded inputs (two independent Gaussian
    fields), and the copies onto the smaller grids are seen to run."""
    N, L, nb = 128, 1000.0, 12
    kF = 2 * math.pi / L
    edges = [kF * (0.5 + 41.9 * i / nb) for i in range(nb + 1)]
    a = spt.linear_field(N, L, 3, COSMO, 41, kcut_lin=kF * 60)
    b = spt.linear_field(N, L, 3, COSMO, 42, kcut_lin=kF * 60)
    a = inputs.half_to_full(inputs.full_to_half(a).astype(np.complex64))
    b = inputs.half_to_full(inputs.full_to_half(b).astype(np.complex64))
    plan = g.Plan(N, 3, L)
    g.profile_begin()
    E, nt = g.bispectrum(plan, to_dev(a), to_dev(b), edges)
    torch.cuda.synchronize()
    stats = g.profile_end()
    assert stats.get("shell_grid", (0,))[0] >= 5          # one copy per distinct smaller grid
    Er, ntr = estimators.bispectrum_equilateral(a, b, L, edges)
    assert np.allclose(nt.cpu().numpy(), ntr, rtol=1e-6, atol=1e-3)
    sel = ntr > 0.5
    E = E.cpu().numpy()
    assert sel.all()
    assert np.all(np.abs(E - Er) <= 1e-4 * np.abs(Er).max())


@pytest.mark.parametrize("N,L,nb", [(32, 250.0, 5), (48, 300.0, 6)])
def test_triple_and_one_loop_bispectrum_match_oracle(N, L, nb):
    """E[a, b, c] for three different fields and the one-loop bispectrum of
    Eq. bk_1loop (GPU: 6 E[1,2,3] + E[2,2,2] + 3 E[1,1,4]; oracle: the ten
    ordered terms) on the oracle's fields rounded to FP32; E within 1e-4 of
    its scale, N_tri within FP32 rounding of the cubes."""
    n_max = 4
    plan = g.Plan(N, n_max, L)
    ref1 = spt.linear_field(N, L, n_max, COSMO, 29)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    dk, _ = spt.run_orders(ref1, L, n_max)
    r = [ref1] + [inputs.half_to_full(inputs.full_to_half(dk[n]).astype(np.complex64)) for n in (2, 3, 4)]
    dev = [to_dev(x) for x in r]
    kc = 2 * math.pi / L * N / (n_max + 1)
    edges = [kc * i / nb for i in range(nb + 1)]
    E, nt = g.bispectrum_triple(plan, dev[0], dev[1], dev[2], edges)
    Er, ntr = estimators.bispectrum_triple(r[0], r[1], r[2], L, edges)
    assert np.allclose(nt.cpu().numpy(), ntr, rtol=1e-6, atol=1e-3)
    sel = ntr > 0.5
    E = E.cpu().numpy()
    assert np.all(np.abs(E[sel] - Er[sel]) <= 1e-4 * np.abs(Er[sel]).max())
    B, _ = g.bispectrum_one_loop(plan, *dev, edges)
    Br, _ = estimators.bispectrum_one_loop(*r, L, edges)
    B = B.cpu().numpy()
    assert np.all(np.abs(B[sel] - Br[sel]) <= 1e-4 * np.abs(Br[sel]).max())


def test_triple_estimator_with_repeated_field_is_the_two_field_estimator():
    """E[a, a, b] of the triple form equals E[a, b] of gridspt_bispectrum bit for
    bit (same terms a a b, same sums, same sum J^3), in every z-pass variant."""
    N, L, nb = 64, 400.0, 6
    kc = 2 * math.pi / L * N / 4
    edges = [kc * i / nb for i in range(nb + 1)]
    outs = []
    for choice in ([0] * 5, [0, 0, 0, 2, 0]):
        p1, p2 = g.Plan(N, 3, L), g.Plan(N, 3, L)
        for pl in (p1, p2):
            g.set_tuning(pl, choice)
        d1 = g.make_linear_field(p1, [8])
        sp = g.run_orders(p1, d1)
        two = g.bispectrum(p1, d1[0], sp[0, 0, 0], edges)
        tri = g.bispectrum_triple(p2, d1[0], d1[0], sp[0, 0, 0], edges)
        assert torch.equal(two[0], tri[0]) and torch.equal(two[1], tri[1])
        outs.append([t.clone() for t in g.bispectrum_triple(p2, d1[0], sp[0, 0, 0], sp[0, 1, 0], edges)])
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_bispectrum_reuses_shell_normalisation_across_calls():
    """The first call stores sum J^3 per shell in the plan; repeated calls with
    the same shells reuse it and agree bit for bit; new shells recompute."""
    N, L, nb = 48, 300.0, 6
    plan = g.Plan(N, 3, L)
    d1 = g.make_linear_field(plan, [4])
    sp = g.run_orders(plan, d1)
    kc = 2 * math.pi / L * N / 4
    e1 = [kc * i / nb for i in range(nb + 1)]
    e2 = [kc * (0.5 + i) / (nb + 1) for i in range(nb + 1)]
    first = [t.clone() for t in g.bispectrum(plan, d1[0], sp[0, 0, 0], e1)]
    again = g.bispectrum(plan, d1[0], sp[0, 0, 0], e1)
    assert torch.equal(first[0], again[0]) and torch.equal(first[1], again[1])
    other = g.bispectrum(plan, d1[0], sp[0, 0, 0], e2)
    fresh = g.bispectrum(g.Plan(N, 3, L), d1[0], sp[0, 0, 0], e2)
    assert torch.equal(other[0], fresh[0]) and torch.equal(other[1], fresh[1])


def test_fp64_accumulator_matches_compensated_and_oracle():
    """accum="fp64" (products and sums in FP64) against the default compensated
    FP32 sums (FP32 products) on the same inputs: power within 1e-6 of the bin's
    sqrt(P_11 P_22) (the FP32 rounding of the products, ~1e-8, is all that
    separates them), the bispectrum within 1e-6 of its scale (same FP32 terms,
    Kahan FP32 chains against FP64 sums); both against the oracle estimators at
    the usual bars."""
    N, L, n_max = 48, 300.0, 3
    ref1 = spt.linear_field(N, L, n_max, COSMO, 17)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    dk, _ = spt.run_orders(ref1, L, 2)
    d2 = inputs.half_to_full(inputs.full_to_half(dk[2]).astype(np.complex64))
    a, b = to_dev(ref1), to_dev(d2)
    pe = _bins_linear(L, 20)
    kc = 2 * math.pi / L * N / (n_max + 1)
    be = [kc * i / 8 for i in range(9)]
    out = {}
    for acc in ("compensated", "fp64"):
        plan = g.Plan(N, n_max, L, accum=acc)
        p, nk = g.power(plan, a, b, pe)
        E, nt = g.bispectrum(plan, a, b, be)
        out[acc] = (p.cpu().numpy(), nk.cpu().numpy(), E.cpu().numpy(), nt.cpu().numpy())
        g.check(plan)
    pc, nkc, Ec, ntc = out["compensated"]
    pf, nkf, Ef, ntf = out["fp64"]
    assert np.array_equal(nkc, nkf)
    sel = nkc > 0
    # cross spectrum of delta_1 and delta_2: its bins scatter around zero, so the
    # difference is taken relative to sqrt(P_11 P_22) of the bin
    p11, _ = estimators.power(ref1, ref1, L, pe)
    p22, _ = estimators.power(d2, d2, L, pe)
    scale = np.sqrt(p11 * p22)
    assert np.all(np.abs(pf[sel] - pc[sel]) <= 1e-6 * scale[sel])
    assert np.allclose(ntf, ntc, rtol=1e-6, atol=1e-9)          # Kahan FP32 chains vs FP64: ~1e-8
    assert np.all(np.abs(Ef - Ec) <= 1e-6 * np.abs(Ec).max())
    pr, _ = estimators.power(ref1, d2, L, pe)
    assert np.all(np.abs(pf[sel] - pr[sel]) <= 1e-5 * np.abs(pr[sel]))
    Er, ntr = estimators.bispectrum_equilateral(ref1, d2, L, be)
    s = ntr > 0.5
    assert np.all(np.abs(Ef[s] - Er[s]) <= 1e-4 * np.abs(Er[s]).max())
