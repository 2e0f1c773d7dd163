"""Divergence-form sources on the GPU (plan form "divergence"; not in the paper).

A_n = div sum_m delta_m u_{n-m} and B_n = (1/2) lap sum_m u_m . u_{n-m} rewrite
the nine-term sources of Eq. recursion_formula exactly (theta = div u, u curl
free); the GPU forms them from four real fields per order. Checked against
the FP64 oracle's divergence form at every mode (same tolerances as the
nine-term parity: RMS relative error <= 1e-5 at n = 2, <= 1e-4 up to n = 5),
and against the oracle's nine-term form on the modes below delta_1's cut,
where the two forms agree exactly; above the cut the grid products fold and
the forms differ by design.
"""
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import cosmology, spt  # noqa: E402
from paper_1807_04215_gb300 import gridspt as g  # noqa: E402
from tests import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
COSMO = cosmology.DEFAULT_COSMO


def to_dev(full):
    return torch.from_numpy(inputs.full_to_half(full).astype(np.complex64)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def rms_rel(got_half, ref_full, sel=None):
    """Parseval-weighted RMS relative error of a half spectrum vs a full grid,
    over the modes selected by `sel` (full-grid boolean, or all)."""
    N = ref_full.shape[0]
    ref = ref_full[:, :, : N // 2]
    w = np.full(ref.shape, 2.0)
    w[:, :, 0] = 1.0
    if sel is not None:
        w = w * sel[:, :, : N // 2]
    return math.sqrt(np.sum(w * np.abs(got_half - ref) ** 2) / np.sum(w * np.abs(ref) ** 2))


def _case(N, L, n_max, seed, kcut_nl=0.0):
    plan = g.Plan(N, n_max, L, kcut_nl=kcut_nl, form="divergence")
    ref1 = spt.linear_field(N, L, n_max, COSMO, seed)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))   # FP32-rounded input
    sp = g.run_orders(plan, to_dev(ref1)[None])
    return plan, ref1, sp


@pytest.mark.parametrize("N,L,n_max,seed", [(32, 250.0, 5, 51), (48, 300.0, 5, 52), (64, 500.0, 3, 53),
                                             (24, 150.0, 4, 54)])
def test_divergence_form_matches_oracle(N, L, n_max, seed):
    plan, ref1, sp = _case(N, L, n_max, seed)
    dk, tk = spt.run_orders_divergence(ref1, L, n_max)
    nine_d, nine_t = spt.run_orders(ref1, L, n_max)
    sx, sy, sz = spt.wave_indices(N)
    r = spt.cut_ratio(N, L, n_max, None)
    band = (sx * sx + sy * sy + sz * sz) < r * r
    report = {}
    for n in range(2, n_max + 1):
        tol = 1e-5 if n == 2 else 1e-4
        for which, ref, nine in ((0, dk[n], nine_d[n]), (1, tk[n], nine_t[n])):
            got = host(sp[0, n - 2, which])
            e_all, e_band = rms_rel(got, ref), rms_rel(got, nine, band)
            report[f"{'delta' if which == 0 else 'theta'}_{n}"] = [float(f"{e_all:.2e}"), float(f"{e_band:.2e}")]
            assert e_all < tol, (n, which)
            assert e_band < tol, (n, which, "in band vs nine-term form")
            assert got[0, 0, 0] == 0                 # A_n(0) = i 0 . V, B_n(0) = 0 exactly
    print(f"DIVERGENCE_{N}_L{L:g}_NMAX{n_max} " + json.dumps(report))


def test_divergence_form_with_nonlinear_cut():
    N, L, n_max = 32, 250.0, 4
    kF = 2 * math.pi / L
    plan, ref1, sp = _case(N, L, n_max, 55, kcut_nl=kF * 9.5)
    dk, tk = spt.run_orders_divergence(ref1, L, n_max, kcut_nl=kF * 9.5)
    for n in range(2, n_max + 1):
        for which, ref in ((0, dk[n]), (1, tk[n])):
            assert rms_rel(host(sp[0, n - 2, which]), ref) < 1e-4, (n, which)


def test_divergence_form_single_plane_wave_closed_form():
    """Zel'dovich closed form of one wave. Bound: the field parity bar (1e-5 at
    n = 2, 1e-4 above) relative to (A/2)^n 2^n. B = (1/2) lap(u . u) takes the
    Laplacian of a product whose norm sits at large scales (u ~ theta / k), so
    its FP32 rounding reaches the high harmonics multiplied by k^2; the
    nine-term form multiplies O(delta) fields and meets 1e-5 here."""
    N, L, A = 32, 100.0, 0.1
    plan = g.Plan(N, 5, L, form="divergence")
    sp = g.run_orders(plan, to_dev(inputs.plane_waves(N, [((1, 0, 0), A)]))[None])
    for n in range(2, 6):
        exp = np.zeros((N, N, N // 2), complex)
        for m in range(n % 2, n + 1, 2):
            j = (n - m) // 2
            v = (-1) ** j * m ** n * (A / 2) ** n / (math.factorial(j) * math.factorial(m + j))
            exp[m % N, 0, 0] = v
            exp[-m % N, 0, 0] = v
        tol = (1e-5 if n == 2 else 1e-4) * (A / 2) ** n * 2 ** n
        for which in (0, 1):
            assert np.abs(host(sp[0, n - 2, which]) - exp).max() < tol, (n, which)


def test_divergence_form_resume_graph_and_workspace():
    N, L, n_max = 64, 400.0, 5
    plan = g.Plan(N, n_max, L, batch=2, form="divergence")
    assert plan.workspace_size() == (4 * n_max + 7) * 4 * N ** 3
    d1 = g.make_linear_field(plan, [61, 62])
    full = g.run_orders(plan, d1)
    part = full.clone()
    part[:, 2:] = 0
    g.run_orders(plan, d1, start_order=4, spectra=part)
    assert torch.equal(full, part)
    b = g.Batch([plan], [d1])
    out = b.launch()[0]
    torch.cuda.synchronize()
    assert torch.equal(out, full)
    b.close()
    for choice in ([1] * 5, [0, 0, 2, 2, 2], [0, 0, 3, 2, 2]):      # tile variants regroup work only
        g.set_tuning(plan, choice)
        assert torch.equal(g.run_orders(plan, d1), full)
