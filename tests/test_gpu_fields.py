"""Field-level outputs on the GPU against the FP64 oracle: the summed density
field delta_SPT = W(kR) sum D^i delta_i (Sec. III.A) and the cross-correlation
coefficient (Eqs. r_corr_nthPT, r_corr_sum_nth), on the oracle's fields
rounded to FP32. delta_SPT: every mode within 1e-6 of the largest (FP32 sums
and filter); r: within 1e-6 absolute (FP32 products, FP64 shell sums)."""
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


def _fields(N, L, n_max, seed):
    ref1 = spt.linear_field(N, L, n_max, COSMO, seed)
    ref1 = inputs.half_to_full(inputs.full_to_half(ref1).astype(np.complex64))
    dk, _ = spt.run_orders(ref1, L, n_max)
    full = [ref1] + [inputs.half_to_full(inputs.full_to_half(dk[n]).astype(np.complex64)) for n in range(2, n_max + 1)]
    return full


def _dev(full):
    return torch.from_numpy(inputs.full_to_half(full).astype(np.complex64)).cuda()


@pytest.mark.parametrize("N,L,n_max,n,z,R", [(32, 250.0, 5, 5, 1.0, 8.0), (48, 300.0, 4, 3, 0.0, 0.0),
                                              (24, 150.0, 3, 1, 0.5, 12.0)])
def test_sum_orders_matches_oracle(N, L, n_max, n, z, R):
    plan = g.Plan(N, n_max, L)
    full = _fields(N, L, n_max, 71)
    spectra = torch.zeros(plan.half_shape(n_max - 1, 2), dtype=torch.complex64, device="cuda")
    for m in range(2, n_max + 1):
        spectra[m - 2, 0] = _dev(full[m - 1])
    D = g.growth_factor(z)
    got = g.sum_orders(plan, _dev(full[0]), spectra, n, D, R).cpu().numpy().astype(np.complex128)
    ref = spt.sum_orders(full[:n], D, R, L)[:, :, : N // 2]
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


def test_cross_correlation_matches_oracle():
    N, L, n_max = 48, 300.0, 4
    plan = g.Plan(N, n_max, L)
    full = _fields(N, L, n_max, 72)
    kF = 2 * math.pi / L
    edges = [kF * e for e in (0.5, 2.5, 5.5, 9.5, 14.5, 23.5)]
    sum3 = spt.sum_orders(full[:3], 1.0, 0.0, L)
    for a, b in ((full[0], full[2]), (full[1], full[3]), (full[0], sum3)):
        got = g.cross_correlation(plan, _dev(a), _dev(b), edges).cpu().numpy()
        ref = estimators.cross_correlation(a, b, L, edges)
        assert np.abs(got - ref).max() < 1e-6
    one = g.cross_correlation(plan, _dev(full[1]), _dev(full[1]), edges).cpu().numpy()
    assert np.abs(one - 1.0).max() < 1e-12


def test_cutoff_scan_matches_oracle():
    """The paper's two-cut scheme (k_cut,1 on delta_1, k_cut,2 = 4/3 k_cut,1 on
    every higher order) through the scan driver: P_2-loop within 3e-5 of its
    scale and B_1-loop within 1e-4 of its scale of the oracle, which draws the
    same delta_1 from the same seed (end to end: GPU fields in FP32)."""
    from paper_1807_04215_gb300 import cutoff_scan
    N, L, kc, seed = 32, 250.0, 0.11, 3
    res = cutoff_scan.scan(N, L, [kc], seeds=(seed,))[0]
    d1 = spt.linear_field(N, L, 5, COSMO, seed, kcut_lin=kc)
    dk, _ = spt.run_orders(d1, L, 5, kcut_nl=4.0 / 3.0 * kc)
    pe, be = res["pk_edges"], res["bk_edges"]
    p2 = 2 * estimators.power(d1, dk[5], L, pe)[0] + 2 * estimators.power(dk[2], dk[4], L, pe)[0] + \
        estimators.power(dk[3], dk[3], L, pe)[0]
    got = np.array(res["P_2loop"])
    assert np.abs(got - p2).max() <= 3e-5 * np.abs(p2).max()
    b1, nt = estimators.bispectrum_one_loop(d1, dk[2], dk[3], dk[4], L, be)
    got = np.array(res["B_1loop"])
    sel = nt > 0.5
    assert np.abs(got[sel] - b1[sel]).max() <= 1e-4 * np.abs(b1[sel]).max()
