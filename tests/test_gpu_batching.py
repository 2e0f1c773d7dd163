"""Launch batching and autotuning (not part of the paper's method): a CUDA
graph of the whole recursion and a mixed-size batch in one graph launch must
reproduce the eager launches bit for bit; tile variants chosen by the
autotuner must not change any result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1807_04215_gb300 import gridspt as g  # noqa: E402

pytestmark = pytest.mark.gpu


def test_single_plan_graph_equals_eager():
    plan = g.Plan(64, 5, 500.0, batch=2)
    d1 = g.make_linear_field(plan, [11, 12])
    eager = g.run_orders(plan, d1)
    b = g.Batch([plan], [d1])
    out = b.launch()[0]
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    out.zero_()
    b.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)          # replay recomputes everything
    b.close()


def test_mixed_size_batch_one_launch_equals_separate_runs():
    sizes = [(32, 250.0), (48, 375.0), (64, 500.0)]   # same cell size, as in the mixed workload
    plans = [g.Plan(n, 5, L, batch=2) for n, L in sizes]
    d1s = [g.make_linear_field(p, [100 + i, 200 + i]) for i, p in enumerate(plans)]
    ref = [g.run_orders(p, d) for p, d in zip(plans, d1s)]
    b = g.Batch(plans, d1s)
    outs = b.launch()
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)
    b.close()


@pytest.mark.parametrize("N,n_max", [(32, 5), (64, 5), (128, 3), (192, 5), (256, 5), (512, 5)])
def test_tile_variants_give_identical_results(N, n_max):
    """Tile widths, cp.async prefetch, the TMA-staged y pass (y variant 2), the
    column-pair y pass (y variant 3), the prefetching y pass (y variant 4) and
    the paired-output x and y passes (x variants 2, 3; y variants 5, 6), the
    warp-row z passes (z expansion and
    z forward variant 2: one row per 2 .. 32 lanes for power-of-two N, the tile
    kernels for N = 192) only regroup work: results are bit-identical.
    n_max = 5 runs the z expansion store-only, with one target and with two
    targets."""
    plan = g.Plan(N, n_max, 4.0 * N)
    d1 = g.make_linear_field(plan, [5])
    results = []
    for choice in ([0] * 5, [1] * 5, [0, 0, 2, 0, 0], [0, 0, 3, 0, 0], [0, 0, 4, 0, 0], [0, 0, 0, 2, 0],
                   [0, 0, 0, 0, 2], [1, 1, 4, 2, 2], [0, 2, 5, 0, 0], [0, 3, 6, 0, 0]):
        g.set_tuning(plan, choice)
        assert g.get_tuning(plan) == choice
        results.append(g.run_orders(plan, d1).clone())
        g.check(plan)
    ref = results[0]
    for r in results[1:]:
        assert torch.equal(ref, r)
    del results
    ch = g.autotune(plan)
    assert len(ch) == 5 and all(0 <= c < k for c, k in zip(ch, (2, 4, 7, 3, 3)))
    assert g.get_tuning(plan) == ch
    assert torch.equal(g.run_orders(plan, d1), ref)
    del ref
    torch.cuda.empty_cache()


@pytest.mark.parametrize("N", [64, 256])
def test_variants_identical_with_the_higher_order_cut(N):
    """With k_cut,2 every order m >= 2 has the band of that cut: the x and y
    passes move only band columns and every z launch (store-only, one target,
    two targets) reads only kz < band, zero-filling its row buffers in the
    warp-row form and its tiles in the tile form. All variants agree bit for
    bit, and the spectra vanish outside the band columns."""
    L = 4.0 * N
    kF = 2 * np.pi / L
    kc = kF * N / 6
    plan = g.Plan(N, 5, L, kcut_lin=kc, kcut_nl=4.0 / 3.0 * kc)
    d1 = g.make_linear_field(plan, [6])
    results = []
    for choice in ([0] * 5, [1, 1, 1, 1, 1], [1, 1, 3, 2, 2], [1, 1, 4, 2, 2], [1, 2, 5, 2, 2], [1, 3, 6, 2, 2]):
        g.set_tuning(plan, choice)
        results.append(g.run_orders(plan, d1).clone())
        g.check(plan)
    for r in results[1:]:
        assert torch.equal(results[0], r)
    B = int(np.floor(np.sqrt(np.floor((4.0 / 3.0 * N / 6) ** 2)))) + 1
    B += B & 1
    sy = torch.from_numpy(np.fft.fftfreq(N, 1.0 / N).astype(np.int64)).cuda()
    outside = (sy.abs() >= B)[None, :, None] | (torch.arange(N // 2, device="cuda") >= B)[None, None, :]
    for m in range(2, 6):
        for w in range(2):
            assert torch.all(results[0][0, m - 2, w][outside.expand(N, N, N // 2)] == 0)
    del results


@pytest.mark.parametrize("N", [32, 64, 256])
def test_bispectrum_identical_for_warp_row_z_pass(N):
    """The bispectrum's z pass in warp-row form (z expansion variant 2) forms
    the same terms, per-row shuffle trees and row order as the tile kernel:
    E and N_tri are bitwise equal, with and without the cached J^3 sums."""
    L = 4.0 * N
    kc = 2 * np.pi / L * N / 6
    edges = [kc * i / 8 for i in range(9)]
    out = []
    for choice in ([0] * 5, [0, 0, 3, 2, 0]):
        plan = g.Plan(N, 5, L)
        g.set_tuning(plan, choice)
        d1 = g.make_linear_field(plan, [9])
        sp = g.run_orders(plan, d1)
        first = g.bispectrum(plan, d1[0], sp[0, 0, 0], edges)       # J^3 formed
        second = g.bispectrum(plan, d1[0], sp[0, 0, 0], edges)      # J^3 from the cache
        out.append([t.clone() for t in first] + [t.clone() for t in second])
    for a, b in zip(*out):
        assert torch.equal(a, b)
