"""P-term emulator end to end on a small workload: GridSPT (64^3, L = 250
Mpc/h, n_max = 5, 2 seeds) makes the training set on a Latin hypercube, the
network is trained with the library's kernels, and GridSPT measures its error on
held-out points and serves as the fallback outside the training box. Also
measures what the network gains: cosmologies per second vs. the grid method
on the same GPU."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1807_04215_gb300 import emulator as E  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    cfg = E.GridConfig(n=64, box=250.0, seeds=(1, 2), k_lo=0.03, k_hi=0.6, nbins=12)
    grid = E.GridSPTTerms(cfg)
    tr = E.latin_hypercube(64, 5)
    ho = E.latin_hypercube(8, 7)
    ytr = grid.many(tr)
    yho = grid.many(ho)
    mask = grid.nk.cpu().numpy() > 0
    emu = E.train(tr, ytr, mask, steps=4000)
    return cfg, grid, emu, ho, yho, mask


def test_emulator_reproduces_gridspt_on_heldout_points(trained):
    cfg, grid, emu, ho, yho, mask = trained
    err = E.errors(emu.predict(ho), yho, mask)
    for name, e in err.items():
        assert e["scale_max"] < 0.03, (name, e)
        assert e["rel_rms"] < 0.03, (name, e)


def test_sigma8_scaling_is_exact_in_gridspt(trained):
    """P_ij scales as sigma_8^(i+j) with fixed seeds (what the target scaling uses)."""
    cfg, grid, emu, ho, yho, mask = trained
    p = np.array([0.8, 0.96, 0.2])
    a = grid(p)
    b = grid(p * np.array([0.5, 1.0, 1.0]))
    for t, (i, j) in enumerate(E.TERMS):
        assert np.allclose(b[t], a[t] * 0.5 ** (i + j), rtol=1e-6, atol=1e-12 * np.abs(a[t]).max())


def test_fallback_outside_box_uses_gridspt(trained):
    cfg, grid, emu, ho, yho, mask = trained
    pts = np.array([[0.8, 0.96, 0.2], [1.3, 0.96, 0.2]])
    res, ok = emu.predict_or_fallback(pts, grid)
    assert ok.tolist() == [True, False]
    assert np.array_equal(res[1], grid(pts[1]))


def test_emulator_throughput_gain(trained):
    cfg, grid, emu, ho, yho, mask = trained
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p in ho[:4]:
        grid(p)
    torch.cuda.synchronize()
    t_grid = (time.perf_counter() - t0) / 4
    pts = E.latin_hypercube(4096, 3)
    emu.predict(pts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emu.predict(pts)
    torch.cuda.synchronize()
    t_emu = (time.perf_counter() - t0) / 4096
    assert t_grid / t_emu > 100
