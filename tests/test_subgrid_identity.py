"""Identities behind the work the library skips (CPU, FP64, on the oracle).

Smaller-grid bispectrum:

Every vector of a shell whose components satisfy |s_a| < B can be stored on a
grid of size S; the sum over the S^3 cells of a product of three shell fields
keeps the triangles s_1 + s_2 + s_3 = 0 (mod S in each component). When
S > 3 (B - 1) no other sum is a multiple of S, so the sums are those of the
N^3 grid times (S/N)^3 and E, N_tri are unchanged; at S = 3 (B - 1) wrapped
triangles enter. Checked with the oracle's FFT shell estimator on both grids.

Band-limited orders: products of fields whose modes have components at most
a c1 and b c1 have components at most (a + b) c1; while that stays below N/2
nothing wraps, so the higher orders vanish outside their band.
"""
import math

import numpy as np

from oracle import estimators
from tests import inputs


def _on_grid(a, S):
    """The modes of a full N^3 spectrum with every component in (-S/2, S/2),
    placed on an S^3 grid (Nyquist planes of the small grid zero)."""
    N = a.shape[0]
    s = np.fft.fftfreq(S, 1.0 / S).astype(int)
    idx = s % N
    out = a[np.ix_(idx, idx, idx)].copy()
    out[S // 2, :, :] = 0
    out[:, S // 2, :] = 0
    out[:, :, S // 2] = 0
    return out


def test_shell_sums_on_smaller_grids_equal_the_full_grid():
    N, L = 48, 300.0
    kF = 2 * math.pi / L
    a = np.fft.fftn(inputs.random_real((N, N, N), 1))
    b = np.fft.fftn(inputs.random_real((N, N, N), 2))
    # shells [lo, hi) in units of k_F; B - 1 = largest component, grid = smallest supported S > 3 (B - 1)
    for lo, hi, S in [(0.5, 4.0, 12), (4.0, 7.0, 24), (7.0, 10.0, 32)]:
        edges = [kF * lo, kF * hi]
        E, nt = estimators.bispectrum_equilateral(a, b, L, edges)
        Es, nts = estimators.bispectrum_equilateral(_on_grid(a, S), _on_grid(b, S), L, edges)
        assert nt[0] > 0.5
        assert abs(nts[0] - nt[0]) <= 1e-9 * nt[0]
        assert abs(Es[0] - E[0]) <= 1e-10 * abs(E[0])


def test_a_grid_of_three_times_the_band_wraps_triangles_in():
    """Shell 3.5 <= |s| < 4.5 holds s = (4, 0, 0): B - 1 = 4, so S = 12 = 3 (B - 1)
    also counts the wrapped triangles (4, 0, 0) x 3 = (12, 0, 0); S = 16 does not."""
    N, L = 48, 300.0
    kF = 2 * math.pi / L
    a = np.fft.fftn(inputs.random_real((N, N, N), 3))
    edges = [kF * 3.5, kF * 4.5]
    E, nt = estimators.bispectrum_equilateral(a, a, L, edges)
    _, nt16 = estimators.bispectrum_equilateral(_on_grid(a, 16), _on_grid(a, 16), L, edges)
    _, nt12 = estimators.bispectrum_equilateral(_on_grid(a, 12), _on_grid(a, 12), L, edges)
    assert abs(nt16[0] - nt[0]) <= 1e-9 * nt[0]
    assert nt12[0] > nt[0] + 0.5


def test_orders_formed_from_a_band_limited_field_vanish_outside_their_band():
    """The identity behind the library's band-limited passes of orders m >= 2:
    with every component of delta_1's modes at most c1, delta_m and theta_m
    vanish at every mode with a component above m c1 as long as m c1 < N/2 (no
    product of the recursion up to order m wraps around the grid). The
    oracle's FP64 recursion on 32^3, with the default cut N/6 (c1 = 5: orders 2
    and 3 have a band inside the grid) and with a linear cut at 3.5 k_F (c1 = 3:
    every order up to 5)."""
    from oracle import cosmology, spt
    N, L, n_max = 32, 250.0, 5
    kF = 2 * math.pi / L
    s = np.abs(np.fft.fftfreq(N, 1.0 / N).astype(int))
    comp = np.maximum(np.maximum(s[:, None, None], s[None, :, None]), s[None, None, :])
    for kcut, c1, banded in [(None, 5, (2, 3)), (3.5 * kF, 3, (2, 3, 4, 5))]:
        d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, 3, kcut_lin=kcut)
        dk, tk = spt.run_orders(d1, L, n_max)
        for m in banded:
            assert 2 * m * c1 < N
            outside = comp > m * c1
            assert outside.sum() > 0
            for f in (dk[m], tk[m]):
                assert np.abs(f[outside]).max() <= 1e-12 * np.abs(f).max(), (kcut, m)


def test_truncating_each_order_keeps_every_order_below_the_linear_cut():
    """The identity behind the library's truncate option: cutting every order j
    >= 2 at min(j, n_max + 1 - j) K_c right after it is formed leaves delta_n,
    theta_n at |k| <= K_c as the full recursion has them. A mode of delta_n below
    K_c sums products of an order-j mode and an order-(n - j) mode within
    (n - j) K_c of it, so the order-j factor lies below (n + 1 - j) K_c <=
    (n_max + 1 - j) K_c, besides its own band j K_c. Checked with the oracle's
    own steps (derived fields, sources, forward transform) and the cut
    inserted, against its untruncated recursion, FP64 on 32^3."""
    from oracle import cosmology, spt
    N, L, n_max = 32, 250.0, 5
    d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, 7)
    dk, tk = spt.run_orders(d1, L, n_max)
    nyq = spt.nyquist_mask(N)
    sx, sy, sz = spt.wave_indices(N)
    s2 = (sx * sx + sy * sy + sz * sz).astype(np.float64)
    r = N / (n_max + 1)
    delta, theta, fields = [None, d1.copy()], [None, d1.copy()], {}
    for n in range(2, n_max + 1):
        fields[n - 1] = spt.derived_fields(delta[n - 1], theta[n - 1], L)
        A, B = spt.sources(fields, n)
        cdA, cdB, ctA, ctB = spt.recursion_coefficients(n)
        dn, tn = spt.forward(cdA * A + cdB * B), spt.forward(ctA * A + ctB * B)
        cut = math.floor((min(n, n_max + 1 - n) * r) ** 2)
        for f in (dn, tn):
            f[nyq] = 0.0
            f[s2 > cut] = 0.0
        delta.append(dn)
        theta.append(tn)
    inb = s2 <= math.floor(r * r)
    for n in range(2, n_max + 1):
        for full, cut_run in ((dk[n], delta[n]), (tk[n], theta[n])):
            scale = np.abs(full[inb]).max()
            assert np.abs(full[inb] - cut_run[inb]).max() <= 1e-12 * scale, n
