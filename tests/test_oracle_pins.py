"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the planted mistake it is meant to catch. None compares the
oracle with a retyped copy of itself: the expected values come from closed
forms (Zel'dovich plane wave, textbook F_2/G_2), brute-force mode sums with the
independent Fourier-kernel recursion, published known-answer vectors,
invariants (mass conservation, Hermitian symmetry, exact 2^n scaling, zero
padding) or an independent quadrature.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology, cutout, estimators, kernels, rng, spt
from tests import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ generator
def test_philox_known_answers():
    """Published Philox4x32-10 vectors (catches a wrong constant, word order or round count)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(v, 16) for v in r]
        out = rng.philox4x32_10(np.array(vals[0:4]), np.array(vals[4:6]))
        assert [int(v) for v in out] == vals[6:10]


def test_mode_key_two_complement():
    lo, hi = rng.mode_key(np.array([-1]), np.array([0]), np.array([1]))
    packed = int(lo[0]) | (int(hi[0]) << 32)
    assert packed & 0x1FFFFF == 0x1FFFFF          # -1 in 21-bit two's complement
    assert (packed >> 21) & 0x1FFFFF == 0
    assert (packed >> 42) & 0x1FFFFF == 1


# ------------------------------------------------------------- DFT convention
def test_transform_pair_matches_naive_sums():
    """Sec. II.C transform pair against the triple sums written out
    (catches a sign flip or a missing 1/N^3)."""
    N = 6
    a_k = inputs.random_complex((N, N, N), 1)
    j = np.arange(N)
    ph = np.exp(2j * math.pi * np.outer(j, j) / N)  # e^{+i k x}, [x, k]
    naive_x = np.einsum("xa,yb,zc,abc->xyz", ph, ph, ph, a_k)
    assert np.allclose(spt.backward(a_k), naive_x, rtol=0, atol=1e-12 * np.abs(naive_x).max())
    a_x = inputs.random_complex((N, N, N), 2)
    naive_k = np.einsum("xa,yb,zc,xyz->abc", ph.conj(), ph.conj(), ph.conj(), a_x) / N ** 3
    assert np.allclose(spt.forward(a_x), naive_k, rtol=0, atol=1e-12 * np.abs(naive_k).max())


# ------------------------------------------------------------------ cosmology
def test_sigma8_normalisation_by_independent_quadrature():
    """sigma_8 of the normalised spectrum by adaptive quadrature in k (not the
    oracle's Simpson in ln k): catches a wrong window, measure or 2 pi^2."""
    c = dict(cosmology.DEFAULT_COSMO)
    A = cosmology.amplitude(c)
    R = 8.0

    def integrand(k):
        x = k * R
        w = 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3 if x > 1e-3 else 1.0
        return k * k * float(cosmology.linear_pk(np.array([k]), c, A)[0]) * w * w

    pts = [1e-3, 1e-2, 0.05, 0.1, 0.3, 1.0, 3.0, 10.0]
    total = 0.0
    edges = [1e-6] + pts + [200.0]
    for lo, hi in zip(edges[:-1], edges[1:]):
        total += integrate.quad(integrand, lo, hi, limit=400, epsabs=0, epsrel=1e-11)[0]
    sigma8 = math.sqrt(total / (2 * math.pi ** 2))
    assert abs(sigma8 - 0.8) < 1e-6


def _bbks_constants():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "bbks1986_transfer.txt"))
            if l.strip() and not l.startswith("#")]
    return {k: float(v) for k, v in rows}


def _bbks_taylor_by_hand(a, b, c, d):
    """Taylor coefficients t1, t2, t3 of T(q) = 1 + t1 q + t2 q^2 + t3 q^3 + ...
    at q -> 0, expanded by hand from the published form. With
    P = 1 + b q + c^2 q^2 + d^3 q^3 + ..., (1 + x)^(-1/4) = 1 - x/4 + 5 x^2/32
    - 15 x^3/128 gives P^(-1/4) = 1 + p1 q + p2 q^2 + p3 q^3 with
        p1 = -b/4,  p2 = -c^2/4 + 5 b^2/32,  p3 = -d^3/4 + 5 b c^2/16 - 15 b^3/128,
    and ln(1 + a q)/(a q) = 1 - a q/2 + a^2 q^2/3 - a^3 q^3/4; their product
    has t1 = p1 - a/2, t2 = p2 - a p1/2 + a^2/3, t3 = p3 - a p2/2 + a^2 p1/3 - a^3/4."""
    p1 = -b / 4.0
    p2 = -c * c / 4.0 + 5.0 * b * b / 32.0
    p3 = -d ** 3 / 4.0 + 5.0 * b * c * c / 16.0 - 15.0 * b ** 3 / 128.0
    return (p1 - a / 2.0,
            p2 - a * p1 / 2.0 + a * a / 3.0,
            p3 - a * p2 / 2.0 + a * a * p1 / 3.0 - a ** 3 / 4.0)


def _taylor_fit(T, h=2e-3, deg=7):
    """Coefficients of q^0..q^3 of T near 0: a polynomial fit in the scaled
    variable y = q/h - 1 over (0, 2h] at Chebyshev nodes, re-expanded in q (the
    nearest singularity of the BBKS form is at |q| = 0.063, so the truncation
    error of degree 7 on q <= 2h is far below the tolerances used)."""
    y = np.cos(np.linspace(0.0, math.pi, 401))[:-1]
    q = h * (1.0 + y)
    P = np.polynomial.Polynomial(np.polynomial.polynomial.polyfit(y, T(q), deg))
    return P(np.polynomial.Polynomial([-1.0, 1.0 / h])).coef[:4]


def _bbks_pins_hold(T, consts):
    c0, c1, c2, c3 = _taylor_fit(T)
    t1, t2, t3 = _bbks_taylor_by_hand(consts["a"], consts["b"], consts["c"], consts["d"])
    a, e = consts["a"], consts["e"]
    qb = np.array([1e9])
    lim = T(qb)[0] * qb[0] ** 2 / math.log(a * qb[0])
    return (abs(c0 - 1.0) < 1e-12 and abs(c1 / t1 - 1.0) < 1e-9 and abs(c2 / t2 - 1.0) < 1e-7
            and abs(c3 / t3 - 1.0) < 1e-5 and abs(lim * a * e - 1.0) < 1e-2)


def test_bbks_taylor_coefficients_and_large_q_limit():
    """T(q) of the oracle against the published BBKS constants
    (tests/golden/bbks1986_transfer.txt): its q, q^2 and q^3 Taylor coefficients
    at q -> 0 (expanded by hand; they fix a, b, then c through c^2 and d through
    d^3) and its q -> inf limit T q^2 / ln(a q) -> 1/(a e) (fixes e). Catches a
    wrong value of any of the five constants."""
    assert _bbks_pins_hold(cosmology.bbks_transfer, _bbks_constants())


@pytest.mark.parametrize("typo", [("16.1", "16.2"), ("5.46", "5.47"), ("3.89", "3.98"),
                                  ("(5.46 * qq) ** 3", "(5.46 * qq) ** 2"), ("6.71", "6.17")])
def test_bbks_pins_catch_a_planted_typo(typo):
    """The pins above reject a copy of the oracle's T(q) with one constant or
    exponent mistyped (the mistake is planted in a copy of the oracle's source,
    on the CPU)."""
    import inspect
    src = inspect.getsource(cosmology.bbks_transfer)
    assert typo[0] in src
    scope = {"np": np}
    exec(src.replace(typo[0], typo[1], 1), scope)
    assert not _bbks_pins_hold(scope["bbks_transfer"], _bbks_constants())


# ---------------------------------------------------------- initial field
def test_linear_field_hermitian_cut_and_real():
    N, L, n_max = 24, 300.0, 3
    d = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, seed=11)
    idx = (-np.arange(N)) % N
    assert np.array_equal(d, np.conj(d[idx][:, idx][:, :, idx]))
    assert d[0, 0, 0] == 0
    assert not np.any(d[spt.nyquist_mask(N)])
    sx, sy, sz = spt.wave_indices(N)
    s2 = sx ** 2 + sy ** 2 + sz ** 2
    r = N / (n_max + 1)
    assert not np.any(d[s2 > r * r])
    assert np.all(d[(s2 <= r * r) & (s2 > 0)] != 0)
    x = spt.backward(d)
    assert np.abs(x.imag).max() < 1e-12 * np.abs(x.real).max()


def test_linear_field_gaussian_statistics():
    """L^3 |delta|^2 / P(k) has mean 1 and Re/Im parts are N(0, 1/2) after
    normalising: catches a missing 1/sqrt(2), L^3 or a wrong Box-Muller."""
    N, L, n_max = 48, 500.0, 1
    c = cosmology.DEFAULT_COSMO
    d = spt.linear_field(N, L, n_max, c, seed=3)
    k, s2 = estimators.mode_k(N, L)
    sel = (d != 0)
    ratio = L ** 3 * np.abs(d[sel]) ** 2 / cosmology.linear_pk(k[sel], c)
    n = ratio.size // 2  # pairs are not independent
    assert abs(ratio.mean() - 1.0) < 5.0 / math.sqrt(n)
    z = d[sel] / np.sqrt(cosmology.linear_pk(k[sel], c) / L ** 3)
    assert abs(z.real.std() ** 2 - 0.5) < 5 * 0.5 * math.sqrt(2.0 / n)
    assert abs(z.real.mean()) < 5 * math.sqrt(0.5 / n)


def test_linear_field_shared_modes_across_grids():
    """Keying by wavevector: the same seed and box on N and 2N share the
    common in-band modes exactly."""
    c = cosmology.DEFAULT_COSMO
    a = spt.linear_field(16, 200.0, 3, c, seed=5, kcut_lin=2 * math.pi / 200.0 * 3.5)
    b = spt.linear_field(32, 200.0, 3, c, seed=5, kcut_lin=2 * math.pi / 200.0 * 3.5)
    s = spt.signed_index(16)
    ii = s % 32
    assert np.array_equal(a, b[np.ix_(ii, ii, ii)])


# ------------------------------------------------------- recursion pins
def test_single_plane_wave_all_orders():
    """1D wave: planar SPT is Zel'dovich; delta_n(+-m k_F) =
    (-1)^j m^n (A/2)^n / (j! (m+j)!), n = m + 2j, theta_n = delta_n, zero
    elsewhere. Catches a wrong recursion coefficient or a dropped term at any order."""
    N, L, A = 16, 100.0, 0.1
    d1 = inputs.plane_waves(N, [((1, 0, 0), A)])
    dk, tk = spt.run_orders(d1, L, 5)
    for n in range(1, 6):
        exp = np.zeros((N, N, N))
        for m in range(n % 2, n + 1, 2):
            j = (n - m) // 2
            v = (-1) ** j * m ** n * (A / 2) ** n / (math.factorial(j) * math.factorial(m + j))
            exp[m % N, 0, 0] = v
            exp[-m % N, 0, 0] = v
        scale = (A / 2) ** n
        assert np.abs(dk[n] - exp).max() < 1e-12 * scale, n
        assert np.abs(tk[n] - exp).max() < 1e-12 * scale, n


def test_fourier_recursion_reduces_to_textbook_f2():
    g = inputs.rng(4)
    for _ in range(20):
        q1, q2 = g.standard_normal(3), g.standard_normal(3)
        F, G = kernels.fg_sym(q1, q2)
        Fc, Gc = kernels.f2_closed(q1, q2)
        assert abs(F - Fc) < 1e-13 and abs(G - Gc) < 1e-13


def test_two_plane_waves_second_order():
    """delta_2(k1+k2) = F_2 A1 A2 / 2 and theta_2 = G_2 A1 A2 / 2 with the
    textbook F_2, G_2; also k1-k2 and 2 k1 (catches a transposed tensor index
    or a sign error in u = -i k theta / k^2)."""
    N, L = 16, 200.0
    kF = 2 * math.pi / L
    s1, s2 = np.array([1, 0, 0]), np.array([1, 2, 0])
    A1, A2 = 0.07, 0.05
    d1 = inputs.plane_waves(N, [(tuple(s1), A1), (tuple(s2), A2)])
    dk, tk = spt.run_orders(d1, L, 2)
    for t, (qa, qb), amp in [(s1 + s2, (s1, s2), A1 * A2 / 2), (s1 - s2, (s1, -s2), A1 * A2 / 2),
                             (2 * s1, (s1, s1), A1 * A1 / 4)]:
        F, G = kernels.f2_closed(kF * qa, kF * qb)
        idx = tuple(int(c) % N for c in t)
        assert abs(dk[2][idx] - F * amp) < 1e-14
        assert abs(tk[2][idx] - G * amp) < 1e-14


def _mode_sum(d1, L, order, kernel_index):
    """Brute-force delta_n(k) (or theta_n) = sum over ordered n-tuples of nonzero
    linear modes of F_n^s(q_1..q_n) prod delta_1(q_i), for sparse delta_1."""
    N = d1.shape[0]
    kF = 2 * math.pi / L
    nz = np.argwhere(d1 != 0)
    s = spt.signed_index(N)
    out = {}
    for tup in itertools.product(range(len(nz)), repeat=order):
        qs = [kF * np.array([s[c] for c in nz[i]], float) for i in tup]
        tot = sum(np.array([s[c] for c in nz[i]]) for i in tup)
        fg = kernels.fg_sym(*qs)[kernel_index]
        val = fg * np.prod([d1[tuple(nz[i])] for i in tup])
        key = tuple(int(c) for c in tot)
        out[key] = out.get(key, 0) + val
    return out


def test_three_plane_waves_third_order_mode_sum():
    """delta_3 and theta_3 at every mode equal the ordered triple mode sum with
    the symmetrised F_3 / G_3 of the Fourier recursion (no aliasing at N=24)."""
    N, L = 24, 300.0
    d1 = inputs.plane_waves(N, [((1, 0, 0), 0.05), ((1, 1, 0), 0.04), ((0, 1, 2), 0.03)])
    dk, tk = spt.run_orders(d1, L, 3)
    for which, arr in [(0, dk[3]), (1, tk[3])]:
        exp = _mode_sum(d1, L, 3, which)
        got_max = 0.0
        full = np.zeros_like(arr)
        for key, v in exp.items():
            full[tuple(c % N for c in key)] += v
        scale = np.abs(full).max()
        assert np.abs(arr - full).max() < 1e-12 * scale
        got_max = np.abs(arr).max()
        assert got_max > 0


def test_random_field_second_order_mode_sum():
    """Random band-limited delta_1 on 12^3: grid delta_2 equals the pair mode sum
    with textbook F_2 at every mode |k| < K_c (exact in band)."""
    N, L, n_max = 12, 150.0, 3
    d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, seed=21)
    dk, tk = spt.run_orders(d1, L, 2)
    kF = 2 * math.pi / L
    s = spt.signed_index(N)
    nz = np.argwhere(d1 != 0)
    qv = np.array([[s[c] for c in p] for p in nz])
    amp = np.array([d1[tuple(p)] for p in nz])
    r = N / (n_max + 1)
    expF = {}
    expG = {}
    for i in range(len(nz)):
        for j in range(len(nz)):
            t = qv[i] + qv[j]
            if t @ t >= r * r:
                continue
            key = tuple(int(c) for c in t)
            if not np.any(qv[i] + qv[j]):
                F = G = 0.0   # F_2(q, -q) = G_2(q, -q) = 0
            else:
                F, G = kernels.f2_closed(kF * qv[i], kF * qv[j])
            expF[key] = expF.get(key, 0) + F * amp[i] * amp[j]
            expG[key] = expG.get(key, 0) + G * amp[i] * amp[j]
    scale = np.abs(dk[2]).max()
    for key in expF:
        idx = tuple(c % N for c in key)
        assert abs(dk[2][idx] - expF[key]) < 1e-12 * scale
        assert abs(tk[2][idx] - expG[key]) < 1e-12 * scale


# ------------------------------------------------------------- invariants
@pytest.fixture(scope="module")
def random_orders():
    N, L, n_max = 16, 200.0, 5
    d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, seed=8)
    return N, L, n_max, d1, spt.run_orders(d1, L, n_max)


def test_mass_conservation_every_order(random_orders):
    N, L, n_max, d1, (dk, tk) = random_orders
    for n in range(2, n_max + 1):
        scale = np.abs(dk[n]).max()
        assert abs(dk[n][0, 0, 0]) < 1e-12 * scale
        assert abs(tk[n][0, 0, 0]) < 1e-12 * scale


def test_hermitian_every_order(random_orders):
    N, L, n_max, d1, (dk, tk) = random_orders
    idx = (-np.arange(N)) % N
    for n in range(2, n_max + 1):
        for a in (dk[n], tk[n]):
            mirror = np.conj(a[idx][:, idx][:, :, idx])
            assert np.abs(a - mirror).max() < 1e-13 * np.abs(a).max()


def test_exact_power_of_two_scaling(random_orders):
    """delta_1 -> 2 delta_1 gives delta_n -> 2^n delta_n bit for bit (Sec. II.B
    growth-factor expansion: delta_n scales as D_+^n)."""
    N, L, n_max, d1, (dk, tk) = random_orders
    dk2, tk2 = spt.run_orders(2.0 * d1, L, n_max)
    for n in range(2, n_max + 1):
        assert np.array_equal(dk2[n], 2.0 ** n * dk[n])
        assert np.array_equal(tk2[n], 2.0 ** n * tk[n])


def test_zero_padding_invariance_in_band():
    """The same band-limited delta_1 on 12^3 and on the 4x zero-padded 48^3 grid
    gives equal delta_n, theta_n at every |k| < K_c (alias cut is exact in band)."""
    N, L, n_max = 12, 150.0, 5
    d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, seed=17)
    big = np.zeros((4 * N,) * 3, dtype=complex)
    s = spt.signed_index(N)
    ii = s % (4 * N)
    big[np.ix_(ii, ii, ii)] = d1
    dk, tk = spt.run_orders(d1, L, n_max)
    dkb, tkb = spt.run_orders(big, L, n_max)
    sx, sy, sz = spt.wave_indices(N)
    band = (sx ** 2 + sy ** 2 + sz ** 2) < (N / (n_max + 1)) ** 2
    for n in range(2, n_max + 1):
        small = dk[n][band]
        large = dkb[n][np.ix_(ii, ii, ii)][band]
        assert np.abs(small - large).max() < 1e-10 * np.abs(large).max(), n
        small = tk[n][band]
        large = tkb[n][np.ix_(ii, ii, ii)][band]
        assert np.abs(small - large).max() < 1e-10 * np.abs(large).max(), n


def test_translation_covariance():
    """delta_1(k) e^{-i k.d} -> delta_n(k) e^{-i k.d} for a grid shift d."""
    N, L, n_max = 12, 150.0, 4
    d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, seed=2)
    sx, sy, sz = spt.wave_indices(N)
    ph = np.exp(-2j * math.pi * (2 * sx + 5 * sy - 3 * sz) / N)
    dk, _ = spt.run_orders(d1, L, n_max)
    dks, _ = spt.run_orders(d1 * ph, L, n_max)
    for n in range(2, n_max + 1):
        assert np.abs(dks[n] - dk[n] * ph).max() < 1e-12 * np.abs(dk[n]).max()


# ------------------------------------------------------------- estimators
def test_power_on_hand_built_spectrum():
    """A spectrum with a(k) = sqrt(c_i / L^3) on shell i (and b = a) gives
    P = c_i and N_k equal to a direct count of integer vectors."""
    N, L = 16, 100.0
    kF = 2 * math.pi / L
    edges = [kF * (b + 0.5) for b in range(6)]
    vals = [3.0, 5.0, 7.0, 11.0, 13.0]
    sx, sy, sz = spt.wave_indices(N)
    r = np.sqrt(sx ** 2 + sy ** 2 + sz ** 2)
    a = np.zeros((N, N, N), complex)
    for i, v in enumerate(vals):
        a[(r >= i + 0.5) & (r < i + 1.5)] = math.sqrt(v / L ** 3)
    p, nk = estimators.power(a, a, L, edges)
    assert np.allclose(p, vals, rtol=1e-14)
    for i in range(5):
        cnt = sum(1 for x in range(-8, 8) for y in range(-8, 8) for z in range(-8, 8)
                  if (i + 0.5) ** 2 <= x * x + y * y + z * z < (i + 1.5) ** 2)
        assert nk[i] == cnt
    # cross term: Re part only
    b = 1j * a
    p2, _ = estimators.power(a, b, L, edges)
    assert np.abs(p2).max() < 1e-14


def test_bispectrum_fft_estimator_equals_triangle_enumeration():
    N, L = 12, 120.0
    kF = 2 * math.pi / L
    a = spt.linear_field(N, L, 3, cosmology.DEFAULT_COSMO, seed=31)
    b = spt.linear_field(N, L, 3, cosmology.DEFAULT_COSMO, seed=32)
    edges = [kF * e for e in (0.5, 1.5, 2.5, 3.5)]
    E, nt = estimators.bispectrum_equilateral(a, b, L, edges)
    Eb, ntb = estimators.bispectrum_brute(a, b, L, edges)
    assert np.allclose(nt, ntb, rtol=1e-12, atol=1e-9)
    assert np.allclose(E, Eb, rtol=1e-10, atol=0)
    # independent count of closed ordered triangles of integer vectors per shell
    for i in range(3):
        lo, hi = (i + 0.5) ** 2, (i + 1.5) ** 2
        vecs = [(x, y, z) for x in range(-5, 6) for y in range(-5, 6) for z in range(-5, 6)
                if lo <= x * x + y * y + z * z < hi]
        vs = set(vecs)
        cnt = sum(1 for p in vecs for q in vecs
                  if (-(p[0] + q[0]), -(p[1] + q[1]), -(p[2] + q[2])) in vs)
        assert round(nt[i]) == cnt


# ------------------------------------------------------------ emulator MLP
def test_mlp_backward_matches_finite_differences():
    """The oracle's analytic gradient against central differences of its own
    forward pass (catches a transposed weight or a wrong SiLU derivative)."""
    from oracle import mlp
    H, O, B = 7, 5, 6
    g = inputs.rng(3)
    theta = g.standard_normal(mlp.n_params(H, O)) * 0.5
    x = g.standard_normal((B, 3))
    t = g.standard_normal((B, O))
    mask = (g.random((B, O)) > 0.2).astype(float)
    y, acts = mlp.forward(x, theta, H, O)
    L, dy = mlp.masked_mse(y, t, mask)
    grad = mlp.backward(x, theta, H, O, acts, dy)
    h = 1e-6
    for i in g.choice(theta.size, 40, replace=False):
        e = np.zeros_like(theta)
        e[i] = h
        Lp = mlp.masked_mse(mlp.forward(x, theta + e, H, O)[0], t, mask)[0]
        Lm = mlp.masked_mse(mlp.forward(x, theta - e, H, O)[0], t, mask)[0]
        assert abs((Lp - Lm) / (2 * h) - grad[i]) < 1e-7 * max(1.0, abs(grad[i]))


def test_silu_and_derivative_closed_values():
    from oracle import mlp
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.silu(np.array([1.0]))[0] - 1.0 / (1.0 + math.exp(-1.0))) < 1e-15
    assert abs(mlp.silu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    # large |z|: SiLU -> z (slope 1) and -> 0 (slope 0)
    assert abs(mlp.silu_grad(np.array([40.0]))[0] - 1.0) < 1e-12
    assert abs(mlp.silu_grad(np.array([-40.0]))[0]) < 1e-12


def test_adam_first_step_is_sign_step():
    """With m = v = 0, the bias-corrected first Adam step is lr * g / (|g| + eps)."""
    from oracle import mlp
    th = np.array([1.0, -2.0, 0.5])
    gr = np.array([0.3, -4.0, 1e-3])
    new, m, v = mlp.adam_step(th, gr, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(new, th - 0.01 * gr / (np.abs(gr) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_rounding_ties_and_range():
    from oracle import mlp
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -7]))[0] == 1.0 + 2.0 ** -7
    x = inputs.rng(1).standard_normal(1000)
    assert np.max(np.abs(mlp.bf16_round(x) / x - 1)) <= 2.0 ** -8


# ------------------------------------------------------- block evaluation (cutout)
def test_cutout_modes_equal_full_grid_draw():
    """The in-band canonical modes drawn one by one equal the full-grid field
    at those modes, and the grid holds nothing else (its other half is their
    conjugates)."""
    N, L, n_max, seed = 24, 150.0, 3, 17
    full = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, seed)
    sx, sy, sz, val = cutout.linear_modes(N, L, n_max, cosmology.DEFAULT_COSMO, seed)
    assert np.array_equal(full[sx % N, sy % N, sz % N], val)
    assert np.array_equal(full[-sx % N, -sy % N, -sz % N], np.conj(val))
    assert np.count_nonzero(full) == 2 * val.size


def test_cutout_second_order_plane_wave_closed_form():
    """One wave delta_1 = A cos(k.x): delta_2 = theta_2 = A^2 cos(2 k.x) (the
    Zel'dovich solution of a single wave), at a block that wraps around the box."""
    N, L, A = 32, 100.0, 0.3
    s = np.array([1]), np.array([2]), np.array([3])
    d2, t2 = cutout.second_order_at_block(*s, np.array([A / 2 + 0j]), N, L, origin=(29, 5, 30), size=4)
    a = (29 + np.arange(4)) % N
    b = (5 + np.arange(4)) % N
    c = (30 + np.arange(4)) % N
    ph = 2 * math.pi * (a[:, None, None] + 2 * b[None, :, None] + 3 * c[None, None, :]) / N
    exp = A * A * np.cos(2 * ph)
    assert np.max(np.abs(d2 - exp)) < 1e-13
    assert np.max(np.abs(t2 - exp)) < 1e-13


def test_cutout_second_order_equals_full_grid_oracle():
    """Direct mode sums at a block equal the full-grid recursion (FFT based) at
    the same cells for a random band-limited field."""
    N, L, n_max, seed = 16, 120.0, 5, 23
    d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, seed)
    ref = spt.real_space_orders(d1, L, 2)[2]
    sx, sy, sz, val = cutout.linear_modes(N, L, n_max, cosmology.DEFAULT_COSMO, seed)
    origin = (13, 2, 9)
    d2, t2 = cutout.second_order_at_block(sx, sy, sz, val, N, L, origin, size=6)
    idx = [(o + np.arange(6)) % N for o in origin]
    for got, full in ((d2, ref[0]), (t2, ref[1])):
        want = full[np.ix_(*idx)]
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


# ------------------------------------------------------ divergence-form sources
def test_divergence_form_equals_direct_form_in_band():
    """A_n = div V_n, B_n = (1/2) nabla^2 S_n is an exact rewriting of the
    nine-term sources: modes below delta_1's cut agree to rounding at every
    order; orders 2 and 3 (products spanning at most 3 K_c <= k_Ny at
    n_max = 5) agree at every mode; delta_n(0) is exactly zero."""
    N, L, n_max = 24, 150.0, 5
    d1 = spt.linear_field(N, L, n_max, cosmology.DEFAULT_COSMO, 5)
    dk, tk = spt.run_orders(d1, L, n_max)
    vk, wk = spt.run_orders_divergence(d1, L, n_max)
    sx, sy, sz = spt.wave_indices(N)
    r = spt.cut_ratio(N, L, n_max, None)
    band = (sx * sx + sy * sy + sz * sz) < r * r
    for n in range(2, n_max + 1):
        for a, b in ((dk[n], vk[n]), (tk[n], wk[n])):
            scale = np.abs(a[band]).max()
            assert np.abs(a[band] - b[band]).max() <= 1e-13 * scale
            if n <= 3:
                assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
            assert b[0, 0, 0] == 0


def test_divergence_form_single_plane_wave_all_orders():
    """Zel'dovich closed form of one wave (no folding) in the divergence form."""
    N, L, A = 32, 100.0, 0.1
    d1 = inputs.plane_waves(N, [((1, 0, 0), A)])
    dk, tk = spt.run_orders_divergence(d1, L, 5)
    for n in range(2, 6):
        exp = np.zeros((N, N, N), complex)
        for m in range(n % 2, n + 1, 2):
            j = (n - m) // 2
            v = (-1) ** j * m ** n * (A / 2) ** n / (math.factorial(j) * math.factorial(m + j))
            exp[m % N, 0, 0] = v
            exp[-m % N, 0, 0] = v
        assert np.abs(dk[n] - exp).max() < 1e-15
        assert np.abs(tk[n] - exp).max() < 1e-15


# ------------------------------------------------------- one-loop bispectrum
def test_triple_shell_estimator_equals_triangle_enumeration():
    """E[a, b, c] from the FFT shell estimator = the direct sum over closed
    triangles a(k1) b(k2) c(k3) / N_tri, three different random fields."""
    N, L = 12, 100.0
    f = [spt.forward(inputs.random_real((N, N, N), 300 + i)) for i in range(3)]
    for x in f:
        x[spt.nyquist_mask(N)] = 0
    kF = 2 * math.pi / L
    edges = [kF * 0.5, kF * 1.5, kF * 2.5]
    E, nt = estimators.bispectrum_triple(*f, L, edges)
    Eb, ntb = estimators.bispectrum_triple_brute(*f, L, edges)
    assert np.allclose(nt, ntb, rtol=0, atol=1e-9)
    assert np.allclose(E, Eb, rtol=1e-10, atol=1e-12 * np.abs(Eb).max())
    Ea, _ = estimators.bispectrum_equilateral(f[0], f[2], L, edges)     # E[a, a, c]
    Et, _ = estimators.bispectrum_triple(f[0], f[0], f[2], L, edges)
    assert np.allclose(Ea, Et, rtol=1e-12)


def test_one_loop_bispectrum_equals_enumeration_of_its_definition():
    """Eq. bk_1loop summed term by term over enumerated closed triangles
    equals the oracle's shell-estimator form (four different fields)."""
    N, L = 12, 100.0
    d = [spt.forward(inputs.random_real((N, N, N), 310 + i)) for i in range(4)]
    for x in d:
        x[spt.nyquist_mask(N)] = 0
    kF = 2 * math.pi / L
    edges = [kF * 0.5, kF * 1.5, kF * 2.5]
    B, nt = estimators.bispectrum_one_loop(*d, L, edges)
    d1, d2, d3, d4 = d
    Bb = 0.0
    for a, b, c in [(d1, d2, d3), (d1, d3, d2), (d2, d1, d3), (d2, d3, d1), (d3, d1, d2), (d3, d2, d1),
                    (d2, d2, d2), (d1, d1, d4), (d1, d4, d1), (d4, d1, d1)]:
        Bb = Bb + estimators.bispectrum_triple_brute(a, b, c, L, edges)[0]
    assert np.allclose(B, Bb, rtol=1e-10, atol=1e-12 * np.abs(Bb).max())


# ------------------------------------------------- summed fields, correlation
def test_growth_factor_eds_and_ode():
    """D_+(z)/D_+(0): Einstein-de Sitter gives a = 1/(1+z) exactly; for LCDM the
    integral form equals the growing solution of the linear growth ODE
    D'' + (3/a + dlnE/da) D' - 1.5 Om / (a^5 E^2) D = 0 integrated from deep in
    matter domination (D = a there)."""
    from scipy.integrate import solve_ivp
    eds = dict(cosmology.DEFAULT_COSMO, omega_m=1.0)
    for z in (0.0, 0.5, 1.0, 3.0):
        assert abs(cosmology.growth_factor(z, eds) - 1.0 / (1.0 + z)) < 1e-10
    om = 0.3
    E = lambda a: math.sqrt(om / a ** 3 + 1 - om)
    dlnE = lambda a: -1.5 * om / a ** 4 / E(a) ** 2

    def rhs(a, y):
        D, dD = y
        return [dD, -(3.0 / a + dlnE(a)) * dD + 1.5 * om / (a ** 5 * E(a) ** 2) * D]

    a0 = 1e-4
    sol = solve_ivp(rhs, (a0, 1.0), [a0, 1.0], rtol=1e-11, atol=1e-14, dense_output=True)
    c = dict(cosmology.DEFAULT_COSMO, omega_m=om)
    for z in (0.5, 1.0, 2.0):
        ode = sol.sol(1.0 / (1.0 + z))[0] / sol.sol(1.0)[0]
        assert abs(cosmology.growth_factor(z, c) - ode) < 1e-6


def test_sum_orders_smooths_a_plane_wave_by_the_gaussian():
    """One wave per order: the smoothed sum is sum_i D^i A_i e^{-k^2 R^2/2} cos(k.x)
    at every cell (direct evaluation in real space)."""
    N, L, R, D = 16, 100.0, 7.0, 0.6
    waves = [((1, 2, 0), 0.3), ((2, 0, 1), 0.2)]
    f1 = inputs.plane_waves(N, [waves[0]])
    f2 = inputs.plane_waves(N, [waves[1]])
    got = spt.backward(spt.sum_orders([f1, f2], D, R, L)).real
    j = np.arange(N)
    x, y, z = np.meshgrid(j, j, j, indexing="ij")
    exp = 0.0
    for i, ((s, A)) in enumerate(waves, start=1):
        k2 = (2 * math.pi / L) ** 2 * sum(c * c for c in s)
        exp = exp + D ** i * A * math.exp(-0.5 * k2 * R * R) * np.cos(2 * math.pi * (s[0] * x + s[1] * y + s[2] * z) / N)
    assert np.abs(got - exp).max() < 1e-13


def test_cross_correlation_limits_and_definition():
    N, L = 16, 120.0
    a = spt.forward(inputs.random_real((N, N, N), 41))
    b = spt.forward(inputs.random_real((N, N, N), 42))
    kF = 2 * math.pi / L
    edges = [kF * e for e in (0.5, 2.5, 4.5, 7.5)]
    assert np.allclose(estimators.cross_correlation(a, 3.0 * a, L, edges), 1.0, atol=1e-14)
    assert np.allclose(estimators.cross_correlation(a, -a, L, edges), -1.0, atol=1e-14)
    r = estimators.cross_correlation(a, b, L, edges)
    assert np.all(np.abs(r) <= 1.0)
    # against the estimator's power spectra: r = P_ab / sqrt(P_aa P_bb)
    pab = estimators.power(a, b, L, edges)[0]
    paa = estimators.power(a, a, L, edges)[0]
    pbb = estimators.power(b, b, L, edges)[0]
    assert np.allclose(r, pab / np.sqrt(paa * pbb), rtol=1e-12)
