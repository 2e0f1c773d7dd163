"""GridSPT in plain FP64 on full complex grids (oracle side).

Follows the paper step by step:

* DFT convention of Sec. II.C (the discrete transform pair defined there):
  a(x) = sum_k a(k) e^{i k.x},  a(k) = N^-3 sum_x a(x) e^{-i k.x},
  k = (2 pi / L) s with signed integer s, x_j = j L / N.
* Step (1): Gaussian delta_0(k) from P_0(k); Eq. ``recursion_n=1``: delta_1 = theta_1.
* Steps (2) and (5): multiply the order-m spectra by 1, i k, -i k / k^2 and
  k_i k_j / k^2 (u = grad nabla^-2 theta, Eq. ``u_and_theta``) and
  transform back to real space.
* Steps (3) and (6): Eq. ``recursion_formula``,
      (delta_n, theta_n) = 2/((2n+3)(n-1)) [[n+1/2, 1], [3/2, n]] (A_n, B_n),
      A_n = sum_{m=1}^{n-1} grad delta_m . u_{n-m} + delta_m theta_{n-m},
      B_n = sum_{m=1}^{n-1} d_j(u_m)_k d_k(u_{n-m})_j + u_m . grad theta_{n-m},
  evaluated cell by cell with all nine tensor terms written out.
* Step (4): forward transform of delta_n and theta_n.

Readings where the paper is silent (each listed with its reason in the design
notes): the alias cut is applied to delta_1 only, at |k| <= k_cut (default
2 k_Ny / (n_max + 1)); modes with any component at the Nyquist index -N/2 are
zero in every spectrum; the k = 0 mode of delta_1 and every 1/k^2 multiplier at
k = 0 are zero.

Everything is FP64 on the full N^3 complex grid (numpy's FFT as the transform
primitive), with no blocking, fusion or symmetry shortcuts.
"""
import math

import numpy as np

from . import cosmology, rng


# --------------------------------------------------------------------------- grid
def signed_index(N):
    n = np.arange(N)
    return np.where(n < N // 2, n, n - N)


def wave_indices(N):
    s = signed_index(N)
    return np.meshgrid(s, s, s, indexing="ij")


def nyquist_mask(N):
    sx, sy, sz = wave_indices(N)
    h = -(N // 2)
    return (sx == h) | (sy == h) | (sz == h)


def cut_ratio(N, L, n_max, kcut):
    """k_cut / k_F. Default cut 2 k_Ny / (n_max + 1) gives N / (n_max + 1)."""
    if kcut is None or kcut <= 0:
        return N / (n_max + 1)
    return kcut * L / (2.0 * math.pi)


def backward(fk):
    """a(x) = sum_k a(k) e^{+i k.x} on the full grid."""
    N = fk.shape[0]
    return np.fft.ifftn(fk) * float(N) ** 3


def forward(fx):
    """a(k) = N^-3 sum_x a(x) e^{-i k.x}."""
    N = fx.shape[0]
    return np.fft.fftn(fx) / float(N) ** 3


def to_real(fx, what="field"):
    """Backward transforms of Hermitian spectra are real; check and drop Im."""
    scale = np.max(np.abs(fx.real)) if fx.size else 0.0
    if scale > 0:
        assert np.max(np.abs(fx.imag)) <= 1e-9 * scale, f"{what}: non-Hermitian spectrum"
    return fx.real.copy()


# --------------------------------------------------------------- initial field
def linear_field(N, L, n_max, cosmo, seed, kcut_lin=None, A=None):
    """delta_1(k) = sqrt(P(|k|) / L^3) (g1 + i g2) / sqrt(2), Hermitian.

    Each mode pair {s, -s} draws one Philox output keyed by the canonical member
    c (c_z > 0, or c_z = 0 and c_y > 0, or c_z = c_y = 0 and c_x > 0); the other
    member is the complex conjugate. g1 + i g2 = sqrt(-2 ln u1) e^{2 pi i u2}
    (Box-Muller). Zero: k = 0, any Nyquist component, and |s|^2 > (k_cut/k_F)^2.
    """
    sx, sy, sz = wave_indices(N)
    s2 = (sx * sx + sy * sy + sz * sz).astype(np.float64)
    r = cut_ratio(N, L, n_max, kcut_lin)
    valid = (s2 > 0) & (s2 <= r * r) & ~nyquist_mask(N)
    canon = (sz > 0) | ((sz == 0) & (sy > 0)) | ((sz == 0) & (sy == 0) & (sx > 0))
    cx = np.where(canon, sx, -sx)[valid]
    cy = np.where(canon, sy, -sy)[valid]
    cz = np.where(canon, sz, -sz)[valid]
    u1, u2 = rng.mode_uniforms(seed, cx, cy, cz)
    g = np.sqrt(-2.0 * np.log(u1)) * (np.cos(2.0 * math.pi * u2) + 1j * np.sin(2.0 * math.pi * u2))
    kF = 2.0 * math.pi / L
    k = kF * np.sqrt(s2[valid])
    amp = np.sqrt(cosmology.linear_pk(k, cosmo, A) / L ** 3)
    val = amp * g / math.sqrt(2.0)
    val = np.where(canon[valid], val, np.conj(val))
    d = np.zeros((N, N, N), dtype=np.complex128)
    d[valid] = val
    return d


# ------------------------------------------------------------- derived fields
def derived_fields(delta_k, theta_k, L):
    """Real-space fields of one order from its two spectra (steps (2)/(5)).

    Returns a dict: 'd' = delta, 't' = theta, 'gd'[a] = d_a delta,
    'gt'[a] = d_a theta, 'u'[a] = u_a, 'du'[a][b] = d_a u_b (all nine)."""
    N = delta_k.shape[0]
    kF = 2.0 * math.pi / L
    sx, sy, sz = wave_indices(N)
    kv = [kF * sx, kF * sy, kF * sz]
    k2 = kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2
    inv_k2 = np.zeros_like(k2)
    inv_k2[k2 > 0] = 1.0 / k2[k2 > 0]
    out = {
        "d": to_real(backward(delta_k), "delta"),
        "t": to_real(backward(theta_k), "theta"),
        "gd": [to_real(backward(1j * kv[a] * delta_k), "grad delta") for a in range(3)],
        "gt": [to_real(backward(1j * kv[a] * theta_k), "grad theta") for a in range(3)],
        "u": [to_real(backward(-1j * kv[a] * inv_k2 * theta_k), "u") for a in range(3)],
        "du": [[to_real(backward(kv[a] * kv[b] * inv_k2 * theta_k), "grad u")
                for b in range(3)] for a in range(3)],
    }
    return out


def recursion_coefficients(n):
    c = 2.0 / ((2 * n + 3) * (n - 1))
    return c * (n + 0.5), c * 1.0, c * 1.5, c * n


def sources(fields, n):
    """A_n and B_n of Eq. recursion_formula at every cell (literal sums)."""
    A = 0.0
    B = 0.0
    for m in range(1, n):
        fm, fr = fields[m], fields[n - m]
        for a in range(3):
            A = A + fm["gd"][a] * fr["u"][a]
        A = A + fm["d"] * fr["t"]
        for j in range(3):
            for k in range(3):
                B = B + fm["du"][j][k] * fr["du"][k][j]
        for a in range(3):
            B = B + fm["u"][a] * fr["gt"][a]
    return A, B


def run_orders(delta1_k, L, n_max, kcut_nl=None):
    """All orders 1..n_max. Returns (delta_k, theta_k) lists indexed by order
    (index 0 unused). delta1_k must already be Hermitian with zero Nyquist modes."""
    N = delta1_k.shape[0]
    nyq = nyquist_mask(N)
    sx, sy, sz = wave_indices(N)
    s2 = (sx * sx + sy * sy + sz * sz).astype(np.float64)
    delta = [None, delta1_k.copy()]
    theta = [None, delta1_k.copy()]          # Eq. recursion_n=1
    fields = {}
    for n in range(2, n_max + 1):
        fields[n - 1] = derived_fields(delta[n - 1], theta[n - 1], L)
        A, B = sources(fields, n)
        cdA, cdB, ctA, ctB = recursion_coefficients(n)
        dn = forward(cdA * A + cdB * B)
        tn = forward(ctA * A + ctB * B)
        dn[nyq] = 0.0
        tn[nyq] = 0.0
        if kcut_nl is not None and kcut_nl > 0:
            r = kcut_nl * L / (2.0 * math.pi)
            dn[s2 > r * r] = 0.0
            tn[s2 > r * r] = 0.0
        delta.append(dn)
        theta.append(tn)
    return delta, theta


def run_orders_divergence(delta1_k, L, n_max, kcut_nl=None):
    """Eq. recursion_formula with its sources rewritten in divergence form.

    With u = grad nabla^-2 theta (Eq. u_and_theta), theta = div u and u curl free:
        grad delta_m . u_r + delta_m theta_r = div (delta_m u_r),
        sum over the ordered pairs (m, r) of [d_j u_{m,k} d_k u_{r,j} + u_m . grad theta_r]
            = (1/2) nabla^2 sum_m u_m . u_{n-m},
    so A_n = div V_n and B_n = (1/2) nabla^2 S_n with V_n = sum_m delta_m u_{n-m},
    S_n = sum_m u_m . u_{n-m} formed cell by cell. V_n and S_n are transformed
    forward, A_n(k) = i k . V_n(k) and B_n(k) = -(k^2 / 2) S_n(k) taken in
    k-space, and delta_n, theta_n follow from the same 2x2 recursion. Modes
    |k| < k_cut of delta_1's cut agree with ``run_orders`` to rounding (the
    identities hold exactly for products that do not fold); above it the
    folded parts of the products differ between the two forms.
    Returns (delta_k, theta_k) lists indexed by order like ``run_orders``."""
    N = delta1_k.shape[0]
    kF = 2.0 * math.pi / L
    nyq = nyquist_mask(N)
    sx, sy, sz = wave_indices(N)
    s2 = (sx * sx + sy * sy + sz * sz).astype(np.float64)
    kv = [kF * sx, kF * sy, kF * sz]
    k2 = kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2
    inv_k2 = np.zeros_like(k2)
    inv_k2[k2 > 0] = 1.0 / k2[k2 > 0]
    delta = [None, delta1_k.copy()]
    theta = [None, delta1_k.copy()]          # Eq. recursion_n=1
    d_x, u_x = {}, {}
    for n in range(2, n_max + 1):
        m = n - 1
        d_x[m] = to_real(backward(delta[m]), "delta")
        u_x[m] = [to_real(backward(-1j * kv[a] * inv_k2 * theta[m]), "u") for a in range(3)]
        V = [0.0, 0.0, 0.0]
        S = 0.0
        for m in range(1, n):
            r = n - m
            for a in range(3):
                V[a] = V[a] + d_x[m] * u_x[r][a]
                S = S + u_x[m][a] * u_x[r][a]
        A = sum(1j * kv[a] * forward(V[a]) for a in range(3))
        B = -0.5 * k2 * forward(S)
        cdA, cdB, ctA, ctB = recursion_coefficients(n)
        dn = cdA * A + cdB * B
        tn = ctA * A + ctB * B
        dn[nyq] = 0.0
        tn[nyq] = 0.0
        if kcut_nl is not None and kcut_nl > 0:
            rr = kcut_nl * L / (2.0 * math.pi)
            dn[s2 > rr * rr] = 0.0
            tn[s2 > rr * rr] = 0.0
        delta.append(dn)
        theta.append(tn)
    return delta, theta


def real_space_orders(delta1_k, L, n_max, kcut_nl=None):
    """delta_n(x) and theta_n(x) as formed by the recursion before the forward
    transform (step (3)/(6) output), for n = 2..n_max."""
    N = delta1_k.shape[0]
    delta_k, theta_k = run_orders(delta1_k, L, n_max, kcut_nl)
    out = {}
    fields = {}
    for n in range(2, n_max + 1):
        fields[n - 1] = derived_fields(delta_k[n - 1], theta_k[n - 1], L)
        A, B = sources(fields, n)
        cdA, cdB, ctA, ctB = recursion_coefficients(n)
        out[n] = (cdA * A + cdB * B, ctA * A + ctB * B)
    return out


def sum_orders(fields_k, D, R, L):
    """delta_SPT(k) = W(k R) sum_{i=1}^{n} D^i delta_i(k) (Sec. III.A), with the
    Gaussian filter W(x) = exp(-x^2 / 2) the paper applies before looking at
    the fields (R = 0: no filter). fields_k: [delta_1, ..., delta_n] full grids."""
    N = fields_k[0].shape[0]
    kF = 2.0 * math.pi / L
    sx, sy, sz = wave_indices(N)
    k2 = kF * kF * (sx * sx + sy * sy + sz * sz).astype(np.float64)
    out = np.zeros_like(fields_k[0])
    for i, f in enumerate(fields_k, start=1):
        out = out + D ** i * f
    return out * np.exp(-0.5 * k2 * R * R)
