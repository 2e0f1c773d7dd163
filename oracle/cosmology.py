"""Linear power spectrum for the initial field (oracle side, FP64).

The paper draws the initial field from a linear spectrum P_0(k) (Sec. II.C,
step 1) computed for a WMAP5 cosmology (Sec. III) whose transfer function it
does not give. The reading used here: a BBKS fit (Bardeen, Bond, Kaiser &
Szalay 1986, Eq. G3) with shape parameter Gamma,

    T(q) = ln(1 + 2.34 q) / (2.34 q) * [1 + 3.89 q + (16.1 q)^2 + (5.46 q)^3
           + (6.71 q)^4]^(-1/4),      q = k / Gamma  (k in h/Mpc),

    P(k) = A k^{n_s} T(k/Gamma)^2,

with A fixed by sigma_8: sigma_R^2 = (1/2pi^2) int k^2 P(k) W(kR)^2 dk at
R = 8 Mpc/h, W(x) = 3 (sin x - x cos x) / x^3.
"""
import math

import numpy as np

SIGMA_R = 8.0  # Mpc/h


def bbks_transfer(q):
    q = np.asarray(q, dtype=np.float64)
    out = np.ones_like(q)
    nz = q > 0
    qq = q[nz]
    poly = 1.0 + 3.89 * qq + (16.1 * qq) ** 2 + (5.46 * qq) ** 3 + (6.71 * qq) ** 4
    out[nz] = np.log1p(2.34 * qq) / (2.34 * qq) * poly ** -0.25
    return out


def tophat_window(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-3
    xs = x[small]
    out[small] = 1.0 - xs ** 2 / 10.0 + xs ** 4 / 280.0
    xl = x[~small]
    out[~small] = 3.0 * (np.sin(xl) - xl * np.cos(xl)) / xl ** 3
    return out


def shape_gamma(cosmo):
    g = cosmo.get("gamma", 0.0)
    return g if g > 0 else cosmo["omega_m"] * cosmo["h"]


def unnormalised_pk(k, cosmo):
    """k^{n_s} T^2(k / Gamma) with A = 1."""
    k = np.asarray(k, dtype=np.float64)
    return k ** cosmo["n_s"] * bbks_transfer(k / shape_gamma(cosmo)) ** 2


def sigma_r_squared_unit(cosmo, R=SIGMA_R, n_intervals=1 << 16):
    """(1/2pi^2) int k^3 P_{A=1}(k) W(kR)^2 dlnk by composite Simpson in ln k
    over [1e-5, 1e3] h/Mpc."""
    lo, hi = math.log(1e-5), math.log(1e3)
    lnk = np.linspace(lo, hi, n_intervals + 1)
    k = np.exp(lnk)
    f = k ** 3 * unnormalised_pk(k, cosmo) * tophat_window(k * R) ** 2
    h = (hi - lo) / n_intervals
    w = np.ones(n_intervals + 1)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return h / 3.0 * np.dot(w, f) / (2.0 * math.pi ** 2)


def amplitude(cosmo):
    """A such that sigma_8 of A k^{n_s} T^2 equals cosmo['sigma8']."""
    return cosmo["sigma8"] ** 2 / sigma_r_squared_unit(cosmo)


def linear_pk(k, cosmo, A=None):
    if A is None:
        A = amplitude(cosmo)
    return A * unnormalised_pk(k, cosmo)


DEFAULT_COSMO = {"omega_m": 0.3, "h": 0.7, "n_s": 0.96, "sigma8": 0.8, "gamma": 0.0}


def growth_factor(z, cosmo, n_intervals=1 << 16):
    """Linear growth factor D_+(z) / D_+(0) of a flat LCDM background (the
    D_+ of Sec. II.A and of delta_SPT = sum D_+^i delta_i, Sec. III.A):
        D(a) = (5 Omega_m / 2) E(a) int_0^a da' / (a' E(a'))^3,
        E(a) = sqrt(Omega_m a^-3 + 1 - Omega_m)   (Heath 1977),
    the integral by composite Simpson in a (the integrand vanishes like
    a'^(3/2) at a' -> 0)."""
    om = cosmo["omega_m"]

    def D(a):
        x = np.linspace(0.0, a, n_intervals + 1)
        with np.errstate(divide="ignore", invalid="ignore"):
            E = np.sqrt(om / x ** 3 + 1.0 - om)
            f = np.where(x > 0, 1.0 / (x * E) ** 3, 0.0)
        h = a / n_intervals
        integral = h / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())
        return 2.5 * om * math.sqrt(om / a ** 3 + 1.0 - om) * integral

    return D(1.0 / (1.0 + z)) / D(1.0)
