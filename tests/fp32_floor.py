"""The rounding floor of FP32 fields, measured on the CPU (test code only).

The library keeps every field in FP32 (real-space products, transforms and
spectra); its P-term and field errors against the FP64 oracle are therefore
bounded below by what FP32 storage and arithmetic do to the recursion, whatever
the kernels. This module measures that floor with the oracle's own steps, so
that a GPU error can be compared with it:

* ``recursion_rounded_real``: the oracle's FP64 recursion in which only the
  real-space delta_n(x), theta_n(x) of each order are rounded to FP32 before
  their forward transform (the least rounding any implementation that forms
  the products in FP32 real-space fields must do);
* ``recursion_fp32``: the same steps with FP32 fields throughout: FP32 spectra
  and multipliers, single-precision transforms (scipy.fft on complex64), FP32
  products and sums (an independent FP32 implementation of the recursion).

The noise these leave in delta_n(k) is close to white (rounding of fields
whose power sits at high k), so it is described by one level per order,
s_n^2 = mean |e_n(k)|^2 over the modes below delta_1's cut. A binned P-term
error of such noise has standard deviation (the estimator's sum over the full
grid counts every pair {k, -k} twice)

    sigma_b(P_ij) = f sqrt(L^3 / N_b) (s_j sqrt(P_ii,b) + s_i sqrt(P_jj,b)),

f = 2 for the paper's cross terms (P_13 = 2 P(delta_1, delta_3)), and for
i = j, f = 1 with both terms present (2 s_i sqrt(P_ii,b)). The bar of a bin is
max(1e-5 |P_b|, z sigma_b): where FP32 rounding alone moves a bin by more than
1e-5 of its value, the 1e-5 bar measures FP32, not the path.

Imports the oracle (allowed for tests); the library never sees this module.
"""
import math
import os

import numpy as np
import scipy.fft as sfft

from oracle import estimators, spt

WORKERS = os.cpu_count() or 8


def _r32(x):
    return x.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(x) else \
        x.astype(np.float32).astype(np.float64)


def recursion_rounded_real(delta1_k, L, n_max):
    """Oracle recursion (FP64) with delta_n(x), theta_n(x) rounded to FP32
    before each forward transform. Returns delta_k indexed by order."""
    N = delta1_k.shape[0]
    nyq = spt.nyquist_mask(N)
    delta, theta, fields = [None, delta1_k], [None, delta1_k], {}
    for n in range(2, n_max + 1):
        fields[n - 1] = spt.derived_fields(delta[n - 1], theta[n - 1], L)
        A, B = spt.sources(fields, n)
        cdA, cdB, ctA, ctB = spt.recursion_coefficients(n)
        dn = spt.forward(_r32(cdA * A + cdB * B))
        tn = spt.forward(_r32(ctA * A + ctB * B))
        dn[nyq] = 0.0
        tn[nyq] = 0.0
        delta.append(dn)
        theta.append(tn)
    return delta


def recursion_fp32(delta1_k, L, n_max):
    """The recursion with FP32 fields, FP32 transforms and FP32 products.
    Returns delta_k indexed by order (complex128 holding FP32 values)."""
    N = delta1_k.shape[0]
    kF = np.float32(2.0 * math.pi / L)
    sx, sy, sz = spt.wave_indices(N)
    kv = [kF * s.astype(np.float32) for s in (sx, sy, sz)]
    k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]
    ik2 = np.zeros_like(k2)
    ik2[k2 > 0] = np.float32(1.0) / k2[k2 > 0]
    nyq = spt.nyquist_mask(N)
    cells = np.float32(N) ** 3

    def bw(fk):
        return (sfft.ifftn(fk.astype(np.complex64), workers=WORKERS) * cells).real.astype(np.float32)

    def fw(fx):
        return (sfft.fftn(fx.astype(np.float32), workers=WORKERS) / cells).astype(np.complex64)

    one_i = np.complex64(1j)
    delta = [None, delta1_k.astype(np.complex64)]
    theta = [None, delta1_k.astype(np.complex64)]
    F = {}
    for n in range(2, n_max + 1):
        m = n - 1
        dk, tk = delta[m], theta[m]
        F[m] = {"d": bw(dk), "t": bw(tk),
                "gd": [bw(one_i * kv[a] * dk) for a in range(3)],
                "gt": [bw(one_i * kv[a] * tk) for a in range(3)],
                "u": [bw(-one_i * kv[a] * ik2 * tk) for a in range(3)],
                "du": [[bw(kv[a] * kv[b] * ik2 * tk) for b in range(3)] for a in range(3)]}
        A = np.zeros((N, N, N), np.float32)
        B = np.zeros((N, N, N), np.float32)
        for mm in range(1, n):
            fm, fr = F[mm], F[n - mm]
            for a in range(3):
                A += fm["gd"][a] * fr["u"][a]
            A += fm["d"] * fr["t"]
            for j in range(3):
                for k in range(3):
                    B += fm["du"][j][k] * fr["du"][k][j]
            for a in range(3):
                B += fm["u"][a] * fr["gt"][a]
        cdA, cdB, ctA, ctB = (np.float32(c) for c in spt.recursion_coefficients(n))
        dn, tn = fw(cdA * A + cdB * B), fw(ctA * A + ctB * B)
        dn[nyq] = 0
        tn[nyq] = 0
        delta.append(dn)
        theta.append(tn)
    return [None] + [d.astype(np.complex128) for d in delta[1:]]


def inband_mask(N, n_max, kcut_ratio=None):
    """Modes |s|^2 <= floor(r^2), r = k_cut / k_F (default N / (n_max + 1))."""
    r = N / (n_max + 1) if kcut_ratio is None else kcut_ratio
    sx, sy, sz = spt.wave_indices(N)
    return (sx * sx + sy * sy + sz * sz) <= math.floor(r * r)


def noise_levels(got, ref, mask, orders):
    """s_n = RMS over the masked modes of got[n] - ref[n] (full grids)."""
    return {n: float(np.sqrt(np.mean(np.abs(got[n] - ref[n])[mask] ** 2))) for n in orders}


def pterm_sigma(ref, s, i, j, L, edges):
    """Standard deviation per bin of the error of P_ij (with the paper's factor
    2 for i != j) caused by white noise of levels s[n] in delta_n (s[1] = 0:
    both sides use the same initial field)."""
    pii, nk = estimators.power(ref[i], ref[i], L, edges)
    pjj, _ = estimators.power(ref[j], ref[j], L, edges)
    si, sj = s.get(i, 0.0), s.get(j, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        root = np.where(nk > 0, np.sqrt(L ** 3 / np.maximum(nk, 1)), 0.0)
    f = 1.0 if i == j else 2.0
    return f * root * (sj * np.sqrt(np.abs(pii)) + si * np.sqrt(np.abs(pjj)))


def pterm_bar(p_ref, sigma, nk, rel=1e-5, z=6.0, mask_frac=1e-3):
    """Per-bin bar max(rel |P|, z sigma) over the bins with N_k > 0 and
    |P| > mask_frac max |P|; returns (selected bins, bar, floor_used)."""
    sel = (nk > 0) & (np.abs(p_ref) > mask_frac * np.abs(p_ref).max())
    bar = np.maximum(rel * np.abs(p_ref), z * sigma)
    return sel, bar, z * sigma > rel * np.abs(p_ref)
