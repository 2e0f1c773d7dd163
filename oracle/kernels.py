"""Analytic Fourier-space SPT kernels F_n, G_n (oracle side, FP64).

Eq. ``PT_recursion_fourier`` (Sec. II.B) with the Einstein-de Sitter
coefficients that the real-space recursion (Eq. ``recursion_formula``) implies:

  F_n = sum_{m=1}^{n-1} G_m(q_1..q_m) [(2n+1) alpha(k1,k2) F_{n-m}(q_{m+1}..q_n)
                                      + 2 beta(k1,k2) G_{n-m}(q_{m+1}..q_n)] / ((2n+3)(n-1))
  G_n = sum_{m=1}^{n-1} G_m(q_1..q_m) [3 alpha(k1,k2) F_{n-m}(...)
                                      + 2n beta(k1,k2) G_{n-m}(...)] / ((2n+3)(n-1))

with k1 = q_1+..+q_m, k2 = q_{m+1}+..+q_n, alpha(k1,k2) = (k1+k2).k1 / k1^2,
beta(k1,k2) = |k1+k2|^2 (k1.k2) / (2 k1^2 k2^2), F_1 = G_1 = 1. The symmetrised
kernel averages over all orderings of the arguments. Used only to pin the grid
recursion (plane-wave and mode-sum tests), never by the GPU library.
"""
import itertools
import math

import numpy as np


def _alpha(k1, k2):
    n1 = np.dot(k1, k1)
    if n1 == 0:
        return 0.0
    return np.dot(k1 + k2, k1) / n1


def _beta(k1, k2):
    n1, n2 = np.dot(k1, k1), np.dot(k2, k2)
    if n1 == 0 or n2 == 0:
        return 0.0
    k12 = k1 + k2
    return np.dot(k12, k12) * np.dot(k1, k2) / (2.0 * n1 * n2)


def _fg(qs):
    n = len(qs)
    if n == 1:
        return 1.0, 1.0
    F = G = 0.0
    for m in range(1, n):
        k1 = np.sum(qs[:m], axis=0)
        k2 = np.sum(qs[m:], axis=0)
        _, Gm = _fg(qs[:m])
        Fr, Gr = _fg(qs[m:])
        a, b = _alpha(k1, k2), _beta(k1, k2)
        F += Gm * ((2 * n + 1) * a * Fr + 2.0 * b * Gr)
        G += Gm * (3.0 * a * Fr + 2.0 * n * b * Gr)
    d = (2 * n + 3) * (n - 1)
    return F / d, G / d


def fg_sym(*qs):
    """Symmetrised (F_n, G_n) at wavevectors q_1..q_n (3-vectors)."""
    qs = [np.asarray(q, dtype=np.float64) for q in qs]
    F = G = 0.0
    perms = list(itertools.permutations(range(len(qs))))
    for p in perms:
        f, g = _fg([qs[i] for i in p])
        F += f
        G += g
    return F / len(perms), G / len(perms)


def f2_closed(q1, q2):
    """Textbook EdS F_2 and G_2 in terms of mu and the magnitude ratio."""
    q1 = np.asarray(q1, float)
    q2 = np.asarray(q2, float)
    a, b = math.sqrt(np.dot(q1, q1)), math.sqrt(np.dot(q2, q2))
    mu = np.dot(q1, q2) / (a * b)
    F = 5.0 / 7.0 + 0.5 * mu * (a / b + b / a) + 2.0 / 7.0 * mu * mu
    G = 3.0 / 7.0 + 0.5 * mu * (a / b + b / a) + 4.0 / 7.0 * mu * mu
    return F, G
