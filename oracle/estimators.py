"""Shell estimators (oracle side, FP64, full complex grid).

Power (Sec. III.B.1, Eqs. ``pk_lin``, ``pk_1loop``, ``pk_2loop``): for a bin
[e_i, e_{i+1}) (lower edge inclusive) the estimator is

    P_ab(i) = L^3 / N_i * sum_{k in bin} Re[a(k) b*(k)],

summed over every mode of the full grid with k = k_F sqrt(|s|^2) != 0, N_i the
number of such modes. The paper prints the sums without the volume factor L^3
and without saying how N_k is counted; with this reading <P_11> = P_0(k).
The paper's cross terms carry 2 Re[...]: P_13 = 2 P(delta_1, delta_3).

Bispectrum (Eq. ``bk_tree``, measured with an FFT shell estimator): for an
equilateral shell b, with I_b[f](x) = sum_{k in b} f(k) e^{i k.x} and
J_b(x) = sum_{k in b} e^{i k.x},

    E_b[a, a, b] = L^6 sum_x I_b[a](x)^2 I_b[b](x) / sum_x J_b(x)^3,
    N_tri(b)     = sum_x J_b(x)^3 / N^3   (closed ordered triangles),

and B_tree = 3 E_b[delta_1, delta_1, delta_2] (three equal permutations).

One-loop bispectrum (Eq. ``bk_1loop``): with the triple-product form
E_b[a, b, c] = L^6 sum_x I_b[a] I_b[b] I_b[c] / sum_x J_b^3, each term of the
equation is one E_b over an ordered assignment of fields to (k1, k2, k3):
B_1-loop = sum of the six orderings of (delta_1, delta_2, delta_3) + E[delta_2,
delta_2, delta_2] + the three orderings of (delta_1, delta_1, delta_4).
"""
import math

import numpy as np

from .spt import backward, wave_indices


def mode_k(N, L):
    sx, sy, sz = wave_indices(N)
    s2 = (sx * sx + sy * sy + sz * sz).astype(np.float64)
    return (2.0 * math.pi / L) * np.sqrt(s2), s2


def bin_index(k, s2, edges):
    """Index i with edges[i] <= k < edges[i+1]; -1 outside or at k = 0."""
    edges = np.asarray(edges, dtype=np.float64)
    idx = np.searchsorted(edges, k, side="right") - 1
    idx[(idx >= len(edges) - 1) | (s2 == 0)] = -1
    return idx


def power(a_k, b_k, L, edges):
    N = a_k.shape[0]
    k, s2 = mode_k(N, L)
    idx = bin_index(k, s2, edges)
    nb = len(edges) - 1
    prod = (a_k * np.conj(b_k)).real
    sums = np.zeros(nb)
    counts = np.zeros(nb, dtype=np.int64)
    sel = idx >= 0
    np.add.at(sums, idx[sel], prod[sel])
    np.add.at(counts, idx[sel], 1)
    p = np.zeros(nb)
    nz = counts > 0
    p[nz] = L ** 3 * sums[nz] / counts[nz]
    return p, counts


def bispectrum_equilateral(a_k, b_k, L, edges):
    N = a_k.shape[0]
    k, s2 = mode_k(N, L)
    idx = bin_index(k, s2, edges)
    nb = len(edges) - 1
    E = np.zeros(nb)
    ntri = np.zeros(nb)
    for i in range(nb):
        mask = (idx == i).astype(np.float64)
        Ia = backward(a_k * mask).real
        Ib = backward(b_k * mask).real
        J = backward(mask.astype(np.complex128)).real
        sj3 = np.sum(J ** 3)
        ntri[i] = sj3 / float(N) ** 3
        if ntri[i] > 0.5:
            E[i] = L ** 6 * np.sum(Ia * Ia * Ib) / sj3
    return E, ntri


def bispectrum_brute(a_k, b_k, L, edges):
    """Direct triangle enumeration: E = L^6 sum_{k1+k2+k3=0} a(k1) a(k2) b(k3) / N_tri
    over ordered triples in the shell. Only for shells well below N/3 (no wrap)."""
    N = a_k.shape[0]
    k, s2 = mode_k(N, L)
    idx = bin_index(k, s2, edges)
    sx, sy, sz = wave_indices(N)
    nb = len(edges) - 1
    E = np.zeros(nb)
    ntri = np.zeros(nb)
    for i in range(nb):
        pts = np.argwhere(idx == i)
        acc = 0.0 + 0.0j
        cnt = 0
        member = idx == i
        for p1 in pts:
            for p2 in pts:
                s3 = [-(sx[tuple(p1)] + sx[tuple(p2)]), -(sy[tuple(p1)] + sy[tuple(p2)]),
                      -(sz[tuple(p1)] + sz[tuple(p2)])]
                if max(abs(c) for c in s3) >= N // 2:
                    continue
                p3 = tuple(int(c) % N for c in s3)
                if member[p3]:
                    acc += a_k[tuple(p1)] * a_k[tuple(p2)] * b_k[p3]
                    cnt += 1
        ntri[i] = cnt
        if cnt:
            E[i] = L ** 6 * acc.real / cnt
    return E, ntri


def bispectrum_triple(a_k, b_k, c_k, L, edges):
    """E_b[a, b, c] = L^6 sum_x I_b[a] I_b[b] I_b[c] / sum_x J_b^3 per shell, and
    N_tri (as in ``bispectrum_equilateral``)."""
    N = a_k.shape[0]
    k, s2 = mode_k(N, L)
    idx = bin_index(k, s2, edges)
    nb = len(edges) - 1
    E = np.zeros(nb)
    ntri = np.zeros(nb)
    for i in range(nb):
        mask = (idx == i).astype(np.float64)
        Ia = backward(a_k * mask).real
        Ib = backward(b_k * mask).real
        Ic = backward(c_k * mask).real
        J = backward(mask.astype(np.complex128)).real
        sj3 = np.sum(J ** 3)
        ntri[i] = sj3 / float(N) ** 3
        if ntri[i] > 0.5:
            E[i] = L ** 6 * np.sum(Ia * Ib * Ic) / sj3
    return E, ntri


def bispectrum_triple_brute(a_k, b_k, c_k, L, edges):
    """Direct enumeration: L^6 sum_{k1+k2+k3=0} a(k1) b(k2) c(k3) / N_tri over
    ordered triples in the shell (shells well below N/3 only)."""
    N = a_k.shape[0]
    k, s2 = mode_k(N, L)
    idx = bin_index(k, s2, edges)
    sx, sy, sz = wave_indices(N)
    nb = len(edges) - 1
    E = np.zeros(nb)
    ntri = np.zeros(nb)
    for i in range(nb):
        pts = np.argwhere(idx == i)
        member = idx == i
        acc = 0.0 + 0.0j
        cnt = 0
        for p1 in pts:
            for p2 in pts:
                s3 = [-(sx[tuple(p1)] + sx[tuple(p2)]), -(sy[tuple(p1)] + sy[tuple(p2)]),
                      -(sz[tuple(p1)] + sz[tuple(p2)])]
                if max(abs(c) for c in s3) >= N // 2:
                    continue
                p3 = tuple(int(c) % N for c in s3)
                if member[p3]:
                    acc += a_k[tuple(p1)] * b_k[tuple(p2)] * c_k[p3]
                    cnt += 1
        ntri[i] = cnt
        if cnt:
            E[i] = L ** 6 * acc.real / cnt
    return E, ntri


def bispectrum_one_loop(d1, d2, d3, d4, L, edges):
    """Eq. ``bk_1loop`` (D_+ = 1) in equilateral shells: the ten ordered terms."""
    terms = [(d1, d2, d3), (d1, d3, d2), (d2, d1, d3), (d2, d3, d1), (d3, d1, d2), (d3, d2, d1),
             (d2, d2, d2), (d1, d1, d4), (d1, d4, d1), (d4, d1, d1)]
    B = 0.0
    for a, b, c in terms:
        E, ntri = bispectrum_triple(a, b, c, L, edges)
        B = B + E
    return B, ntri


def cross_correlation(a_k, b_k, L, edges):
    """r(bin) = sum Re[a b*] / sqrt(sum |a|^2 sum |b|^2) over the modes of each
    bin (Eqs. r_corr_nthPT and r_corr_sum_nth; the printed Re[a b] reads as
    the cross-spectrum Re[a b*]); 0 for an empty bin."""
    N = a_k.shape[0]
    k, s2 = mode_k(N, L)
    idx = bin_index(k, s2, edges)
    nb = len(edges) - 1
    r = np.zeros(nb)
    for i in range(nb):
        m = idx == i
        if m.any():
            ab = np.sum((a_k[m] * np.conj(b_k[m])).real)
            aa = np.sum(np.abs(a_k[m]) ** 2)
            bb = np.sum(np.abs(b_k[m]) ** 2)
            r[i] = ab / math.sqrt(aa * bb) if aa > 0 and bb > 0 else 0.0
    return r
