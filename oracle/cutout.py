"""Second-order fields at a small block of cells of a large grid (oracle side).

Test infrastructure only. On grids too large for the full-grid oracle (1024^3
in FP64), the second order can still be evaluated exactly at a few cells:

* delta_1(k) is drawn mode by mode exactly as in ``spt.linear_field`` (the
  draw of Sec. II.C step (1) is keyed by the wavevector, so only the in-band
  modes |s|^2 <= (k_cut / k_F)^2 need to be enumerated);
* each derived field of order 1 is the inverse transform of Sec. II.C at the
  chosen cells, written out as its defining sum over modes,
      f(x) = sum_k c_f(k) delta_1(k) e^{i k.x}
           = sum_{canonical k} 2 Re[c_f(k) delta_1(k) e^{i k.x}],
  with c_f = 1, i k_a (gradients), -i k_a / k^2 (u_a, Eq. ``u_and_theta``) and
  k_a k_b / k^2 (d_a u_b); every c_f satisfies c_f(-k) = conj c_f(k), and
  delta_1(-k) = conj delta_1(k), which gives the second form;
* A_2, B_2 of Eq. ``recursion_formula`` at n = 2 with theta_1 = delta_1
  (Eq. ``recursion_n=1``), all nine tensor terms, then delta_2, theta_2 with
  the 2x2 recursion coefficients.

The sums over modes run in chunks: a table of the phases e^{i k.x} of a chunk
of modes at the block's cells (separable over the three axes) multiplied by
the matrix of weighted mode amplitudes (a matrix product is the only library
step). FP64 throughout.
"""
import math

import numpy as np

from . import cosmology, rng, spt


def linear_modes(N, L, n_max, cosmo, seed, kcut_lin=None):
    """Canonical in-band modes of delta_1 and their amplitudes.

    Returns (sx, sy, sz, value): integer wavevectors s with |s|^2 <= r^2
    (r = k_cut / k_F), s != 0, no Nyquist component, and canonical (s_z > 0, or
    s_z = 0 and s_y > 0, or s_z = s_y = 0 and s_x > 0); value = delta_1(k) of
    ``spt.linear_field`` (the other member of each pair is its conjugate)."""
    r = spt.cut_ratio(N, L, n_max, kcut_lin)
    ri = int(math.floor(r))
    h = N // 2
    rng_s = np.arange(-min(ri, h - 1), min(ri, h - 1) + 1)
    out = [[], [], []]
    for z in range(0, min(ri, h - 1) + 1):
        gx, gy = np.meshgrid(rng_s, rng_s, indexing="ij")
        s2 = gx * gx + gy * gy + z * z
        keep = (s2 > 0) & (s2 <= r * r)
        if z == 0:
            keep &= (gy > 0) | ((gy == 0) & (gx > 0))
        out[0].append(gx[keep])
        out[1].append(gy[keep])
        out[2].append(np.full(int(keep.sum()), z))
    sx, sy, sz = (np.concatenate(a).astype(np.int64) for a in out)
    u1, u2 = rng.mode_uniforms(seed, sx, sy, sz)
    g = np.sqrt(-2.0 * np.log(u1)) * (np.cos(2.0 * math.pi * u2) + 1j * np.sin(2.0 * math.pi * u2))
    kF = 2.0 * math.pi / L
    k = kF * np.sqrt((sx * sx + sy * sy + sz * sz).astype(np.float64))
    amp = np.sqrt(cosmology.linear_pk(k, cosmo) / L ** 3)
    return sx, sy, sz, amp * g / math.sqrt(2.0)


def first_order_fields_at_block(sx, sy, sz, d1, N, L, origin, size=8, chunk=1 << 15):
    """The 13 distinct derived fields of order 1 (theta_1 = delta_1) at the
    cells origin + (a, b, c), 0 <= a, b, c < size: a dict like
    ``spt.derived_fields`` with arrays of shape (size, size, size)."""
    kF = 2.0 * math.pi / L
    names = ["d"] + [f"g{a}" for a in range(3)] + [f"u{a}" for a in range(3)] + \
            [f"du{a}{b}" for a in range(3) for b in range(a, 3)]
    acc = np.zeros((len(names), size ** 3), dtype=np.complex128)
    off = np.arange(size)
    for lo in range(0, sx.size, chunk):
        x, y, z = sx[lo:lo + chunk], sy[lo:lo + chunk], sz[lo:lo + chunk]
        d = d1[lo:lo + chunk]
        kv = [kF * x, kF * y, kF * z]
        k2 = kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2
        w = [d]
        w += [1j * kv[a] * d for a in range(3)]
        w += [-1j * kv[a] / k2 * d for a in range(3)]
        w += [kv[a] * kv[b] / k2 * d for a in range(3) for b in range(a, 3)]
        W = np.stack(w, axis=0)                                        # [13, m]
        base = np.exp(2j * math.pi * (x * origin[0] + y * origin[1] + z * origin[2]) / N)
        ex = np.exp(2j * math.pi * np.outer(x, off) / N)                # [m, size]
        ey = np.exp(2j * math.pi * np.outer(y, off) / N)
        ez = np.exp(2j * math.pi * np.outer(z, off) / N)
        ph = (base[:, None, None, None] * ex[:, :, None, None] * ey[:, None, :, None] * ez[:, None, None, :])
        acc += W @ ph.reshape(x.size, -1)                               # sum over the chunk's modes
    vals = 2.0 * acc.real.reshape(len(names), size, size, size)         # canonical member + its conjugate
    f = dict(zip(names, vals))
    du = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(a, 3):
            du[a][b] = du[b][a] = f[f"du{a}{b}"]
    g = [f[f"g{a}"] for a in range(3)]
    return {"d": f["d"], "t": f["d"], "gd": g, "gt": g, "u": [f[f"u{a}"] for a in range(3)], "du": du}


def second_order_at_block(sx, sy, sz, d1, N, L, origin, size=8):
    """delta_2(x), theta_2(x) at the block (Eq. recursion_formula, n = 2)."""
    f = first_order_fields_at_block(sx, sy, sz, d1, N, L, origin, size)
    A, B = spt.sources({1: f}, 2)
    cdA, cdB, ctA, ctB = spt.recursion_coefficients(2)
    return cdA * A + cdB * B, ctA * A + ctB * B
