"""Philox4x32-10 counter-based generator (oracle side).

Written from the published definition in J. K. Salmon, M. A. Moraes,
R. O. Dror and D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11 (Sec. 4, the Philox-4x32 bijection): a 4-word counter and a 2-word key;
each of the 10 rounds multiplies words 0 and 2 by two fixed 32-bit constants,
takes the high and low halves of the 64-bit products, and mixes them with the
other two counter words and the key; the key is advanced by two Weyl constants
between rounds.

The GridSPT paper draws its initial Gaussian field without saying how
(Sec. II.C, step 1); this generator is the reading used by both the oracle and
the GPU library, each with its own implementation.

Pinned by the known-answer vectors of the generator's authors
(tests/golden/philox4x32_10_kat.txt).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Apply the 10-round Philox-4x32 bijection.

    counter: uint array [..., 4] of 32-bit words; key: uint array [..., 2].
    Returns a uint64 array [..., 4] holding 32-bit results.
    """
    c = np.asarray(counter, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
        p0 = _M0 * c0          # exact: both factors < 2**32, product < 2**64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def mode_key(sx, sy, sz):
    """Pack a signed integer wavevector into the 2-word counter prefix.

    Each component is stored as a 21-bit two's-complement field
    (bits 0-20: x, 21-41: y, 42-62: z) of a 64-bit integer, split into low and
    high 32-bit words. Keying the draw by the wavevector (not the array index)
    makes grids of different size with the same box share their common modes.
    """
    m21 = np.int64(0x1FFFFF)
    px = np.asarray(sx, dtype=np.int64) & m21
    py = np.asarray(sy, dtype=np.int64) & m21
    pz = np.asarray(sz, dtype=np.int64) & m21
    packed = (px | (py << np.int64(21)) | (pz << np.int64(42))).astype(np.uint64)
    return packed & _MASK32, packed >> np.uint64(32)


def mode_uniforms(seed, sx, sy, sz):
    """Two uniforms in (0, 1) for each wavevector, from counter (key_lo, key_hi, 0, 0)
    under key (seed_lo, seed_hi): u = (r + 1/2) * 2**-32 for output words 0 and 1."""
    lo, hi = mode_key(sx, sy, sz)
    zero = np.zeros_like(lo)
    ctr = np.stack([lo, hi, zero, zero], axis=-1)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    key = np.broadcast_to(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64),
                          lo.shape + (2,))
    r = philox4x32_10(ctr, key)
    u1 = (r[..., 0].astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (r[..., 1].astype(np.float64) + 0.5) * 2.0 ** -32
    return u1, u2
