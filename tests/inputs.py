"""Seeded synthetic inputs shared by the oracle tests and the GPU tests.

Holds no arithmetic of the method: only random arrays, plane-wave spectra built
by setting individual modes, and layout slicing between the full complex grid
used by the oracle and the half-spectrum layout float2[N][N][N/2] used by the
library (the kz = N/2 plane is zero there by construction and not stored).
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def random_complex(shape, seed):
    g = rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def random_real(shape, seed):
    return rng(seed).standard_normal(shape)


def plane_waves(N, waves):
    """Full-grid spectrum of sum_i A_i cos(2 pi s_i . j / N): modes +-s_i get A_i / 2."""
    d = np.zeros((N, N, N), dtype=np.complex128)
    for s, A in waves:
        d[s[0] % N, s[1] % N, s[2] % N] += A / 2.0
        d[-s[0] % N, -s[1] % N, -s[2] % N] += A / 2.0
    return d


def full_to_half(full):
    """[N][N][N] complex -> [N][N][N/2] (kz = 0..N/2-1)."""
    N = full.shape[-1]
    return np.ascontiguousarray(full[..., : N // 2])


def half_to_full(half):
    """[..., N, N, N/2] -> [..., N, N, N] using a(-k) = conj a(k); kz = N/2 plane zero."""
    N = half.shape[-2]
    M = half.shape[-1]
    assert M == N // 2
    out = np.zeros(half.shape[:-1] + (N,), dtype=np.complex128)
    out[..., :M] = half
    # kz = -j for j = 1..M-1 (indices N-j) from the conjugate of (-kx, -ky, j)
    idx = (-np.arange(N)) % N
    src = half[..., idx, :, :][..., :, idx, :]
    for j in range(1, M):
        out[..., N - j] = np.conj(src[..., j])
    return out
