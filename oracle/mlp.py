"""FP64 reference of the P-term emulator's network (oracle side).

The emulator is not part of the GridSPT paper: the workload adds a small
multilayer perceptron mapping (sigma_8, n_s, Gamma) to binned P-terms,
3 -> H -> H -> O with SiLU activations (SiLU(z) = z / (1 + e^{-z})) and a
linear output layer, trained with Adam (Kingma & Ba, ICLR 2015) on a masked
mean-squared error. This module writes those definitions out in plain numpy
FP64; it is test infrastructure only.

Parameter vector layout (row-major [in][out] weights), shared by the GPU
kernels' documented ABI: W1[3][H], b1[H], W2[H][H], b2[H], W3[H][O], b3[O].
Optional rounding hook `rnd` (e.g. to bfloat16) is applied to the weights and
to the stored activations, to mirror a lower-precision storage format.
"""
import numpy as np


def sizes(H, O, I=3):
    return [(I, H), (H,), (H, H), (H,), (H, O), (O,)]


def unpack(theta, H, O, I=3):
    out, k = [], 0
    for shp in sizes(H, O, I):
        n = int(np.prod(shp))
        out.append(theta[k:k + n].reshape(shp))
        k += n
    return out


def n_params(H, O, I=3):
    return sum(int(np.prod(s)) for s in sizes(H, O, I))


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def ident(a):
    return a


def forward(x, theta, H, O, rnd=ident):
    """Returns y and the activations (z1, a1, z2, a2) needed by backward."""
    W1, b1, W2, b2, W3, b3 = [rnd(p) for p in unpack(theta, H, O, x.shape[1])]
    z1 = x @ W1 + b1
    a1 = rnd(silu(z1))
    z2 = a1 @ W2 + b2
    a2 = rnd(silu(z2))
    y = a2 @ W3 + b3
    return y, (z1, a1, z2, a2)


def masked_mse(y, t, mask):
    """L = sum(mask (y - t)^2) / sum(mask); returns (L, dL/dy)."""
    cnt = mask.sum()
    d = (y - t) * mask
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def backward(x, theta, H, O, acts, dy, rnd=ident):
    """Gradient of sum(dy * y) with respect to theta (same layout)."""
    W1, b1, W2, b2, W3, b3 = [rnd(p) for p in unpack(theta, H, O, x.shape[1])]
    z1, a1, z2, a2 = acts
    gW3 = a2.T @ dy
    gb3 = dy.sum(axis=0)
    d2 = (dy @ W3.T) * silu_grad(z2)
    gW2 = a1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * silu_grad(z1)
    gW1 = x.T @ d1
    gb1 = d1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step count t >= 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (ties to even), via FP32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
