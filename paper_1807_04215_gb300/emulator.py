"""Emulator of binned GridSPT P-terms (not part of the paper's method).

Maps the linear-spectrum parameters (sigma_8, n_s, Gamma) to the loop terms
P22, P13, P33, P24, P15 in log k-bins, with a 3 -> 128 -> 128 -> (5 x bins)
SiLU network whose forward, backward, loss and Adam kernels are the library's
own (gridspt_mlp_*). Training targets are made by GridSPT itself; GridSPT
also measures the emulator's error and is the fallback outside the box it
was trained on.

Target scaling: with the seeds held fixed, every delta_n is proportional to
sigma_8^n, so P_ij = sigma_8^(i+j) * P_ij(sigma_8 = 1) exactly. The network
learns the standardised sigma_8 = 1 terms (a smooth function of n_s and
Gamma); predictions multiply the power back in.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import gridspt as g

TERMS = [(2, 2), (1, 3), (3, 3), (2, 4), (1, 5)]          # P22, P13, P33, P24, P15
TERM_NAMES = ["P22", "P13", "P33", "P24", "P15"]
BOX = {"sigma8": (0.6, 1.0), "n_s": (0.90, 1.02), "gamma": (0.15, 0.25)}
KEYS = ["sigma8", "n_s", "gamma"]


def latin_hypercube(n, seed):
    """n points, one per stratum in every dimension (strata shuffled per
    dimension, uniform position inside each stratum)."""
    r = np.random.default_rng(seed)
    u = np.empty((n, 3))
    for d in range(3):
        u[:, d] = (r.permutation(n) + r.random(n)) / n
    lo = np.array([BOX[k][0] for k in KEYS])
    hi = np.array([BOX[k][1] for k in KEYS])
    return lo + u * (hi - lo)


def log_edges(lo, hi, nb):
    return [lo * (hi / lo) ** (i / nb) for i in range(nb + 1)]


@dataclass
class GridConfig:
    n: int = 256
    box: float = 1000.0
    n_max: int = 5
    seeds: tuple = (1, 2, 3, 4)
    k_lo: float = 0.01
    k_hi: float = 0.3
    nbins: int = 32


class GridSPTTerms:
    """P-terms of GridSPT at given cosmologies, averaged over a fixed seed set."""

    def __init__(self, cfg: GridConfig):
        self.cfg = cfg
        self.plan = g.Plan(cfg.n, cfg.n_max, cfg.box, batch=len(cfg.seeds))
        self.edges = log_edges(cfg.k_lo, cfg.k_hi, cfg.nbins)
        self.d1 = torch.empty(self.plan.half_shape(len(cfg.seeds)), dtype=torch.complex64, device="cuda")
        self.spec = torch.empty(self.plan.half_shape(len(cfg.seeds), cfg.n_max - 1, 2), dtype=torch.complex64,
                                device="cuda")
        self.ws = torch.empty(self.plan.workspace_size(), dtype=torch.uint8, device="cuda")
        self.pws = torch.empty(g.power_workspace_size(self.plan, cfg.nbins), dtype=torch.uint8, device="cuda")
        self.out = torch.empty(len(cfg.seeds), len(TERMS), cfg.nbins, dtype=torch.float64, device="cuda")
        self.nk = torch.empty(cfg.nbins, dtype=torch.int64, device="cuda")

    def __call__(self, point):
        s8, ns, gam = (float(v) for v in point)
        cosmo = dict(omega_m=0.3, h=0.7, n_s=ns, sigma8=s8, gamma=gam)
        g.make_linear_field(self.plan, self.cfg.seeds, cosmo, out=self.d1)
        g.run_orders(self.plan, self.d1, spectra=self.spec, ws=self.ws)
        for b in range(len(self.cfg.seeds)):
            dl = {1: self.d1[b], **{n: self.spec[b, n - 2, 0] for n in range(2, self.cfg.n_max + 1)}}
            for t, (i, j) in enumerate(TERMS):
                g.power(self.plan, dl[i], dl[j], self.edges, ws=self.pws, out=self.out[b, t], nk=self.nk)
        fac = torch.tensor([1.0 if i == j else 2.0 for i, j in TERMS], dtype=torch.float64, device="cuda")
        return (self.out.mean(dim=0) * fac[:, None]).cpu().numpy()   # [5, nbins]

    def many(self, points):
        return np.stack([self(p) for p in points])


@dataclass
class Emulator:
    net: "g.MLP"
    x_lo: np.ndarray
    x_hi: np.ndarray
    mu: np.ndarray
    sd: np.ndarray
    mask: np.ndarray                       # [5 * nbins] outputs learned (bins with modes, not identically 0)
    powers: np.ndarray = field(default_factory=lambda: np.array([i + j for i, j in TERMS], dtype=float))

    def _xin(self, pts):
        return 2.0 * (pts - self.x_lo) / (self.x_hi - self.x_lo) - 1.0

    def predict(self, pts, out=None):
        """Emulated P-terms [n, 5, nbins] (device forward pass, host rescaling)."""
        pts = np.asarray(pts, dtype=np.float64)
        x = torch.from_numpy(self._xin(pts).astype(np.float32)).cuda()
        y = self.net.forward(x, y=out).double().cpu().numpy()
        y = np.where(self.mask[None, :], y * self.sd + self.mu, 0.0)
        nb = self.mu.size // 5
        return y.reshape(-1, 5, nb) * (pts[:, :1, None] ** self.powers[None, :, None])

    def inside(self, pts):
        pts = np.atleast_2d(pts)
        return np.all((pts >= self.x_lo) & (pts <= self.x_hi), axis=1)

    def predict_or_fallback(self, pts, grid: GridSPTTerms):
        """Emulator inside the training box, GridSPT outside it."""
        pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
        res = np.empty((len(pts), 5, self.mu.size // 5))
        ok = self.inside(pts)
        if ok.any():
            res[ok] = self.predict(pts[ok])
        for i in np.flatnonzero(~ok):
            res[i] = grid(pts[i])
        return res, ok


def train(points, targets, nk_mask, hidden=128, steps=20000, lr=2e-3, lr_end=2e-5, bf16=True, seed=0,
          log_every=0):
    """Fit the network to GridSPT targets [n, 5, nbins] at points [n, 3]."""
    pts = np.asarray(points, dtype=np.float64)
    n, nt, nb = targets.shape
    powers = np.array([i + j for i, j in TERMS], dtype=float)
    scaled = targets / (pts[:, :1, None] ** powers[None, :, None])
    flat = scaled.reshape(n, nt * nb)
    # learn bins that hold modes and are not identically zero (terms with delta_1
    # vanish above the cut on delta_1)
    mask = np.repeat(nk_mask[None, :], nt, axis=0).reshape(-1).astype(bool) & np.any(flat != 0, axis=0)
    mu = flat.mean(axis=0)
    sd = flat.std(axis=0)
    sd[~mask | (sd == 0)] = 1.0
    y_std = np.where(mask[None, :], (flat - mu) / sd, 0.0)
    x_lo = np.array([BOX[k][0] for k in KEYS])
    x_hi = np.array([BOX[k][1] for k in KEYS])
    net = g.MLP(3, hidden, nt * nb, bf16=bf16, seed=seed)
    emu = Emulator(net, x_lo, x_hi, mu, sd, mask)
    x = torch.from_numpy(emu._xin(pts).astype(np.float32)).cuda()
    t = torch.from_numpy(y_std.astype(np.float32)).cuda()
    m = torch.from_numpy(np.repeat(mask[None, :], n, axis=0).astype(np.float32)).cuda()
    act = torch.empty(n, 4 * hidden, dtype=torch.float32, device="cuda")
    y = torch.empty(n, nt * nb, dtype=torch.float32, device="cuda")
    dy = torch.empty_like(y)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = torch.empty(net.ws_bytes(n), dtype=torch.uint8, device="cuda")
    history = []
    t0 = time.perf_counter()
    for it in range(steps):
        # cosine decay from lr to lr_end
        cur = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * it / max(steps - 1, 1)))
        net.forward(x, y=y, act=act)
        net.mse(y, t, m, dy, loss)
        net.backward(x, act, dy, ws)
        net.adam(cur)
        if log_every and it % log_every == 0:
            history.append((it, float(loss.item())))
    torch.cuda.synchronize()
    emu.train_seconds = time.perf_counter() - t0
    emu.history = history
    emu.final_loss = float(loss.item())
    return emu


def errors(pred, ref, nk_mask):
    """Per-term emulator errors against GridSPT, {term: dict}:
    rel_rms, rel_max: |pred - ref| / |ref| over bins that hold modes and where
        the term keeps one sign over all points (at a zero crossing the
        relative error is undefined);
    scale_rms, scale_max: |pred - ref| / max_k |ref| of the same point, over
        every bin that holds modes."""
    out = {}
    for t, name in enumerate(TERM_NAMES):
        r = ref[:, t, :]
        live = nk_mask.astype(bool) & np.any(r != 0, axis=0)
        one_sign = live & (np.all(r > 0, axis=0) | np.all(r < 0, axis=0))
        e_rel = np.abs(pred[:, t, one_sign] - r[:, one_sign]) / np.abs(r[:, one_sign])
        scale = np.abs(r[:, live]).max(axis=1, keepdims=True)
        e_sc = np.abs(pred[:, t, live] - r[:, live]) / scale
        out[name] = dict(rel_rms=float(np.sqrt(np.mean(e_rel ** 2))), rel_max=float(e_rel.max()),
                         scale_rms=float(np.sqrt(np.mean(e_sc ** 2))), scale_max=float(e_sc.max()),
                         bins_rel=int(one_sign.sum()), bins=int(live.sum()))
    return out
