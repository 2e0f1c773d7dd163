"""Cutoff scan of the two-loop power spectrum and the one-loop bispectrum.

The paper filters the linear field at k_cut,1 and every higher order at
k_cut,2 (Sec. II.C), and studies how P_2-loop and B_1-loop depend on the cut
below and above k_crit = (2 pi / L)(N / 3) (Sec. III.B.3). This driver runs
that scheme through the library: for each cut it forms delta_1..delta_5 for a
set of seeds (plan kcut_lin = k_cut,1, kcut_nl = k_cut,2), then

    P_2-loop(k) = 2 P[delta_1, delta_5] + 2 P[delta_2, delta_4] + P[delta_3, delta_3]
                  (Eq. pk_2loop, D_+ = 1),
    B_1-loop(k) = 6 E[1,2,3] + E[2,2,2] + 3 E[1,1,4]   (Eq. bk_1loop, equilateral),

averaged over the seeds. Every statistic is computed by the library's kernels.

    python -m paper_1807_04215_gb300.cutoff_scan --n 256 --box 1000 --cuts 0.5,0.75,1.0 --ratio 1.3333
"""
import argparse
import json
import math

import numpy as np
import torch

from . import gridspt as g


def scan(n, box, cuts, ratio=4.0 / 3.0, seeds=(1, 2, 3, 4), pk_edges=None, bk_edges=None, n_max=5):
    """For each k_cut,1 in `cuts` (h/Mpc; k_cut,2 = ratio * k_cut,1) return a dict
    with the seed-averaged P_2-loop per power bin and B_1-loop per shell."""
    kF = 2 * math.pi / box
    kny = kF * n / 2
    if pk_edges is None:
        pk_edges = [0.01 * (0.9 * kny / 0.01) ** (i / 24) for i in range(25)]
    if bk_edges is None:
        top = 0.66 * kny                       # shells below 2 k_Ny / 3
        bk_edges = [top * i / 12 for i in range(13)]
    out = []
    for kc in cuts:
        plan = g.Plan(n, n_max, box, batch=len(seeds), kcut_lin=kc, kcut_nl=ratio * kc)
        d1 = g.make_linear_field(plan, list(seeds))
        sp = g.run_orders(plan, d1)
        p2, b1 = 0.0, 0.0
        for b in range(len(seeds)):
            d = {1: d1[b], **{m: sp[b, m - 2, 0] for m in range(2, n_max + 1)}}
            p15, _ = g.power(plan, d[1], d[5], pk_edges)
            p24, _ = g.power(plan, d[2], d[4], pk_edges)
            p33, nk = g.power(plan, d[3], d[3], pk_edges)
            p2 = p2 + (2 * p15 + 2 * p24 + p33).cpu().numpy()
            bb, nt = g.bispectrum_one_loop(plan, d[1], d[2], d[3], d[4], bk_edges)
            b1 = b1 + bb.cpu().numpy()
        out.append({"kcut_lin": kc, "kcut_nl": ratio * kc,
                    "k_crit": kF * n / 3,
                    "pk_edges": list(pk_edges), "P_2loop": (p2 / len(seeds)).tolist(),
                    "bk_edges": list(bk_edges), "B_1loop": (b1 / len(seeds)).tolist(),
                    "N_tri": nt.cpu().numpy().tolist()})
        del plan, d1, sp
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--box", type=float, default=1000.0)
    ap.add_argument("--cuts", default="0.5,0.75,1.0")
    ap.add_argument("--ratio", type=float, default=4.0 / 3.0)
    ap.add_argument("--seeds", default="1,2,3,4")
    a = ap.parse_args()
    res = scan(a.n, a.box, [float(c) for c in a.cuts.split(",")], a.ratio,
               tuple(int(s) for s in a.seeds.split(",")))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
