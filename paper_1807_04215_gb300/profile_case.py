"""Small, self-contained invocations of the library for profilers (ncu).

    python -m paper_1807_04215_gb300.profile_case CASE [--n N] [--nmax K] [--reps R] [--tuning a,b,c,d,e]

CASE is one of:
  c2r      backward transforms of 4 random half spectra (x, y, z passes)
  r2c      forward transforms of 4 random real fields
  orders   one realisation: initial field and orders 2..nmax (L = 2000 N / 512)
  power    the six P-terms of one realisation (32 log bins, 0.01-0.4 h/Mpc)
  bispec   the equilateral bispectrum of one realisation (16 shells)
Each case runs `reps` times (default 2) so that a profiler can skip the first.
--stats prints the library's per-kind launches, event time and algorithmic
bytes of the last repetition (JSON).
"""
import argparse
import json
import math

import torch

from . import gridspt as g


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["c2r", "r2c", "orders", "power", "bispec"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--nmax", type=int, default=5)
    ap.add_argument("--tuning", default="", help="tile variants per pass, e.g. 0,0,1,0,0")
    ap.add_argument("--stats", action="store_true", help="print per-kind stats of the last repetition")
    a = ap.parse_args()
    N = a.n
    L = 2000.0 * N / 512
    n_max = a.nmax
    plan = g.Plan(N, n_max, L)
    if a.tuning:
        g.set_tuning(plan, [int(v) for v in a.tuning.split(",")])
    gen = torch.Generator(device="cuda").manual_seed(0)
    if a.case in ("c2r", "r2c"):
        spec = torch.randn(4, N, N, N // 2, dtype=torch.complex64, device="cuda", generator=gen)
        real = torch.empty(4, N, N, N, dtype=torch.float32, device="cuda")
        for _ in range(a.reps):
            if a.case == "c2r":
                g.c2r(plan, spec, out=real)
            else:
                g.r2c(plan, real.normal_(generator=gen), out=spec)
    else:
        d1 = g.make_linear_field(plan, [1000])
        spectra = g.run_orders(plan, d1) if a.case != "orders" else None
        edges = [0.01 * 40.0 ** (i / 32) for i in range(33)]
        kc = 2 * math.pi / L * N / (n_max + 1)
        bedges = [kc * i / 16 for i in range(17)]
        for rep in range(a.reps):
            if a.stats and rep == a.reps - 1:
                torch.cuda.synchronize()
                g.profile_begin()
            if a.case == "orders":
                g.make_linear_field(plan, [1000], out=d1)
                spectra = g.run_orders(plan, d1)
            elif a.case == "power":
                dl = {1: d1[0], **{n: spectra[0, n - 2, 0] for n in range(2, n_max + 1)}}
                for i, j in [(1, 1), (1, 3), (2, 2), (1, 5), (2, 4), (3, 3)]:
                    if j <= n_max:
                        g.power(plan, dl[i], dl[j], edges)
            else:
                g.bispectrum(plan, d1[0], spectra[0, 0, 0], bedges)
    torch.cuda.synchronize()
    if a.stats and a.case not in ("c2r", "r2c"):
        st = g.profile_end()
        print(json.dumps({k: {"launches": v[0], "ms": round(v[1], 4), "GB": round(v[2] / 1e9, 4)} for k, v in st.items()}))
    print("ok", a.case, N)


if __name__ == "__main__":
    main()
