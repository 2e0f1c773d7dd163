"""Throughput benchmark of the GridSPT hot path on GB300.

Workload: 16 realisations of a 512^3 grid, L = 2000 Mpc/h, n_max = 5, FP32
fields (BBKS LCDM, Omega_m = 0.3, h = 0.7, n_s = 0.96, sigma_8 = 0.8, seeds
1000 + r). One step = for every realisation of the batch: Gaussian initial
field, orders 2..5 of the recursion, the six P-terms P11, P13, P22, P15, P24,
P33 in 32 log bins over 0.01-0.4 h/Mpc, and the tree-level equilateral
bispectrum in 16 shells over [0, K_c). Metric: Mcells*orders/s =
batch * N^3 * n_max / step time. Every field (512 MiB) is larger than the
129 MB L2, so no L2 flush is needed between steps.

`--impl reference` times the FP64 CPU oracle instead (bounded sample, see
cpu_baseline). Under torchrun each rank runs its own realisations (replicas:
no data exchange) and rank 0 reports the aggregate.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcells*orders/s to 5th order at 512^3 FP32"
UNIT = "Mcells*orders/s"
N_GRID, BOX, N_MAX = 512, 2000.0, 5
FALLBACK_HBM_GBS = 6800.0
# DRAM traffic / algorithmic bytes measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) for the kernels as they stand, on the launches of one
# realisation of this workload (512^3); traffic per launch is reported as this
# ratio times the launch's algorithmic bytes. A kernel changed since its
# capture has no entry (traffic null).
NCU_TRAFFIC_RATIO = {"z_expand": 1.008, "y_expand": 1.024, "x_fwd_expand": 1.039}


def log_edges(lo, hi, nb):
    return [lo * (hi / lo) ** (i / nb) for i in range(nb + 1)]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for key in ("hbm_gbs", "hbm_GBps", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------- replica helpers
def rank_seeds(rank, per_rank):
    """Realisations are independent: rank r runs seeds 1000 + r * B .. + B - 1."""
    return [1000 + rank * per_rank + i for i in range(per_rank)]


def max_over_ranks(value, dist, device):
    """Slowest rank's time (the job is done when every replica is done)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(world, per_rank, n, n_max, ms):
    """Whole-job Mcells*orders/s: all ranks' realisations over the slowest rank's time."""
    return world * per_rank * n ** 3 * n_max / 1e6 / (ms / 1e3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- oracle arm
def cpu_model():
    """The host CPU's model name (lscpu / /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_worker(args):
    """One worker of the oracle sample: realisations of an n^3 grid (same cell
    size as the workload) for about target_s seconds; returns their count."""
    n, target_s, seed0 = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import cosmology, spt
    L = BOX * n / N_GRID
    A = cosmology.amplitude(cosmology.DEFAULT_COSMO)
    reps, t0 = 0, time.perf_counter()
    while True:
        d1 = spt.linear_field(n, L, N_MAX, cosmology.DEFAULT_COSMO, seed0 + reps, A=A)
        spt.run_orders(d1, L, N_MAX)
        reps += 1
        if time.perf_counter() - t0 >= target_s:
            return reps


def oracle_sample(target_s=12.0, n=64, workers=1):
    """FP64 oracle on a bounded sample of the workload: realisations of an n^3
    grid with the same cell size (L = 2000 n / 512 Mpc/h), orders 1..5 (initial
    field + recursion), for about target_s seconds, on `workers` host cores (one
    process each, started with spawn; numpy's transforms are single threaded).
    Returns (Mcells*orders/s, seconds, realisations, cpu_baseline record)."""
    t0 = time.perf_counter()
    if workers <= 1:
        reps = _oracle_worker((n, target_s, 1000))
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            reps = sum(pool.map(_oracle_worker, [(n, target_s, 1000 + 100000 * w) for w in range(workers)]))
    el = time.perf_counter() - t0
    value = reps * n ** 3 * N_MAX / el / 1e6
    L = BOX * n / N_GRID
    return value, el, reps, {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                             "sample": f"{reps} realisation(s) of {n}^3, L={L:g} Mpc/h (same cell size), n_max=5, "
                                       f"IC + recursion, numpy FP64, {workers} process(es), {el:.1f} s"}


def workload_config(n, batch, world):
    """The `config` object of both arms' JSON lines (the workload, by its sizes)."""
    L = BOX * n / N_GRID
    return {"workload": f"gridspt-{n}^3-L{L:g}-nmax{N_MAX}", "grid": n, "box_mpc_h": L, "n_max": N_MAX,
            "realisations_per_gpu": batch, "estimators": "6 P-terms x 32 log bins + B_tree x 16 shells",
            "schedule": "recursion per realisation; its estimators on a second stream beside the next one",
            "l2": "inputs larger than L2 (512 MiB fields), no flush", "parallelism": f"replicas{world}"}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on all host cores, a bounded sample
    of the workload per step (the workload's `config`; the sample is described
    in `cpu_baseline`)."""
    if rank != 0:
        return
    workers = os.cpu_count() or 1
    vals = []
    for _ in range(args.warmup):
        oracle_sample(target_s=0.0)
    t_all = time.perf_counter()
    cb = None
    for _ in range(args.steps):
        v, el, reps, cb = oracle_sample(target_s=max(1.0, 30.0 / max(args.steps, 1)), workers=workers)
        vals.append(v)
    total = time.perf_counter() - t_all
    value = statistics.median(vals)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.n, args.batch, args.gpus),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_mem_bytes():
    """Available host memory (MemAvailable), or None."""
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except Exception:
        pass
    return None


def run_cpu_sweep(args):
    """The oracle at 64^3, 128^3 and 256^3 (same cell size as the workload) on
    one core and on every core: Mcells*orders/s per size (one JSON line). One
    realisation of the FP64 oracle holds about 2 GB per 2 M cells (its derived
    fields on full complex grids); the all-core run starts no more processes
    than half the available host memory holds."""
    out = {"cpu_model": cpu_model(), "nproc": os.cpu_count(), "sizes": {}}
    avail = host_mem_bytes()
    for n, t in ((64, 10.0), (128, 20.0), (256, 1.0)):
        per = 2.0e9 * n ** 3 / 2 ** 21
        workers = os.cpu_count() or 1
        if avail:
            workers = max(1, min(workers, int(0.5 * avail / per)))
        one = oracle_sample(target_s=t, n=n, workers=1)
        allc = oracle_sample(target_s=t, n=n, workers=workers)
        out["sizes"][f"{n}^3"] = {"one_core": round(one[0], 3), "all_cores": round(allc[0], 3),
                                  "processes": workers,
                                  "one_core_s_per_realisation": round(one[1] / one[2], 2),
                                  "all_cores_realisations": allc[2]}
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------- GPU arm
def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:   # NVTX markers are optional annotations
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def run_gpu(args, rank, world):
    import torch
    from paper_1807_04215_gb300 import gridspt as g

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    N, B = args.n, args.batch
    L = BOX * N / N_GRID
    plan = g.Plan(N, N_MAX, L, batch=B)
    seeds = rank_seeds(rank, B)
    d1 = torch.empty(plan.half_shape(B), dtype=torch.complex64, device="cuda")
    spectra = torch.empty(plan.half_shape(B, N_MAX - 1, 2), dtype=torch.complex64, device="cuda")
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device="cuda")
    pedges = log_edges(0.01, 0.4, 32)
    kc = 2 * math.pi / L * N / (N_MAX + 1)
    bedges = [kc * i / 16 for i in range(17)]
    pws = torch.empty(g.power_workspace_size(plan, 32), dtype=torch.uint8, device="cuda")
    bws = torch.empty(g.bispectrum_workspace_size(plan, 16), dtype=torch.uint8, device="cuda")
    pout = torch.empty(B, 6, 32, dtype=torch.float64, device="cuda")
    nk = torch.empty(32, dtype=torch.int64, device="cuda")
    bout = torch.empty(B, 2, 16, dtype=torch.float64, device="cuda")

    def delta(b, n, src):
        return src[b] if n == 1 else spectra[b, n - 2, 0]

    def estimators_one(b, src):
        for t, (i, j) in enumerate([(1, 1), (1, 3), (2, 2), (1, 5), (2, 4), (3, 3)]):
            g.power(plan, delta(b, i, src), delta(b, j, src), pedges, ws=pws, out=pout[b, t], nk=nk)
        E, nt = g.bispectrum(plan, src[b], spectra[b, 0, 0], bedges, ws=bws)
        bout[b, 0].copy_(E)
        bout[b, 1].copy_(nt)

    # The recursion runs realisation by realisation on the main stream; the
    # estimators of realisation b run on a second stream once b's spectra are
    # written, alongside the recursion of b + 1 (their many small, partly
    # latency-bound launches fill gaps of the large passes). Separate scratch:
    # ws for the recursion, pws / bws for the estimators.
    plan1 = g.Plan(N, N_MAX, L, batch=1)
    est_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(B)]
    est_done = torch.cuda.Event()

    def orders_and_estimators(src):
        main = torch.cuda.current_stream()
        est_stream.wait_stream(main)                     # inputs of this step are in place
        for b in range(B):
            g.run_orders(plan1, src[b:b + 1], spectra=spectra[b:b + 1], ws=ws)
            ready[b].record(main)
            with torch.cuda.stream(est_stream):
                est_stream.wait_event(ready[b])
                estimators_one(b, src)
        est_done.record(est_stream)
        main.wait_event(est_done)                        # the step ends when both streams are done

    def step():
        g.make_linear_field(plan, seeds, out=d1)
        orders_and_estimators(d1)

    tuning = g.autotune(plan, scratch=ws)
    g.set_tuning(plan1, tuning)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev) if rank == 0 else None
    g.profile_begin()
    torch.cuda.synchronize()
    nvtx_push("timed_step")       # lets a profiler select exactly the timed launches
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    nvtx_pop()
    prof = g.profile_end()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
    if dist:
        dist.barrier()

    # end to end through the public API: delta_1(k) from pinned host memory in,
    # binned statistics read back to the host, every step. The next step's
    # input is copied on a second stream into a second device buffer while the
    # current step computes (double buffering), and each step's statistics are
    # copied into one of two pinned host buffers; the host waits for step s's
    # read-back after queueing step s + 1, so the GPU never idles on the host.
    # Every step's copy in and read-back stay inside the timed region.
    host_d1 = torch.empty_like(d1, device="cpu").pin_memory()
    host_d1.copy_(d1.cpu())
    host_out = [torch.empty(B * 6 * 32 + B * 2 * 16, dtype=torch.float64).pin_memory() for _ in range(2)]
    d2h_done = [torch.cuda.Event(), torch.cuda.Event()]
    d1b = [d1, torch.empty_like(d1)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    released = [torch.cuda.Event(), torch.cuda.Event()]

    def issue_copy(k):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(released[k])          # the buffer's previous step is done with it
            d1b[k].copy_(host_d1, non_blocking=True)
            copied[k].record(copy_stream)

    def e2e_run(nsteps):
        issue_copy(0)
        for st in range(nsteps):
            k = st % 2
            if st + 1 < nsteps:
                issue_copy(1 - k)                        # next step's input, overlapped
            stream.wait_event(copied[k])
            orders_and_estimators(d1b[k])
            released[k].record(stream)
            host_out[k][: B * 192].copy_(pout.view(-1), non_blocking=True)
            host_out[k][B * 192:].copy_(bout.view(-1), non_blocking=True)
            d2h_done[k].record(stream)
            if st >= 1:
                d2h_done[1 - k].synchronize()            # the previous step's statistics are on the host
        d2h_done[(nsteps - 1) % 2].synchronize()         # and the last step's

    e2e_run(2)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_run(args.steps)
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / args.steps, dist, "cuda")

    # end to end from the library's own host input, the seeds (a host array the
    # initial-field call takes), to the binned statistics read back to the host
    def e2e_seeds_run(nsteps):
        for st in range(nsteps):
            k = st % 2
            g.make_linear_field(plan, seeds, out=d1)
            orders_and_estimators(d1)
            host_out[k][: B * 192].copy_(pout.view(-1), non_blocking=True)
            host_out[k][B * 192:].copy_(bout.view(-1), non_blocking=True)
            d2h_done[k].record(stream)
            if st >= 1:
                d2h_done[1 - k].synchronize()
        d2h_done[(nsteps - 1) % 2].synchronize()

    e2e_seeds_run(2)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_seeds_run(args.steps)
    e2e_seeds_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / args.steps, dist, "cuda")
    del d1b[1]
    # the host -> device link rate of the same copy alone (it varies between
    # machines and dominates the difference between e2e and the device timing)
    ev0.record(stream)
    d1.copy_(host_d1, non_blocking=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    h2d_gbps = d1.numel() * 8 / (ev0.elapsed_time(ev1) / 1e3) / 1e9

    # the same recursion (all B realisations) captured once as a CUDA graph and replayed
    graph = g.Batch([plan], [d1], spectra=[spectra], wss=[ws])
    graph.launch()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        graph.launch()
    ev1.record(stream)
    torch.cuda.synchronize()
    graph_ms = ev0.elapsed_time(ev1) / args.steps
    graph.close()
    del ws
    div = variant_section(args, N, L, B, d1, spectra, stream, form="divergence") if rank == 0 else None
    trunc = variant_section(args, N, L, B, d1, spectra, stream, truncate=True) if rank == 0 else None
    mixed = mixed_batch(args) if rank == 0 and not args.quick else None
    fftcmp = cufft_comparator(N, L, tuning) if rank == 0 else None
    emu = emulator_section(args) if rank == 0 and not args.quick else None
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    work = world * B * N ** 3 * N_MAX / 1e6
    value = aggregate_throughput(world, B, N, N_MAX, ms)
    # dominant kernel by summed device time, among the kinds launched on the main
    # stream (the estimator kinds' event times include the time they share the
    # GPU with the recursion on the second stream)
    rec_kinds = ("ic", "x_expand", "x_fwd_expand", "y_expand", "z_expand", "y_fwd", "x_fwd", "z_r2c", "product")
    kname, (nl, kms, kbytes) = max(((k, v) for k, v in prof.items() if k in rec_kinds), key=lambda kv: kv[1][1])
    peak, src = peaks()
    achieved = kbytes / (kms / 1e3) / 1e9
    breakdown = {k: {"launches": v[0], "ms_per_step": round(v[1] / args.steps, 3),
                     "GBps": round(v[2] / (v[1] / 1e3) / 1e9, 1) if v[1] > 0 else None}
                 for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    cpu_value, el, reps, cb = oracle_sample(target_s=10.0, workers=os.cpu_count() or 1)
    one = oracle_sample(target_s=6.0, workers=1)
    cb["one_core"] = {"value": one[0], "sample": one[3]["sample"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(N, B, world),
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak,
                     "peak_source": src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": (round(NCU_TRAFFIC_RATIO[kname] * kbytes / nl / 1e9, 3) if kname in NCU_TRAFFIC_RATIO
                                 else None),
                     "traffic_unit": "GB per launch", "algorithmic_per_launch": round(kbytes / nl / 1e9, 3)},
        "recursion_ms_per_realisation": round(sum(prof[k][1] for k in rec_kinds if k in prof) / args.steps / B, 3),
        "kernels": breakdown,
        "kernels_note": ("event times per launch on its own stream; the estimator kinds (power, shell_*, "
                         "bispec_final) run on a second stream beside the recursion, so theirs include "
                         "the time they share the GPU with it"),
        "clocks": clk,
        "e2e": {"value": work / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(d1.numel() * 8), "d2h_bytes_per_step": int(host_out[0].numel() * 8),
                "ms_per_step": e2e_ms, "h2d_GBps": round(h2d_gbps, 1),
                "path": "delta_1(k) from pinned host -> run_orders -> estimators -> host; each step's copy "
                        "in overlaps the previous step's compute (two device buffers, copy stream); each "
                        "step's read-back is awaited once the next step is queued (two pinned buffers)"},
        "e2e_seeds": {"value": work / (e2e_seeds_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": 8 * B,
                      "d2h_bytes_per_step": int(host_out[0].numel() * 8), "ms_per_step": e2e_seeds_ms,
                      "path": "seeds (host array, the initial-field call's input) -> make_linear_field -> "
                              "run_orders -> estimators -> statistics read back to pinned host memory"},
        "cpu_baseline": cb,
        "autotune": tuning,
        "recursion_graph": {"ms_per_launch": round(graph_ms, 3), "realisations": B,
                            "value": round(B * N ** 3 * (N_MAX - 1) / graph_ms / 1e3, 1),
                            "unit": "Mcells*orders/s (orders 2..5, one graph launch, IC excluded)"},
        "mixed_batch": mixed,
        "fft_vs_cufft": fftcmp,
        "emulator": emu,
        "divergence_form": div,
        "truncated_orders": trunc,
    }
    # kernels launched per timed region: recorded launches plus the final-reduction kernels
    # of the estimators (one per power call and per bispectrum shell)
    extra = args.steps * B * (6 + 16)
    line["gpu_launches"] = int(sum(v[0] for v in prof.values())) + extra
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def variant_section(args, N, L, B, d1, spectra, stream, **plan_kw):
    """The same B realisations (orders 2..5, IC excluded) with a plan option that
    keeps the modes below delta_1's cut and changes the others (so not the
    headline): the sources in divergence form (form="divergence": A_n = div sum
    delta_m u_{n-m}, B_n = lap sum u_m . u_{n-m} / 2, four real fields per order)
    or every order j cut at min(j, n_max + 1 - j) K_c (truncate=True). Reports
    the RMS relative difference to the nine-term spectra on the modes below
    delta_1's cut, where both equal them up to rounding."""
    import torch
    from paper_1807_04215_gb300 import gridspt as g
    plan = g.Plan(N, N_MAX, L, batch=B, **plan_kw)
    tuning = g.autotune(plan)          # its own scratch: larger than this form's workspace
    torch.cuda.empty_cache()
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device="cuda")
    spd = torch.empty_like(spectra)
    for _ in range(args.warmup):
        g.run_orders(plan, d1, spectra=spd, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.profile_begin()
    e0.record(stream)
    for _ in range(args.steps):
        g.run_orders(plan, d1, spectra=spd, ws=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = g.profile_end()
    ms = e0.elapsed_time(e1) / args.steps
    s = torch.arange(N, device="cuda")
    s = torch.where(s < N // 2, s, s - N)
    s2 = s[:, None, None] ** 2 + s[None, :, None] ** 2 + s[None, None, : N // 2] ** 2
    band = (s2 < (N / (N_MAX + 1)) ** 2).to(torch.float64)
    w = torch.full((N, N, N // 2), 2.0, dtype=torch.float64, device="cuda")
    w[:, :, 0] = 1.0
    w = w * band
    worst = 0.0
    for n in range(2, N_MAX + 1):
        a, b = spectra[0, n - 2], spd[0, n - 2]
        num = (w * (a - b).abs().double() ** 2).sum()
        den = (w * a.abs().double() ** 2).sum()
        worst = max(worst, float(torch.sqrt(num / den)))
    gbytes = sum(v[2] for v in prof.values()) / args.steps / B / 1e9
    del ws, spd
    torch.cuda.empty_cache()
    return {"ms_per_realisation": round(ms / B, 3), "realisations": B,
            "value": round(B * N ** 3 * (N_MAX - 1) / ms / 1e3, 1),
            "unit": "Mcells*orders/s (orders 2..5, IC excluded)",
            "algorithmic_GB_per_realisation": round(gbytes, 2),
            "avg_GBps": round(gbytes * B / (ms / 1e3), 1),
            "autotune": tuning,
            "in_band_rms_rel_vs_full": float(f"{worst:.2e}")}


def mixed_batch(args):
    """Uneven batch: 128^3, 192^3 and 256^3 grids (L = 500, 750, 1000 Mpc/h, same
    cell size), 4 seeds each, n_max = 5: the whole recursion of all twelve
    realisations as one CUDA graph launch vs. the same work launched eagerly."""
    import torch
    from paper_1807_04215_gb300 import gridspt as g
    sizes = [(128, 500.0), (192, 750.0), (256, 1000.0)]
    plans = [g.Plan(n, N_MAX, L, batch=4) for n, L in sizes]
    for p in plans:
        g.autotune(p)
    d1s = [g.make_linear_field(p, [2000 + 10 * i + j for j in range(4)]) for i, p in enumerate(plans)]
    batch = g.Batch(plans, d1s)
    eager_sp = [torch.empty_like(x) for x in batch.spectra]
    eager_ws = [torch.empty(p.workspace_size(), dtype=torch.uint8, device="cuda") for p in plans]
    for _ in range(3):
        batch.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for _ in range(reps):
        batch.launch()
    e1.record()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / reps
    for p, d, sp, w in zip(plans, d1s, eager_sp, eager_ws):
        g.run_orders(p, d, spectra=sp, ws=w)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        for p, d, sp, w in zip(plans, d1s, eager_sp, eager_ws):
            g.run_orders(p, d, spectra=sp, ws=w)
    e1.record()
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1) / reps
    same = all(torch.equal(a, b) for a, b in zip(batch.spectra, eager_sp))
    cells = sum(4 * n ** 3 for n, _ in sizes)
    batch.close()
    # the same twelve realisations as ONE launch of the persistent work-queue
    # kernel; and with one plan (own workspace) per realisation, so that all
    # twelve chains can run concurrently
    def queue_ms(multi):
        for _ in range(3):
            multi.launch()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            multi.launch()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    multi = g.Multi(plans, d1s, wss=eager_ws)
    q_ms = queue_ms(multi)
    q_same = all(torch.equal(a, b) for a, b in zip(multi.spectra, eager_sp))
    multi.close()
    del eager_ws
    torch.cuda.empty_cache()
    singles, sd1 = [], []
    for i, (n, L) in enumerate(sizes):
        for j in range(4):
            p1 = g.Plan(n, N_MAX, L)
            g.set_tuning(p1, g.get_tuning(plans[i]))
            singles.append(p1)
            sd1.append(d1s[i][j:j + 1].contiguous())
    multi12 = g.Multi(singles, sd1)
    q12_ms = queue_ms(multi12)
    q12_same = all(torch.equal(multi12.spectra[4 * i + j], eager_sp[i][j:j + 1])
                   for i in range(3) for j in range(4))
    multi12.close()
    return {"grids": "128^3, 192^3, 256^3 x 4 seeds, n_max=5", "graph_ms": round(graph_ms, 3),
            "eager_ms": round(eager_ms, 3), "value": round(cells * N_MAX / graph_ms / 1e3, 1), "unit": UNIT,
            "bitwise_equal_to_eager": bool(same),
            "persistent_queue": {"ms": round(q_ms, 3), "value": round(cells * N_MAX / q_ms / 1e3, 1),
                                 "launches": 1, "chains": 3, "bitwise_equal_to_eager": bool(q_same)},
            "persistent_queue_12_chains": {"ms": round(q12_ms, 3), "value": round(cells * N_MAX / q12_ms / 1e3, 1),
                                           "launches": 1, "chains": 12,
                                           "bitwise_equal_to_eager": bool(q12_same)}}


def cufft_comparator(N, L, tuning):
    """Timing comparator only, not on the library's path: the library's 3D
    backward (C2R) and forward (R2C) transforms of four N^3 fields against
    cuFFT's (through torch.fft, which calls cuFFT) on the same fields, after
    warm-up (cuFFT's plans are cached by torch). Both unnormalised on the
    backward side; cuFFT's half spectrum keeps the kz = N/2 plane, which the
    library omits (zero by construction). Inputs of 2 GiB: larger than L2. The
    library's transforms use the tile variants the autotuner chose for the
    workload."""
    import torch
    from paper_1807_04215_gb300 import gridspt as g
    plan = g.Plan(N, N_MAX, L)
    g.set_tuning(plan, tuning)
    gen = torch.Generator(device="cuda").manual_seed(0)
    F = 4
    spec = torch.randn(F, N, N, N // 2, dtype=torch.complex64, device="cuda", generator=gen)
    real = torch.empty(F, N, N, N, dtype=torch.float32, device="cuda")
    spec_cu = torch.zeros(F, N, N, N // 2 + 1, dtype=torch.complex64, device="cuda")
    spec_cu[..., : N // 2] = spec
    dims = (-3, -2, -1)

    def per_field_ms(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return round(e0.elapsed_time(e1) / reps / F, 4)

    out = {"fields": f"{F} x {N}^3 FP32", "comparator": "cuFFT through torch.fft (timing only)",
           "library_tuning": list(tuning)}
    out["library_c2r_ms_per_field"] = per_field_ms(lambda: g.c2r(plan, spec, out=real))
    out["cufft_c2r_ms_per_field"] = per_field_ms(lambda: torch.fft.irfftn(spec_cu, s=(N, N, N), dim=dims,
                                                                           norm="forward"))
    out["library_r2c_ms_per_field"] = per_field_ms(lambda: g.r2c(plan, real, out=spec))
    out["cufft_r2c_ms_per_field"] = per_field_ms(lambda: torch.fft.rfftn(real, dim=dims))
    del spec, real, spec_cu
    torch.cuda.empty_cache()
    return out


def emulator_section(args):
    """P-term emulator: 256-point Latin hypercube over (sigma_8, n_s, Gamma),
    GridSPT at 256^3, L = 1000 Mpc/h, n_max = 5, 4 seeds per point, P22, P13,
    P33, P24, P15 in 32 log bins over 0.01-0.3 h/Mpc; 3-128-128-160 SiLU network
    (bf16 weights and activations, FP32 accumulation) trained with the
    library's kernels; its error measured by GridSPT on 32 held-out points."""
    import numpy as np
    import torch
    from paper_1807_04215_gb300 import emulator as E
    cfg = E.GridConfig()
    grid = E.GridSPTTerms(cfg)
    tr = E.latin_hypercube(256, 5)
    ho = E.latin_hypercube(32, 7)
    grid(tr[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ytr = grid.many(tr)
    torch.cuda.synchronize()
    grid_s_per_point = (time.perf_counter() - t0) / len(tr)
    yho = grid.many(ho)
    mask = grid.nk.cpu().numpy() > 0
    emu = E.train(tr, ytr, mask, steps=args.emu_steps)
    err = E.errors(emu.predict(ho), yho, mask)
    # throughput: emulator forward at batch 4096 vs GridSPT per cosmology
    xq = E.latin_hypercube(4096, 11)
    out = torch.empty(4096, 160, dtype=torch.float32, device="cuda")
    xin = torch.from_numpy(emu._xin(xq).astype(np.float32)).cuda()
    for _ in range(3):
        emu.net.forward(xin, y=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        emu.net.forward(xin, y=out)
    e1.record()
    torch.cuda.synchronize()
    emu_s_per_point = e0.elapsed_time(e1) / 20 / 1e3 / 4096
    return {"err_rel_rms": {k: round(v["rel_rms"], 5) for k, v in err.items()},
            "err_rel_max": {k: round(v["rel_max"], 5) for k, v in err.items()},
            "err_scale_max": {k: round(v["scale_max"], 5) for k, v in err.items()},
            "train_points": 256, "heldout_points": 32, "train_steps": args.emu_steps,
            "train_s": round(emu.train_seconds, 2),
            "gridspt_ms_per_cosmology": round(1e3 * grid_s_per_point, 3),
            "emulator_us_per_cosmology_b4096": round(1e6 * emu_s_per_point, 5),
            "speedup": round(grid_s_per_point / emu_s_per_point, 1)}


def run_case(args):
    """Small, self-contained invocations of the library for a profiler (ncu):
    one case, repeated `reps` times so that a profiler can skip the first.
      c2r      backward transforms of 4 random half spectra (x, y, z passes)
      r2c      forward transforms of 4 random real fields
      orders   one realisation: initial field and orders 2..n_max (L = 2000 N / 512)
      power    the six P-terms of one realisation (32 log bins, 0.01-0.4 h/Mpc)
      bispec   the equilateral bispectrum of one realisation (16 shells)
    --stats prints the library's per-kind launches, event time and algorithmic
    bytes of the last repetition (JSON)."""
    import torch
    from paper_1807_04215_gb300 import gridspt as g
    N, n_max = args.n, args.nmax
    L = BOX * N / N_GRID
    plan = g.Plan(N, n_max, L)
    if args.tuning:
        g.set_tuning(plan, [int(v) for v in args.tuning.split(",")])
    gen = torch.Generator(device="cuda").manual_seed(0)
    if args.case in ("c2r", "r2c"):
        spec = torch.randn(4, N, N, N // 2, dtype=torch.complex64, device="cuda", generator=gen)
        real = torch.empty(4, N, N, N, dtype=torch.float32, device="cuda")
        for _ in range(args.reps):
            if args.case == "c2r":
                g.c2r(plan, spec, out=real)
            else:
                g.r2c(plan, real.normal_(generator=gen), out=spec)
    else:
        d1 = g.make_linear_field(plan, [1000])
        spectra = g.run_orders(plan, d1) if args.case != "orders" else None
        edges = log_edges(0.01, 0.4, 32)
        kc = 2 * math.pi / L * N / (n_max + 1)
        bedges = [kc * i / 16 for i in range(17)]
        for rep in range(args.reps):
            if args.stats and rep == args.reps - 1:
                torch.cuda.synchronize()
                g.profile_begin()
            if args.case == "orders":
                g.make_linear_field(plan, [1000], out=d1)
                spectra = g.run_orders(plan, d1)
            elif args.case == "power":
                dl = {1: d1[0], **{n: spectra[0, n - 2, 0] for n in range(2, n_max + 1)}}
                for i, j in [(1, 1), (1, 3), (2, 2), (1, 5), (2, 4), (3, 3)]:
                    if j <= n_max:
                        g.power(plan, dl[i], dl[j], edges)
            else:
                g.bispectrum(plan, d1[0], spectra[0, 0, 0], bedges)
    torch.cuda.synchronize()
    if args.stats and args.case not in ("c2r", "r2c"):
        st = g.profile_end()
        print(json.dumps({k: {"launches": v[0], "ms": round(v[1], 4), "GB": round(v[2] / 1e9, 4)}
                          for k, v in st.items()}))
    print("ok", args.case, N)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--quick", action="store_true", help="skip the mixed-batch and emulator sections")
    ap.add_argument("--emu-steps", type=int, default=20000)
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="time the FP64 oracle at 64^3, 128^3, 256^3 on one and on all host cores")
    ap.add_argument("--case", choices=["c2r", "r2c", "orders", "power", "bispec"],
                    help="run one small library case for a profiler instead of the benchmark")
    ap.add_argument("--reps", type=int, default=2, help="--case: repetitions")
    ap.add_argument("--nmax", type=int, default=N_MAX, help="--case: highest order")
    ap.add_argument("--tuning", default="", help="--case: tile variants per pass, e.g. 1,1,1,2,2")
    ap.add_argument("--stats", action="store_true", help="--case: per-kind stats of the last repetition")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    if args.cpu_sweep:
        run_cpu_sweep(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
