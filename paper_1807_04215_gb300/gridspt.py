"""Python binding of libgridspt.so with the C-ABI's names (include/gridspt.h).

Tensors are torch CUDA tensors used only as device memory: half spectra are
complex64 [..., N, N, N/2] (interleaved re/im = float2), real fields float32
[..., N, N, N]. Each function checks shapes, allocates outputs and scratch
with torch, and passes raw pointers plus the current torch stream to the
library; every step of the computation runs in the library's CUDA kernels.
"""
import ctypes
import math
from dataclasses import dataclass

import torch

from . import _lib

DEFAULT_COSMO = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma8=0.8, gamma=0.0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


@dataclass
class Desc:
    n: int
    n_max: int
    box: float
    batch: int = 1
    kcut_lin: float = 0.0
    kcut_nl: float = 0.0


class Plan:
    """Owns a gridspt_plan (twiddle table on the current device)."""

    FORMS = {"nine_term": 0, "divergence": 1}
    ACCUMS = {"compensated": 0, "fp64": 1}

    def __init__(self, n, n_max, box, batch=1, kcut_lin=0.0, kcut_nl=0.0, form="nine_term", truncate=False,
                 accum="compensated"):
        """form: "nine_term" (the paper's bilinear sources) or "divergence"
        (A_n = div sum delta_m u_{n-m}, B_n = lap sum u_m . u_{n-m} / 2; equal in
        band, four real fields per order). truncate: cut every order j >= 2 at
        min(j, n_max + 1 - j) K_c (outputs at |k| <= K_c unchanged; nine-term
        form only). accum: shell sums of the estimators, "compensated" (FP32
        with carried rounding error, finished in FP64) or "fp64"."""
        self.lib = _lib.load()
        if form not in self.FORMS:
            raise ValueError(f"form must be one of {sorted(self.FORMS)}")
        if accum not in self.ACCUMS:
            raise ValueError(f"accum must be one of {sorted(self.ACCUMS)}")
        self.desc = Desc(n, n_max, box, batch, kcut_lin, kcut_nl)
        self.form = form
        self.truncate = bool(truncate)
        self.accum = accum
        d = _lib.GridsptDesc(n, n_max, batch, self.FORMS[form], box, kcut_lin, kcut_nl, int(bool(truncate)),
                             self.ACCUMS[accum])
        h = ctypes.c_void_p()
        _lib.check("gridspt_plan_create", self.lib.gridspt_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.n, self.m, self.n_max, self.batch, self.box = n, n // 2, n_max, batch, box

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.check("gridspt_plan_destroy", self.lib.gridspt_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- shapes
    def half_shape(self, *lead):
        return tuple(lead) + (self.n, self.n, self.m)

    def workspace_size(self):
        b = ctypes.c_size_t()
        _lib.check("gridspt_workspace_size", self.lib.gridspt_workspace_size(self.handle, ctypes.byref(b)))
        return b.value

    def _check_half(self, t, lead, name):
        exp = self.half_shape(*lead)
        if t.dtype != torch.complex64 or tuple(t.shape) != exp or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name}: expected contiguous CUDA complex64 {exp}, got {t.dtype} {tuple(t.shape)}")


def linear_amplitude(cosmo=None):
    lib = _lib.load()
    c = _lib.GridsptCosmo(**(cosmo or DEFAULT_COSMO))
    A = ctypes.c_double()
    _lib.check("gridspt_linear_amplitude", lib.gridspt_linear_amplitude(ctypes.byref(c), ctypes.byref(A)))
    return A.value


def growth_factor(z, cosmo=None):
    """D_+(z) / D_+(0) of a flat LCDM background (gridspt_growth_factor)."""
    lib = _lib.load()
    c = _lib.GridsptCosmo(**(cosmo or DEFAULT_COSMO))
    D = ctypes.c_double()
    _lib.check("gridspt_growth_factor", lib.gridspt_growth_factor(ctypes.byref(c), float(z), ctypes.byref(D)))
    return D.value


def make_linear_field(plan, seeds, cosmo=None, out=None):
    seeds = [int(s) for s in seeds]
    if len(seeds) != plan.batch:
        raise ValueError(f"need {plan.batch} seeds")
    if out is None:
        out = torch.empty(plan.half_shape(plan.batch), dtype=torch.complex64, device="cuda")
    plan._check_half(out, (plan.batch,), "out")
    c = _lib.GridsptCosmo(**(cosmo or DEFAULT_COSMO))
    arr = (ctypes.c_uint64 * len(seeds))(*seeds)
    _lib.check("gridspt_make_linear_field",
               plan.lib.gridspt_make_linear_field(plan.handle, ctypes.byref(c), arr, _ptr(out), _stream()))
    return out


def run_orders(plan, delta1, start_order=2, spectra=None, ws=None):
    plan._check_half(delta1, (plan.batch,), "delta1")
    if spectra is None:
        spectra = torch.empty(plan.half_shape(plan.batch, plan.n_max - 1, 2), dtype=torch.complex64, device="cuda")
    plan._check_half(spectra, (plan.batch, plan.n_max - 1, 2), "spectra")
    need = plan.workspace_size()
    if ws is None:
        ws = torch.empty(max(need, 16), dtype=torch.uint8, device="cuda")
    _lib.check("gridspt_run_orders",
               plan.lib.gridspt_run_orders(plan.handle, _ptr(delta1), start_order, _ptr(spectra), _ptr(ws),
                                           ws.numel() * ws.element_size(), _stream()))
    return spectra


class Batch:
    """gridspt_batch: the recursion of several plans (sizes may differ) captured
    as one CUDA graph; launch() replays it with one graph launch. Keeps the
    tensors it was built on alive (their addresses are baked into the graph)."""

    def __init__(self, plans, delta1s, spectra=None, wss=None, start_orders=None):
        self.lib = _lib.load()
        n = len(plans)
        spectra = list(spectra) if spectra is not None else [
            torch.empty(p.half_shape(p.batch, p.n_max - 1, 2), dtype=torch.complex64, device="cuda") for p in plans]
        wss = list(wss) if wss is not None else [
            torch.empty(max(p.workspace_size(), 16), dtype=torch.uint8, device="cuda") for p in plans]
        starts = list(start_orders) if start_orders is not None else [2] * n
        for p, d, sp in zip(plans, delta1s, spectra):
            p._check_half(d, (p.batch,), "delta1")
            p._check_half(sp, (p.batch, p.n_max - 1, 2), "spectra")
        self.keep = (plans, list(delta1s), spectra, wss)
        arr = lambda T, xs: (T * n)(*xs)  # noqa: E731
        h = ctypes.c_void_p()
        _lib.check("gridspt_batch_create", self.lib.gridspt_batch_create(
            arr(ctypes.c_void_p, [p.handle.value for p in plans]), n,
            arr(ctypes.c_void_p, [d.data_ptr() for d in delta1s]), arr(ctypes.c_int32, starts),
            arr(ctypes.c_void_p, [x.data_ptr() for x in spectra]), arr(ctypes.c_void_p, [w.data_ptr() for w in wss]),
            arr(ctypes.c_size_t, [w.numel() for w in wss]), ctypes.byref(h)))
        self.handle = h
        self.spectra = spectra

    def launch(self):
        _lib.check("gridspt_batch_launch", self.lib.gridspt_batch_launch(self.handle, _stream()))
        return self.spectra

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.check("gridspt_batch_destroy", self.lib.gridspt_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """gridspt_multi: the recursion of several plans (sizes may differ) as one
    launch of the persistent work-queue kernel (gridspt_run_orders_multi per
    launch()). Keeps the tensors it was built on alive (the queue holds their
    addresses)."""

    def __init__(self, plans, delta1s, spectra=None, wss=None, start_orders=None):
        self.lib = _lib.load()
        n = len(plans)
        spectra = list(spectra) if spectra is not None else [
            torch.empty(p.half_shape(p.batch, p.n_max - 1, 2), dtype=torch.complex64, device="cuda") for p in plans]
        wss = list(wss) if wss is not None else [
            torch.empty(max(p.workspace_size(), 16), dtype=torch.uint8, device="cuda") for p in plans]
        starts = list(start_orders) if start_orders is not None else [2] * n
        for p, d, sp in zip(plans, delta1s, spectra):
            p._check_half(d, (p.batch,), "delta1")
            p._check_half(sp, (p.batch, p.n_max - 1, 2), "spectra")
        self.keep = (plans, list(delta1s), spectra, wss)
        arr = lambda T, xs: (T * n)(*xs)  # noqa: E731
        h = ctypes.c_void_p()
        _lib.check("gridspt_multi_create", self.lib.gridspt_multi_create(
            arr(ctypes.c_void_p, [p.handle.value for p in plans]), n,
            arr(ctypes.c_void_p, [d.data_ptr() for d in delta1s]), arr(ctypes.c_int32, starts),
            arr(ctypes.c_void_p, [x.data_ptr() for x in spectra]), arr(ctypes.c_void_p, [w.data_ptr() for w in wss]),
            arr(ctypes.c_size_t, [w.numel() for w in wss]), ctypes.byref(h)))
        self.handle = h
        self.spectra = spectra

    def launch(self):
        _lib.check("gridspt_run_orders_multi", self.lib.gridspt_run_orders_multi(self.handle, _stream()))
        return self.spectra

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.check("gridspt_multi_destroy", self.lib.gridspt_multi_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check(plan):
    """gridspt_check: raises GridsptError with status 5 (GRIDSPT_E_TIMEOUT) if a
    bounded device wait gave up, 6 (GRIDSPT_E_NUMERIC) if an estimator result
    was NaN or infinite since the last check."""
    _lib.check("gridspt_check", plan.lib.gridspt_check(plan.handle, _stream()))


def autotune(plan, scratch=None):
    """Time the tile variants of every transform pass and keep the fastest;
    returns the choices [column pass, x, y, z expansion, z forward]."""
    b = ctypes.c_size_t()
    _lib.check("gridspt_autotune_scratch_size", plan.lib.gridspt_autotune_scratch_size(plan.handle, ctypes.byref(b)))
    if scratch is None:
        scratch = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    ch = (ctypes.c_int32 * 5)()
    _lib.check("gridspt_autotune", plan.lib.gridspt_autotune(plan.handle, _ptr(scratch), scratch.numel(), ch,
                                                              _stream()))
    return list(ch)


def set_tuning(plan, choices):
    ch = (ctypes.c_int32 * 5)(*[int(c) for c in choices])
    _lib.check("gridspt_set_tuning", plan.lib.gridspt_set_tuning(plan.handle, ch))


def get_tuning(plan):
    ch = (ctypes.c_int32 * 5)()
    _lib.check("gridspt_get_tuning", plan.lib.gridspt_get_tuning(plan.handle, ch))
    return list(ch)


def c2r(plan, spec, out=None):
    lead = tuple(spec.shape[:-3])
    count = int(math.prod(lead)) if lead else 1
    plan._check_half(spec, lead, "spec")
    if out is None:
        out = torch.empty(lead + (plan.n,) * 3, dtype=torch.float32, device="cuda")
    _lib.check("gridspt_c2r", plan.lib.gridspt_c2r(plan.handle, _ptr(spec), _ptr(out), count, _stream()))
    return out


def r2c(plan, field, out=None):
    lead = tuple(field.shape[:-3])
    count = int(math.prod(lead)) if lead else 1
    if field.dtype != torch.float32 or not field.is_contiguous() or tuple(field.shape[-3:]) != (plan.n,) * 3:
        raise ValueError("field: expected contiguous float32 [..., N, N, N]")
    if out is None:
        out = torch.empty(plan.half_shape(*lead), dtype=torch.complex64, device="cuda")
    _lib.check("gridspt_r2c", plan.lib.gridspt_r2c(plan.handle, _ptr(field), _ptr(out), count, _stream()))
    return out


def _edges(edges):
    e = [float(x) for x in edges]
    return (ctypes.c_double * len(e))(*e), len(e) - 1


def power_workspace_size(plan, nbins):
    b = ctypes.c_size_t()
    _lib.check("gridspt_power_workspace_size",
               plan.lib.gridspt_power_workspace_size(plan.handle, nbins, ctypes.byref(b)))
    return b.value


def power(plan, a, b, edges, ws=None, out=None, nk=None):
    """P(i) = L^3 / N_i sum Re[a b*] over shell i; returns (p, n_k) device tensors."""
    plan._check_half(a, (), "a")
    plan._check_half(b, (), "b")
    e, nb = _edges(edges)
    if out is None:
        out = torch.empty(nb, dtype=torch.float64, device="cuda")
    if nk is None:
        nk = torch.empty(nb, dtype=torch.int64, device="cuda")
    if ws is None:
        ws = torch.empty(power_workspace_size(plan, nb), dtype=torch.uint8, device="cuda")
    _lib.check("gridspt_power",
               plan.lib.gridspt_power(plan.handle, _ptr(a), _ptr(b), nb, e, _ptr(out), _ptr(nk), _ptr(ws),
                                      ws.numel(), _stream()))
    return out, nk


def power_noalloc(plan, a, b, edges, out=None, nk=None):
    """gridspt_power_noalloc: the shell power estimator with the library's own
    static scratch, for callers that must not allocate device memory (the
    caller passes only inputs and outputs)."""
    plan._check_half(a, (), "a")
    plan._check_half(b, (), "b")
    e, nb = _edges(edges)
    if out is None:
        out = torch.empty(nb, dtype=torch.float64, device="cuda")
    if nk is None:
        nk = torch.empty(nb, dtype=torch.int64, device="cuda")
    _lib.check("gridspt_power_noalloc",
               plan.lib.gridspt_power_noalloc(plan.handle, _ptr(a), _ptr(b), nb, e, _ptr(out), _ptr(nk),
                                              _stream()))
    return out, nk


def bispectrum_workspace_size(plan, nbins):
    b = ctypes.c_size_t()
    _lib.check("gridspt_bispectrum_workspace_size",
               plan.lib.gridspt_bispectrum_workspace_size(plan.handle, nbins, ctypes.byref(b)))
    return b.value


def bispectrum(plan, a, b, edges, ws=None):
    """Equilateral shell triple product E = L^6 sum I_a^2 I_b / sum J^3 and N_tri per
    shell; B_tree = 3 E for a = delta_1, b = delta_2."""
    plan._check_half(a, (), "a")
    plan._check_half(b, (), "b")
    e, nb = _edges(edges)
    E = torch.empty(nb, dtype=torch.float64, device="cuda")
    nt = torch.empty(nb, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = torch.empty(bispectrum_workspace_size(plan, nb), dtype=torch.uint8, device="cuda")
    _lib.check("gridspt_bispectrum",
               plan.lib.gridspt_bispectrum(plan.handle, _ptr(a), _ptr(b), nb, e, _ptr(E), _ptr(nt), _ptr(ws),
                                           ws.numel(), _stream()))
    return E, nt


def sum_orders(plan, delta1, spectra, n, D=1.0, R=0.0, out=None):
    """delta_SPT(k) = exp(-k^2 R^2 / 2) sum_{i<=n} D^i delta_i(k) for one
    realisation: delta1 [N][N][N/2], spectra [n_max-1][2][N][N][N/2]."""
    plan._check_half(delta1, (), "delta1")
    if n >= 2:
        plan._check_half(spectra, (plan.n_max - 1, 2), "spectra")
    if out is None:
        out = torch.empty(plan.half_shape(), dtype=torch.complex64, device="cuda")
    plan._check_half(out, (), "out")
    _lib.check("gridspt_sum_orders",
               plan.lib.gridspt_sum_orders(plan.handle, _ptr(delta1), _ptr(spectra) if n >= 2 else None, int(n),
                                           float(D), float(R), _ptr(out), _stream()))
    return out


def cross_correlation(plan, a, b, edges, ws=None):
    """Cross-correlation coefficient r = P_ab / sqrt(P_aa P_bb) per bin."""
    plan._check_half(a, (), "a")
    plan._check_half(b, (), "b")
    e, nb = _edges(edges)
    if ws is None:
        size = ctypes.c_size_t()
        _lib.check("gridspt_cross_correlation_workspace_size",
                   plan.lib.gridspt_cross_correlation_workspace_size(plan.handle, nb, ctypes.byref(size)))
        ws = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    r = torch.empty(nb, dtype=torch.float64, device="cuda")
    _lib.check("gridspt_cross_correlation",
               plan.lib.gridspt_cross_correlation(plan.handle, _ptr(a), _ptr(b), nb, e, _ptr(r), _ptr(ws), ws.numel(),
                                                  _stream()))
    return r


def bispectrum_triple(plan, a, b, c, edges, ws=None):
    """Equilateral shell triple product E = L^6 sum I_a I_b I_c / sum J^3 and N_tri
    per shell (gridspt_bispectrum_triple)."""
    for t, name in ((a, "a"), (b, "b"), (c, "c")):
        plan._check_half(t, (), name)
    e, nb = _edges(edges)
    E = torch.empty(nb, dtype=torch.float64, device="cuda")
    nt = torch.empty(nb, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = torch.empty(bispectrum_workspace_size(plan, nb), dtype=torch.uint8, device="cuda")
    _lib.check("gridspt_bispectrum_triple",
               plan.lib.gridspt_bispectrum_triple(plan.handle, _ptr(a), _ptr(b), _ptr(c), nb, e, _ptr(E), _ptr(nt),
                                                  _ptr(ws), ws.numel(), _stream()))
    return E, nt


def bispectrum_one_loop(plan, d1, d2, d3, d4, edges, ws=None):
    """One-loop bispectrum of Eq. bk_1loop (D_+ = 1) in equilateral shells:
    B = 6 E[d1, d2, d3] + E[d2, d2, d2] + 3 E[d1, d1, d4] (the ten ordered terms
    of the equation collapse to these three sums when all |k_i| share a shell).
    Returns (B, N_tri)."""
    e, nb = _edges(edges)
    if ws is None:
        ws = torch.empty(bispectrum_workspace_size(plan, nb), dtype=torch.uint8, device="cuda")
    e123, nt = bispectrum_triple(plan, d1, d2, d3, edges, ws)
    e222, _ = bispectrum_triple(plan, d2, d2, d2, edges, ws)
    e114, _ = bispectrum_triple(plan, d1, d1, d4, edges, ws)
    return 6.0 * e123 + e222 + 3.0 * e114, nt


def default_kcut(n, n_max, box):
    """2 k_Ny / (n_max + 1) in h/Mpc."""
    return 2.0 * math.pi / box * n / (n_max + 1)


def profile_begin():
    lib = _lib.load()
    _lib.check("gridspt_profile_begin", lib.gridspt_profile_begin())


def profile_end():
    """{kernel kind: (launches, ms, algorithmic bytes)} recorded since profile_begin."""
    lib = _lib.load()
    cap = 32
    arr = (_lib.GridsptKernelStat * cap)()
    n = ctypes.c_int32()
    _lib.check("gridspt_profile_end", lib.gridspt_profile_end(arr, cap, ctypes.byref(n)))
    return {arr[i].name.decode(): (arr[i].launches, arr[i].ms, arr[i].bytes) for i in range(n.value)}


# ---------------------------------------------------------------- emulator MLP
class MLP:
    """Device buffers and kernel calls of the emulator network (C-ABI
    gridspt_mlp_*): FP32 master parameters, the bf16 (or FP32) copy read by
    forward/backward, Adam moments and the device step counter."""

    def __init__(self, n_in=3, hidden=128, n_out=160, bf16=True, seed=0):
        self.lib = _lib.load()
        self.I, self.H, self.O, self.bf16 = n_in, hidden, n_out, int(bool(bf16))
        c = ctypes.c_int64()
        _lib.check("gridspt_mlp_param_count", self.lib.gridspt_mlp_param_count(n_in, hidden, n_out, ctypes.byref(c)))
        self.n = c.value
        # Glorot-uniform weights, zero biases (initial values from a seeded torch generator)
        gen = torch.Generator().manual_seed(seed)
        parts = []
        for fi, fo in ((n_in, hidden), (hidden, hidden), (hidden, n_out)):
            lim = math.sqrt(6.0 / (fi + fo))
            parts += [(torch.rand(fi * fo, generator=gen) * 2 - 1) * lim, torch.zeros(fo)]
        self.master = torch.cat(parts).to(torch.float32).cuda()
        self.lowp = torch.empty(self.n, dtype=torch.bfloat16 if self.bf16 else torch.float32, device="cuda")
        self.m = torch.zeros(self.n, dtype=torch.float32, device="cuda")
        self.v = torch.zeros(self.n, dtype=torch.float32, device="cuda")
        self.step = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.grad = torch.zeros(self.n, dtype=torch.float32, device="cuda")
        self.sync_lowp()

    def sync_lowp(self):
        _lib.check("gridspt_mlp_convert", self.lib.gridspt_mlp_convert(_ptr(self.master), _ptr(self.lowp), self.bf16,
                                                                        self.n, _stream()))

    def forward(self, x, y=None, act=None):
        B = x.shape[0]
        if y is None:
            y = torch.empty(B, self.O, dtype=torch.float32, device="cuda")
        _lib.check("gridspt_mlp_forward", self.lib.gridspt_mlp_forward(
            _ptr(x), B, self.I, self.H, self.O, _ptr(self.lowp), self.bf16, _ptr(y), _ptr(act), _stream()))
        return y

    def ws_bytes(self, B):
        b = ctypes.c_size_t()
        _lib.check("gridspt_mlp_backward_workspace_size",
                   self.lib.gridspt_mlp_backward_workspace_size(B, self.I, self.H, self.O, ctypes.byref(b)))
        return b.value

    def backward(self, x, act, dy, ws):
        _lib.check("gridspt_mlp_backward", self.lib.gridspt_mlp_backward(
            _ptr(x), x.shape[0], self.I, self.H, self.O, _ptr(self.lowp), self.bf16, _ptr(act), _ptr(dy),
            _ptr(self.grad), _ptr(ws), ws.numel(), _stream()))
        return self.grad

    def mse(self, y, t, mask, dy, loss=None):
        _lib.check("gridspt_mlp_mse", self.lib.gridspt_mlp_mse(_ptr(y), _ptr(t), _ptr(mask), y.numel(), _ptr(dy),
                                                                _ptr(loss), _stream()))

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        _lib.check("gridspt_mlp_adam", self.lib.gridspt_mlp_adam(
            _ptr(self.master), _ptr(self.lowp), self.bf16, _ptr(self.grad), _ptr(self.m), _ptr(self.v),
            _ptr(self.step), self.n, ctypes.c_float(lr), ctypes.c_float(b1), ctypes.c_float(b2), ctypes.c_float(eps),
            _stream()))
