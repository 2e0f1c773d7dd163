// Host runtime behind include/gridspt.h: argument validation, plan tables,
// the order-by-order schedule of the Sec. II.C recipe, and the estimator
// drivers. Every step of the path runs in the CUDA kernels; this file only
// validates, computes host scalars (FP64 spectrum normalisation, integer bin
// thresholds) and enqueues launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <functional>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gridspt.h"
#include "gridspt_internal.h"

using namespace gridspt;

struct gridspt_plan_s {
    gridspt_desc d;
    Geo geo;
    float2* tw = nullptr;   // device: N entries, then the tables of the smaller sizes (sub_off)
    long long sub_off[kNumSizes] = {};   // offset in tw of the table of kSizes[i] < N, else -1
    long long s2_lin;       // keep 0 < |s|^2 <= s2_lin in delta_1
    double r_lin = 0.0;     // the linear cut K_c / k_F
    long long s2_nl;        // < 0: no cut on higher orders
    int device = 0;
    long long pb_top = -1;  // cache of the last power-launch byte count (profiling only)
    double pb_modes = 0.0;
    double* j3 = nullptr;   // device [kMaxBins]: sum_x J^3 per bispectrum shell (data independent)
    double* ic_table = nullptr;   // device [ic_s2 + 1]: mode amplitude per |s|^2 (same allocation as j3)
    long long ic_s2 = 0;
    int* status = nullptr;  // device status word (bounded waits that gave up)
    int j3_nb = 0;          // shells the cache holds (0: empty) and their thresholds
    int j3_thr[kMaxBins + 1] = {};
};

namespace {

thread_local char g_err[512] = "";

gridspt_status fail(gridspt_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

gridspt_status cuda_fail(cudaError_t e, const char* where) {
    return fail(GRIDSPT_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Host-side fault injection for tests (no GPU fault is ever caused): the
// environment variable GRIDSPT_FAULT_INJECT holds a comma-separated list of
//   plan_alloc  - the plan's second device allocation reports out-of-memory
//   launch      - every kernel launch reports a launch failure without launching
bool fault_inject(const char* what) {
    const char* v = std::getenv("GRIDSPT_FAULT_INJECT");
    if (!v || !*v) return false;
    const size_t n = std::strlen(what);
    for (const char* q = v; (q = std::strstr(q, what)) != nullptr; q += n) {
        const bool start = q == v || q[-1] == ',';
        const bool end = q[n] == 0 || q[n] == ',';
        if (start && end) return true;
    }
    return false;
}

// ------------------------------------------------------------- profiling
enum ProfKind {
    PK_IC, PK_XEXP, PK_XEXP_FWD, PK_YEXP, PK_ZEXP, PK_Y_FWD, PK_X_FWD, PK_ZR2C,
    PK_PRODUCT, PK_POWER, PK_BISPEC, PK_BX, PK_BY, PK_BZ, PK_MLP_FWD, PK_MLP_BWD, PK_MLP_OPT, PK_FIELDS,
    PK_BGATHER, PK_QUEUE, PK_COUNT
};
const char* const kProfNames[PK_COUNT] = {
    "ic", "x_expand", "x_fwd_expand", "y_expand", "z_expand", "y_fwd", "x_fwd", "z_r2c",
    "product", "power", "bispec_final", "shell_x", "shell_y", "shell_z", "mlp_forward", "mlp_backward",
    "mlp_update", "sum_orders", "shell_grid", "work_queue"};
constexpr size_t kMaxProfRecs = 65536;

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes;
};
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
};
Profiler g_prof;
thread_local bool t_capturing = false;   // launches being captured into a graph are not profiled

cudaEvent_t prof_event() {
    if (!g_prof.pool.empty()) {
        cudaEvent_t e = g_prof.pool.back();
        g_prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch through `f`, bracketed by events on `s` while profiling is on.
template <class F>
cudaError_t prof_launch(int kind, double bytes, cudaStream_t s, F&& f) {
    if (fault_inject("launch")) return cudaErrorLaunchFailure;
    std::unique_lock<std::mutex> lk(g_prof.mu);
    if (!g_prof.on || t_capturing || g_prof.recs.size() >= kMaxProfRecs) {
        lk.unlock();
        return f();
    }
    cudaEvent_t a = prof_event(), b = prof_event();
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(a, s);
    if (e != cudaSuccess) return e;
    e = f();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(b, s);
    if (e != cudaSuccess) return e;
    g_prof.recs.push_back({kind, a, b, bytes});
    return cudaSuccess;
}

#define CKP(kind, bytes, s, call, where)                                              \
    do {                                                                              \
        cudaError_t e_ = prof_launch((kind), (bytes), (s), [&]() { return (call); }); \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);                           \
    } while (0)

// Stage recording for the persistent work queue (gridspt_run_orders_multi):
// while t_queue is set, the launch sites of the recursion append a stage
// (kind, grid, arguments, work estimate) instead of launching.
thread_local std::vector<QStage>* t_queue = nullptr;

QStage q_stage(const Geo& g, int kind, double cost) {
    QStage q{};
    q.kind = kind;
    q.N = g.N;
    q.dep = -1;
    q.tw = g.tw;
    q.kF = kDerivUnit;
    q.inv_kF2 = 1.0f / (kDerivUnit * kDerivUnit);
    q.cost = cost;
    return q;
}

#define CKQ(kind, bytes, s, call, where, stage)          \
    do {                                                 \
        if (t_queue) {                                   \
            QStage q_ = (stage);                         \
            queue_tiles(q_);                             \
            t_queue->push_back(q_);                      \
        } else {                                         \
            CKP(kind, bytes, s, call, where);            \
        }                                                \
    } while (0)

long long field_floats(const gridspt_plan_s* p) { return (long long)p->geo.N * p->geo.N * p->geo.N; }
long long field_c(const gridspt_plan_s* p) { return (long long)p->geo.N * p->geo.N * p->geo.M; }

int order_base(int m) { return m == 1 ? 0 : 13 + 17 * (m - 2); }
// Accumulate-ahead workspace (fields of 4 N^3 bytes): the real derived fields
// of the orders that later pairs still need (2m <= n_max), two accumulator
// fields (A, B) per target order n >= 4, then the expansion scratch
// (7 x-fields + 12 xy-fields).
constexpr int kExpScratch = 7 + 12;
int stored_orders(int n_max) { return n_max / 2; }
int total_derived(int n_max) { return n_max >= 2 ? order_base(stored_orders(n_max) + 1) : 0; }
int acc_base(int n_max) { return total_derived(n_max); }
int n_acc(int n_max) { return n_max >= 4 ? 2 * (n_max - 3) : 0; }
int scratch_base(int n_max) { return acc_base(n_max) + n_acc(n_max); }
int workspace_fields(int n_max) { return n_max >= 2 ? scratch_base(n_max) + kExpScratch : 0; }

// Divergence-form workspace: the real fields delta, u_x, u_y, u_z of orders
// 1..n_max-1 (every later order needs them), the sources V_x, V_y, V_z, S of
// the order being formed (transformed in place), then the expansion scratch
// (3 x-fields, 4 xy-fields).
int div_order_base(int m) { return 4 * (m - 1); }
int div_src_base(int n_max) { return 4 * (n_max - 1); }
int div_scratch_base(int n_max) { return div_src_base(n_max) + 4; }
int div_workspace_fields(int n_max) { return n_max >= 2 ? div_scratch_base(n_max) + 3 + 4 : 0; }

// s2 threshold: smallest integer t >= 0 with kF * sqrt(t) >= e (FP64), so that
// "t <= |s|^2" is exactly the FP64 test "e <= kF sqrt(|s|^2)".
long long s2_threshold(double e, double kF) {
    if (!(e > 0.0)) return 0;
    double r = e / kF;
    long long t = (long long)std::floor(r * r);
    if (t < 0) t = 0;
    while (t > 0 && kF * std::sqrt((double)(t - 1)) >= e) --t;
    while (kF * std::sqrt((double)t) < e) ++t;
    return t;
}

// ---------------------------------------------------------------- spectrum
double bbks(double q) {
    if (q <= 0.0) return 1.0;
    const double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
    return std::log1p(2.34 * q) / (2.34 * q) * std::pow(poly, -0.25);
}
double gamma_of(const gridspt_cosmo* c) { return c->gamma > 0 ? c->gamma : c->omega_m * c->h; }
double tophat(double x) {
    if (std::fabs(x) < 1e-3) return 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
    return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}
// sigma_8^2 for A = 1: (1/2pi^2) int k^3 k^ns T^2 W(8k)^2 dlnk, Simpson, 65536 intervals on [1e-5, 1e3].
double sigma8_sq_unit(const gridspt_cosmo* c) {
    const int n = 1 << 16;
    const double lo = std::log(1e-5), hi = std::log(1e3), h = (hi - lo) / n, G = gamma_of(c);
    double s = 0.0;
    for (int i = 0; i <= n; ++i) {
        const double k = std::exp(lo + h * i);
        const double t = bbks(k / G), w = tophat(8.0 * k);
        const double f = k * k * k * std::pow(k, c->n_s) * t * t * w * w;
        s += f * (i == 0 || i == n ? 1.0 : (i % 2 ? 4.0 : 2.0));
    }
    return h / 3.0 * s / (2.0 * M_PI * M_PI);
}

gridspt_status check_plan(gridspt_plan p) {
    if (!p) return fail(GRIDSPT_E_INVALID, "plan is NULL");
    return GRIDSPT_OK;
}

gridspt_status set_device(const gridspt_plan_s* p) {
    int cur = -1;
    CK(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != p->device) return fail(GRIDSPT_E_INVALID, "plan was created on device %d, current is %d", p->device, cur);
    return GRIDSPT_OK;
}

}  // namespace

extern "C" {

const char* gridspt_last_error(void) { return g_err; }

gridspt_status gridspt_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto& r : g_prof.recs) {
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.recs.clear();
    g_prof.on = true;
    return GRIDSPT_OK;
}

gridspt_status gridspt_profile_end(gridspt_kernel_stat* stats, int32_t capacity, int32_t* count) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = false;
    double ms[PK_COUNT] = {0}, bytes[PK_COUNT] = {0};
    int launches[PK_COUNT] = {0};
    gridspt_status st = GRIDSPT_OK;
    for (auto& r : g_prof.recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && st == GRIDSPT_OK) st = cuda_fail(e, "profile event");
        ms[r.kind] += t;
        bytes[r.kind] += r.bytes;
        launches[r.kind] += 1;
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.recs.clear();
    int n = 0;
    for (int k = 0; k < PK_COUNT; ++k) {
        if (!launches[k]) continue;
        if (stats && n < capacity) {
            std::memset(&stats[n], 0, sizeof(stats[n]));
            std::snprintf(stats[n].name, sizeof(stats[n].name), "%s", kProfNames[k]);
            stats[n].launches = launches[k];
            stats[n].ms = ms[k];
            stats[n].bytes = bytes[k];
        }
        ++n;
    }
    if (count) *count = std::min(n, capacity);
    return st;
}

gridspt_status gridspt_plan_create(const gridspt_desc* d, gridspt_plan* out) {
    g_err[0] = 0;
    if (!d || !out) return fail(GRIDSPT_E_INVALID, "desc/out is NULL");
    *out = nullptr;
    if (!supported_n(d->n)) return fail(GRIDSPT_E_INVALID, "n=%d: need even N = 2^a or 3*2^a, 8 <= N <= 1024", d->n);
    if (d->n_max < 1 || d->n_max > kMaxOrder) return fail(GRIDSPT_E_INVALID, "n_max=%d outside [1, %d]", d->n_max, kMaxOrder);
    if (d->batch < 1) return fail(GRIDSPT_E_INVALID, "batch=%d < 1", d->batch);
    if (!(d->box > 0.0) || !std::isfinite(d->box)) return fail(GRIDSPT_E_INVALID, "box must be > 0");
    if (d->form != GRIDSPT_FORM_NINE_TERM && d->form != GRIDSPT_FORM_DIVERGENCE)
        return fail(GRIDSPT_E_INVALID, "form=%d: must be GRIDSPT_FORM_NINE_TERM (0) or GRIDSPT_FORM_DIVERGENCE (1)",
                    d->form);
    if (d->truncate != 0 && d->truncate != 1) return fail(GRIDSPT_E_INVALID, "truncate=%d: must be 0 or 1", d->truncate);
    if (d->truncate && d->form != GRIDSPT_FORM_NINE_TERM)
        return fail(GRIDSPT_E_INVALID, "truncate=1 needs the nine-term form");
    if (d->accum != GRIDSPT_ACCUM_COMPENSATED && d->accum != GRIDSPT_ACCUM_FP64)
        return fail(GRIDSPT_E_INVALID, "accum=%d: must be GRIDSPT_ACCUM_COMPENSATED (0) or GRIDSPT_ACCUM_FP64 (1)",
                    d->accum);
    gridspt_plan_s* p = new (std::nothrow) gridspt_plan_s();
    if (!p) return fail(GRIDSPT_E_NOMEM, "host allocation failed");
    p->d = *d;
    const int N = d->n;
    p->geo.N = N;
    p->geo.M = N / 2;
    p->geo.kF = 2.0 * M_PI / d->box;
    p->geo.accum = d->accum == GRIDSPT_ACCUM_FP64 ? kAccumFp64 : kAccumCompensated;
    const double r = d->kcut_lin > 0 ? d->kcut_lin * d->box / (2.0 * M_PI) : (double)N / (d->n_max + 1);
    p->s2_lin = (long long)std::floor(r * r);
    p->r_lin = r;
    if (d->kcut_nl > 0) {
        const double rn = d->kcut_nl * d->box / (2.0 * M_PI);
        p->s2_nl = (long long)std::floor(rn * rn);
    } else {
        p->s2_nl = -1;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
    // roots of unity of size N, then of every smaller supported size (the
    // bispectrum evaluates band-limited shells on smaller grids)
    std::vector<float2> tw;
    auto roots = [&tw](int n) {
        for (int j = 0; j < n; ++j) {
            const double a = 2.0 * M_PI * (double)j / (double)n;
            tw.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
    };
    roots(N);
    for (int i = 0; i < kNumSizes; ++i) {
        p->sub_off[i] = kSizes[i] < N ? (long long)tw.size() : -1;
        if (kSizes[i] < N) roots(kSizes[i]);
    }
    e = cudaMalloc(&p->tw, sizeof(float2) * tw.size());
    if (e != cudaSuccess) { delete p; return fail(GRIDSPT_E_NOMEM, "twiddle table: %s", cudaGetErrorString(e)); }
    // one small block: the shell cache (kMaxBins doubles), the status word (4
    // ints) and the initial field's amplitude table (|s|^2 = 0..ic_s2)
    p->ic_s2 = std::min<long long>(p->s2_lin, 3LL * (N / 2) * (N / 2));
    e = fault_inject("plan_alloc") ? cudaErrorMemoryAllocation
                                   : cudaMalloc(&p->j3, sizeof(double) * (kMaxBins + 2 + p->ic_s2 + 1));
    if (e != cudaSuccess) {
        cudaFree(p->tw);
        delete p;
        return fail(GRIDSPT_E_NOMEM, "shell cache: %s", cudaGetErrorString(e));
    }
    p->status = reinterpret_cast<int*>(p->j3 + kMaxBins);
    p->ic_table = p->j3 + kMaxBins + 2;
    p->geo.status = p->status;
    e = cudaMemset(p->status, 0, sizeof(int));
    if (e != cudaSuccess) { cudaFree(p->tw); cudaFree(p->j3); delete p; return cuda_fail(e, "status word"); }
    e = cudaMemcpy(p->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(p->tw); cudaFree(p->j3); delete p; return cuda_fail(e, "twiddle upload"); }
    p->geo.tw = p->tw;
    *out = p;
    return GRIDSPT_OK;
}

gridspt_status gridspt_plan_destroy(gridspt_plan p) {
    if (!p) return GRIDSPT_OK;
    cudaError_t e = cudaSuccess;
    if (p->tw) {
        e = cudaDeviceSynchronize();
        cudaError_t e2 = cudaFree(p->tw);
        if (e == cudaSuccess) e = e2;
        e2 = p->j3 ? cudaFree(p->j3) : cudaSuccess;
        if (e == cudaSuccess) e = e2;
    }
    delete p;
    if (e != cudaSuccess) return cuda_fail(e, "plan_destroy");
    return GRIDSPT_OK;
}

gridspt_status gridspt_workspace_size(gridspt_plan p, size_t* bytes) {
    if (check_plan(p) || !bytes) return fail(GRIDSPT_E_INVALID, "plan/bytes is NULL");
    const int nf = p->d.form == GRIDSPT_FORM_DIVERGENCE ? div_workspace_fields(p->d.n_max) : workspace_fields(p->d.n_max);
    *bytes = (size_t)nf * (size_t)field_floats(p) * sizeof(float);
    return GRIDSPT_OK;
}

gridspt_status gridspt_linear_amplitude(const gridspt_cosmo* c, double* A) {
    if (!c || !A) return fail(GRIDSPT_E_INVALID, "cosmo/A is NULL");
    if (!(c->sigma8 > 0) || !(gamma_of(c) > 0)) return fail(GRIDSPT_E_INVALID, "sigma8 and Gamma must be > 0");
    *A = c->sigma8 * c->sigma8 / sigma8_sq_unit(c);
    return GRIDSPT_OK;
}

gridspt_status gridspt_make_linear_field(gridspt_plan p, const gridspt_cosmo* c, const uint64_t* seeds,
                                         void* delta1_k, gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (!c || !seeds || !delta1_k) return fail(GRIDSPT_E_INVALID, "NULL argument");
    if (!aligned16(delta1_k)) return fail(GRIDSPT_E_INVALID, "delta1_k not 16-byte aligned");
    if (gridspt_status st = set_device(p)) return st;
    double A = 0.0;
    if (gridspt_status st = gridspt_linear_amplitude(c, &A)) return st;
    IcArgs a{};
    a.amp = A;
    a.n_s = c->n_s;
    a.gamma = gamma_of(c);
    a.inv_vol = 1.0 / (p->d.box * p->d.box * p->d.box);
    a.s2_cut = p->ic_s2;
    a.table = p->ic_table;
    a.kF = p->geo.kF;
    CK(launch_ic_table(a, (cudaStream_t)stream), "ic amplitude table");
    for (int b = 0; b < p->d.batch; ++b) {
        a.out = static_cast<float2*>(delta1_k) + (long long)b * field_c(p);
        a.seed = seeds[b];
        CKP(PK_IC, 4.0 * (double)field_floats(p), (cudaStream_t)stream, launch_ic(p->geo, a, (cudaStream_t)stream),
            "ic launch");
    }
    return GRIDSPT_OK;
}

namespace {

// The x-, y- and z-expansion output lists of order m (see derive_order).
void expansion_codes(int m, XExpArgs& xa, YZExpArgs& ya, YZExpArgs& za) {
    const int I = 1, NI = 2;  // z-pass constants i and -i
    if (m == 1) {
        const int xc[5] = {x_code(XK_POW, 0, XS_DELTA), x_code(XK_POW, 1, XS_DELTA), x_code(XK_POW, 0, XS_PHI),
                           x_code(XK_POW, 1, XS_PHI), x_code(XK_POW, 2, XS_PHI)};
        const int yc[9] = {y_code(0, 0, 0), y_code(0, 1, 1), y_code(1, 0, 2), y_code(2, 0, 3), y_code(2, 1, 4),
                           y_code(2, 2, 5), y_code(3, 0, 6), y_code(3, 1, 7), y_code(4, 0, 8)};
        const int zc[13] = {z_code(0, 0, 0, 0), z_code(0, 1, I, 3), z_code(1, 0, I, 2), z_code(2, 0, I, 1),
                            z_code(3, 1, NI, 6), z_code(3, 2, 0, 9), z_code(4, 0, NI, 5), z_code(4, 1, 0, 12),
                            z_code(5, 0, 0, 8), z_code(6, 0, NI, 4), z_code(6, 1, 0, 11), z_code(7, 0, 0, 10),
                            z_code(8, 0, 0, 7)};
        xa.nout = 5;
        ya.nout = 9;
        za.nout = 13;
        for (int i = 0; i < 5; ++i) xa.codes[i] = xc[i];
        for (int i = 0; i < 9; ++i) ya.codes[i] = yc[i];
        for (int i = 0; i < 13; ++i) za.codes[i] = zc[i];
    } else {
        const int xc[7] = {x_code(XK_POW, 0, XS_DELTA), x_code(XK_POW, 1, XS_DELTA), x_code(XK_POW, 0, XS_THETA),
                           x_code(XK_POW, 1, XS_THETA), x_code(XK_POW, 0, XS_PHI), x_code(XK_POW, 1, XS_PHI),
                           x_code(XK_POW, 2, XS_PHI)};
        const int yc[12] = {y_code(0, 0, 0), y_code(0, 1, 1), y_code(1, 0, 2), y_code(2, 0, 3),
                            y_code(2, 1, 4), y_code(3, 0, 5), y_code(4, 0, 6), y_code(4, 1, 7),
                            y_code(4, 2, 8), y_code(5, 0, 9), y_code(5, 1, 10), y_code(6, 0, 11)};
        const int zc[17] = {z_code(0, 0, 0, 0), z_code(0, 1, I, 4), z_code(1, 0, I, 3), z_code(2, 0, I, 2),
                            z_code(3, 0, 0, 1), z_code(3, 1, I, 7), z_code(4, 0, I, 6), z_code(5, 0, I, 5),
                            z_code(6, 1, NI, 10), z_code(6, 2, 0, 13), z_code(7, 0, NI, 9), z_code(7, 1, 0, 16),
                            z_code(8, 0, 0, 12), z_code(9, 0, NI, 8), z_code(9, 1, 0, 15), z_code(10, 0, 0, 14),
                            z_code(11, 0, 0, 11)};
        xa.nout = 7;
        ya.nout = 12;
        za.nout = 17;
        for (int i = 0; i < 7; ++i) xa.codes[i] = xc[i];
        for (int i = 0; i < 12; ++i) ya.codes[i] = yc[i];
        for (int i = 0; i < 17; ++i) za.codes[i] = zc[i];
    }
}

// Recursion coefficients of order n times N^-3: (delta_n, theta_n) =
// c_n [(n + 1/2) A + B, 3/2 A + n B] / N^3 (Eq. recursion_formula).
void recursion_coefs(const gridspt_plan_s* p, int n, float* cdA, float* cdB, float* ctA, float* ctB) {
    const double inv_cells = 1.0 / (double)field_floats(p);
    const double c = 2.0 / ((2.0 * n + 3.0) * (n - 1.0));
    *cdA = (float)(c * (n + 0.5) * inv_cells);
    *cdB = (float)(c * inv_cells);
    *ctA = (float)(c * 1.5 * inv_cells);
    *ctB = (float)(c * n * inv_cells);
}

// Partner fields of produced slot s (order m >= 2, 17 slots) in the stored
// order j (13 slots for j = 1, where theta_1 = delta_1, else 17), with the
// coefficients of both ordered pairs (m, j) and (j, m) in A and B.
void pair_table(int j, PairTarget& T) {
    auto f = [&](int slot17) {   // stored field index of canonical slot
        if (j >= 2) return slot17;
        if (slot17 <= 1) return 0;                 // delta, theta
        if (slot17 <= 4) return 1 + (slot17 - 2);  // grad delta
        if (slot17 <= 7) return 1 + (slot17 - 5);  // grad theta = grad delta
        if (slot17 <= 10) return 4 + (slot17 - 8); // u
        return 7 + (slot17 - 11);                  // d_a u_b
    };
    for (int sl = 0; sl < 17; ++sl) {
        T.pcount[sl] = 0;
        auto add = [&](int slot17, float ca, float cb) {
            const int fi = f(slot17);
            for (int q = 0; q < T.pcount[sl]; ++q)
                if (T.pfield[sl][q] == fi) {   // aliased partner: merge coefficients
                    T.pcoef_a[sl][q] += ca;
                    T.pcoef_b[sl][q] += cb;
                    return;
                }
            T.pfield[sl][T.pcount[sl]] = fi;
            T.pcoef_a[sl][T.pcount[sl]] = ca;
            T.pcoef_b[sl][T.pcount[sl]] = cb;
            ++T.pcount[sl];
        };
        if (sl == 0) add(1, 1.f, 0.f);                       // delta_m theta_j
        else if (sl == 1) add(0, 1.f, 0.f);                  // delta_j theta_m
        else if (sl <= 4) add(8 + (sl - 2), 1.f, 0.f);       // grad delta_m . u_j
        else if (sl <= 7) add(8 + (sl - 5), 0.f, 1.f);       // u_j . grad theta_m
        else if (sl <= 10) {                                 // grad delta_j . u_m, u_m . grad theta_j
            add(2 + (sl - 8), 1.f, 0.f);
            add(5 + (sl - 8), 0.f, 1.f);
        } else if (sl <= 13) add(sl, 0.f, 2.f);              // diagonal d_a u_a, both orders
        else add(sl, 0.f, 4.f);                              // off-diagonal (symmetric) x both orders
    }
}

// The diagonal pair (1, 1) of order 2 (Eq. recursion_formula with m = n - m =
// 1) as a target of order 1's own z pass: every product of two order-1 fields
// is added when the later of the two is formed (the earlier one is read back
// from the rows this launch has just stored; a square uses the formed field
// itself, pfield -1). Order-1 stored fields: 0 delta (= theta), 1..3 grad delta
// (= grad theta), 4..6 u, 7..9 d_a u_a, 10..12 the off-diagonal d_a u_b.
// A = delta theta + grad delta . u, B = u . grad theta + sum_ab (d_a u_b)^2.
void diag1_table(const YZExpArgs& za, PairTarget& T) {
    int pos[17];
    for (int sl = 0; sl < 17; ++sl) pos[sl] = -1;
    for (int f = 0; f < za.nout; ++f) pos[za.codes[f] >> 16] = f;
    for (int sl = 0; sl < 17; ++sl) T.pcount[sl] = 0;
    auto term = [&](int a, int b, float ca, float cb) {
        const int late = pos[a] >= pos[b] ? a : b, early = late == a ? b : a;
        const int q = T.pcount[late]++;
        T.pfield[late][q] = a == b ? -1 : early;
        T.pcoef_a[late][q] = ca;
        T.pcoef_b[late][q] = cb;
    };
    term(0, 0, 1.f, 0.f);                                   // delta_1 theta_1
    for (int a = 0; a < 3; ++a) term(1 + a, 4 + a, 1.f, 1.f);  // grad delta . u and u . grad theta
    for (int t = 0; t < 3; ++t) term(7 + t, 7 + t, 0.f, 1.f);  // (d_a u_a)^2
    for (int t = 0; t < 3; ++t) term(10 + t, 10 + t, 0.f, 2.f);  // 2 (d_a u_b)^2, a < b
}

// z pass of order m fused with the pair products (m, j), j < m, m + j <= n_max,
// for the targets n' = m + j >= start. Stores the order's real fields when a
// later order needs them (2m <= n_max). More than two targets are split over
// several launches (the z expansion is then repeated).
gridspt_status zexp_pairs(const gridspt_plan_s* p, int m, const YZExpArgs& za, float* ws, int start,
                          const std::vector<float2*>& spec_delta, cudaStream_t s) {
    const int n_max = p->d.n_max;
    const long long cells = field_floats(p);
    const double fb = 4.0 * (double)cells;
    std::vector<int> js;
    for (int j = 1; j < m && m + j <= n_max; ++j)
        if (m + j >= start) js.push_back(j);
    const bool store = 2 * m <= n_max;
    size_t first = 0;
    do {
        ZPairArgs a{};
        a.z = za;
        a.cells = cells;
        a.store = (store && first == 0) ? ws + (long long)order_base(m) * cells : nullptr;
        a.ntargets = 0;
        const double fz = za.band > 0 ? (double)za.band / p->geo.M : 1.0;             // band-limited inputs
        double bytes = fb * za.nout * (a.store ? 1 : 0) + fb * fz * (m == 1 ? 9 : 12);   // stores + xy-field inputs
        // a launch holds at most kMaxPairTargets targets and kMaxPartners partner
        // fields per output over all its targets (order 1 supplies at most one
        // partner per output, higher orders two)
        int partners = 0;
        if (m == 1 && n_max >= 2 && start <= 2 && a.store) {   // the diagonal pair (1, 1): all of order 2
            PairTarget& T = a.t[a.ntargets++];
            T.partner = a.store;
            diag1_table(za, T);
            T.out_a = reinterpret_cast<float*>(spec_delta[2]);
            T.out_b = reinterpret_cast<float*>(spec_delta[2] + field_c(p));
            recursion_coefs(p, 2, &T.ca0, &T.ca1, &T.cb0, &T.cb1);
            partners = 1;
            bytes += fb * 2;   // delta_2, theta_2 written; the partners are this launch's own stores
        }
        for (size_t q = first; q < js.size() && a.ntargets < kMaxPairTargets; ++q, ++first) {
            const int j = js[q], n = m + j;
            if (partners + (j == 1 ? 1 : 2) > kMaxPartners) break;
            partners += j == 1 ? 1 : 2;
            PairTarget& T = a.t[a.ntargets++];
            T.partner = ws + (long long)order_base(j) * cells;
            pair_table(j, T);
            // the first contribution to target n comes from order ceil(n / 2)
            // (the diagonal pair for even n), every later one reads the partial sums
            const int first_m = (n + 1) / 2;
            float* acc = ws + (long long)(acc_base(n_max) + 2 * (n - 4)) * cells;
            if (first_m < m) {
                T.acc_in_a = acc;
                T.acc_in_b = acc + cells;
            }
            if (j == 1) {   // last pair of target n: write delta_n, theta_n
                T.out_a = reinterpret_cast<float*>(spec_delta[n]);
                T.out_b = reinterpret_cast<float*>(spec_delta[n] + field_c(p));
                recursion_coefs(p, n, &T.ca0, &T.ca1, &T.cb0, &T.cb1);
            } else {
                T.out_a = acc;
                T.out_b = acc + cells;
                T.ca0 = 1.f;
                T.ca1 = 0.f;
                T.cb0 = 0.f;
                T.cb1 = 1.f;
            }
            bytes += fb * (j == 1 ? 13 : 17) + fb * 2 + (T.acc_in_a ? fb * 2 : 0);
        }
        for (int sl = 0; sl < 17; ++sl) {   // the kernels stage at most kMaxPartners partner tiles
            int c = 0;
            for (int t = 0; t < a.ntargets; ++t)
                for (int q = 0; q < a.t[t].pcount[sl]; ++q) c += a.t[t].pfield[sl][q] >= 0 ? 1 : 0;
            if (c > kMaxPartners) return fail(GRIDSPT_E_INVALID, "internal: %d partner fields for one output", c);
        }
        if (!a.store && a.ntargets == 0) break;
        if (a.ntargets == 0) {   // store only: the plain z expansion
            YZExpArgs zs = za;
            zs.out = reinterpret_cast<float2*>(a.store);
            ZPairArgs zq{};
            zq.z = zs;
            zq.cells = cells;
            CKQ(PK_ZEXP, bytes, s, launch_zexp(p->geo, zs, s), "z expansion",
                [&]() { QStage q = q_stage(p->geo, Q_Z, bytes); q.z = zq; return q; }());
            break;
        }
        CKQ(PK_ZEXP, bytes, s, launch_zexp_pairs(p->geo, a, s), "z expansion and pair products",
            [&]() { QStage q = q_stage(p->geo, Q_Z, bytes); q.z = a; return q; }());
    } while (first < js.size());
    return GRIDSPT_OK;
}

// Order 1 from delta_1, whose modes above the linear cut (|s|^2 > s2_lin, Sec.
// II.C step (1)) are zero: the x pass applies that cut to its input and moves
// only the columns with |ky|, kz < band; the y pass forms only kz < band
// columns; the z pass reads only kz < band. band = floor(sqrt(s2_lin)) + 1
// bounds every component of an in-band wavevector. The skipped columns hold
// zeros in the full computation, so the fields are the same.
void set_band(const gridspt_plan_s* p, int band, XExpArgs& xa, YZExpArgs& ya, YZExpArgs& za, double* fx,
              double* fy_in, double* fy_out) {
    band += band & 1;                    // even: the z pass copies rows in kz pairs
    if (band >= p->geo.M) return;
    const double N = p->geo.N, M = p->geo.M;
    xa.band = ya.band = za.band = band;
    *fx = (2.0 * band - 1.0) * band / (N * M);
    *fy_in = (2.0 * band - 1.0) / N * band / M;
    *fy_out = band / M;
}

void order1_band(const gridspt_plan_s* p, XExpArgs& xa, YZExpArgs& ya, YZExpArgs& za, double* fx, double* fy_in,
                 double* fy_out) {
    xa.s2_in = p->s2_lin;
    set_band(p, (int)std::floor(std::sqrt((double)p->s2_lin)) + 1, xa, ya, za, fx, fy_in, fy_out);
}

// Cut on an order m >= 2 formed in this call (< 0: none): the higher-order cut
// s2_nl and, with truncate, |s| <= min(m, n_max + 1 - m) K_c / k_F, all that
// the orders above m use of it for their modes below K_c.
long long order_cut(const gridspt_plan_s* p, int m) {
    long long c = p->s2_nl;
    if (p->d.truncate) {
        const double rt = std::min(m, p->d.n_max + 1 - m) * p->r_lin;
        const long long t = (long long)std::floor(rt * rt);
        c = c < 0 ? t : std::min(c, t);
    }
    return c;
}

// Band of an order m >= 2 formed in this call (0: none). Every component of
// an order-1 mode is at most c1 = floor(sqrt(s2_lin)); a product of fields of
// orders a + b = m then has components at most m c1, and while m c1 < N/2 no
// product of the recursion up to order m wraps around the grid, so
// delta_m(k), theta_m(k) vanish at every mode with a component |s_a| > m c1.
// That holds when every lower order was formed here too (start == 2); stored
// lower orders are not assumed band limited. With a cut on order m
// (order_cut >= 0: the higher-order cut, or truncate) the finalising pass
// zeroes every |s|^2 above it, which bounds the components by the cut's
// floor(sqrt) whatever the products did.
int order_band(const gridspt_plan_s* p, int m, int start) {
    const long long c1 = (long long)std::floor(std::sqrt((double)p->s2_lin));
    long long c = (start == 2 && 2 * m * c1 < p->geo.N) ? m * c1 : -1;
    const long long cut = order_cut(p, m);
    if (cut >= 0) {
        const long long cn = (long long)std::floor(std::sqrt((double)cut));
        c = c < 0 ? cn : std::min(c, cn);
    }
    return c < 0 ? 0 : (int)(c + 1);
}

// Derived fields of order m from its spectra (Sec. II.C steps (2)/(5)),
// written to ws at the order's slot, through the factorised x, y and z
// expansion passes. With fwd, the spectra buffers hold the y-transformed
// product output and the x pass first completes the forward transform
// (writing delta_m(k), theta_m(k) in place).
//
// Order m >= 2, 17 real fields in slot order [delta, theta, d delta (3),
// d theta (3), u (3), d_a u_b (xx, yy, zz, xy, xz, yz)], phi = theta / k^2:
//   x-fields: X0 delta, X1 kx delta, X2 theta, X3 kx theta, X4 phi, X5 kx phi, X6 kx^2 phi
//   xy-fields: Y0 X0, Y1 ky X0, Y2 X1, Y3 X2, Y4 ky X2, Y5 X3, Y6 X4, Y7 ky X4, Y8 ky^2 X4,
//              Y9 X5, Y10 ky X5, Y11 X6
//   real: delta = Y0, d_z delta = i kz Y0, d_y delta = i Y1, d_x delta = i Y2, theta = Y3,
//         d_z theta = i kz Y3, d_y theta = i Y4, d_x theta = i Y5, u_z = -i kz Y6,
//         d_z u_z = kz^2 Y6, u_y = -i Y7, d_y u_z = kz Y7, d_y u_y = Y8, u_x = -i Y9,
//         d_x u_z = kz Y9, d_x u_y = Y10, d_x u_x = Y11.
// Order 1 (theta = delta), 13 fields [delta, d delta (3), u (3), d_a u_b (6)]:
//   x-fields: X0 delta, X1 kx delta, X2 phi, X3 kx phi, X4 kx^2 phi
//   xy-fields: Y0 X0, Y1 ky X0, Y2 X1, Y3 X2, Y4 ky X2, Y5 ky^2 X2, Y6 X3, Y7 ky X3, Y8 X4
gridspt_status derive_order(const gridspt_plan_s* p, int m, float2* dk, float2* tk, float* ws, bool fwd,
                            int start, const std::vector<float2*>& spec_delta, cudaStream_t s) {
    const long long F = field_c(p);
    const double fb = 4.0 * (double)field_floats(p);  // bytes of one field
    float2* xs = reinterpret_cast<float2*>(ws + (long long)scratch_base(p->d.n_max) * field_floats(p));
    float2* ys = xs + 7 * F;
    XExpArgs xa{};
    xa.src0 = dk;
    xa.src1 = tk;
    xa.out = xs;
    xa.out_stride = F;
    xa.fwd_first = fwd ? 1 : 0;
    xa.zero_k0 = fwd ? 1 : 0;   // order m >= 2 formed here: its k = 0 mode is exactly zero
    xa.s2_nl = m >= 2 ? order_cut(p, m) : p->s2_nl;
    YZExpArgs ya{}, za{};
    ya.in = xs;
    ya.in_stride = F;
    ya.out = ys;
    ya.out_stride = F;
    za.in = ys;
    za.in_stride = F;
    za.out = nullptr;
    za.out_stride = F;
    expansion_codes(m, xa, ya, za);
    xa.s2_in = -1;
    const int nin = m == 1 ? 1 : 2;
    double fx = 1.0, fy_in = 1.0, fy_out = 1.0;
    if (m == 1) order1_band(p, xa, ya, za, &fx, &fy_in, &fy_out);
    else if (fwd) {
        if (const int band = order_band(p, m, start)) set_band(p, band, xa, ya, za, &fx, &fy_in, &fy_out);
    }
    const double xbytes = fb * fx * (fwd ? 2 * nin + xa.nout : nin + xa.nout);
    CKQ(fwd ? PK_XEXP_FWD : PK_XEXP, xbytes, s, launch_xexp(p->geo, xa, s), "x expansion",
        [&]() { QStage q = q_stage(p->geo, fwd ? Q_XEXP1 : Q_XEXP0, xbytes); q.x = xa; return q; }());
    if (m >= 2 && xa.band > 0 && fwd)   // the spectra outside the band columns: zeros
        CKQ(PK_XEXP_FWD, fb * 2.0 * (1.0 - fx), s, launch_zero_outside_band(dk, tk, p->geo.N, xa.band, s),
            "zeros outside the band", [&]() {
                QStage q = q_stage(p->geo, Q_ZEROBAND, fb * 2.0 * (1.0 - fx));
                q.data = dk;
                q.data2 = tk;
                q.band = xa.band;
                return q;
            }());
    const double ybytes = fb * (fy_in * xa.nout + fy_out * ya.nout);
    CKQ(PK_YEXP, ybytes, s, launch_yexp(p->geo, ya, s), "y expansion",
        [&]() { QStage q = q_stage(p->geo, Q_YEXP, ybytes); q.y = ya; return q; }());
    return zexp_pairs(p, m, za, ws, start, spec_delta, s);
}

// Backward transform of `count` fields in place (or in -> out): x, y, z passes
// with one output per input, optionally with a shell mask (bispectrum).
gridspt_status backward_fields(const gridspt_plan_s* p, const float2* in0, const float2* in1, float2* out,
                               long long out_stride, int count, bool shell, long long lo, long long hi,
                               int band, bool skip_z, cudaStream_t s) {
    const double fb = 4.0 * (double)field_floats(p);
    XExpArgs xa{};
    xa.src0 = const_cast<float2*>(in0);
    xa.src1 = const_cast<float2*>(in1);
    xa.out = out;
    xa.out_stride = out_stride;
    xa.s2_nl = -1;
    xa.shell_lo = lo;
    xa.shell_hi = hi;
    xa.band = band;
    xa.nout = count;
    const int srcs[3] = {XS_DELTA, in1 == in0 ? XS_DELTA : XS_THETA, XS_ONE};
    for (int f = 0; f < count; ++f) xa.codes[f] = x_code(shell ? XK_SHELL : XK_POW, 0, srcs[f]);
    YZExpArgs ya{};
    ya.in = out;
    ya.in_stride = out_stride;
    ya.out = out;
    ya.out_stride = out_stride;
    ya.nout = count;
    ya.band = band;
    for (int f = 0; f < count; ++f) ya.codes[f] = y_code(f, 0, f);
    YZExpArgs za = ya;
    za.band = 0;
    for (int f = 0; f < count; ++f) za.codes[f] = z_code(f, 0, 0, f);
    const int nin = in1 == in0 ? 1 : 2;
    // algorithmic bytes: with a band B only the band columns move
    const double N = p->geo.N, M = p->geo.M;
    const double fx = band > 0 ? (2.0 * band - 1.0) * band / (N * M) : 1.0;   // x columns
    const double fy_in = band > 0 ? (2.0 * band - 1.0) / N * band / M : 1.0;   // y inputs
    const double fy_out = band > 0 ? band / M : 1.0;                         // y outputs
    CKP(shell ? PK_BX : PK_XEXP, fb * fx * (nin + count), s, launch_xexp(p->geo, xa, s), "x pass");
    CKP(shell ? PK_BY : PK_YEXP, fb * count * (fy_in + fy_out), s, launch_yexp(p->geo, ya, s), "y pass");
    if (!skip_z) CKP(shell ? PK_BZ : PK_ZEXP, 2 * fb * count, s, launch_zexp(p->geo, za, s), "z pass");
    return GRIDSPT_OK;
}

}  // namespace

}  // extern "C"

namespace {

// Divergence form, one order m: the x pass (forward from the sources V, S when
// `src` is set, writing delta_m(k), theta_m(k); else backward from the given
// spectra) makes the x-fields delta, phi, kx phi (phi = theta / k^2); the y pass
// the xy-fields delta, ky phi, phi, kx phi; the z pass stores delta and
// u = -i k phi (Eq. u_and_theta) as real fields of order m. At m = n_max only
// the forward x pass runs.
gridspt_status derive_order_div(const gridspt_plan_s* p, int m, float2* dk, float2* tk, float* ws, const float2* src,
                                cudaStream_t s) {
    const long long F = field_c(p), cells = field_floats(p);
    const double fb = 4.0 * (double)cells;
    const int n_max = p->d.n_max;
    float2* xs = reinterpret_cast<float2*>(ws + (long long)div_scratch_base(n_max) * cells);
    float2* ys = xs + 3 * F;
    XExpArgs xa{};
    xa.src0 = dk;
    xa.src1 = tk;
    xa.out = xs;
    xa.out_stride = F;
    xa.s2_nl = p->s2_nl;
    if (src) {
        const double c = 2.0 / ((2.0 * m + 3.0) * (m - 1.0));   // Eq. recursion_formula (N^-3 is in the sources)
        xa.fwd_first = 1;
        xa.div_in = src;
        xa.div_stride = F;
        xa.cdA = (float)(c * (m + 0.5));
        xa.cdB = (float)c;
        xa.ctA = (float)(c * 1.5);
        xa.ctB = (float)(c * m);
    }
    if (m < n_max) {
        xa.nout = 3;
        xa.codes[0] = x_code(XK_POW, 0, XS_DELTA);
        xa.codes[1] = x_code(XK_POW, 0, XS_PHI);
        xa.codes[2] = x_code(XK_POW, 1, XS_PHI);
    }
    xa.s2_in = -1;
    YZExpArgs ya{}, za{};
    double fx = 1.0, fy_in = 1.0, fy_out = 1.0;
    if (m == 1) order1_band(p, xa, ya, za, &fx, &fy_in, &fy_out);
    const int nin = src ? 4 : (m == 1 ? 1 : 2);
    CKP(src ? (m < n_max ? PK_XEXP_FWD : PK_X_FWD) : PK_XEXP, fb * fx * (nin + (src ? 2 : 0) + xa.nout), s,
        launch_xexp(p->geo, xa, s), "x pass (divergence form)");
    if (m == n_max) return GRIDSPT_OK;
    ya.in = xs;
    ya.in_stride = F;
    ya.out = ys;
    ya.out_stride = F;
    ya.nout = 4;
    ya.codes[0] = y_code(0, 0, 0);   // delta
    ya.codes[1] = y_code(1, 1, 1);   // ky phi
    ya.codes[2] = y_code(1, 0, 2);   // phi
    ya.codes[3] = y_code(2, 0, 3);   // kx phi
    const int NI = 2;                // z-pass constant -i
    za.in = ys;
    za.in_stride = F;
    za.out = reinterpret_cast<float2*>(ws + (long long)div_order_base(m) * cells);
    za.out_stride = F;
    za.nout = 4;
    za.codes[0] = z_code(0, 0, 0, 0);    // delta
    za.codes[1] = z_code(3, 0, NI, 1);   // u_x = -i kx phi
    za.codes[2] = z_code(1, 0, NI, 2);   // u_y = -i ky phi
    za.codes[3] = z_code(2, 1, NI, 3);   // u_z = -i kz phi
    const double fz = za.band > 0 ? (double)za.band / p->geo.M : 1.0;
    CKP(PK_YEXP, fb * (3 * fy_in + 4 * fy_out), s, launch_yexp(p->geo, ya, s), "y expansion (divergence form)");
    CKP(PK_ZEXP, fb * (4 * fz + 4), s, launch_zexp(p->geo, za, s), "z expansion (divergence form)");
    return GRIDSPT_OK;
}

// Orders 1..n_max of one realisation in divergence form (see derive_order_div).
gridspt_status run_orders_div(const gridspt_plan_s* p, float2* d1, const std::function<float2*(int, int)>& spec,
                              int start_order, float* w, cudaStream_t s) {
    const int n_max = p->d.n_max;
    const long long F = field_c(p), cells = field_floats(p);
    const double fb = 4.0 * (double)cells;
    float2* src = reinterpret_cast<float2*>(w + (long long)div_src_base(n_max) * cells);
    for (int m = 1; m <= n_max; ++m) {
        const bool given = m == 1 || m < start_order;
        float2* dk = m == 1 ? d1 : spec(m, 0);
        float2* tk = m == 1 ? d1 : spec(m, 1);
        if (!given) {
            ProductDivArgs pa{};
            pa.ws = w;
            pa.cells = cells;   // order q's fields at div_order_base(q) = 4 (q - 1)
            pa.n = m;
            pa.out = reinterpret_cast<float*>(src);
            pa.scale = (float)(1.0 / (double)cells);
            CKP(PK_PRODUCT, fb * 4.0 * m, s, launch_product_div(p->geo, pa, s), "divergence-form sources");
            CKP(PK_ZR2C, 8 * fb, s, launch_zr2c(p->geo, src, src, F, 4, 1.0f, 0, s), "z r2c (divergence form)");
            CKP(PK_Y_FWD, 8 * fb, s, launch_colpass_fwd(p->geo, src, F, 4, 1, 0, -1, 0, s),
                "y pass fwd (divergence form)");
        } else if (m == n_max) {
            break;
        }
        if (gridspt_status st = derive_order_div(p, m, dk, tk, w, given ? nullptr : src, s)) return st;
    }
    return GRIDSPT_OK;
}

gridspt_status run_orders_impl(gridspt_plan p, const void* delta1_k, int32_t start_order, void* spectra,
                               void* ws, size_t ws_bytes, gridspt_stream stream) {
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    const int n_max = p->d.n_max;
    if (!delta1_k || (!spectra && n_max >= 2)) return fail(GRIDSPT_E_INVALID, "NULL argument");
    if (!aligned16(delta1_k) || !aligned16(spectra) || !aligned16(ws))
        return fail(GRIDSPT_E_INVALID, "pointers must be 16-byte aligned");
    if (n_max < 2) return GRIDSPT_OK;
    if (start_order < 2 || start_order > n_max) return fail(GRIDSPT_E_INVALID, "start_order=%d outside [2, %d]", start_order, n_max);
    size_t need = 0;
    gridspt_workspace_size(p, &need);
    if (!ws || ws_bytes < need) return fail(GRIDSPT_E_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (gridspt_status st = set_device(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const long long F = field_c(p);
    float* w = static_cast<float*>(ws);
    for (int b = 0; b < p->d.batch; ++b) {
        float2* d1 = const_cast<float2*>(static_cast<const float2*>(delta1_k)) + (long long)b * F;
        auto spec = [&](int n, int which) {
            return static_cast<float2*>(spectra) + ((long long)(b * (n_max - 1) + (n - 2)) * 2 + which) * F;
        };
        if (p->d.form == GRIDSPT_FORM_DIVERGENCE) {
            if (gridspt_status st = run_orders_div(p, d1, spec, start_order, w, s)) return st;
            continue;
        }
        std::vector<float2*> spec_delta(n_max + 1, nullptr);
        for (int n = 2; n <= n_max; ++n) spec_delta[n] = spec(n, 0);
        const double fb = 4.0 * (double)field_floats(p);
        // Orders m = 1..n_max. Below start_order the spectra are given; from there
        // on delta_m, theta_m arrive as real fields from the pair products of
        // the lower orders and are transformed forward first.
        for (int m = 1; m <= n_max; ++m) {
            const bool given = m == 1 || m < start_order;
            float2* dk = m == 1 ? d1 : spec(m, 0);
            float2* tk = m == 1 ? d1 : spec(m, 1);
            if (!given) {
                auto col = [&](int kind) {
                    QStage q = q_stage(p->geo, kind, 4 * fb);
                    q.data = dk;
                    q.fstride = F;
                    q.count = 2;
                    q.scale = 1.0f;
                    q.s2 = order_cut(p, m);
                    q.zero_k0 = 1;
                    return q;
                };
                // A band-limited order below n_max: its x pass reads only the band
                // columns (|ky|, kz < band) and its spectra are zeroed outside them
                // after it, so the z pass writes only kz < band and the y pass
                // transforms only those columns and writes only their band rows.
                int fband = 0;
                if (m < n_max) {
                    const int b = order_band(p, m, start_order);
                    if (b > 0 && b + (b & 1) < p->geo.M) fband = b + (b & 1);
                }
                const double fo = fband ? (double)fband / p->geo.M : 1.0;
                const double fr = fband ? (2.0 * fband - 1.0) / p->geo.N : 1.0;
                CKQ(PK_ZR2C, (2 + 2 * fo) * fb, s, launch_zr2c(p->geo, dk, dk, F, 2, 1.0f, fband, s), "z r2c",
                    col(Q_ZR2C));
                CKQ(PK_Y_FWD, 2 * fo * (1 + fr) * fb, s, launch_colpass_fwd(p->geo, dk, F, 2, 1, 0, -1, fband, s),
                    "y pass fwd", col(Q_COLY));
                if (m == n_max) {
                    CKQ(PK_X_FWD, 4 * fb, s, launch_colpass_fwd(p->geo, dk, F, 2, 0, 2, order_cut(p, m), 0, s),
                        "x pass fwd", col(Q_COLX));
                    break;
                }
            }
            if (m == n_max) break;
            if (gridspt_status st = derive_order(p, m, dk, tk, w, !given, start_order, spec_delta, s)) return st;
            if (m >= 2 && 2 * m <= n_max && 2 * m >= start_order) {   // diagonal pair (m, m) of order 2m
                // ((1, 1) is a target of order 1's z pass)
                ProductArgs pa{};
                pa.ws = w;
                pa.cells = field_floats(p);
                for (int q = 1; q <= kMaxOrder; ++q) pa.base[q] = order_base(q);
                pa.n = 2 * m;
                pa.diag_only = m;
                if (2 * m == 2) {   // order 2 has no other pair: write delta_2, theta_2
                    pa.out_delta = reinterpret_cast<float*>(spec(2, 0));
                    pa.out_theta = reinterpret_cast<float*>(spec(2, 1));
                    recursion_coefs(p, 2, &pa.cdA, &pa.cdB, &pa.ctA, &pa.ctB);
                } else {            // first (partial) contribution to order 2m
                    float* acc = w + (long long)(acc_base(n_max) + 2 * (2 * m - 4)) * field_floats(p);
                    pa.out_delta = acc;
                    pa.out_theta = acc + field_floats(p);
                    pa.cdA = 1.f;
                    pa.cdB = 0.f;
                    pa.ctA = 0.f;
                    pa.ctB = 1.f;
                }
                CKQ(PK_PRODUCT, fb * (m == 1 ? 13 + 2 : 17 + 2), s, launch_product(p->geo, pa, s), "diagonal pair",
                    [&]() { QStage q = q_stage(p->geo, Q_PRODUCT, fb * (m == 1 ? 13 + 2 : 17 + 2)); q.pr = pa; return q; }());
            }
        }
    }
    return GRIDSPT_OK;
}

}  // namespace

extern "C" {

gridspt_status gridspt_run_orders(gridspt_plan p, const void* delta1_k, int32_t start_order, void* spectra,
                                  void* ws, size_t ws_bytes, gridspt_stream stream) {
    g_err[0] = 0;
    return run_orders_impl(p, delta1_k, start_order, spectra, ws, ws_bytes, stream);
}

// ------------------------------------------------------------ batch graphs
}  // extern "C"

struct gridspt_batch_s {
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

gridspt_status gridspt_batch_create(const gridspt_plan* plans, int32_t count, const void* const* delta1_k,
                                    const int32_t* start_order, void* const* spectra, void* const* ws,
                                    const size_t* ws_bytes, gridspt_batch* out) {
    g_err[0] = 0;
    if (!plans || count < 1 || !delta1_k || !start_order || !spectra || !ws || !ws_bytes || !out)
        return fail(GRIDSPT_E_INVALID, "NULL argument or count < 1");
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return fail(GRIDSPT_E_INVALID, "plans[%d] is NULL", i);
        for (int j = 0; j < i; ++j)
            if (ws[j] && ws[j] == ws[i]) return fail(GRIDSPT_E_INVALID, "branches %d and %d share a workspace", j, i);
    }
    std::vector<cudaStream_t> st(count + 1, nullptr);
    std::vector<cudaEvent_t> ev(count + 1, nullptr);
    cudaGraph_t graph = nullptr;
    gridspt_status res = GRIDSPT_OK;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        for (auto x : ev) if (x) cudaEventDestroy(x);
        for (auto x : st) if (x) cudaStreamDestroy(x);
        if (graph) cudaGraphDestroy(graph);
    };
    for (int i = 0; i <= count && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "batch streams");
    }
    e = cudaStreamBeginCapture(st[0], cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "begin capture");
    }
    t_capturing = true;
    e = cudaEventRecord(ev[0], st[0]);   // fork
    for (int i = 0; i < count && e == cudaSuccess && res == GRIDSPT_OK; ++i) {
        e = cudaStreamWaitEvent(st[i + 1], ev[0], 0);
        if (e != cudaSuccess) break;
        res = run_orders_impl(plans[i], delta1_k[i], start_order[i], spectra[i], ws[i], ws_bytes[i],
                              (gridspt_stream)st[i + 1]);
        if (res != GRIDSPT_OK) break;
        e = cudaEventRecord(ev[i + 1], st[i + 1]);   // join
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st[0], ev[i + 1], 0);
    }
    t_capturing = false;
    cudaError_t e2 = cudaStreamEndCapture(st[0], &graph);
    if (res != GRIDSPT_OK) {
        cleanup();
        return res;
    }
    if (e == cudaSuccess) e = e2;
    gridspt_batch b = nullptr;
    if (e == cudaSuccess) {
        b = new (std::nothrow) gridspt_batch_s();
        if (!b) {
            cleanup();
            return fail(GRIDSPT_E_NOMEM, "host allocation failed");
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
    }
    cleanup();
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "batch capture");
    }
    *out = b;
    return GRIDSPT_OK;
}

gridspt_status gridspt_batch_launch(gridspt_batch b, gridspt_stream stream) {
    g_err[0] = 0;
    if (!b || !b->exec) return fail(GRIDSPT_E_INVALID, "batch is NULL");
    CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "graph launch");
    return GRIDSPT_OK;
}

gridspt_status gridspt_batch_destroy(gridspt_batch b) {
    if (!b) return GRIDSPT_OK;
    cudaError_t e = b->exec ? cudaGraphExecDestroy(b->exec) : cudaSuccess;
    delete b;
    if (e != cudaSuccess) return cuda_fail(e, "batch destroy");
    return GRIDSPT_OK;
}

// ------------------------------------------------------- persistent queue
}  // extern "C"

struct gridspt_multi_s {
    void* dev = nullptr;         // stages, then first tickets, then the queue header
    QStage* stages = nullptr;
    long long* starts = nullptr;
    int* hdr = nullptr;
    int nst = 0;
    long long total = 0;
    int* status = nullptr;       // status word of plans[0]
    int device = 0;
};

namespace {
constexpr long long kQueueWaitNs = 1000000000LL;   // a tile gives up waiting after 1 s
}

extern "C" {

gridspt_status gridspt_multi_create(const gridspt_plan* plans, int32_t count, const void* const* delta1_k,
                                    const int32_t* start_order, void* const* spectra, void* const* ws,
                                    const size_t* ws_bytes, gridspt_multi* out) {
    g_err[0] = 0;
    if (!plans || count < 1 || !delta1_k || !spectra || !ws || !ws_bytes || !out)
        return fail(GRIDSPT_E_INVALID, "NULL argument or count < 1");
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        const gridspt_plan_s* p = plans[i];
        if (!p) return fail(GRIDSPT_E_INVALID, "plans[%d] is NULL", i);
        if (p->d.form != GRIDSPT_FORM_NINE_TERM)
            return fail(GRIDSPT_E_UNSUPPORTED, "plans[%d]: the work queue runs the nine-term form only", i);
        if (!queue_supported_n(p->geo.N))
            return fail(GRIDSPT_E_UNSUPPORTED, "plans[%d]: N=%d; the work queue supports N = 64, 96, 128, 192, 256",
                        i, p->geo.N);
        if (p->device != plans[0]->device) return fail(GRIDSPT_E_INVALID, "plans on different devices");
        for (int j = 0; j < i; ++j)
            if (ws[j] && ws[j] == ws[i]) return fail(GRIDSPT_E_INVALID, "plans %d and %d share a workspace", j, i);
    }
    // record every launch of each plan's run_orders as a stage (its chain)
    std::vector<std::vector<QStage>> chains(count);
    for (int i = 0; i < count; ++i) {
        t_queue = &chains[i];
        const gridspt_status st = run_orders_impl(plans[i], delta1_k[i], start_order ? start_order[i] : 2,
                                                  spectra[i], ws[i], ws_bytes[i], nullptr);
        t_queue = nullptr;
        if (st != GRIDSPT_OK) return st;
    }
    // z passes of N = 3 * 2^a with two pair targets become two stages of one
    // target each (the z expansion is repeated; each target's sums are those
    // of the two-target pass, term by term)
    for (auto& ch : chains) {
        std::vector<QStage> out;
        for (const QStage& st : ch) {
            if (st.kind == Q_Z && st.z.ntargets == 2 && st.N % 3 == 0) {
                QStage a = st, b = st;
                a.z.ntargets = 1;
                b.z.ntargets = 1;
                b.z.t[0] = st.z.t[1];
                b.z.store = nullptr;
                out.push_back(a);
                out.push_back(b);
            } else {
                out.push_back(st);
            }
        }
        ch.swap(out);
    }
    // interleave the chains by cumulative work: the next stage comes from the
    // chain that has been given the least work so far
    std::vector<QStage> q;
    std::vector<size_t> pos(count, 0);
    std::vector<int> last(count, -1);
    std::vector<double> cum(count, 0.0);
    for (;;) {
        int best = -1;
        for (int i = 0; i < count; ++i)
            if (pos[i] < chains[i].size() && (best < 0 || cum[i] < cum[best])) best = i;
        if (best < 0) break;
        QStage s = chains[best][pos[best]++];
        s.dep = last[best];
        last[best] = (int)q.size();
        cum[best] += s.cost > 0 ? s.cost : 1.0;
        q.push_back(s);
    }
    const int nst = (int)q.size();
    // tiles per ticket: about four tickets per resident block in a stage's
    // share of the GPU, at most 8 tiles (fewer atomics and waits per tile,
    // small enough that a stage's last tickets do not leave the GPU idle)
    int sms = 1;
    if (gridspt_status st = set_device(plans[0])) return st;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plans[0]->device), "SM count");
    const long long blocks = 2LL * sms;
    std::vector<long long> starts(nst + 1, 0);
    for (int i = 0; i < nst; ++i) {
        q[i].chunk = std::max<long long>(1, std::min<long long>(8, q[i].ntiles / (8 * blocks)));
        q[i].nticks = (q[i].ntiles + q[i].chunk - 1) / q[i].chunk;
        q[i].tile0 = starts[i];
        starts[i + 1] = starts[i] + q[i].nticks;
    }
    if (fault_inject("queue_stall") && nst > 1) q[nst / 2].nosignal = 1;
    gridspt_multi m = new (std::nothrow) gridspt_multi_s();
    if (!m) return fail(GRIDSPT_E_NOMEM, "host allocation failed");
    m->nst = nst;
    m->total = starts[nst];
    m->status = plans[0]->status;
    m->device = plans[0]->device;
    const size_t b_st = align256(sizeof(QStage) * (size_t)nst);
    const size_t b_so = align256(sizeof(long long) * (size_t)(nst + 1));
    const size_t b_hd = align256(sizeof(int) * (size_t)(4 + nst));
    if (gridspt_status st = set_device(plans[0])) { delete m; return st; }
    cudaError_t e = cudaMalloc(&m->dev, b_st + b_so + b_hd);
    if (e != cudaSuccess) {
        delete m;
        return fail(GRIDSPT_E_NOMEM, "work queue: %s", cudaGetErrorString(e));
    }
    char* base = static_cast<char*>(m->dev);
    m->stages = reinterpret_cast<QStage*>(base);
    m->starts = reinterpret_cast<long long*>(base + b_st);
    m->hdr = reinterpret_cast<int*>(base + b_st + b_so);
    e = cudaMemcpy(m->stages, q.data(), sizeof(QStage) * (size_t)nst, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->starts, starts.data(), sizeof(long long) * (size_t)(nst + 1),
                                         cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->dev);
        delete m;
        return cuda_fail(e, "work queue upload");
    }
    *out = m;
    return GRIDSPT_OK;
}

gridspt_status gridspt_run_orders_multi(gridspt_multi m, gridspt_stream stream) {
    g_err[0] = 0;
    if (!m || !m->dev) return fail(GRIDSPT_E_INVALID, "multi is NULL");
    int cur = -1;
    CK(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != m->device) CK(cudaSetDevice(m->device), "cudaSetDevice");
    double bytes = 0.0;
    if (g_prof.on) {   // the algorithmic bytes of every stage, counted once per launch
        static thread_local std::vector<QStage> host;
        host.resize((size_t)m->nst);
        CK(cudaMemcpy(host.data(), m->stages, sizeof(QStage) * (size_t)m->nst, cudaMemcpyDeviceToHost),
           "work queue read-back");
        for (const QStage& q : host) bytes += q.cost;
    }
    CKP(PK_QUEUE, bytes, (cudaStream_t)stream,
        launch_queue(m->stages, m->starts, m->nst, m->total, m->hdr, m->status, kQueueWaitNs, (cudaStream_t)stream),
        "work-queue launch");
    return GRIDSPT_OK;
}

gridspt_status gridspt_multi_destroy(gridspt_multi m) {
    if (!m) return GRIDSPT_OK;
    cudaError_t e = cudaSuccess;
    if (m->dev) {
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(m->device);
        e = cudaDeviceSynchronize();
        cudaError_t e2 = cudaFree(m->dev);
        if (e == cudaSuccess) e = e2;
        if (cur >= 0) cudaSetDevice(cur);
    }
    delete m;
    if (e != cudaSuccess) return cuda_fail(e, "multi destroy");
    return GRIDSPT_OK;
}

// ------------------------------------------------------------- autotuner
gridspt_status gridspt_autotune_scratch_size(gridspt_plan p, size_t* bytes) {
    if (check_plan(p) || !bytes) return fail(GRIDSPT_E_INVALID, "plan/bytes is NULL");
    *bytes = 29 * (size_t)field_floats(p) * sizeof(float);   // 2 spectra + 7 + 12 + 17 expansion fields (overlapping)
    return GRIDSPT_OK;
}

gridspt_status gridspt_set_tuning(gridspt_plan p, const int32_t* choices) {
    g_err[0] = 0;
    if (check_plan(p) || !choices) return fail(GRIDSPT_E_INVALID, "plan/choices is NULL");
    for (int i = 0; i < TV_COUNT; ++i)
        if (choices[i] < 0 || choices[i] >= kTuneVariants[i])
            return fail(GRIDSPT_E_INVALID, "choice %d must be in [0, %d)", i, kTuneVariants[i]);
    for (int i = 0; i < TV_COUNT; ++i) p->geo.var[i] = choices[i];
    return GRIDSPT_OK;
}

gridspt_status gridspt_get_tuning(gridspt_plan p, int32_t* choices) {
    if (check_plan(p) || !choices) return fail(GRIDSPT_E_INVALID, "plan/choices is NULL");
    for (int i = 0; i < TV_COUNT; ++i) choices[i] = p->geo.var[i];
    return GRIDSPT_OK;
}

gridspt_status gridspt_autotune(gridspt_plan p, void* scratch, size_t scratch_bytes, int32_t* choices_out,
                                gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    size_t need = 0;
    gridspt_autotune_scratch_size(p, &need);
    if (!scratch || scratch_bytes < need || !aligned16(scratch))
        return fail(GRIDSPT_E_INVALID, "scratch must be 16-byte aligned and >= %zu bytes", need);
    if (gridspt_status st = set_device(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const long long F = field_c(p);
    float2* f0 = static_cast<float2*>(scratch);
    CK(cudaMemsetAsync(scratch, 0, need, s), "scratch clear");
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a), "event");
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_fail(e, "event");
    }
    // per pass, on scratch fields: the x and y expansions of orders 1 .. n_max - 1
    // as a run from delta_1 launches them (order 1 and the band-limited orders
    // move only their band columns, so the timing weighs the variants as the
    // run does); the z expansion of an order >= 2 (12 -> 17, store-only and
    // fused with pair products); the forward passes of delta_n, theta_n
    auto run = [&](const Geo& g, int pass) -> cudaError_t {
        XExpArgs xa{};
        YZExpArgs ya{}, za{};
        expansion_codes(2, xa, ya, za);
        switch (pass) {
            case TV_COLPASS: return launch_colpass_fwd(g, f0, F, 2, 1, 0, -1, 0, s);
            case TV_XEXP:
            case TV_YEXP: {
                const int top = p->d.n_max > 2 ? p->d.n_max - 1 : 1;
                for (int m = 1; m <= top; ++m) {
                    XExpArgs xm{};
                    YZExpArgs ym{}, zm{};
                    expansion_codes(m, xm, ym, zm);
                    double fx = 1.0, fyi = 1.0, fyo = 1.0;
                    if (m == 1) order1_band(p, xm, ym, zm, &fx, &fyi, &fyo);
                    else if (const int band = order_band(p, m, 2)) set_band(p, band, xm, ym, zm, &fx, &fyi, &fyo);
                    cudaError_t em;
                    if (pass == TV_XEXP) {   // order 1 backward only, orders >= 2 forward first
                        xm.src0 = f0;
                        xm.src1 = m == 1 ? f0 : f0 + F;
                        xm.out = f0 + 2 * F;
                        xm.out_stride = F;
                        xm.s2_nl = m == 1 ? -1 : order_cut(p, m);
                        xm.fwd_first = m >= 2;
                        xm.zero_k0 = m >= 2;
                        em = launch_xexp(g, xm, s);
                    } else {
                        ym.in = f0;
                        ym.in_stride = F;
                        ym.out = f0 + 7 * F;
                        ym.out_stride = F;
                        em = launch_yexp(g, ym, s);
                    }
                    if (em != cudaSuccess) return em;
                }
                return cudaSuccess;
            }
            case TV_ZEXP: {
                za.in = f0;
                za.in_stride = F;
                za.out = f0 + 12 * F;
                za.out_stride = F;
                cudaError_t ez = launch_zexp(g, za, s);
                if (ez != cudaSuccess) return ez;
                // and the form fused with pair products: one target, order-1
                // partners in fields 0..12, partial sums in from fields 13, 14,
                // outputs to fields 15, 16 (nothing written is read in the launch)
                ZPairArgs pa{};
                pa.z = za;
                pa.cells = field_floats(p);
                pa.ntargets = 1;
                PairTarget& T = pa.t[0];
                T.partner = reinterpret_cast<const float*>(f0);
                pair_table(1, T);
                T.acc_in_a = reinterpret_cast<const float*>(f0 + 13 * F);
                T.acc_in_b = reinterpret_cast<const float*>(f0 + 14 * F);
                T.out_a = reinterpret_cast<float*>(f0 + 15 * F);
                T.out_b = reinterpret_cast<float*>(f0 + 16 * F);
                T.ca0 = T.cb1 = 1.f;
                T.ca1 = T.cb0 = 0.f;
                return launch_zexp_pairs(g, pa, s);
            }
            default: return launch_zr2c(g, f0, f0, F, 2, 1.0f, 0, s);
        }
    };
    int best[TV_COUNT];
    for (int pass = 0; pass < TV_COUNT && e == cudaSuccess; ++pass) {
        float tbest = 0.f;
        best[pass] = 0;
        for (int v = 0; v < kTuneVariants[pass] && e == cudaSuccess; ++v) {
            Geo g = p->geo;
            g.var[pass] = v;
            e = run(g, pass);   // warm-up
            if (e == cudaErrorNotSupported) {   // variant not built for this size
                e = cudaSuccess;
                continue;
            }
            if (e == cudaSuccess) e = cudaEventRecord(a, s);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = run(g, pass);
            if (e == cudaSuccess) e = cudaEventRecord(b, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
            if (e == cudaSuccess && (v == 0 || t < tbest)) {
                tbest = t;
                best[pass] = v;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    for (int i = 0; i < TV_COUNT; ++i) {
        p->geo.var[i] = best[i];
        if (choices_out) choices_out[i] = best[i];
    }
    return GRIDSPT_OK;
}

gridspt_status gridspt_check(gridspt_plan p, gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    CK(cudaStreamSynchronize((cudaStream_t)stream), "check: stream synchronize");
    int st = 0;
    CK(cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost), "check: read status");
    if (st) {
        CK(cudaMemset(p->status, 0, sizeof(int)), "check: reset status");
        if (st & (kStatusWaitTma | kStatusWaitSelftest | kStatusWaitQueue))
            return fail(GRIDSPT_E_TIMEOUT, "a bounded device-side wait gave up (status %d); results of the calls "
                                           "since the last check are invalid", st);
        return fail(GRIDSPT_E_NUMERIC, "an estimator produced a NaN or infinite result since the last check "
                                       "(status %d): an input spectrum holds non-finite values", st);
    }
    return GRIDSPT_OK;
}

gridspt_status gridspt_selftest_bounded_wait(gridspt_plan p, gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    CK(launch_wait_selftest(p->status, (cudaStream_t)stream), "bounded-wait self-test");
    return GRIDSPT_OK;
}

// ---------------------------------------------------------- emulator MLP
}  // extern "C"
namespace {
gridspt_status mlp_dims(int32_t in, int32_t hidden, int32_t out) {
    if (in < 1 || in > 8 || hidden < 1 || hidden > 256 || out < 1 || out > 256)
        return fail(GRIDSPT_E_INVALID, "mlp dims in=%d hidden=%d out=%d outside [1,8] x [1,256] x [1,256]", in,
                    hidden, out);
    return GRIDSPT_OK;
}
}  // namespace
extern "C" {

gridspt_status gridspt_mlp_param_count(int32_t in, int32_t hidden, int32_t out, int64_t* count) {
    if (gridspt_status st = mlp_dims(in, hidden, out)) return st;
    if (!count) return fail(GRIDSPT_E_INVALID, "count is NULL");
    *count = mlp_params(in, hidden, out);
    return GRIDSPT_OK;
}

gridspt_status gridspt_mlp_forward(const float* x, int32_t batch, int32_t in, int32_t hidden, int32_t out,
                                   const void* params, int32_t bf16, float* y, float* act, gridspt_stream stream) {
    g_err[0] = 0;
    if (gridspt_status st = mlp_dims(in, hidden, out)) return st;
    if (!x || !params || !y || batch < 1) return fail(GRIDSPT_E_INVALID, "NULL argument or batch < 1");
    CKP(PK_MLP_FWD, 4.0 * batch * (in + out) + (bf16 ? 2.0 : 4.0) * mlp_params(in, hidden, out), (cudaStream_t)stream,
        launch_mlp_forward(x, batch, in, hidden, out, params, bf16, y, act, (cudaStream_t)stream), "mlp forward");
    return GRIDSPT_OK;
}

gridspt_status gridspt_mlp_backward_workspace_size(int32_t batch, int32_t in, int32_t hidden, int32_t out,
                                                   size_t* bytes) {
    if (gridspt_status st = mlp_dims(in, hidden, out)) return st;
    if (!bytes || batch < 1) return fail(GRIDSPT_E_INVALID, "NULL argument or batch < 1");
    *bytes = sizeof(float) * (size_t)mlp_bwd_blocks(batch) * (size_t)mlp_params(in, hidden, out);
    return GRIDSPT_OK;
}

gridspt_status gridspt_mlp_backward(const float* x, int32_t batch, int32_t in, int32_t hidden, int32_t out,
                                    const void* params, int32_t bf16, const float* act, const float* dy, float* grad,
                                    void* ws, size_t ws_bytes, gridspt_stream stream) {
    g_err[0] = 0;
    size_t need = 0;
    if (gridspt_status st = gridspt_mlp_backward_workspace_size(batch, in, hidden, out, &need)) return st;
    if (!x || !params || !act || !dy || !grad) return fail(GRIDSPT_E_INVALID, "NULL argument");
    if (!ws || ws_bytes < need) return fail(GRIDSPT_E_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, need);
    CKP(PK_MLP_BWD, 4.0 * batch * (in + 4 * hidden + out) + 4.0 * mlp_params(in, hidden, out), (cudaStream_t)stream,
        launch_mlp_backward(x, batch, in, hidden, out, params, bf16, act, dy, static_cast<float*>(ws), grad,
                            (cudaStream_t)stream),
        "mlp backward");
    return GRIDSPT_OK;
}

gridspt_status gridspt_mlp_mse(const float* y, const float* target, const float* mask, int64_t n, float* dy,
                               float* loss, gridspt_stream stream) {
    g_err[0] = 0;
    if (!y || !target || !mask || !dy || n < 1) return fail(GRIDSPT_E_INVALID, "NULL argument or n < 1");
    CKP(PK_MLP_OPT, 16.0 * n, (cudaStream_t)stream, launch_mlp_mse(y, target, mask, n, dy, loss, (cudaStream_t)stream),
        "mlp mse");
    return GRIDSPT_OK;
}

gridspt_status gridspt_mlp_adam(float* master, void* params_lowp, int32_t bf16, const float* grad, float* m, float* v,
                                int32_t* step, int64_t n, float lr, float beta1, float beta2, float eps,
                                gridspt_stream stream) {
    g_err[0] = 0;
    if (!master || !grad || !m || !v || !step || n < 1) return fail(GRIDSPT_E_INVALID, "NULL argument or n < 1");
    CKP(PK_MLP_OPT, 20.0 * n, (cudaStream_t)stream,
        launch_mlp_adam(master, params_lowp, bf16, grad, m, v, step, n, lr, beta1, beta2, eps, (cudaStream_t)stream),
        "mlp adam");
    return GRIDSPT_OK;
}

gridspt_status gridspt_mlp_convert(const float* master, void* params_lowp, int32_t bf16, int64_t n,
                                   gridspt_stream stream) {
    g_err[0] = 0;
    if (!master || !params_lowp || n < 1) return fail(GRIDSPT_E_INVALID, "NULL argument or n < 1");
    CK(launch_mlp_convert(master, params_lowp, bf16, n, (cudaStream_t)stream), "mlp convert");
    return GRIDSPT_OK;
}

gridspt_status gridspt_c2r(gridspt_plan p, const void* in_k, float* out_x, int32_t count, gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (!in_k || !out_x || count < 1) return fail(GRIDSPT_E_INVALID, "NULL argument or count < 1");
    if (!aligned16(in_k) || !aligned16(out_x)) return fail(GRIDSPT_E_INVALID, "pointers must be 16-byte aligned");
    if (gridspt_status st = set_device(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const long long F = field_c(p);
    for (int f = 0; f < count; ++f) {
        const float2* in = static_cast<const float2*>(in_k) + f * F;
        if (gridspt_status st = backward_fields(p, in, in, reinterpret_cast<float2*>(out_x) + f * F, F, 1, false, 0, 0,
                                                0, false, s))
            return st;
    }
    return GRIDSPT_OK;
}

gridspt_status gridspt_r2c(gridspt_plan p, const float* in_x, void* out_k, int32_t count, gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (!in_x || !out_k || count < 1) return fail(GRIDSPT_E_INVALID, "NULL argument or count < 1");
    if (!aligned16(in_x) || !aligned16(out_k)) return fail(GRIDSPT_E_INVALID, "pointers must be 16-byte aligned");
    if (gridspt_status st = set_device(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const long long F = field_c(p);
    float2* o = static_cast<float2*>(out_k);
    const float scale = (float)(1.0 / (double)field_floats(p));
    CK(launch_zr2c(p->geo, reinterpret_cast<const float2*>(in_x), o, F, count, scale, 0, s), "z r2c");
    CK(launch_colpass_fwd(p->geo, o, F, count, 1, 0, -1, 0, s), "y pass");
    CK(launch_colpass_fwd(p->geo, o, F, count, 0, 1, -1, 0, s), "x pass");
    return GRIDSPT_OK;
}

namespace {

// Algorithmic bytes of one power launch: each stored mode below the top edge
// read once from each input (8 bytes per mode and input).
double power_bytes(gridspt_plan_s* p, long long top, bool same) {
    if (!g_prof.on) return 0.0;
    if (p->pb_top == top) return 8.0 * p->pb_modes * (same ? 1 : 2);
    const int N = p->geo.N, M = p->geo.M;
    long long modes = 0;
    for (int kx = 0; kx < N; ++kx)
        for (int ky = 0; ky < N; ++ky) {
            const long long sx = kx < N / 2 ? kx : kx - N, sy = ky < N / 2 ? ky : ky - N;
            const long long rem = top - sx * sx - sy * sy;
            if (rem <= 0) continue;
            long long kz = (long long)std::sqrt((double)rem);
            while (kz * kz >= rem) --kz;
            while ((kz + 1) * (kz + 1) < rem) ++kz;
            modes += std::min<long long>(kz + 1, M);
        }
    p->pb_top = top;
    p->pb_modes = (double)modes;
    return 8.0 * (double)modes * (same ? 1 : 2);
}

gridspt_status make_bins(const gridspt_plan_s* p, int nbins, const double* edges, double kmax, BinSpec* bs) {
    if (nbins < 1 || nbins > kMaxBins) return fail(GRIDSPT_E_INVALID, "nbins=%d outside [1, %d]", nbins, kMaxBins);
    if (!edges) return fail(GRIDSPT_E_INVALID, "edges is NULL");
    for (int i = 0; i < nbins; ++i)
        if (!(edges[i] < edges[i + 1]) || !(edges[i] >= 0.0))
            return fail(GRIDSPT_E_INVALID, "edges must be non-negative and increasing");
    if (!std::isfinite(edges[nbins])) return fail(GRIDSPT_E_INVALID, "edges must be finite");
    bs->nbins = nbins;
    // thresholds above every mode of the grid (3 (N/2)^2) are clamped there: the
    // callers reject a last edge above the Nyquist wavenumber
    const long long cap = 3LL * (p->geo.N / 2) * (p->geo.N / 2) + 1;
    for (int i = 0; i <= nbins; ++i) {
        const double r = edges[i] / p->geo.kF;
        bs->thr[i] = r * r >= (double)cap ? (int)cap : (int)s2_threshold(edges[i], p->geo.kF);
    }
    (void)kmax;
    return GRIDSPT_OK;
}

}  // namespace

gridspt_status gridspt_power_workspace_size(gridspt_plan p, int32_t nbins, size_t* bytes) {
    if (check_plan(p) || !bytes) return fail(GRIDSPT_E_INVALID, "plan/bytes is NULL");
    if (nbins < 1 || nbins > kMaxBins) return fail(GRIDSPT_E_INVALID, "nbins=%d outside [1, %d]", nbins, kMaxBins);
    *bytes = (size_t)power_blocks(p->geo) * 2 * nbins * sizeof(double);
    return GRIDSPT_OK;
}

gridspt_status gridspt_power(gridspt_plan p, const void* a_k, const void* b_k, int32_t nbins, const double* edges,
                             double* p_out, int64_t* nk_out, void* ws, size_t ws_bytes, gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (!a_k || !b_k || !p_out) return fail(GRIDSPT_E_INVALID, "NULL argument");
    if (!aligned16(a_k) || !aligned16(b_k) || !aligned16(ws)) return fail(GRIDSPT_E_INVALID, "pointers must be 16-byte aligned");
    BinSpec bs{};
    if (gridspt_status st = make_bins(p, nbins, edges, 0, &bs)) return st;
    const long long half = p->geo.N / 2;
    if (bs.thr[nbins] > half * half) return fail(GRIDSPT_E_INVALID, "last edge above the Nyquist wavenumber");
    size_t need = 0;
    gridspt_power_workspace_size(p, nbins, &need);
    if (!ws || ws_bytes < need) return fail(GRIDSPT_E_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (gridspt_status st = set_device(p)) return st;
    const double vol = p->d.box * p->d.box * p->d.box;
    CKP(PK_POWER, power_bytes(p, bs.thr[nbins], a_k == b_k), (cudaStream_t)stream,
        launch_power(p->geo, static_cast<const float2*>(a_k), static_cast<const float2*>(b_k), bs,
                     static_cast<double*>(ws), p_out, nk_out, vol, (cudaStream_t)stream), "power launch");
    return GRIDSPT_OK;
}

}  // extern "C"


extern "C" {

gridspt_status gridspt_growth_factor(const gridspt_cosmo* c, double z, double* D) {
    g_err[0] = 0;
    if (!c || !D) return fail(GRIDSPT_E_INVALID, "cosmo/D is NULL");
    const double om = c->omega_m;
    if (!(om > 0.0 && om <= 1.0) || !(z > -1.0) || !std::isfinite(z))
        return fail(GRIDSPT_E_INVALID, "need 0 < omega_m <= 1 and z > -1");
    // D(a) = 5/2 Om E(a) int_0^a da' (a' E(a'))^-3, E = sqrt(Om a^-3 + 1 - Om): composite Simpson
    auto growth = [om](double a) {
        const int n = 1 << 16;
        const double h = a / n;
        double sum = 0.0;
        for (int i = 1; i <= n; ++i) {   // f(0) = 0
            const double x = i * h;
            const double e = std::sqrt(om / (x * x * x) + 1.0 - om);
            const double f = 1.0 / ((x * e) * (x * e) * (x * e));
            sum += (i == n ? 1.0 : (i % 2 ? 4.0 : 2.0)) * f;
        }
        return 2.5 * om * std::sqrt(om / (a * a * a) + 1.0 - om) * (h / 3.0) * sum;
    };
    *D = growth(1.0 / (1.0 + z)) / growth(1.0);
    return GRIDSPT_OK;
}

gridspt_status gridspt_sum_orders(gridspt_plan p, const void* delta1_k, const void* spectra, int32_t n, double D,
                                  double R, void* out_k, gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (n < 1 || n > p->d.n_max) return fail(GRIDSPT_E_INVALID, "n=%d outside [1, %d]", n, p->d.n_max);
    if (!delta1_k || !out_k || (n >= 2 && !spectra)) return fail(GRIDSPT_E_INVALID, "NULL argument");
    if (!aligned16(delta1_k) || !aligned16(out_k) || (spectra && !aligned16(spectra)))
        return fail(GRIDSPT_E_INVALID, "pointers must be 16-byte aligned");
    if (!std::isfinite(D) || !(R >= 0.0) || !std::isfinite(R)) return fail(GRIDSPT_E_INVALID, "need finite D, R >= 0");
    if (gridspt_status st = set_device(p)) return st;
    const long long F = field_c(p);
    SumOrdersArgs a{};
    a.n = n;
    a.N = p->geo.N;
    a.out = static_cast<float2*>(out_k);
    a.r2kf2 = (float)((R * p->geo.kF) * (R * p->geo.kF));
    double c = 1.0;
    for (int i = 1; i <= n; ++i) {
        c *= D;
        a.coef[i - 1] = (float)c;
        a.field[i - 1] = i == 1 ? static_cast<const float2*>(delta1_k)
                                : static_cast<const float2*>(spectra) + (long long)(i - 2) * 2 * F;
    }
    CKP(PK_FIELDS, 4.0 * (double)field_floats(p) * (n + 1), (cudaStream_t)stream,
        launch_sum_orders(a, (cudaStream_t)stream), "summed orders");
    return GRIDSPT_OK;
}

gridspt_status gridspt_cross_correlation_workspace_size(gridspt_plan p, int32_t nbins, size_t* bytes) {
    if (check_plan(p) || !bytes) return fail(GRIDSPT_E_INVALID, "plan/bytes is NULL");
    size_t pw = 0;
    if (gridspt_status st = gridspt_power_workspace_size(p, nbins, &pw)) return st;
    *bytes = align256(pw) + align256(3 * (size_t)nbins * sizeof(double));
    return GRIDSPT_OK;
}

gridspt_status gridspt_cross_correlation(gridspt_plan p, const void* a_k, const void* b_k, int32_t nbins,
                                         const double* edges, double* r_out, void* ws, size_t ws_bytes,
                                         gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (!a_k || !b_k || !r_out || !ws) return fail(GRIDSPT_E_INVALID, "NULL argument");
    size_t need = 0, pw = 0;
    if (gridspt_status st = gridspt_cross_correlation_workspace_size(p, nbins, &need)) return st;
    if (ws_bytes < need) return fail(GRIDSPT_E_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, need);
    gridspt_power_workspace_size(p, nbins, &pw);
    char* base = static_cast<char*>(ws);
    double* pp = reinterpret_cast<double*>(base + align256(pw));
    const struct { const void* x; const void* y; double* out; } terms[3] = {
        {a_k, b_k, pp}, {a_k, a_k, pp + nbins}, {b_k, b_k, pp + 2 * nbins}};
    for (const auto& t : terms)
        if (gridspt_status st = gridspt_power(p, t.x, t.y, nbins, edges, t.out, nullptr, ws, align256(pw), stream))
            return st;
    CK(launch_rcorr(pp, pp + nbins, pp + 2 * nbins, nbins, r_out, (cudaStream_t)stream), "correlation coefficient");
    return GRIDSPT_OK;
}

gridspt_status gridspt_power_noalloc(gridspt_plan p, const void* a_k, const void* b_k, int32_t nbins,
                                     const double* edges, double* p_out, int64_t* nk_out,
                                     gridspt_stream stream) {
    g_err[0] = 0;
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (!a_k || !b_k || !p_out) return fail(GRIDSPT_E_INVALID, "NULL argument");
    if (!aligned16(a_k) || !aligned16(b_k)) return fail(GRIDSPT_E_INVALID, "pointers must be 16-byte aligned");
    BinSpec bs{};
    if (gridspt_status st = make_bins(p, nbins, edges, 0, &bs)) return st;
    const long long half = p->geo.N / 2;
    if (bs.thr[nbins] > half * half) return fail(GRIDSPT_E_INVALID, "last edge above the Nyquist wavenumber");
    if (!power_static_fits(p->geo, nbins))
        return fail(GRIDSPT_E_INVALID, "%d blocks x %d bins of partial sums exceed the %zu-byte static scratch",
                    power_blocks(p->geo), nbins, power_static_scratch_bytes());
    if (gridspt_status st = set_device(p)) return st;
    double* scratch = nullptr;
    CK(power_static_scratch(&scratch), "static scratch address");
    const double vol = p->d.box * p->d.box * p->d.box;
    CKP(PK_POWER, power_bytes(p, bs.thr[nbins], a_k == b_k), (cudaStream_t)stream,
        launch_power(p->geo, static_cast<const float2*>(a_k), static_cast<const float2*>(b_k), bs, scratch,
                     p_out, nk_out, vol, (cudaStream_t)stream), "power launch");
    return GRIDSPT_OK;
}

gridspt_status gridspt_bispectrum_workspace_size(gridspt_plan p, int32_t nbins, size_t* bytes) {
    if (check_plan(p) || !bytes) return fail(GRIDSPT_E_INVALID, "plan/bytes is NULL");
    if (nbins < 1 || nbins > kMaxBins) return fail(GRIDSPT_E_INVALID, "nbins=%d outside [1, %d]", nbins, kMaxBins);
    *bytes = 4 * align256((size_t)field_floats(p) * sizeof(float)) + align256((size_t)shell_blocks(p->geo) * 2 * sizeof(double));
    return GRIDSPT_OK;
}

}  // extern "C"

namespace {

// Geometry of the grid of size S <= N that shares the plan's box (same k_F,
// tile variants and status word) for the band-limited bispectrum shells.
bool sub_geo(const gridspt_plan_s* p, int S, Geo* out) {
    *out = p->geo;
    if (S == p->geo.N) return true;
    for (int i = 0; i < kNumSizes; ++i) {
        if (kSizes[i] == S && p->sub_off[i] >= 0) {
            out->tw = p->tw + p->sub_off[i];
            out->N = S;
            out->M = S / 2;
            return true;
        }
    }
    return false;                       // no table of that size in the plan
}

// Grid on which a shell with every component |s_a| < band is evaluated: the
// smallest supported size S > 3 (band - 1) (then no sum s_1 + s_2 + s_3 of
// three shell vectors other than 0 is a multiple of S in any component), or N.
int shell_grid(int N, int band) {
    for (int i = 0; i < kNumSizes; ++i)
        if (kSizes[i] < N && kSizes[i] > 3 * (band - 1)) return kSizes[i];
    return N;
}

// Shell fields of one bispectrum shell on grid g: I_a, I_b (, I_c) and,
// without a cached sum J^3, J, transformed along x (pruned to |ky|, kz < band)
// and y into out[f] (stride fstride); the z pass follows fused with the sums.
// a, b, c are half spectra of grid g.
gridspt_status shell_fields(const Geo& geo, const float2* a, const float2* b, const float2* c, bool has_j,
                            long long lo, long long hi, int band, float2* out, long long fstride, cudaStream_t s) {
    const double N = geo.N, M = geo.M;
    const double fb = 4.0 * N * N * N;
    const double fx = band > 0 ? (2.0 * band - 1.0) * band / (N * M) : 1.0;   // x columns
    const double fy_in = band > 0 ? (2.0 * band - 1.0) / N * band / M : 1.0;   // y inputs
    const double fy_out = band > 0 ? band / M : 1.0;                         // y outputs
    auto xpass = [&](const float2* s0, const float2* s1, int first, int count, const int* srcs) -> gridspt_status {
        XExpArgs xa{};
        xa.src0 = const_cast<float2*>(s0);
        xa.src1 = const_cast<float2*>(s1);
        xa.out = out + first * fstride;
        xa.out_stride = fstride;
        xa.s2_nl = -1;
        xa.shell_lo = lo;
        xa.shell_hi = hi;
        xa.band = band;
        xa.nout = count;
        for (int f = 0; f < count; ++f) xa.codes[f] = x_code(XK_SHELL, 0, srcs[f]);
        CKP(PK_BX, fb * fx * ((s0 == s1 ? 1 : 2) + count), s, launch_xexp(geo, xa, s), "x pass");
        return GRIDSPT_OK;
    };
    int nf = 0;
    if (!c) {
        const int srcs[3] = {XS_DELTA, b == a ? XS_DELTA : XS_THETA, XS_ONE};
        if (gridspt_status st = xpass(a, b, 0, has_j ? 3 : 2, srcs)) return st;
        nf = has_j ? 3 : 2;
    } else {
        const int s_ab[2] = {XS_DELTA, b == a ? XS_DELTA : XS_THETA};
        const int s_cj[2] = {XS_DELTA, XS_ONE};
        if (gridspt_status st = xpass(a, b, 0, 2, s_ab)) return st;
        if (gridspt_status st = xpass(c, c, 2, has_j ? 2 : 1, s_cj)) return st;
        nf = has_j ? 4 : 3;
    }
    YZExpArgs ya{};
    ya.in = out;
    ya.in_stride = fstride;
    ya.out = out;
    ya.out_stride = fstride;
    ya.nout = nf;
    ya.band = band;
    for (int f = 0; f < nf; ++f) ya.codes[f] = y_code(f, 0, f);
    CKP(PK_BY, fb * nf * (fy_in + fy_out), s, launch_yexp(geo, ya, s), "y pass");
    return GRIDSPT_OK;
}

// E = L^6 sum I_a^2 I_b / sum J^3 (c == NULL) or L^6 sum I_a I_b I_c / sum J^3.
// Each shell is evaluated on the smallest grid that holds its products
// without aliasing (shell_grid): the inputs are copied onto that grid once per
// grid size (the shells come in increasing order) into the workspace's field
// area, which holds 3 inputs and 4 shell fields of any smaller supported size.
gridspt_status bispectrum_impl(gridspt_plan p, const void* a_k, const void* b_k, const void* c_k, int32_t nbins,
                               const double* edges, double* e_out, double* ntri_out, void* ws, size_t ws_bytes,
                               gridspt_stream stream) {
    if (check_plan(p)) return GRIDSPT_E_INVALID;
    if (!a_k || !b_k || !e_out || !ntri_out) return fail(GRIDSPT_E_INVALID, "NULL argument");
    if (!aligned16(a_k) || !aligned16(b_k) || (c_k && !aligned16(c_k)) || !aligned16(ws))
        return fail(GRIDSPT_E_INVALID, "pointers must be 16-byte aligned");
    BinSpec bs{};
    if (gridspt_status st = make_bins(p, nbins, edges, 0, &bs)) return st;
    const long long maxs2 = (long long)bs.thr[nbins] - 1;
    if (9 * maxs2 >= (long long)p->geo.N * p->geo.N)
        return fail(GRIDSPT_E_INVALID, "last edge must lie below 2 k_Ny / 3 (shell vectors |s| < N/3)");
    size_t need = 0;
    gridspt_bispectrum_workspace_size(p, nbins, &need);
    if (!ws || ws_bytes < need) return fail(GRIDSPT_E_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (gridspt_status st = set_device(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = p->geo.N;
    const size_t fb = align256((size_t)field_floats(p) * sizeof(float));
    char* base = static_cast<char*>(ws);
    double* partial = reinterpret_cast<double*>(base + 4 * fb);
    const double L = p->d.box;
    const int G = shell_blocks(p->geo);
    // sum J^3 per shell is data independent: reuse it when the shells match the cached ones
    bool cached = p->j3_nb == nbins;
    for (int i = 0; cached && i <= nbins; ++i) cached = p->j3_thr[i] == bs.thr[i];
    const int triple = c_k ? 1 : 0;
    const int nf = 2 + triple + (cached ? 0 : 1);
    // distinct inputs (a field passed twice is copied once, so the x pass
    // still sees equal pointers)
    const float2* in0[3] = {static_cast<const float2*>(a_k), static_cast<const float2*>(b_k),
                            static_cast<const float2*>(c_k)};
    const float2* uniq[3] = {};
    int slot[3] = {0, 0, 0}, nin = 0;
    for (int f = 0; f < (c_k ? 3 : 2); ++f) {
        int j = 0;
        while (j < nin && uniq[j] != in0[f]) ++j;
        if (j == nin) uniq[nin++] = in0[f];
        slot[f] = j;
    }
    int have = 0;                       // grid size the workspace's inputs are on (0: none)
    for (int i = 0; i < nbins; ++i) {
        if (bs.thr[i + 1] <= 1) {   // shell holds no mode with k > 0
            CK(cudaMemsetAsync(e_out + i, 0, sizeof(double), s), "bispectrum empty shell");
            CK(cudaMemsetAsync(ntri_out + i, 0, sizeof(double), s), "bispectrum empty shell");
            if (!cached) CK(cudaMemsetAsync(p->j3 + i, 0, sizeof(double), s), "bispectrum empty shell");
            continue;
        }
        // every mode of the shell has |s_a| < band in each component
        const int band = (int)std::floor(std::sqrt((double)(bs.thr[i + 1] - 1))) + 1;
        int S = shell_grid(N, band);
        Geo geo{};
        if (!sub_geo(p, S, &geo)) return fail(GRIDSPT_E_INVALID, "internal: no transform table for grid %d", S);
        const size_t fs = align256((size_t)S * S * S * sizeof(float));
        if (S < N && (7 * fs > 4 * fb || shell_blocks(geo) > G)) {
            S = N;
            sub_geo(p, S, &geo);
        }
        const float2* in[3] = {in0[0], in0[1], in0[2]};
        float2* fields = reinterpret_cast<float2*>(base);
        long long fstride = (long long)(fb / sizeof(float2));
        if (S < N) {
            float2* small = reinterpret_cast<float2*>(base);
            const long long sstride = (long long)(fs / sizeof(float2));
            if (S != have) {
                CKP(PK_BGATHER, 2.0 * nin * (double)S * S * S * 4.0, s,
                    launch_subgrid(N, S, uniq, nin, small, sstride, s), "bispectrum sub-grid copy");
                have = S;
            }
            for (int f = 0; f < (c_k ? 3 : 2); ++f) in[f] = small + slot[f] * sstride;
            fields = small + 3 * sstride;
            fstride = sstride;
        } else {
            have = 0;                   // the full-size shell fields overwrite the copies
        }
        if (gridspt_status st = shell_fields(geo, in[0], in[1], c_k ? in[2] : nullptr, !cached, bs.thr[i],
                                             bs.thr[i + 1], band, fields, fstride, s))
            return st;
        const double fbytes = 4.0 * (double)S * S * S;
        const int Gs = shell_blocks(geo);
        CKP(PK_BZ, fbytes * nf * ((double)band / geo.M), s,
            launch_zshell(geo, fields, fstride, band, nf, triple, partial, s), "bispectrum z pass and sums");
        CKP(PK_BISPEC, 16.0 * Gs, s,
            launch_bispec_final(geo, partial, Gs, cached ? 2 : 3, p->j3 + i, e_out + i, ntri_out + i,
                                L * L * L * L * L * L, s),
            "bispectrum final sum");
    }
    if (!cached) {
        p->j3_nb = nbins;
        for (int i = 0; i <= nbins; ++i) p->j3_thr[i] = bs.thr[i];
    }
    return GRIDSPT_OK;
}

}  // namespace

extern "C" {

gridspt_status gridspt_bispectrum(gridspt_plan p, const void* a_k, const void* b_k, int32_t nbins,
                                  const double* edges, double* e_out, double* ntri_out, void* ws,
                                  size_t ws_bytes, gridspt_stream stream) {
    g_err[0] = 0;
    return bispectrum_impl(p, a_k, b_k, nullptr, nbins, edges, e_out, ntri_out, ws, ws_bytes, stream);
}

gridspt_status gridspt_bispectrum_triple(gridspt_plan p, const void* a_k, const void* b_k, const void* c_k,
                                         int32_t nbins, const double* edges, double* e_out, double* ntri_out,
                                         void* ws, size_t ws_bytes, gridspt_stream stream) {
    g_err[0] = 0;
    if (!c_k) return fail(GRIDSPT_E_INVALID, "NULL argument");
    return bispectrum_impl(p, a_k, b_k, c_k, nbins, edges, e_out, ntri_out, ws, ws_bytes, stream);
}

}  // extern "C"
