/*
 * gridspt.h -- C ABI of the GB300 GridSPT library (libgridspt.so).
 *
 * GridSPT (Taruya, Nishimichi & Jeong, arXiv:1807.04215) generates standard
 * perturbation theory density and velocity-divergence fields order by order on
 * a periodic grid: a Gaussian linear field delta_1 = theta_1 (Eq.
 * recursion_n=1), then for n = 2..n_max the real-space recursion of Eq.
 * recursion_formula (Sec. II.B), with spectral derivatives and inverse
 * Laplacians taken in Fourier space and products in real space, following the
 * recipe of Sec. II.C. Power spectra (Eqs. pk_lin, pk_1loop, pk_2loop) and the
 * equilateral bispectrum (Eq. bk_tree) are measured from the spectra.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid: N points per side, N even, N = 2^a or 3 * 2^a, 8 <= N <= 1024; box
 *   side L (Mpc/h). Signed wavevector index s, k = (2 pi / L) s.
 * - Transform pair (Sec. II.C): a(x) = sum_k a(k) e^{i k.x},
 *   a(k) = N^-3 sum_x a(x) e^{-i k.x}.
 * - Real field: float[N][N][N], z fastest (x_j = j L / N).
 * - Half spectrum: float2[N][N][N/2] = (re, im), index [kx][ky][kz] with
 *   kx, ky in FFT order (0..N/2-1, then -N/2..-1) and kz = 0..N/2-1. Modes
 *   with a component at the Nyquist index -N/2 are zero in every spectrum, so
 *   the kz = N/2 plane is omitted; a half spectrum has the same byte size as a
 *   real field (4 N^3 bytes). Modes with kz < 0 follow from a(-k) = conj a(k).
 * - Every data pointer is a DEVICE pointer to caller-owned memory, aligned to
 *   16 bytes. The library never allocates, frees or retains caller memory.
 *   A plan owns a few KB of device tables (allocated in gridspt_plan_create on
 *   the current device, freed in gridspt_plan_destroy) and nothing else.
 * - Streams: `stream` is a cudaStream_t (NULL = legacy default stream). All
 *   compute entry points only enqueue work on `stream` and do not synchronise;
 *   results are valid once the stream has reached them.
 * - Errors: arguments are validated before any launch; on failure nothing is
 *   enqueued and a status != GRIDSPT_OK is returned, with a message available
 *   from gridspt_last_error() (thread-local). Launch failures return
 *   GRIDSPT_E_CUDA. No C++ exception crosses the ABI.
 */
#ifndef GRIDSPT_H
#define GRIDSPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRIDSPT_OK = 0,
    GRIDSPT_E_INVALID = 1,     /* bad argument, size, alignment or workspace */
    GRIDSPT_E_UNSUPPORTED = 2, /* valid request outside what the library supports */
    GRIDSPT_E_NOMEM = 3,       /* plan tables could not be allocated */
    GRIDSPT_E_CUDA = 4,        /* a CUDA runtime call or launch failed */
    GRIDSPT_E_TIMEOUT = 5,     /* a bounded device-side wait gave up (reported by gridspt_check) */
    GRIDSPT_E_NUMERIC = 6      /* an estimator result was NaN or infinite (reported by gridspt_check) */
} gridspt_status;

typedef struct gridspt_plan_s* gridspt_plan;
typedef void* gridspt_stream; /* cudaStream_t */

/* Form of the sources A_n, B_n of Eq. recursion_formula.
 * GRIDSPT_FORM_NINE_TERM: the paper's bilinear terms, A_n = sum_m grad delta_m .
 *   u_{n-m} + delta_m theta_{n-m}, B_n = sum_m d_j u_{m,k} d_k u_{n-m,j} +
 *   u_m . grad theta_{n-m}, from 13 (order 1) or 17 real derived fields per order.
 * GRIDSPT_FORM_DIVERGENCE: the same sources rewritten with theta = div u and u
 *   curl free (Eq. u_and_theta): A_n = div sum_m delta_m u_{n-m}, B_n = (1/2)
 *   lap sum_m u_m . u_{n-m}, the divergence and Laplacian taken in k-space; four
 *   real fields per order (delta, u). Modes below delta_1's cut equal the
 *   nine-term form's to rounding; modes above it, where the grid products fold,
 *   differ between the two forms. Not in the paper. */
enum { GRIDSPT_FORM_NINE_TERM = 0, GRIDSPT_FORM_DIVERGENCE = 1 };

/* Shell-sum accumulation of the power and bispectrum estimators (Eqs. pk_lin,
 * pk_1loop, pk_2loop, bk_tree; the paper does not state a precision). The
 * terms are formed from the FP32 fields either way.
 * GRIDSPT_ACCUM_COMPENSATED (default, 0): FP32 partial sums whose rounding
 *   errors are carried (two-sum in the power scan, Kahan chains in the shell
 *   sums), finished in FP64.
 * GRIDSPT_ACCUM_FP64: every term added in FP64 (power products formed in FP64
 *   from the FP32 inputs; shell products formed in FP32, summed in FP64). */
enum { GRIDSPT_ACCUM_COMPENSATED = 0, GRIDSPT_ACCUM_FP64 = 1 };

/* Problem description (Sec. II.C: box, grid, highest order, sharp-k cuts). */
typedef struct {
    int32_t n;        /* grid points per side */
    int32_t n_max;    /* highest perturbative order, 1..8 */
    int32_t batch;    /* realisations per call of make_linear_field / run_orders */
    int32_t form;     /* GRIDSPT_FORM_NINE_TERM (default, 0) or GRIDSPT_FORM_DIVERGENCE */
    double box;       /* L in Mpc/h, > 0 */
    double kcut_lin;  /* sharp-k cut on delta_1 in h/Mpc (|k| <= kcut kept);
                         <= 0 selects 2 k_Ny / (n_max + 1), k_Ny = pi N / L */
    double kcut_nl;   /* sharp-k cut applied to delta_n, theta_n for n >= 2;
                         <= 0 means none (only the Nyquist modes are zeroed) */
    int32_t truncate; /* 1: every order j >= 2 formed by gridspt_run_orders is cut at
                         min(j, n_max + 1 - j) K_c (|k| kept below it; K_c = the
                         cut on delta_1), which is all that the orders above it
                         need for their modes below K_c: delta_n, theta_n at
                         |k| <= K_c equal those of the full recursion up to
                         rounding, the modes above the cut are zero, and the
                         passes of the cut orders move only their band columns.
                         Nine-term form only. 0 (default): no such cut. */
    int32_t accum;    /* estimator shell sums: GRIDSPT_ACCUM_COMPENSATED (0) or
                         GRIDSPT_ACCUM_FP64 (1) */
} gridspt_desc;

/* Linear spectrum parameters: P(k) = A k^{n_s} T_BBKS(k / Gamma)^2, A fixed by
 * sigma_8 (top-hat radius 8 Mpc/h); gamma <= 0 selects Gamma = omega_m * h. */
typedef struct {
    double omega_m, h, n_s, sigma8, gamma;
} gridspt_cosmo;

/* Create a plan for `desc` on the current CUDA device (host call; allocates
 * and uploads the FP32 twiddle table, computed in FP64 on the host).
 * Returns GRIDSPT_E_INVALID for an unsupported N, n_max, box or batch. */
gridspt_status gridspt_plan_create(const gridspt_desc* desc, gridspt_plan* out);

/* Release the plan's device tables. Safe on NULL. Synchronises the device. */
gridspt_status gridspt_plan_destroy(gridspt_plan plan);

/* Bytes of caller workspace gridspt_run_orders needs, in fields of 4 N^3 bytes
 * (independent of batch). Nine-term form: the real-space derived fields (Sec.
 * II.C steps (2) and (5)) of the orders m with 2m <= n_max (13 for order 1, 17
 * for later orders; the pair products of the other orders are accumulated as
 * soon as those are formed), two partial-sum fields per order n >= 4, and the
 * expansion scratch of 19 fields: 53 fields for n_max = 5. Divergence form:
 * delta and u of orders 1..n_max-1, the four source fields and 7 scratch
 * fields: 4 n_max + 7 (27 for n_max = 5). */
gridspt_status gridspt_workspace_size(gridspt_plan plan, size_t* bytes);

/* Normalisation A of the linear spectrum (host only, FP64 Simpson in ln k). */
gridspt_status gridspt_linear_amplitude(const gridspt_cosmo* cosmo, double* amplitude);

/* Sec. II.C step (1): Gaussian delta_1(k) for each realisation b < batch.
 *   seeds:    HOST uint64[batch], one Philox4x32-10 key per realisation.
 *   delta1_k: device half spectra float2[batch][N][N][N/2] (written).
 * Each mode pair {s, -s} draws two uniforms from Philox4x32-10 (Salmon et al.
 * SC'11) with key = seed and counter = (packed s lo, packed s hi, 0, 0), where
 * the canonical member c of the pair (c_z > 0, or c_z = 0 and c_y > 0, or
 * c_z = c_y = 0 and c_x > 0) is packed as three 21-bit two's-complement
 * fields; u = (r + 1/2) 2^-32, g1 + i g2 = sqrt(-2 ln u1) e^{2 pi i u2},
 * delta(c) = sqrt(P(|k|) / L^3) (g1 + i g2) / sqrt(2), delta(-c) = conj.
 * Zero: k = 0, Nyquist modes and |s|^2 > (kcut_lin / k_F)^2. FP64 arithmetic,
 * stored as FP32. */
gridspt_status gridspt_make_linear_field(gridspt_plan plan, const gridspt_cosmo* cosmo,
                                         const uint64_t* seeds, void* delta1_k,
                                         gridspt_stream stream);

/* Sec. II.C steps (2)-(6) repeated to order n_max (Eq. recursion_formula):
 *   delta1_k: device float2[batch][N][N][N/2] (read only). Its modes with
 *             |s|^2 > (kcut_lin / k_F)^2 (default cut 2 k_Ny / (n_max + 1))
 *             are taken as zero, the cut of Sec. II.C on the linear field, as
 *             gridspt_make_linear_field writes them; the order-1 passes move
 *             only the columns inside that cut.
 *   spectra:  device float2[batch][n_max-1][2][N][N][N/2]; slot [b][n-2][0] is
 *             delta_n(k), [b][n-2][1] is theta_n(k), n = 2..n_max (written for
 *             n >= start_order, read for 2 <= n < start_order). An order n
 *             formed in the call whose modes have every component at most c_n
 *             (c_n = n floor(sqrt(s2_lin)) while 2 c_n < N and all lower orders
 *             were formed in the same call; with kcut_nl at most
 *             floor(sqrt(s2_nl))) is transformed only on the columns
 *             |ky|, kz < B, B = c_n + 1 rounded up to even, when B < N/2, and
 *             is written as exact zeros outside them, where its exact values
 *             vanish. s2_lin = floor((kcut_lin / k_F)^2), likewise s2_nl.
 *             The k = 0 mode of every order formed in the call is written as
 *             zero, its exact value (mass conservation: the k = 0 modes of
 *             the two source terms cancel exactly on the grid), not as the
 *             FP32 rounding residue of the mean of the products, which would
 *             otherwise feed the next orders as a spurious uniform field.
 *   start_order: 2 for a full run; 3..n_max resumes from stored lower orders
 *             (Sec. II.C: only delta_m, theta_m are needed to continue).
 *   ws, ws_bytes: device scratch of at least gridspt_workspace_size bytes.
 * Realisations run one after another on `stream` and reuse ws. */
gridspt_status gridspt_run_orders(gridspt_plan plan, const void* delta1_k, int32_t start_order,
                                  void* spectra, void* ws, size_t ws_bytes,
                                  gridspt_stream stream);

/* Unnormalised backward transform (Sec. II.C pair) of `count` half spectra
 * into real fields: out_x[f](x) = sum_k in_k[f](k) e^{i k.x}. in_k and out_x
 * may be the same buffer (in place); otherwise in_k is left unchanged. */
gridspt_status gridspt_c2r(gridspt_plan plan, const void* in_k, float* out_x, int32_t count,
                           gridspt_stream stream);

/* Forward transform of `count` real fields: out_k = N^-3 sum_x in_x e^{-i k.x},
 * Nyquist modes zeroed. in_x and out_k may be the same buffer. */
gridspt_status gridspt_r2c(gridspt_plan plan, const float* in_x, void* out_k, int32_t count,
                           gridspt_stream stream);

/* Shell power estimator (Sec. III.B.1, Eqs. pk_lin/pk_1loop/pk_2loop):
 *   p_out[i] = L^3 / N_i * sum_{k in bin i} Re[a(k) b*(k)]  over every mode of
 *   the full grid with k = k_F sqrt(|s|^2) != 0 and edges[i] <= k < edges[i+1].
 *   a_k, b_k: device half spectra (one realisation each; b_k may equal a_k).
 *   edges:    HOST double[nbins+1], increasing, edges[nbins] <= k_Ny.
 *   p_out:    device double[nbins]; nk_out: device int64[nbins] (may be NULL).
 *   1 <= nbins <= 64. Products in FP32; runs of up to 32 consecutive modes
 *   of a bin summed in FP32 with each addition's rounding error carried
 *   (two-sum), the runs accumulated in FP64, all reduced in a fixed order
 *   (bitwise repeatable); with accum = GRIDSPT_ACCUM_FP64 the products and
 *   every sum are FP64. A NaN or infinite result sets the plan's status
 *   (gridspt_check then returns GRIDSPT_E_NUMERIC). Cross terms of the paper carry a factor
 *   2: P_13 = 2 * gridspt_power(delta_1, delta_3). ws: device scratch of
 *   gridspt_power_workspace_size bytes (per-block partial sums). */
gridspt_status gridspt_power_workspace_size(gridspt_plan plan, int32_t nbins, size_t* bytes);
gridspt_status gridspt_power(gridspt_plan plan, const void* a_k, const void* b_k, int32_t nbins,
                             const double* edges, double* p_out, int64_t* nk_out, void* ws,
                             size_t ws_bytes, gridspt_stream stream);

/* Allocation-free variant of gridspt_power for callers that cannot allocate
 * device memory when they need a spectrum (their framework's allocator owns the
 * device memory, or they are handed only input and output buffers). The paper
 * has no counterpart: this is a deployment convenience.
 * Same arguments and results as gridspt_power, without ws/ws_bytes: the
 * per-block partial sums live in a static device array compiled into the
 * library, 1,245,184 bytes (1216 blocks x 2 x 64 bins x 8 bytes), held on every
 * GPU that loads the library until the process exits. Requests that would need
 * more (nbins > 64) are rejected with GRIDSPT_E_INVALID and a message.
 * The first call on each device looks up the array's device address (a host
 * call, made with that device current); make that first call before any
 * stream capture. No call allocates or frees memory. All calls on a device
 * share the one array: each call overwrites every partial sum it reads, so no
 * state carries over, but calls that can overlap on the GPU (different
 * streams, no ordering between them) race on it and must be serialised by the
 * caller. */
gridspt_status gridspt_power_noalloc(gridspt_plan plan, const void* a_k, const void* b_k, int32_t nbins,
                                     const double* edges, double* p_out, int64_t* nk_out,
                                     gridspt_stream stream);

/* Linear growth factor D_+(z) / D_+(0) of a flat LCDM background (Omega_Lambda
 * = 1 - omega_m; the D_+ of Sec. II.A that weights order i by D_+^i):
 *   D(a) = (5 Omega_m / 2) E(a) int_0^a da' / (a' E(a'))^3,
 *   E(a) = sqrt(Omega_m a^-3 + 1 - Omega_m), a = 1 / (1 + z),
 * host FP64 (composite Simpson, 2^16 intervals). Requires 0 < omega_m <= 1,
 * z > -1; only cosmo->omega_m is used. */
gridspt_status gridspt_growth_factor(const gridspt_cosmo* cosmo, double z, double* D);

/* Summed density field of Sec. III.A, smoothed with the Gaussian filter the
 * paper applies before comparing fields:
 *   out_k(k) = exp(-k^2 R^2 / 2) sum_{i=1}^{n} D^i delta_i(k)
 * for one realisation. delta1_k: device half spectrum; spectra: device
 * float2[n_max-1][2][N][N][N/2] as gridspt_run_orders writes it for one
 * realisation (may be NULL when n = 1); 1 <= n <= n_max; D: growth factor
 * (e.g. from gridspt_growth_factor), R >= 0 in Mpc/h (0: no filter); out_k:
 * device half spectrum (may not alias the inputs). FP32 sums with D^i formed
 * in FP64 on the host; the filter in FP32. gridspt_c2r gives the field in real
 * space. */
gridspt_status gridspt_sum_orders(gridspt_plan plan, const void* delta1_k, const void* spectra, int32_t n,
                                  double D, double R, void* out_k, gridspt_stream stream);

/* Cross-correlation coefficient per shell (Sec. III.B, Eqs. r_corr_nthPT and
 * r_corr_sum_nth with the cross-spectrum read as Re[a b*]):
 *   r_out[i] = sum Re[a b*] / sqrt(sum |a|^2 sum |b|^2) over the modes of bin i,
 * formed from three gridspt_power spectra (P_ab / sqrt(P_aa P_bb)); 0 for an
 * empty bin. Bins as for gridspt_power; r_out: device double[nbins]; ws:
 * gridspt_cross_correlation_workspace_size bytes of device scratch. */
gridspt_status gridspt_cross_correlation_workspace_size(gridspt_plan plan, int32_t nbins, size_t* bytes);
gridspt_status gridspt_cross_correlation(gridspt_plan plan, const void* a_k, const void* b_k, int32_t nbins,
                                         const double* edges, double* r_out, void* ws, size_t ws_bytes,
                                         gridspt_stream stream);

/* Equilateral FFT shell bispectrum (Sec. III.B.1, Eq. bk_tree, measured with
 * an FFT shell estimator): for shell i,
 *   e_out[i]    = L^6 sum_x I_i[a](x)^2 I_i[b](x) / sum_x J_i(x)^3,
 *   ntri_out[i] = sum_x J_i(x)^3 / N^3  (closed ordered triangles),
 * with I_i[f](x) = sum_{k in shell i} f(k) e^{i k.x}, J_i = I_i[1]. The
 * tree-level bispectrum is B_tree = 3 e_out for a = delta_1, b = delta_2.
 *   edges: HOST double[nbins+1] with edges[nbins] <= 2 k_Ny / 3 (no wrap);
 *   e_out, ntri_out: device double[nbins]; 1 <= nbins <= 64. FP32 fields,
 *   Kahan-compensated FP32 sums over row groups of cells, FP64 across groups,
 *   fixed order (FP64 sums of the same terms with accum = GRIDSPT_ACCUM_FP64);
 *   a NaN or infinite result sets the plan's status (GRIDSPT_E_NUMERIC).
 *   Sums over x run on the smallest supported grid S > 3 (B - 1) (S <= N) for a shell whose vectors have every component |s_a| < B: there
 *   the only sum of three shell vectors that is a multiple of S is zero, so
 *   both sums are those of the N^3 grid times (S/N)^3 and e_out, ntri_out are
 *   unchanged (the inputs are copied onto that grid in the workspace first).
 *   ws: gridspt_bispectrum_workspace_size bytes (4 fields of size N and the
 *   partial sums) of device scratch. sum_x J^3 does not depend on the data: the first call
 *   with a given set of shells computes it and keeps it in the plan (device
 *   memory), later calls with the same shells reuse it, so they must be
 *   ordered after that first call (same stream, or synchronised). */
gridspt_status gridspt_bispectrum_workspace_size(gridspt_plan plan, int32_t nbins, size_t* bytes);
gridspt_status gridspt_bispectrum(gridspt_plan plan, const void* a_k, const void* b_k,
                                  int32_t nbins, const double* edges, double* e_out,
                                  double* ntri_out, void* ws, size_t ws_bytes,
                                  gridspt_stream stream);

/* Triple-product form of the shell estimator for three fields:
 *   e_out[i] = L^6 sum_x I_i[a](x) I_i[b](x) I_i[c](x) / sum_x J_i(x)^3,
 * arguments, workspace, bounds and the cached sum J^3 as for
 * gridspt_bispectrum (which equals this call with b = a and c = b, bit for
 * bit). Each ordered term of the one-loop bispectrum (Eq. bk_1loop) is one
 * such sum; in equilateral shells B_1-loop = 6 E[d1, d2, d3] + E[d2, d2, d2]
 * + 3 E[d1, d1, d4]. */
gridspt_status gridspt_bispectrum_triple(gridspt_plan plan, const void* a_k, const void* b_k,
                                         const void* c_k, int32_t nbins, const double* edges,
                                         double* e_out, double* ntri_out, void* ws, size_t ws_bytes,
                                         gridspt_stream stream);

/* Launch batching (not part of the paper's method): the recursion of one or
 * several plans captured once as a single CUDA graph and replayed with one
 * launch. plans[i] may have different grid sizes, orders and batches; branch i
 * runs exactly the launches of gridspt_run_orders(plans[i], delta1_k[i],
 * start_order[i], spectra[i], ws[i], ws_bytes[i]) (same results, bit for bit),
 * and branches are independent, so realisations of different sizes run
 * concurrently. All pointers are device pointers as in gridspt_run_orders and
 * are baked into the graph: they must stay valid and must not overlap between
 * branches (in particular each branch needs its own workspace). Create,
 * launch and destroy are host calls; create captures on internal streams and
 * synchronises nothing; launch enqueues one graph launch on `stream`. */
typedef struct gridspt_batch_s* gridspt_batch;
gridspt_status gridspt_batch_create(const gridspt_plan* plans, int32_t count, const void* const* delta1_k,
                                    const int32_t* start_order, void* const* spectra, void* const* ws,
                                    const size_t* ws_bytes, gridspt_batch* out);
gridspt_status gridspt_batch_launch(gridspt_batch batch, gridspt_stream stream);
gridspt_status gridspt_batch_destroy(gridspt_batch batch);

/* Persistent work queue (not part of the paper's method): the recursion of one
 * or several plans, whose grid sizes may differ (e.g. 128^3, 192^3 and 256^3
 * realisations), in ONE launch of one persistent kernel.
 *   gridspt_multi_create records, for every plan i, the launches that
 *     gridspt_run_orders(plans[i], delta1_k[i], start_order[i] (NULL: all 2),
 *     spectra[i], ws[i], ws_bytes[i]) would make, as stages of tiles (column
 *     blocks, z row groups, cell blocks), and lays them out in one device-side
 *     queue: a plan's stages form a chain (each waits for its predecessor, so
 *     the realisations of a plan, which share ws[i], run one after another);
 *     chains of different plans are interleaved by their cumulative work.
 *     Host call; allocates and fills the queue's device table (about 1.7 KB a
 *     stage, ~25 stages per realisation at n_max = 5), owned by the returned
 *     object. Pointers are used as in gridspt_run_orders, must stay valid while
 *     the object is used and must not overlap between plans (each plan needs
 *     its own workspace). Supported: the nine-term form with N = 64, 96, 128,
 *     192 or 256 (GRIDSPT_E_UNSUPPORTED otherwise), plans on one device.
 *   gridspt_run_orders_multi enqueues one launch of the persistent kernel on
 *     `stream` (grid: as many 256-thread blocks as fit on the GPU at once). A
 *     block takes the next tile in queue order from a ticket counter, waits
 *     until the tile's predecessor stage has counted all its tiles done, runs
 *     the tile with the arithmetic of the pass's own kernel and counts it
 *     done. Results are bit for bit those of gridspt_run_orders for every plan.
 *     A wait only ever concerns earlier tickets, which running blocks hold, so
 *     it always ends; in addition every wait gives up after 1 s of GPU time:
 *     the block then sets the status word of plans[0] (gridspt_check(plans[0])
 *     returns GRIDSPT_E_TIMEOUT and the results are invalid) and every block
 *     returns. Calls on one object must not overlap on the GPU (they share its
 *     ticket and completion counters).
 *   gridspt_multi_destroy synchronises the device and frees the table. */
typedef struct gridspt_multi_s* gridspt_multi;
gridspt_status gridspt_multi_create(const gridspt_plan* plans, int32_t count, const void* const* delta1_k,
                                    const int32_t* start_order, void* const* spectra, void* const* ws,
                                    const size_t* ws_bytes, gridspt_multi* out);
gridspt_status gridspt_run_orders_multi(gridspt_multi multi, gridspt_stream stream);
gridspt_status gridspt_multi_destroy(gridspt_multi multi);

/* Autotuner for the transform passes (not part of the paper's method). Each
 * pass (0 forward column pass, 1 x expansion, 2 y expansion, 3 z expansion,
 * 4 contiguous-axis forward pass) has two variants for N >= 128 (identical for
 * smaller N). The x expansion has two more (2, 3) that transform two outputs
 * (and the two forward inputs) at a time in a shared exchange. The y
 * expansion has a third, TMA-staged one (N >= 128), a fourth with two
 * adjacent columns per thread (16-byte accesses), a fifth that copies the
 * next input's columns by cp.async during the current input's transforms, and
 * a sixth and seventh (5, 6) that transform two outputs of one input at a
 * time. The z
 * expansion and the contiguous-axis forward pass have a third that runs one z
 * row per group of warp lanes without block-wide barriers (power-of-two
 * N <= 512; other sizes run variant 0 when it is chosen); the z expansion's
 * choice also applies to the pair products fused into it and to the z pass of
 * the bispectrum shells. gridspt_autotune times the
 * variants of every pass on `scratch` (device, >= gridspt_autotune_scratch_size
 * bytes, contents overwritten) with CUDA events on `stream`, keeps the fastest
 * in the plan and writes the choices to choices_out (host int32[5], may be
 * NULL). It synchronises `stream`. gridspt_set_tuning / gridspt_get_tuning
 * store and read the choices (0 or 1; 0..3 for pass 1; 0..6 for pass 2; 0..2 for passes 3 and 4), e.g.
 * from a cache kept by the caller.
 * Results are bitwise identical for all variants: they only change how
 * columns and rows are grouped into thread blocks and warps. */
gridspt_status gridspt_autotune_scratch_size(gridspt_plan plan, size_t* bytes);
gridspt_status gridspt_autotune(gridspt_plan plan, void* scratch, size_t scratch_bytes, int32_t* choices_out,
                                gridspt_stream stream);
gridspt_status gridspt_set_tuning(gridspt_plan plan, const int32_t* choices);
gridspt_status gridspt_get_tuning(gridspt_plan plan, int32_t* choices);

/* P-term emulator network (not part of the paper's method): a multilayer
 * perceptron in -> hidden -> hidden -> out with SiLU after both hidden layers
 * and a linear output, used to emulate binned GridSPT P-terms as a function of
 * (sigma_8, n_s, Gamma). Parameters, one contiguous vector, row-major [in][out]
 * weights: W1[in][hidden], b1[hidden], W2[hidden][hidden], b2[hidden],
 * W3[hidden][out], b3[out]. `bf16` = 1: the parameter copy read by
 * forward/backward is bfloat16 and hidden activations are rounded to bfloat16;
 * 0: FP32. Every product is accumulated in FP32. Limits: 1 <= in <= 8,
 * 1 <= hidden, out <= 256, batch >= 1. All arrays are device arrays.
 *   x [batch][in], y [batch][out] (FP32);
 *   act: NULL, or FP32 [batch][4 * hidden] saved activations (z1, a1, z2, a2)
 *        for gridspt_mlp_backward.
 * gridspt_mlp_backward: grad = d(sum(dy * y)) / d params (FP32, parameter
 * layout), from x, the parameter copy, act and dy [batch][out]; per-block
 * partial gradients in ws are summed in a fixed order (bitwise repeatable).
 * gridspt_mlp_mse: dy = 2 mask (y - t) / sum(mask), loss = sum(mask (y - t)^2)
 * / sum(mask) over n elements (loss: device float, may be NULL).
 * gridspt_mlp_adam: increments the device step counter *step, then one Adam
 * update (Kingma & Ba 2015, bias-corrected) of the FP32 master parameters and
 * moments m, v; writes the updated parameter copy (bf16 or FP32) if
 * params_lowp is not NULL. gridspt_mlp_convert writes that copy from master. */
gridspt_status gridspt_mlp_param_count(int32_t in, int32_t hidden, int32_t out, int64_t* count);
gridspt_status gridspt_mlp_forward(const float* x, int32_t batch, int32_t in, int32_t hidden, int32_t out,
                                   const void* params, int32_t bf16, float* y, float* act, gridspt_stream stream);
gridspt_status gridspt_mlp_backward_workspace_size(int32_t batch, int32_t in, int32_t hidden, int32_t out,
                                                   size_t* bytes);
gridspt_status gridspt_mlp_backward(const float* x, int32_t batch, int32_t in, int32_t hidden, int32_t out,
                                    const void* params, int32_t bf16, const float* act, const float* dy,
                                    float* grad, void* ws, size_t ws_bytes, gridspt_stream stream);
gridspt_status gridspt_mlp_mse(const float* y, const float* target, const float* mask, int64_t n, float* dy,
                               float* loss, gridspt_stream stream);
gridspt_status gridspt_mlp_adam(float* master, void* params_lowp, int32_t bf16, const float* grad, float* m,
                                float* v, int32_t* step, int64_t n, float lr, float beta1, float beta2, float eps,
                                gridspt_stream stream);
gridspt_status gridspt_mlp_convert(const float* master, void* params_lowp, int32_t bf16, int64_t n,
                                   gridspt_stream stream);

/* Launch profiling (tracing aid, not part of the paper's method). Between
 * gridspt_profile_begin and gridspt_profile_end every kernel the library
 * launches is bracketed by two CUDA events recorded on its launch stream, and
 * the algorithmic bytes of the launch (each input field read once, each output
 * written once) are noted. gridspt_profile_end waits for the recorded events
 * and returns, per kernel kind, the number of launches, the summed event time
 * in ms and the summed algorithmic bytes (up to `capacity` entries, `*count`
 * set to the number written). Host calls; not for use inside stream capture.
 * Process-wide; at most 65536 launches are recorded per session. */
typedef struct {
    char name[24];
    int32_t launches;
    int32_t reserved;
    double ms;
    double bytes;
} gridspt_kernel_stat;
gridspt_status gridspt_profile_begin(void);
gridspt_status gridspt_profile_end(gridspt_kernel_stat* stats, int32_t capacity, int32_t* count);

/* Device-side status: synchronises `stream` and reads the plan's status word,
 * which the plan's kernels set since the last check:
 * - GRIDSPT_E_TIMEOUT if a bounded device-side wait (the mbarrier waits of the
 *   TMA-staged passes, or the self-test's) gave up; the results of those calls
 *   are invalid;
 * - else GRIDSPT_E_NUMERIC if a power, cross-correlation or bispectrum result
 *   was NaN or infinite (a non-finite value in an input spectrum inside the
 *   bins reaches the result; values outside every bin are not seen);
 * - GRIDSPT_OK otherwise. The status is reset by the call. */
gridspt_status gridspt_check(gridspt_plan plan, gridspt_stream stream);

/* Failure-detection self-test (not part of the paper's method): launches one
 * block that waits, with the same bounded wait as the TMA-staged passes, on a
 * barrier that is never completed. The wait gives up (about 1 ms), the kernel
 * records the timeout and returns; the next gridspt_check reports
 * GRIDSPT_E_TIMEOUT. Nothing faults or hangs. */
gridspt_status gridspt_selftest_bounded_wait(gridspt_plan plan, gridspt_stream stream);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char* gridspt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GRIDSPT_H */
