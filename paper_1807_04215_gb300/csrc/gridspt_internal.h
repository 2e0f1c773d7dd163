// Internal launcher interface between the host runtime (api.cpp) and the CUDA
// kernels. Host-only C++: no CUDA device code here.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace gridspt {

constexpr int kMaxBins = 64;
constexpr int kMaxOrder = 8;
// Blocks of the power estimator's first kernel (one warp per (kx, ky) row,
// grid-stride): power_blocks() never exceeds this, and the allocation-free
// entry point's static scratch is sized by it.
constexpr int kPowerMaxBlocks = 1216;

// Bits of the plan's device status word (read and cleared by gridspt_check).
constexpr int kStatusWaitTma = 1;       // a bounded mbarrier wait of a TMA-staged pass gave up
constexpr int kStatusWaitSelftest = 2;  // the bounded-wait self-test's wait gave up
constexpr int kStatusNonFinite = 4;     // an estimator produced a NaN or infinite result

// Shell-sum accumulation of the estimators (gridspt_desc.accum).
constexpr int kAccumCompensated = 0;    // FP32 sums with carried rounding error, finished in FP64
constexpr int kAccumFp64 = 1;           // every term added in FP64
constexpr int kMaxDeriveOut = 17;

// Grid geometry shared by every launch. Half spectra are float2[N][N][M],
// M = N / 2 (kz = 0..M-1); real fields float[N][N][N]; both 4 N^3 bytes.
// Transform-pass tile variants chosen by the autotuner (0 = default).
enum TunePass : int { TV_COLPASS = 0, TV_XEXP = 1, TV_YEXP = 2, TV_ZEXP = 3, TV_ZR2C = 4, TV_COUNT = 5 };

struct Geo {
    int N;
    int M;
    double kF;              // 2 pi / L
    const float2* tw;       // device table e^{+2 pi i j / N}, j < N (FP32 from FP64)
    int var[TV_COUNT];      // tile variant per transform pass
    int* status;            // device status word (kStatus* bits)
    int accum;              // estimator shell sums: kAccumCompensated or kAccumFp64
};

// number of tile variants per pass (the autotuner times each; results are
// bitwise equal across them):
//   column pass: 0 wide tile, 1 narrow tile;
//   x expansion: 0 wide tile, 1 narrow tile, 2 narrow and 3 wide tile with
//                two outputs per transform (fft_column_pair);
//   y expansion: 0, 1 tiles, 2 TMA-staged tiles, 3 two columns per thread,
//                4 narrow tile with cp.async prefetch of the next input,
//                5 narrow and 6 wide tile with two outputs per transform;
//   z expansion (and the fused pair products, bispectrum z pass): 0 tile,
//                1 tile with cp.async prefetch, 2 warp rows;
//   z forward pass: 0, 1 tiles, 2 warp rows.
constexpr int kTuneVariants[TV_COUNT] = {2, 4, 7, 3, 3};

// Unit of the wavevector in the derivative multipliers of the expansion
// passes: k_F, i.e. integer wavevectors s. Every source term of Eq.
// recursion_formula pairs one derivative (i k) with one inverse derivative
// (-i k / k^2) or none (d_a d_b / nabla^2, delta theta), so k_F cancels from
// A_n, B_n exactly and the stored derived fields need no physical unit. With
// integer s the cancellations the sources rely on (grad delta . u + delta
// theta and the u-tensor terms at k -> 0, mass and momentum conservation) are
// exact up to the rounding of 1/|s|^2 per mode; a physical k_F would carry
// the FP32 rounding of k_F^2 * (1 / k_F^2) - 1 coherently into every mode and
// leave a relative error growing as 1/k^2 in the low-k part of delta_3, which
// P13 = 2 <delta_1 delta_3> measures.
constexpr float kDerivUnit = 1.0f;

// Factorised spectral derivatives (Sec. II.C steps (2) and (5)). Every
// derived field is c * kx^a * ky^b * kz^g * src(k) with src in {delta, theta,
// phi = theta / k^2} and c in {1, i, -i}. Factors of (ky, kz) commute with the
// transform along x and factors of kz with the transform along y, so the
// backward transform is split into three expansion passes:
//   x pass: kx^a * src (or a shell mask), transformed along x    ("x-fields")
//   y pass: ky^b * x-field, transformed along y                    ("xy-fields")
//   z pass: c * kz^g * xy-field, half-complex -> real along z      (real fields)
// Each pass reads every input once and writes every output once.
constexpr int kMaxExpOut = 17;
enum XKind : int { XK_POW = 0, XK_SHELL = 1 };
enum XSrc : int { XS_DELTA = 0, XS_THETA = 1, XS_PHI = 2, XS_ONE = 3 };
// x pass code: kind | a << 4 | src << 8
constexpr int x_code(int kind, int a, int src) { return kind | (a << 4) | (src << 8); }
// y pass code: input index | b << 8 | output slot << 16
constexpr int y_code(int in, int b, int slot) { return in | (b << 8) | (slot << 16); }
// z pass code: input index | g << 8 | c << 12 | output slot << 16  (c: 0 -> 1, 1 -> i, 2 -> -i)
constexpr int z_code(int in, int g, int c, int slot) { return in | (g << 8) | (c << 12) | (slot << 16); }

struct XExpArgs {
    float2* src0;          // delta spectrum (x-column layout [kx][ky][kz])
    float2* src1;          // theta spectrum (may equal src0)
    float2* out;           // output field f at out + f * out_stride
    long long out_stride;  // float2 elements between output fields
    int nout;
    int codes[kMaxExpOut];
    int fwd_first;         // 1: inputs hold [x][ky][kz] data; transform forward along x,
                           //    finalise (zero Nyquist, optional cut) and store back in place
    long long s2_nl;       // finalise: zero modes with |s|^2 > s2_nl (< 0: no cut)
    int zero_k0;           // finalise: also write the k = 0 mode as zero (orders n >= 2,
                           //    whose k = 0 mode vanishes exactly: mass conservation)
    long long shell_lo;    // XK_SHELL: 0 < |s|^2, lo <= |s|^2 < hi
    long long shell_hi;
    int band;              // > 0: only columns with |ky| < band and kz < band are
                           //      read, transformed and written; the others are left
                           //      untouched (their exact values are zero: the
                           //      caller zeroes them where it needs them)
    long long s2_in = -1;  // backward pass (fwd_first = 0), >= 0: input modes with
                           //      |s|^2 > s2_in are taken as zero (the cut on delta_1)
    // divergence-form sources (fwd_first = 1): when div_in is set, the inputs are
    // the y-transformed V_x, V_y, V_z, S at div_in + q * div_stride (q = 0..3);
    // after the forward x transform A = i k . V, B = -(k^2 / 2) S and
    // src0 = cdA A + cdB B, src1 = ctA A + ctB B are written (then finalised)
    const float2* div_in;
    long long div_stride;
    float cdA, cdB, ctA, ctB;
};

struct YZExpArgs {
    const float2* in;      // input field i at in + i * in_stride
    long long in_stride;
    float2* out;           // output field f at out + f * out_stride
    long long out_stride;
    int nout;
    int codes[kMaxExpOut]; // outputs of the same input must be consecutive; each
                           // is written to out + slot * out_stride
    int band;              // y pass, > 0: inputs nonzero only at |ky| < band and
                           //      kz < band; only kz < band columns are formed.
                           // z pass, > 0 and even: inputs nonzero only at kz < band
                           //      (only those are read); every real output is formed
};

struct IcArgs {
    float2* out;           // one realisation
    uint64_t seed;
    double amp;            // A of P(k) = A k^ns T^2
    double n_s;
    double gamma;
    double inv_vol;        // 1 / L^3
    long long s2_cut;      // keep 0 < |s|^2 <= s2_cut
    double* table;         // [s2_cut + 1]: sqrt(P(k_F sqrt(s2)) / L^3) / sqrt(2), made by launch_ic_table
    double kF;
};

// z expansion fused with accumulate-ahead pair products (Eq. recursion_formula):
// while the real derived fields of order m are formed one by one, each is
// multiplied with its partner fields of stored lower orders j and summed into
// A_{m+j}, B_{m+j}. Target t ends either in accumulator fields (partial) or,
// for its last pair, in delta_n, theta_n.
constexpr int kMaxPairTargets = 2;
constexpr int kMaxPartners = 3;      // partner fields of one output over a launch's targets
struct PairTarget {
    const float* partner;       // stored real fields of order j: field f at partner + f * cells
    const float* acc_in_a;      // partial A, B from earlier pairs (NULL: none)
    const float* acc_in_b;
    float* out_a;               // out_a = ca0 A + ca1 B, out_b = cb0 A + cb1 B
    float* out_b;
    float ca0, ca1, cb0, cb1;
    int pcount[17];             // per produced slot: number of partner fields (0..2)
    int pfield[17][2];          // partner field index in the stored order; -1: the produced field
                                // itself (a square), no partner rows are read
    float pcoef_a[17][2];       // contribution coefficients to A and B
    float pcoef_b[17][2];
};
struct ZPairArgs {
    YZExpArgs z;                // inputs (xy-fields) and output list (slot = derived-field slot)
    float* store;               // real fields of this order (slot s at store + s * cells) or NULL
    long long cells;            // N^3
    int ntargets;
    PairTarget t[kMaxPairTargets];
};
cudaError_t launch_zexp_pairs(const Geo& g, const ZPairArgs& a, cudaStream_t s);

struct ProductArgs {
    const float* ws;       // derived fields; order m field j at ws + (base[m] + j) * cells
    long long cells;       // N^3
    int base[kMaxOrder + 1];
    int n;                 // order being formed
    float* out_delta;      // real field written (4 N^3 bytes)
    float* out_theta;
    float cdA, cdB, ctA, ctB;  // recursion coefficients times N^-3
    int diag_only;             // > 0: only the pair (diag_only, diag_only)
};

struct BinSpec {
    int nbins;
    int thr[kMaxBins + 1]; // bin i holds thr[i] <= |s|^2 < thr[i+1]
};

cudaError_t launch_ic(const Geo& g, const IcArgs& a, cudaStream_t s);
// The mode amplitude of every |s|^2 <= s2_cut into a.table (once per call of
// gridspt_make_linear_field; it depends on the spectrum, not on the seed).
cudaError_t launch_ic_table(const IcArgs& a, cudaStream_t s);
// One block waits on an mbarrier that nothing completes; the bounded wait gives
// up and sets *status (exercises the timeout path without hanging the GPU).
cudaError_t launch_wait_selftest(int* status, cudaStream_t s);
cudaError_t launch_xexp(const Geo& g, const XExpArgs& a, cudaStream_t s);
cudaError_t launch_yexp(const Geo& g, const YZExpArgs& a, cudaStream_t s);
cudaError_t launch_zexp(const Geo& g, const YZExpArgs& a, cudaStream_t s);
// Forward column transform along x (axis 0) or y (axis 1) of `count` fields,
// in place. finalize (x axis): 1 zeroes the Nyquist modes and |s|^2 > s2_nl
// (s2_nl < 0: no cut); 2 also the k = 0 mode (orders n >= 2 of the recursion).
// band > 0 (y axis, 0 < band < N/2): only the columns kz < band are
// transformed and only their rows |ky| < band written; the rest is left as is.
cudaError_t launch_colpass_fwd(const Geo& g, float2* data, long long fstride, int count, int axis,
                               int finalize, long long s2_nl, int band, cudaStream_t s);
// Contiguous-axis real-to-complex with output scale; band > 0 (< N/2): only
// the coefficients kz < band are written.
cudaError_t launch_zr2c(const Geo& g, const float2* in, float2* out, long long fstride, int count,
                        float scale, int band, cudaStream_t s);
cudaError_t launch_product(const Geo& g, const ProductArgs& a, cudaStream_t s);

// Divergence-form sources of order n: V_n = sum_m delta_m u_{n-m} (3 fields) and
// S_n = sum_m u_m . u_{n-m}, times `scale`, from the stored real fields of the
// lower orders (order m: delta, u_x, u_y, u_z at ws + (4 (m - 1) + j) * cells).
struct ProductDivArgs {
    const float* ws;
    long long cells;
    int n;
    float* out;            // V_x, V_y, V_z, S at out + q * cells
    float scale;           // N^-3 (the forward transform is unnormalised)
};
cudaError_t launch_product_div(const Geo& g, const ProductDivArgs& a, cudaStream_t s);

// delta_SPT = W(k R) sum_i coef[i] field[i] over one half spectrum (k_fields.cu)
struct SumOrdersArgs {
    const float2* field[kMaxOrder];
    float coef[kMaxOrder];
    int n;                 // number of fields
    int N;
    float r2kf2;           // (R k_F)^2; 0: no filter
    float2* out;
};
cudaError_t launch_sum_orders(const SumOrdersArgs& a, cudaStream_t s);
// Zero the modes of two half spectra of size N outside the band columns
// (|ky| < band and kz < band, band even, 0 < band < N/2).
cudaError_t launch_zero_outside_band(float2* f0, float2* f1, int N, int band, cudaStream_t s);
// r[i] = pab[i] / sqrt(paa[i] pbb[i]) (0 where the denominator vanishes), nbins <= 64
cudaError_t launch_rcorr(const double* pab, const double* paa, const double* pbb, int nbins, double* r,
                         cudaStream_t s);

// Power: per-block partial sums (2 * nbins doubles per block) then a fixed-order
// final reduction. blocks: number of partial-sum blocks (power_blocks()).
int power_blocks(const Geo& g);
cudaError_t launch_power(const Geo& g, const float2* a, const float2* b, const BinSpec& bins,
                         double* partial, double* p_out, int64_t* nk_out, double volume,
                         cudaStream_t s);
// Bispectrum, one shell: z transform of the xy-fields I_a, I_b (and I_c when
// triple; then J when present; kz < band) fused with the sums of I_a^2 I_b or
// I_a I_b I_c (and J^3), per-block partials, then the fixed-order final
// reduction. nfields counts the data fields and J. sum J^3 does not depend on
// the data: with has_j (nfields 3 in the final kernel's convention) the final
// kernel stores it in *j3_cache, otherwise it reads it from there.
int shell_blocks(const Geo& g);
cudaError_t launch_zshell(const Geo& g, const float2* in, long long in_stride, int band, int nfields, int triple,
                          double* partial, cudaStream_t s);
cudaError_t launch_bispec_final(const Geo& g, const double* partial, int blocks, int nfields, double* j3_cache,
                                double* e_out, double* ntri_out, double vol2, cudaStream_t s);
// Copy the modes of nin half spectra of size N (in[f]) onto a smaller grid of
// size S (out + f * out_stride, half-spectrum layout of size S): mode s with
// every component in (-S/2, S/2) keeps its value, the Nyquist planes of the
// small grid are zero. S <= N, both supported sizes, nin <= 3.
cudaError_t launch_subgrid(int N, int S, const float2* const* in, int nin, float2* out, long long out_stride,
                           cudaStream_t s);

bool supported_n(int N);
// The supported grid sizes in increasing order (kNumSizes of them).
constexpr int kNumSizes = 15;
constexpr int kSizes[kNumSizes] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};

// emulator network (k_mlp.cu)
long long mlp_params(int I, int H, int O);
int mlp_bwd_blocks(int B);
cudaError_t launch_mlp_forward(const float* x, int B, int I, int H, int O, const void* theta, int bf16, float* y,
                               float* act, cudaStream_t s);
cudaError_t launch_mlp_backward(const float* x, int B, int I, int H, int O, const void* theta, int bf16,
                                const float* act, const float* dy, float* part, float* grad, cudaStream_t s);
cudaError_t launch_mlp_mse(const float* y, const float* t, const float* mask, long long n, float* dy, float* loss,
                           cudaStream_t s);
cudaError_t launch_mlp_adam(float* master, void* lowp, int bf16, const float* grad, float* m, float* v, int* step,
                            long long n, float lr, float b1, float b2, float eps, cudaStream_t s);
cudaError_t launch_mlp_convert(const float* src, void* dst, int bf16, long long n, cudaStream_t s);

// ------------------------------------------------ persistent work queue
// The recursion of several plans (grid sizes may differ) as one launch of a
// persistent kernel (k_persistent.cu): every launch that gridspt_run_orders
// would make becomes a stage of tiles in a device-side queue, stages of one
// plan form a chain (each waits for its predecessor), chains of different
// plans are interleaved by their cumulative work. Blocks take tiles in queue
// order from a ticket counter; a tile first waits (bounded) for its stage's
// predecessor to complete, runs, and counts itself done.
enum QKind : int {
    Q_XEXP0 = 0,   // x expansion, backward only (x)
    Q_XEXP1,       // x expansion, forward first (x)
    Q_YEXP,        // y expansion (y)
    Q_Z,           // z expansion, store only or fused pair products (z)
    Q_ZR2C,        // contiguous-axis forward transform (r2c: data, count, scale)
    Q_COLY,        // forward column pass along y (data, count)
    Q_COLX,        // forward column pass along x with finalise (data, count, s2, zero_k0)
    Q_PRODUCT,     // diagonal pair (pr)
    Q_ZEROBAND,    // zeros outside the band columns (data, data2, band)
    Q_KINDS
};
constexpr int kQueueThreads = 256;
constexpr int kStatusWaitQueue = 8;     // a work-queue tile's wait for its predecessor gave up
struct QStage {
    int kind;
    int N;
    int dep;               // stage this one waits for (-1: none)
    int nosignal;          // fault injection: this stage never counts its tiles done
    long long ntiles;
    long long chunk;       // tiles per ticket (set by the host: larger stages take several per ticket)
    long long nticks;      // tickets of the stage, ceil(ntiles / chunk)
    long long tile0;       // first ticket of the stage
    int gx, gy;            // virtual grid of the column passes (tile = bx + gx (by + gy bz))
    int count;             // fields of Q_ZR2C / Q_COLY / Q_COLX
    int zero_k0;           // Q_COLX
    int band;              // Q_ZEROBAND
    long long s2;          // Q_COLX: s2_nl
    float scale;           // Q_ZR2C
    float kF, inv_kF2;
    const float2* tw;
    float2* data;          // Q_ZR2C (in place), Q_COLY, Q_COLX, Q_ZEROBAND (first field)
    float2* data2;         // Q_ZEROBAND (second field)
    long long fstride;
    double cost;           // work estimate (algorithmic bytes), host only
    XExpArgs x;
    YZExpArgs y;
    ZPairArgs z;
    ProductArgs pr;
};
// Supported grid sizes of the queue kernel (its tile bodies are instantiated
// for these); false for the others.
bool queue_supported_n(int N);
// Tiles of a stage whose kind, N and arguments are set (fills gx, gy, ntiles;
// chunk = 1).
void queue_tiles(QStage& st);
// Launch over `nst` stages already in device memory (stages, starts[nst + 1]
// first tickets with starts[nst] = total), with hdr (4 + nst ints, zeroed by
// this call on `s`): ticket counter, abort flag, per-stage done counters.
cudaError_t launch_queue(const QStage* stages, const long long* starts, int nst, long long total, int* hdr,
                         int* status, long long wait_ns, cudaStream_t s);
size_t queue_smem_bytes();

// Library-owned scratch of the allocation-free power entry point
// (k_power_static.cu): device address of the static array on the current
// device (looked up once per device), its size, and whether a request fits.
cudaError_t power_static_scratch(double** out);
size_t power_static_scratch_bytes();
bool power_static_fits(const Geo& g, int nbins);

}  // namespace gridspt
