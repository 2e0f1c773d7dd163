// 3D real<->half-complex transforms of the GridSPT path, as three axis passes.
//
// Layouts (every array is 4 N^3 bytes, no padding):
//   half spectrum / mixed data: float2[N][N][M], M = N / 2, index [x|kx][y|ky][kz]
//   real field:                 float[N][N][N]
// Backward (Sec. II.C synthesis sum a(x) = sum_k a(k) e^{i k.x}), with the
// spectral-derivative multipliers of steps (2)/(5) factorised over the axes:
//   k_xexp  x pass: kx^a * {delta, theta, phi = theta/k^2} (or a shell mask)
//   k_yexp  y pass: ky^b * x-field
//   k_zexp  z pass: c kz^g * xy-field, half-complex -> real
// Forward (analysis sum, N^-3 folded into the producer): k_zr2c, then
// k_colpass along y, then along x (k_colpass with finalise, or k_xexp with
// fwd_first, which also starts the next order's backward expansion).
//
// Column passes stage a tile of TZ adjacent kz columns (TZ * 8 contiguous bytes
// per row of the column) and keep each column in registers (fft_core.cuh).
// The contiguous-axis passes use the half-length complex transform of the
// packed sequence z[m] = x[2m] + i x[2m+1]; the Nyquist coefficient X[N/2] is
// zero in every spectrum of this library and is not stored.
#pragma once
#include <cuda.h>

#include "fft_core.cuh"
#include "gridspt_internal.h"

namespace gridspt {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Tile widths. Variant 0 is the default; variant 1 is the alternative width
// the autotuner also times (only instantiated separately for N >= 128). For
// the z expansion variant 1 keeps the tile width and instead prefetches the
// next input tile with cp.async. Further variants per pass are listed with
// kTuneVariants (TMA-staged, column-pair and prefetching y passes; warp-row z
// passes).
template <int N>
struct Cfg {
    static constexpr int M = N / 2;
    // column passes (length N): TZ adjacent kz columns per block
    static constexpr int EC = fft_elems(N);
    static constexpr int PC = N / EC;
    static constexpr int TZC0 = cmin(16, 1024 / PC);
    static constexpr int TZC1 = N >= 128 ? cmax(4, TZC0 / 2) : TZC0;
    // contiguous-axis passes (length M): TZ rows per block. 16 rows or more:
    // a warp then spans 16 rows of the odd-pitch tile, so column accesses of
    // a warp hit 16 distinct 8-byte bank pairs
    static constexpr int EZ = fft_elems(M);
    static constexpr int PZ = M / EZ;
    static constexpr int TZZ0 = cmin(cmin(64, cmax(16, 256 / PZ)), 1024 / PZ);
    static constexpr int TZZ1 = N >= 128 ? (2 * TZZ0 * PZ <= 1024 ? 2 * TZZ0 : cmax(16, TZZ0 / 2)) : TZZ0;
    static constexpr int PITCH = M + 1;
    // fused z pass with pair products: five tiles (input, exchange, 3 partners)
    // must fit the 227 KB a block may hold; halve the row count until they do
    static constexpr size_t pair_smem(int tz) { return sizeof(float2) * (N + 5 * (size_t)tz * PITCH); }
    static constexpr int TZP = pair_smem(TZZ0) <= 232448 ? TZZ0
                             : pair_smem(TZZ0 / 2) <= 232448 ? TZZ0 / 2 : TZZ0 / 4;
    static_assert(pair_smem(TZP) <= 232448, "fused z pass tiles exceed shared memory");
};

// Shared memory of the column passes (colpass, x and y expansion): the
// lane-major stage-twiddle table of fft_col, then NB exchange buffers of
// col_rows(N) rows of TZ columns (W = 2: column pairs, 16-byte elements), then
// EXTRA float2 (the y pass's prefetch tile). Two buffers (one barrier per
// exchange) whenever they fit the 227 KB a block may hold; a variant whose
// tiles do not fit even with one buffer (the wide column-pair tile of N = 768)
// is not built for that size.
template <int N, int TZ, int W = 1, int EXTRA = 0>
struct ColSm {
    static constexpr int P = N / fft_elems(N);
    static constexpr int TW = (fft_row_tw_total<N>() * P + 1) / 2 * 2;   // 16-byte multiple
    static constexpr int BUF = col_rows(N) * TZ * W;
    static constexpr size_t bytes_nb(int nb) { return sizeof(float2) * (TW + (size_t)nb * BUF + EXTRA); }
    static constexpr bool fits = bytes_nb(1) <= 232448;
    static constexpr int NB = bytes_nb(2) <= 232448 ? 2 : 1;
    static constexpr size_t bytes = bytes_nb(NB);
};

// Shared memory of the forward column pass (one transform per block, so the
// plain fft_column with one exchange buffer and the table of N-th roots).
template <int N, int TZ>
__host__ __device__ constexpr size_t colpass_smem() { return sizeof(float2) * (N + (size_t)N * TZ); }

// Blocks per SM the expansion column passes are compiled for: two 512-thread
// blocks (64 registers a thread) for the narrow tile of power-of-two N >= 512,
// where one block of the natural ~75-86 registers leaves 16 warps per SM; one
// elsewhere (smaller N and radix-3 sizes would spill heavily).
template <int N, int TZ>
__host__ __device__ constexpr int col_min_blocks() {
    return (fft_elems(N) == 8 && N >= 512 && TZ * (N / fft_elems(N)) <= 512) ? 2 : 1;
}

__device__ __forceinline__ int signed_idx(int n, int N) { return n < N / 2 ? n : n - N; }

__device__ __forceinline__ void load_table(float2* tw, const float2* __restrict__ twg, int N) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
}

// Asynchronous 8-byte global -> shared copies (cp.async, Ampere and later);
// src_bytes = 0 fills the destination with zeros.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Hint: bring the 128-byte line of p into L2 (no registers, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Issue (without waiting) the copy of TZ rows of M float2 into a shared tile.
template <int M, int TZ, int PITCH, int NTHR>
__device__ __forceinline__ void tile_prefetch(float2* tile, const float2* src, long long row0, long long rows) {
    constexpr int NV = TZ * M;
    constexpr int PER = (NV + NTHR - 1) / NTHR;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NTHR;
        if (idx < NV) {
            const int r = idx / M, j = idx - r * M;
            const long long row = row0 + r;
            const bool ok = row < rows;
            cp_async8(tile + r * PITCH + j, src + (ok ? row * M + j : 0), ok ? 8 : 0);
        }
    }
    cp_async_commit();
}

// Copy TZ contiguous rows of M float2 between global memory and a shared tile
// of odd pitch PITCH. Consecutive threads move consecutive float2 of a row
// (coalesced, conflict-free); all loads are issued before the shared stores,
// so each thread has TZ * M / NTHR requests in flight. band > 0: only the
// first band entries of each row are read, the rest of the tile row is zero.
template <int M, int TZ, int PITCH, int NTHR>
__device__ __forceinline__ void tile_load(float2* tile, const float2* src, long long row0, long long rows,
                                          int band = 0) {
    constexpr int NV = TZ * M;
    constexpr int PER = (NV + NTHR - 1) / NTHR;
    float2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NTHR;
        const int r = idx / M, j = idx - r * M;
        const long long row = row0 + r;
        v[u] = (idx < NV && row < rows && (band <= 0 || j < band)) ? src[row * M + j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NTHR;
        if (idx < NV) {
            const int r = idx / M, j = idx - r * M;
            tile[r * PITCH + j] = v[u];
        }
    }
}

template <int M, int TZ, int PITCH, int NTHR>
__device__ __forceinline__ void tile_store(float2* dst, const float2* tile, long long row0, long long rows) {
    constexpr int NV = TZ * M;
    constexpr int PER = (NV + NTHR - 1) / NTHR;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NTHR;
        const int r = idx / M, j = idx - r * M;
        const long long row = row0 + r;
        if (idx < NV && row < rows) dst[row * M + j] = tile[r * PITCH + j];
    }
}

// ------------------------------------------------- forward column pass
// The pass bodies below take their block coordinates (bx, by, bz) and shared
// memory explicitly, so that the same code runs as a kernel of its own (block
// coordinates from blockIdx) and as a tile of the persistent work-queue kernel
// (k_persistent.cu); the block has TZ * P threads either way. table_ready:
// the twiddle table already sits at the start of sm (a previous tile of the
// same size and table layout in the same block loaded it, and every thread
// has passed a block barrier since).
// band > 0 (y axis): only the columns kz < band are transformed, and only the
// rows |ky| < band of them are written (a band-limited order, whose x pass
// reads only those and whose spectra are zeroed outside them afterwards).
template <int N, int TZ, int AXIS, bool FIN>
__device__ __forceinline__ void colpass_body(float2* __restrict__ data, long long fstride,
                                             const float2* __restrict__ twg, long long s2_nl, int zero_k0,
                                             int band, int bx, int by, int bz, float2* sm,
                                             bool table_ready = false) {
    constexpr int M = N / 2, E = fft_elems(N), P = N / E;
    float2* tw = sm;
    float2* buf = sm + N;
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    if (!table_ready) load_table(tw, twg, N);
    const int kz = bx * TZ + c;
    const int a = by;
    const bool act = kz < M && (band <= 0 || kz < band);
    constexpr long long estride = AXIS == 0 ? (long long)N * M : (long long)M;
    constexpr long long astride = AXIS == 0 ? (long long)M : (long long)N * M;
    float2* col = data + bz * fstride + a * astride + kz;
    float2 x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = act ? col[(p + P * i) * estride] : make_float2(0.f, 0.f);
    __syncthreads();
    fft_column<N, -1, N>(x, p, buf + c, TZ, tw);
    if constexpr (FIN) {
        const int sy = signed_idx(a, N), sz = kz;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n = p + P * i;
            const int sx = signed_idx(n, N);
            const long long s2 = (long long)sx * sx + (long long)sy * sy + (long long)sz * sz;
            if (n == N / 2 || a == N / 2 || (s2_nl >= 0 && s2 > s2_nl) || (zero_k0 && s2 == 0))
                x[i] = make_float2(0.f, 0.f);
        }
    }
    if (act) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n = p + P * i;
            if (band <= 0 || n < band || n > N - band) col[(p + P * i) * estride] = x[i];
        }
    }
}

template <int N, int TZ, int AXIS, bool FIN>
__global__ void __launch_bounds__(TZ * Cfg<N>::PC)
k_colpass(float2* __restrict__ data, long long fstride, const float2* __restrict__ twg,
          long long s2_nl, int zero_k0, int band) {
    extern __shared__ float2 sm[];
    colpass_body<N, TZ, AXIS, FIN>(data, fstride, twg, s2_nl, zero_k0, band, blockIdx.x, blockIdx.y, blockIdx.z,
                                   sm);
}

// ------------------------------------------------ contiguous axis: R2C
template <int N, int TZ>
__global__ void __launch_bounds__(TZ * Cfg<N>::PZ)
k_zr2c(const float2* in, float2* out, long long fstride, const float2* __restrict__ twg, float scale, int band) {
    constexpr int M = N / 2, E = fft_elems(M), P = M / E, PITCH = Cfg<N>::PITCH;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* tile = sm + N;
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    load_table(tw, twg, N);
    const long long rows = (long long)N * N;
    const long long row0 = (long long)blockIdx.x * TZ;
    const float2* src = in + blockIdx.y * fstride;
    float2* dst = out + blockIdx.y * fstride;
    tile_load<M, TZ, PITCH, TZ * P>(tile, src, row0, rows);
    __syncthreads();
    float2* colp = tile + c * PITCH;
    float2 x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = colp[p + P * i];
    __syncthreads();
    fft_column<M, -1, N>(x, p, colp, 1, tw);
#pragma unroll
    for (int i = 0; i < E; ++i) colp[p + P * i] = x[i];
    __syncthreads();
    const float half = 0.5f * scale;
    constexpr int NV = TZ * M, NTHR = TZ * P, PER = (NV + NTHR - 1) / NTHR;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = tid + u * NTHR;
        const int r = idx / M, k = idx - r * M;
        const long long row = row0 + r;
        if (idx >= NV || row >= rows || (band > 0 && k >= band)) continue;
        const float2 Z = tile[r * PITCH + k];
        const float2 Zr = cconj(tile[r * PITCH + (k ? M - k : 0)]);
        const float2 S = cadd(Z, Zr);                      // 2 E[k]
        const float2 t = cmul(cconj(tw[k]), csub(Z, Zr));  // e^{-2 pi i k/N} 2i O[k]
        // X = E + e^{-2 pi i k / N} O = (S - i t) / 2
        dst[row * M + k] = make_float2(half * (S.x + t.y), half * (S.y - t.x));
    }
}

// ------------------------------------------------------------ x expansion
// Blocks per SM: col_min_blocks (a small spill at 64 registers), except for
// the divergence form, which keeps four input columns in registers.
template <int N, int TZ, int MODE>
__host__ __device__ constexpr int xexp_min_blocks() {
    return MODE != 2 ? col_min_blocks<N, TZ>() : 1;
}

// Inputs: delta(k) and theta(k) columns along kx. Each output f is
// kx^a * src (src = delta, theta, phi = theta / k^2 or 1) or a shell mask times
// src, transformed backward along x. With FWD the inputs first hold the
// y-transformed product output: they are transformed forward along x and
// finalised (delta_n(k), theta_n(k) complete, stored back in place), so the
// spectra are read from HBM once for both directions.
//
// MODE 0: backward x pass only; MODE 1: forward first (FWD above); MODE 2:
// forward first from the divergence-form sources: the four y-transformed
// fields V_x, V_y, V_z, S are transformed forward along x and combined into
// A = i k . V, B = -(k^2 / 2) S, delta = cdA A + cdB B, theta = ctA A + ctB B
// (written to src0, src1 and finalised like MODE 1).
// PAIR: consecutive outputs (and the two forward inputs) are transformed two
// at a time by fft_column_pair (shared twiddle loads and barriers, 16-byte
// exchanges of both transforms' elements; the exchange buffer is twice as
// large). Per output the arithmetic is that of fft_column, bit for bit.
template <int N, int TZ, int MODE, bool PAIR = false>
__device__ __forceinline__ void xexp_body(const XExpArgs& args, const float2* __restrict__ twg, float kF,
                                          float inv_kF2, int bx, int by, float2* sm, bool table_ready = false) {
    constexpr int M = N / 2, E = fft_elems(N), P = N / E;
    using CS = ColSm<N, TZ, PAIR ? 2 : 1>;
    constexpr int NB = CS::NB;
    float2* twl = sm;
    float2* bufA = sm + CS::TW;
    float2* bufB = bufA + CS::BUF;
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    float4* pairA = reinterpret_cast<float4*>(bufA) + c;
    float4* pairB = reinterpret_cast<float4*>(bufB) + c;
    if (!table_ready) col_twiddles<N, N>(twl, twg);
    const int kz = bx * TZ + c;
    const int B = args.band;
    const int ky = (B > 0 && by >= B) ? N - (2 * B - 1 - by) : by;   // band rows: [0, B) and (N - B, N)
    const bool act = kz < M && (B <= 0 || kz < B);
    constexpr long long estride = (long long)N * M;
    const long long colofs = (long long)ky * M + kz;
    const bool two = args.src1 != args.src0;
    float2 xd[E], xt[E];
    const int sy = signed_idx(ky, N), sz = kz;
    const int syz = sy * sy + sz * sz;
    // column `base` of this thread (MODE 0: with the cut on delta_1)
    auto load_col = [&](const float2* base, float2 (&v)[E]) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            v[i] = act ? base[colofs + (p + P * i) * estride] : make_float2(0.f, 0.f);
            if (MODE == 0 && args.s2_in >= 0) {
                const int sx = signed_idx(p + P * i, N);
                if ((long long)(sx * sx + syz) > args.s2_in) v[i] = make_float2(0.f, 0.f);
            }
        }
    };
    if constexpr (MODE == 2) {
        float2 A[E], Bs[E];
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const float2* col = args.div_in + q * args.div_stride + colofs;
            float2 v[E];
#pragma unroll
            for (int i = 0; i < E; ++i) v[i] = act ? col[(p + P * i) * estride] : make_float2(0.f, 0.f);
            fft_col<N, -1, NB>(v, p, bufA + c, bufB + c, TZ, twl);
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int sx = signed_idx(p + P * i, N);
                if (q < 3) {
                    const float kq = kF * (float)(q == 0 ? sx : (q == 1 ? sy : sz));
                    const float2 t = cmul_i<+1>(cscale(v[i], kq));            // i k_q V_q
                    A[i] = q == 0 ? t : cadd(A[i], t);
                } else {
                    const float k2 = kF * kF * (float)(sx * sx + syz);
                    Bs[i] = cscale(v[i], -0.5f * k2);                        // -(k^2 / 2) S
                }
            }
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
            xd[i] = make_float2(fmaf(args.cdA, A[i].x, args.cdB * Bs[i].x), fmaf(args.cdA, A[i].y, args.cdB * Bs[i].y));
            xt[i] = make_float2(fmaf(args.ctA, A[i].x, args.ctB * Bs[i].x), fmaf(args.ctA, A[i].y, args.ctB * Bs[i].y));
        }
    } else if constexpr (MODE == 1) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            xd[i] = act ? args.src0[colofs + (p + P * i) * estride] : make_float2(0.f, 0.f);
            xt[i] = (act && two) ? args.src1[colofs + (p + P * i) * estride] : xd[i];
        }
    } else {
        load_col(args.src0, xd);                          // theta is read when its outputs start
    }
    if constexpr (MODE >= 1) {
        if constexpr (MODE == 1) {
            if (PAIR && two) {
                float2 w[2][E];
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    w[0][i] = xd[i];
                    w[1][i] = xt[i];
                }
                fft_col_pair<N, -1, NB>(w, p, pairA, pairB, TZ, twl);
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    xd[i] = w[0][i];
                    xt[i] = w[1][i];
                }
            } else {
                fft_col<N, -1, NB>(xd, p, bufA + c, bufB + c, TZ, twl);
                if (two) fft_col<N, -1, NB>(xt, p, bufA + c, bufB + c, TZ, twl);
            }
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n = p + P * i;
            const int sx = signed_idx(n, N);
            const long long s2 = (long long)sx * sx + syz;
            if (n == N / 2 || ky == N / 2 || (args.s2_nl >= 0 && s2 > args.s2_nl) || (args.zero_k0 && s2 == 0)) {
                xd[i] = make_float2(0.f, 0.f);
                xt[i] = make_float2(0.f, 0.f);
            }
            if (!two) xt[i] = xd[i];
        }
        if (act) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                args.src0[colofs + (p + P * i) * estride] = xd[i];
                if (two) args.src1[colofs + (p + P * i) * estride] = xt[i];
            }
        }
    }
    // Outputs. One source column is held in registers at a time: delta for the
    // leading delta outputs, then theta, then phi = theta / k^2 (converted in
    // place once, so each element is divided once). Theta is read from memory
    // when its outputs start: MODE 0 reads the input, MODES 1 and 2 re-read the
    // finalised column this thread stored above (its own stores, so the values
    // are those it held).
    // output f before its transform: kx^a * src (or a shell mask times src),
    // src (delta, theta or phi) taken from the column sc
    auto input = [&](int f, const float2 (&sc)[E], float2 (&y)[E]) {
        const int code = args.codes[f];
        const int kind = code & 15, pa = (code >> 4) & 3, src = (code >> 8) & 3;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n = p + P * i;
            const int sx = signed_idx(n, N);
            const int s2 = sx * sx + syz;
            const float2 v0 = src == XS_ONE ? make_float2(1.f, 0.f) : sc[i];
            float2 v = v0;
            if (kind == XK_POW) {
                const float kx = kF * (float)sx;
                if (pa == 1) v = cscale(v, kx);
                else if (pa == 2) v = cscale(v, kx * kx);
            } else {
                const bool in = s2 > 0 && (long long)s2 >= args.shell_lo && (long long)s2 < args.shell_hi;
                if (!in) v = make_float2(0.f, 0.f);
            }
            y[i] = v;
        }
    };
    auto store = [&](int f, const float2 (&y)[E]) {
        if (act) {
            float2* o = args.out + f * args.out_stride + colofs;
#pragma unroll
            for (int i = 0; i < E; ++i) o[(p + P * i) * estride] = y[i];
        }
    };
    auto src_of = [&](int f) { return (args.codes[f] >> 8) & 3; };
    auto is_delta = [&](int f) { return src_of(f) == XS_DELTA; };
    // transform and store outputs f (and f + 1 when paired) from column sc
    auto emit = [&](int f, bool pair, const float2 (&sc)[E]) {
        if (PAIR && pair) {
            float2 y[2][E];
            input(f, sc, y[0]);
            input(f + 1, sc, y[1]);
            fft_col_pair<N, +1, NB>(y, p, pairA, pairB, TZ, twl);
            store(f, y[0]);
            store(f + 1, y[1]);
        } else {
            float2 y[E];
            input(f, sc, y);
            fft_col<N, +1, NB>(y, p, bufA + c, bufB + c, TZ, twl);
            store(f, y);
        }
    };
    int f = 0;
    while (f < args.nout && is_delta(f)) {
        const bool pair = PAIR && f + 1 < args.nout && is_delta(f + 1);
        emit(f, pair, xd);
        f += pair ? 2 : 1;
    }
    if (f < args.nout) {
        float2 xs[E];
        load_col(two ? args.src1 : args.src0, xs);
        bool phi = false;                                 // xs holds theta / k^2
        while (f < args.nout) {
            const int src = src_of(f);
            if (src == XS_DELTA) {                        // a later delta output: re-read delta
                float2 d[E];
                load_col(args.src0, d);
                emit(f, false, d);
                f += 1;
                continue;
            }
            if (src == XS_PHI && !phi) {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int sx = signed_idx(p + P * i, N);
                    const int s2 = sx * sx + syz;
                    const float g = s2 ? inv_kF2 / (float)s2 : 0.f;   // 1 / k^2, 0 at k = 0
                    xs[i] = cscale(xs[i], g);
                }
                phi = true;
            } else if (src == XS_THETA && phi) {          // theta after phi: re-read theta
                load_col(two ? args.src1 : args.src0, xs);
                phi = false;
            }
            const bool pair = PAIR && f + 1 < args.nout && src_of(f + 1) == src;
            emit(f, pair, xs);
            f += pair ? 2 : 1;
        }
    }
}

template <int N, int TZ, int MODE, bool PAIR>
__global__ void __launch_bounds__(TZ * Cfg<N>::PC, PAIR ? 1 : xexp_min_blocks<N, TZ, MODE>())
k_xexp(const __grid_constant__ XExpArgs args, const float2* __restrict__ twg, float kF, float inv_kF2) {
    extern __shared__ __align__(16) float2 sm[];
    xexp_body<N, TZ, MODE, PAIR>(args, twg, kF, inv_kF2, blockIdx.x, blockIdx.y, sm);
}

// ------------------------------------------------------------ y expansion
// Output f = ky^b * x-field[in], transformed backward along y. Outputs of one
// input are consecutive; the input column is loaded once and kept in
// registers. In-place use (out == in, one output per input, same index) is
// safe: a block owns its columns.
//
// PF: the next input's column tile is copied into a second shared buffer by
// cp.async (8-byte, zero-filled where the band excludes it) while the outputs
// of the current input are transformed. Otherwise the next input's column is
// prefetched into L2 (prefetch.global.L2), so its loads wait for L2, not HBM.
// PAIR: two consecutive outputs of the same input are transformed together by
// fft_column_pair (as in xexp_body; bit for bit the same outputs).
template <int N, int TZ, bool PF, bool PAIR = false>
__device__ __forceinline__ void yexp_body(const YZExpArgs& args, const float2* __restrict__ twg, float kF, int bx,
                                          int by, float2* sm, bool table_ready = false) {
    constexpr int M = N / 2, E = fft_elems(N), P = N / E;
    using CS = ColSm<N, TZ, PAIR ? 2 : 1, PF ? N * TZ : 0>;
    constexpr int NB = CS::NB;
    float2* twl = sm;
    float2* bufA = sm + CS::TW;
    float2* bufB = bufA + CS::BUF;
    float2* pre = bufA + NB * CS::BUF;           // PF: next input tile, element (n, c) at n * TZ + c
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    if (!table_ready) col_twiddles<N, N>(twl, twg);
    const int kz = bx * TZ + c;
    const int xr = by;
    const int B = args.band;
    const bool act = kz < M && (B <= 0 || kz < B);
    constexpr long long estride = (long long)M;
    const long long colofs = (long long)xr * N * M + kz;
    float2 xin[E];
    int cur = -1;
    bool have_next = false;
    for (int f = 0; f < args.nout; ++f) {
        const int code = args.codes[f];
        const int in = code & 255, pb = (code >> 8) & 3, slot = code >> 16;
        if (in != cur) {
            if (PF && have_next) {
                cp_async_wait_all();
                __syncthreads();                 // every thread's copies have landed
#pragma unroll
                for (int i = 0; i < E; ++i) xin[i] = pre[(p + P * i) * TZ + c];
            } else {
                const float2* col = args.in + in * args.in_stride + colofs;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int sy = signed_idx(p + P * i, N);
                    const bool live = act && (B <= 0 || (sy < B && -sy < B));
                    xin[i] = live ? col[(p + P * i) * estride] : make_float2(0.f, 0.f);
                }
            }
            cur = in;
            have_next = false;
            if constexpr (!PF) {                 // the next distinct input: prefetched into L2 meanwhile
                int g2 = f + 1;
                while (g2 < args.nout && (args.codes[g2] & 255) == in) ++g2;
                if (g2 < args.nout) {
                    const float2* col = args.in + (args.codes[g2] & 255) * args.in_stride + colofs;
#pragma unroll
                    for (int i = 0; i < E; ++i) {
                        const int sy = signed_idx(p + P * i, N);
                        const bool live = act && (B <= 0 || (sy < B && -sy < B));
                        if (live) prefetch_l2(col + (p + P * i) * estride);
                    }
                }
            }
            if constexpr (PF) {                  // the next distinct input, if any
                int g2 = f + 1;
                while (g2 < args.nout && (args.codes[g2] & 255) == in) ++g2;
                if (g2 < args.nout) {
                    __syncthreads();             // everyone has read the previous prefetch
                    const float2* col = args.in + (args.codes[g2] & 255) * args.in_stride + colofs;
#pragma unroll
                    for (int i = 0; i < E; ++i) {
                        const int sy = signed_idx(p + P * i, N);
                        const bool live = act && (B <= 0 || (sy < B && -sy < B));
                        cp_async8(pre + (p + P * i) * TZ + c, live ? col + (p + P * i) * estride : col, live ? 8 : 0);
                    }
                    cp_async_commit();
                    have_next = true;
                }
            }
        }
        if (PAIR && f + 1 < args.nout && (args.codes[f + 1] & 255) == in) {
            const int code1 = args.codes[f + 1];
            const int pb1 = (code1 >> 8) & 3, slot1 = code1 >> 16;
            float2 y[2][E];
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const float ky = kF * (float)signed_idx(p + P * i, N);
                y[0][i] = pb == 0 ? xin[i] : cscale(xin[i], pb == 1 ? ky : ky * ky);
                y[1][i] = pb1 == 0 ? xin[i] : cscale(xin[i], pb1 == 1 ? ky : ky * ky);
            }
            fft_col_pair<N, +1, NB>(y, p, reinterpret_cast<float4*>(bufA) + c, reinterpret_cast<float4*>(bufB) + c,
                                    TZ, twl);
            if (act) {
                float2* o0 = args.out + slot * args.out_stride + colofs;
                float2* o1 = args.out + slot1 * args.out_stride + colofs;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    o0[(p + P * i) * estride] = y[0][i];
                    o1[(p + P * i) * estride] = y[1][i];
                }
            }
            ++f;                                  // the pair's second output is done too
            continue;
        }
        float2 y[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float ky = kF * (float)signed_idx(p + P * i, N);
            y[i] = pb == 0 ? xin[i] : cscale(xin[i], pb == 1 ? ky : ky * ky);
        }
        fft_col<N, +1, NB>(y, p, bufA + c, bufB + c, TZ, twl);
        if (act) {
            float2* o = args.out + slot * args.out_stride + colofs;
#pragma unroll
            for (int i = 0; i < E; ++i) o[(p + P * i) * estride] = y[i];
        }
    }
}

template <int N, int TZ, bool PF, bool PAIR>
__global__ void __launch_bounds__(TZ * Cfg<N>::PC, (PF || PAIR) ? 1 : col_min_blocks<N, TZ>())
k_yexp(const __grid_constant__ YZExpArgs args, const float2* __restrict__ twg, float kF) {
    extern __shared__ __align__(16) float2 sm[];
    yexp_body<N, TZ, PF, PAIR>(args, twg, kF, blockIdx.x, blockIdx.y, sm);
}

// Column-pair form of k_yexp: each thread holds two adjacent kz columns, so
// global and shared accesses move 16 bytes (both columns) and every twiddle
// load and index computation serves two columns (fft_column_pair); TZ columns
// (TZ / 2 pairs) per block. Same outputs bit for bit.
template <int N, int TZ>
__global__ void __launch_bounds__(TZ / 2 * Cfg<N>::PC)
k_yexp2(YZExpArgs args, const float2* __restrict__ twg, float kF) {
    constexpr int M = N / 2, E = fft_elems(N), P = N / E, TP = TZ / 2;
    static_assert(TZ % 2 == 0 && M % 2 == 0, "column pairs");
    extern __shared__ __align__(16) float2 sm[];
    float2* tw = sm;
    float4* buf = reinterpret_cast<float4*>(sm + N + (N & 1));
    const int tid = threadIdx.x, c2 = tid % TP, p = tid / TP;
    load_table(tw, twg, N);
    const int kz0 = blockIdx.x * TZ + 2 * c2;
    const int xr = blockIdx.y;
    const int B = args.band;
    const bool act0 = kz0 < M && (B <= 0 || kz0 < B);
    const bool act1 = kz0 + 1 < M && (B <= 0 || kz0 + 1 < B);
    constexpr long long estride = (long long)M;
    const long long colofs = (long long)xr * N * M + kz0;
    float2 xin[2][E];
    int cur = -1;
    __syncthreads();
    for (int f = 0; f < args.nout; ++f) {
        const int code = args.codes[f];
        const int in = code & 255, pb = (code >> 8) & 3, slot = code >> 16;
        if (in != cur) {
            const float2* col = args.in + in * args.in_stride + colofs;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int sy = signed_idx(p + P * i, N);
                const bool live = act0 && (B <= 0 || (sy < B && -sy < B));
                const float4 v = live ? *reinterpret_cast<const float4*>(col + (p + P * i) * estride)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                xin[0][i] = make_float2(v.x, v.y);
                xin[1][i] = act1 ? make_float2(v.z, v.w) : make_float2(0.f, 0.f);
            }
            cur = in;
        }
        float2 y[2][E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float ky = kF * (float)signed_idx(p + P * i, N);
#pragma unroll
            for (int h = 0; h < 2; ++h) y[h][i] = pb == 0 ? xin[h][i] : cscale(xin[h][i], pb == 1 ? ky : ky * ky);
        }
        fft_column_pair<N, +1, N>(y, p, buf + c2, TP, tw);
        if (act0) {
            float2* o = args.out + slot * args.out_stride + colofs;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                if (act1)
                    *reinterpret_cast<float4*>(o + (p + P * i) * estride) = make_float4(y[0][i].x, y[0][i].y, y[1][i].x, y[1][i].y);
                else
                    o[(p + P * i) * estride] = y[0][i];
            }
        }
    }
}

// ------------------------------------------------------------ z expansion
// Output f = IFFT_z(c kz^g xy-field[in]) as a real row of N values, via the
// half-length complex transform of the packed row (Nyquist term zero). The
// input tile of 16+ rows is loaded once per input (tin) and kept while its
// outputs are formed in a second tile (tex), which is also the transform's
// exchange buffer.
template <int N, int TZ, bool PREFETCH>
__global__ void __launch_bounds__(TZ * Cfg<N>::PZ, (TZ * Cfg<N>::PZ <= 512) ? 2 : 1)
k_zexp(YZExpArgs args, const float2* __restrict__ twg, float kF) {
    const int B = args.band;                     // > 0: inputs nonzero only at kz < B
    constexpr int M = N / 2, E = fft_elems(M), P = M / E, PITCH = Cfg<N>::PITCH, NT = TZ * P;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    // input tiles (two when the next input is prefetched with cp.async) and the
    // output tile, which is also the transform's exchange buffer
    float2* tin[2] = {sm + N, sm + N + (PREFETCH ? TZ * PITCH : 0)};
    float2* tex = sm + N + (PREFETCH ? 2 : 1) * TZ * PITCH;
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    load_table(tw, twg, N);
    const long long rows = (long long)N * N;
    const long long row0 = (long long)blockIdx.x * TZ;
    if constexpr (PREFETCH)
        tile_prefetch<M, TZ, PITCH, NT>(tin[0], args.in + (args.codes[0] & 255) * args.in_stride, row0, rows);
    int cur = -1, buf = 0;
    for (int f = 0; f < args.nout; ++f) {
        const int code = args.codes[f];
        const int in = code & 255, g = (code >> 8) & 3, cc = (code >> 12) & 3, slot = code >> 16;
        if (in != cur) {
            if constexpr (PREFETCH) {
                if (cur >= 0) buf ^= 1;
                cp_async_wait_all();
                __syncthreads();   // tile complete and visible; the other buffer is no longer read
                int nf = f + 1;    // prefetch the next distinct input while this one's outputs are formed
                while (nf < args.nout && (args.codes[nf] & 255) == in) ++nf;
                if (nf < args.nout)
                    tile_prefetch<M, TZ, PITCH, NT>(tin[buf ^ 1], args.in + (args.codes[nf] & 255) * args.in_stride,
                                                    row0, rows);
            } else {
                __syncthreads();   // previous input no longer read
                tile_load<M, TZ, PITCH, NT>(tin[0], args.in + in * args.in_stride, row0, rows);
                __syncthreads();
            }
            cur = in;
        }
        const float2* colp = tin[buf] + c * PITCH;
        float2 x[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int k = p + P * i;
            float2 Xk = (B <= 0 || k < B) ? colp[k] : make_float2(0.f, 0.f);
            float2 Xm = (k && (B <= 0 || M - k < B)) ? colp[M - k] : make_float2(0.f, 0.f);
            if (g) {
                const float k1 = kF * (float)k, k2 = kF * (float)(M - k);
                Xk = cscale(Xk, g == 1 ? k1 : k1 * k1);
                Xm = cscale(Xm, g == 1 ? k2 : k2 * k2);
            }
            if (cc == 1) {
                Xk = cmul_i<+1>(Xk);
                Xm = cmul_i<+1>(Xm);
            } else if (cc == 2) {
                Xk = cmul_i<-1>(Xk);
                Xm = cmul_i<-1>(Xm);
            }
            Xm = cconj(Xm);                                  // X[k + M] = conj X[M - k]
            const float2 Ev = cadd(Xk, Xm);
            const float2 Ov = cmul(csub(Xk, Xm), tw[k]);     // e^{+2 pi i k / N}
            x[i] = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);    // E + i O
        }
        __syncthreads();                                     // tex free (previous store done reading)
        float2* colx = tex + c * PITCH;
        fft_column<M, +1, N>(x, p, colx, 1, tw);
#pragma unroll
        for (int i = 0; i < E; ++i) colx[p + P * i] = x[i];
        __syncthreads();
        tile_store<M, TZ, PITCH, NT>(args.out + slot * args.out_stride, tex, row0, rows);
    }
    if constexpr (PREFETCH) cp_async_wait_all();
}

// ------------------------------- z expansion fused with pair products
// Forms the real derived fields of one order m like k_zexp and, while each
// field f is in registers, multiplies it with its partner fields g of stored
// lower orders j (loaded tile by tile) and accumulates the pair terms of
// Eq. recursion_formula into A_{m+j}, B_{m+j} held in registers:
//   A += coef_a f g, B += coef_b f g   (coefficients per (f, g), both ordered
//   pairs (m, j) and (j, m) included; see PairTarget). After the last field the
// partial sums from earlier pairs are added and the targets are written as
// accumulator fields or, for a target's last pair, as delta_n, theta_n
// (recursion coefficients and N^-3 folded into ca0.., cb1). The fields of
// order m are stored only when a later order still needs them.
template <int N, int TZ, int NT>
__global__ void __launch_bounds__(TZ * Cfg<N>::PZ, 1)
k_zexp_pairs(ZPairArgs args, const float2* __restrict__ twg, float kF) {
    constexpr int M = N / 2, E = fft_elems(M), P = M / E, PITCH = Cfg<N>::PITCH, NTH = TZ * P;
    constexpr int MAXP = kMaxPartners;         // partner fields of one output over all targets
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* tin = sm + N;                      // input xy-field tile
    float2* tex = tin + TZ * PITCH;            // output tile / exchange buffer
    float2* tpt = tex + TZ * PITCH;            // MAXP partner tiles
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    load_table(tw, twg, N);
    const long long rows = (long long)N * N;
    const long long row0 = (long long)blockIdx.x * TZ;
    const YZExpArgs& z = args.z;
    // z.band > 0: the inputs are nonzero only at kz < band; the input tile is
    // loaded zero-filled beyond it, so the transform needs no per-element test
    constexpr int B = 0;
    // real fields as rows of M float2 (cells 2k, 2k + 1)
    const long long fstride2 = args.cells / 2;
    float2 accA[NT][E], accB[NT][E];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int i = 0; i < E; ++i) accA[t][i] = accB[t][i] = make_float2(0.f, 0.f);
    int cur = -1;
    for (int f = 0; f < z.nout; ++f) {
        const int code = z.codes[f];
        const int in = code & 255, g = (code >> 8) & 3, cc = (code >> 12) & 3, slot = code >> 16;
        __syncthreads();                       // tiles of the previous output no longer read
        // partner tiles of this output: copies issued now, consumed after the transform
        int np = 0;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t >= args.ntargets) break;
            const PairTarget& T = args.t[t];
            for (int q = 0; q < T.pcount[slot]; ++q) {
                if (T.pfield[slot][q] < 0) continue;                // a square: no partner tile
                tile_prefetch<M, TZ, PITCH, NTH>(tpt + np * TZ * PITCH, reinterpret_cast<const float2*>(T.partner) +
                                                                         (long long)T.pfield[slot][q] * fstride2,
                                                 row0, rows);
                ++np;
            }
        }
        if (in != cur) {
            tile_load<M, TZ, PITCH, NTH>(tin, z.in + in * z.in_stride, row0, rows, z.band);
            __syncthreads();
            cur = in;
        }
        const float2* colp = tin + c * PITCH;
        float2 x[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int k = p + P * i;
            float2 Xk = (B <= 0 || k < B) ? colp[k] : make_float2(0.f, 0.f);
            float2 Xm = (k && (B <= 0 || M - k < B)) ? colp[M - k] : make_float2(0.f, 0.f);
            if (g) {
                const float k1 = kF * (float)k, k2 = kF * (float)(M - k);
                Xk = cscale(Xk, g == 1 ? k1 : k1 * k1);
                Xm = cscale(Xm, g == 1 ? k2 : k2 * k2);
            }
            if (cc == 1) {
                Xk = cmul_i<+1>(Xk);
                Xm = cmul_i<+1>(Xm);
            } else if (cc == 2) {
                Xk = cmul_i<-1>(Xk);
                Xm = cmul_i<-1>(Xm);
            }
            Xm = cconj(Xm);
            const float2 Ev = cadd(Xk, Xm);
            const float2 Ov = cmul(csub(Xk, Xm), tw[k]);
            x[i] = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);
        }
        float2* colx = tex + c * PITCH;
        fft_column<M, +1, N>(x, p, colx, 1, tw);   // x[i]: real cells 2n, 2n + 1 of row c, n = p + P i
        cp_async_wait_all();
        if (args.store) {
#pragma unroll
            for (int i = 0; i < E; ++i) colx[p + P * i] = x[i];
        }
        __syncthreads();                           // partner tiles and the output tile are complete
        if (args.store)
            tile_store<M, TZ, PITCH, NTH>(reinterpret_cast<float2*>(args.store) + slot * fstride2, tex, row0, rows);
        np = 0;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t >= args.ntargets) break;
            const PairTarget& T = args.t[t];
            for (int q = 0; q < T.pcount[slot]; ++q) {
                const float ca = T.pcoef_a[slot][q], cb = T.pcoef_b[slot][q];
                const bool sq = T.pfield[slot][q] < 0;
                const float2* pr = tpt + np * TZ * PITCH + c * PITCH;
                if (!sq) ++np;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const float2 gv = sq ? x[i] : pr[p + P * i];
                    const float2 fg = lmul(x[i], gv);
                    accA[t][i] = lfma(ca, fg, accA[t][i]);
                    accB[t][i] = lfma(cb, fg, accB[t][i]);
                }
            }
        }
    }
    // targets: add earlier partial sums, combine, write (via the output tile)
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        if (t >= args.ntargets) break;
        const PairTarget& T = args.t[t];
        if (T.acc_in_a) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __syncthreads();
                tile_load<M, TZ, PITCH, NTH>(tpt, reinterpret_cast<const float2*>(h ? T.acc_in_b : T.acc_in_a),
                                             row0, rows);
                __syncthreads();
                const float2* pr = tpt + c * PITCH;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const float2 v = pr[p + P * i];
                    float2& a = h ? accB[t][i] : accA[t][i];
                    a.x += v.x;
                    a.y += v.y;
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float c0 = h ? T.cb0 : T.ca0, c1 = h ? T.cb1 : T.ca1;
            __syncthreads();
            float2* colx = tex + c * PITCH;
#pragma unroll
            for (int i = 0; i < E; ++i)
                colx[p + P * i] = lfma(c0, accA[t][i], cscale(accB[t][i], c1));
            __syncthreads();
            tile_store<M, TZ, PITCH, NTH>(reinterpret_cast<float2*>(h ? T.out_b : T.out_a), tex, row0, rows);
        }
    }
}

// ------------------------------------- z pass on warp rows (no block barriers)
// The computation of k_zexp (NT = 0, store only) and k_zexp_pairs (NT = 1, 2
// targets) with one z row per P consecutive lanes of a warp (P = M / E <= 32,
// 32 / P rows per warp) instead of block-wide tiles. Each warp runs its rows
// through every output field on its own:
//   * the xy-field input rows are kept in a per-warp buffer while consecutive
//     outputs share them; the next distinct input (that of the next output, or
//     the first of the warp's next row group) is copied into a second buffer by
//     16-byte cp.async while the current output is transformed;
//   * the partner rows of the output are copied into per-warp buffers by
//     16-byte cp.async before the transform and consumed after it;
//   * the transform exchanges through a per-warp padded buffer (fft_row);
//   * stores, accumulator inputs and the targets' outputs go straight between
//     registers and global memory: lane p holds elements p + P i, so every
//     warp access covers whole rows.
// The only block barrier follows the twiddle table set-up. Persistent grid:
// each warp strides over the row groups. Results are bitwise those of the
// tile kernels (same transform arithmetic, same accumulation order).
constexpr int kRowWarps = 8;

template <int N>
struct RowCfg {
    static constexpr int M = N / 2, E = fft_elems(M), P = M / E;
    static constexpr bool ok = (M & (M - 1)) == 0 && P <= 32 && 32 % P == 0;
    static constexpr int RW = ok ? 32 / P : 1;               // rows per warp
    static constexpr int XROW = M + (M >> 4);                 // padded exchange row
    static constexpr int NTW = fft_row_tw_total<M>();
    static constexpr int HDR = ((NTW + E) * P + 1) / 2 * 2;   // twiddle tables, 16-byte multiple
    static constexpr int MAXP = kMaxPartners;
    static constexpr int WIN = RW * M;                        // input rows of a warp
    // per warp: two input buffers (current, next), MAXP partner buffers, exchange rows
    __host__ __device__ static constexpr int wstride(int nt) { return WIN * (2 + (nt ? MAXP : 0)) + RW * XROW; }
    static constexpr size_t smem(int nt) { return sizeof(float2) * (HDR + (size_t)kRowWarps * wstride(nt)); }
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// The same copy, or (read = false) 16 zero bytes written without reading src.
__device__ __forceinline__ void cp_async16z(void* dst, const void* src, bool read) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(read ? 16 : 0)
                 : "memory");
}

// Lane-major twiddle tables of a warp-row kernel from the global table of
// N-th roots (values identical to the tile kernels' shared copy).
template <int N>
__device__ __forceinline__ void zrow_tables(float2* twl, float2* twp, const float2* __restrict__ twg) {
    using C = RowCfg<N>;
    if (threadIdx.x < C::P) {
        fft_row_twiddles<C::M, N>(twl, twg, threadIdx.x);
#pragma unroll
        for (int i = 0; i < C::E; ++i) twp[i * C::P + threadIdx.x] = twg[threadIdx.x + C::P * i];
    }
    __syncthreads();
}

// Body of the warp-row z pass: warp w of the block handles the row groups
// grp0 + w, grp0 + w + gstride, ... (the kernel: grp0 = blockIdx.x * kRowWarps,
// gstride = gridDim.x * kRowWarps; a tile of the persistent queue: one group
// per warp). Inputs, partners and partial sums are read through L2 (cp.async.cg
// and ordinary loads), never through the read-only data path, so the body is
// also correct for fields written earlier in the same launch.
template <int N, int NT, bool BAND>
__device__ __forceinline__ void zrow_body(const ZPairArgs& args, const float2* __restrict__ twg, float kF,
                                          long long grp0, long long gstride, float2* sm, bool table_ready = false) {
    using C = RowCfg<N>;
    constexpr int M = C::M, E = C::E, P = C::P, RW = C::RW, WIN = C::WIN;
    constexpr int NA = NT > 0 ? NT : 1;
    static_assert(C::ok, "warp-row z pass needs P <= 32, 32 % P == 0 and a power-of-two row");
    float2* twl = sm;                                  // [NTW][P] stage twiddles
    float2* twp = twl + C::NTW * P;                    // [E][P] pack twiddles tw[p + P i]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane / P, p = lane - r * P;
    if (!table_ready) zrow_tables<N>(twl, twp, twg);
    float2* wbase = sm + C::HDR + warp * C::wstride(NT);
    float2* wpt = wbase + 2 * WIN;                                                 // [MAXP][RW][M] partners
    float2* xrow = wbase + WIN * (NT ? 2 + C::MAXP : 2) + r * C::XROW;              // this row's exchange buffer
    const YZExpArgs& z = args.z;
    // BAND, z.band > 0 (even): inputs nonzero only at kz < B. Only those are
    // read; the rest of the input buffers is zero-filled by the copies, so the
    // transform needs no per-element test (a separate instance, which keeps
    // the mask's registers out of the launches without a band)
    const int B = BAND ? z.band : 0;
    unsigned inb = 0;            // bit u: this lane's 16-byte piece u of a row window lies at kz < B
#pragma unroll
    for (int u = 0; u < WIN / 64; ++u)
        if (B <= 0 || (2 * (lane + 32 * u)) % M < B) inb |= 1u << u;
    const long long rows = (long long)N * N;
    const long long groups = rows / RW;
    const long long fstride2 = args.cells / 2;
    int buf = 0;                 // wbase + buf * WIN holds the current input rows
    bool have_next = false;      // the other buffer holds (or receives) the next input
    for (long long grp = grp0 + warp; grp < groups; grp += gstride) {
        const long long row0 = grp * RW, row = row0 + r;
        float2 accA[NA][E], accB[NA][E];
#pragma unroll
        for (int t = 0; t < NA; ++t)
#pragma unroll
            for (int i = 0; i < E; ++i) accA[t][i] = accB[t][i] = make_float2(0.f, 0.f);
        int cur = -1;
        for (int f = 0; f < z.nout; ++f) {
            const int code = z.codes[f];
            const int in = code & 255, g = (code >> 8) & 3, cc = (code >> 12) & 3, slot = code >> 16;
            __syncwarp();                                  // earlier reads of the buffers are done
            int np = 0;
            if constexpr (NT > 0) {
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    if (t >= args.ntargets) break;
                    const PairTarget& T = args.t[t];
                    for (int q = 0; q < T.pcount[slot]; ++q) {
                        if (T.pfield[slot][q] < 0) continue;            // a square: no partner rows
                        const float2* src = reinterpret_cast<const float2*>(T.partner) +
                                            (long long)T.pfield[slot][q] * fstride2 + row0 * M;
#pragma unroll
                        for (int u = 0; u < WIN / 64; ++u)
                            cp_async16(wpt + np * WIN + 2 * (lane + 32 * u), src + 2 * (lane + 32 * u));
                        ++np;
                    }
                }
            }
            if (in != cur) {
                if (have_next) {                           // copied during the previous output
                    buf ^= 1;
                } else {                                   // the warp's first input
                    const float4* src = reinterpret_cast<const float4*>(z.in + in * z.in_stride + row0 * M);
                    float4 v[WIN / 64];
#pragma unroll
                    for (int u = 0; u < WIN / 64; ++u)
                        v[u] = ((inb >> u) & 1u) ? src[lane + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < WIN / 64; ++u) reinterpret_cast<float4*>(wbase + buf * WIN)[lane + 32 * u] = v[u];
                    __syncwarp();
                }
                cur = in;
                have_next = false;
            }
            {   // next distinct input into the other buffer (last read two outputs ago at the latest)
                const bool last = f + 1 == z.nout;
                const int nin = last ? (z.codes[0] & 255) : (z.codes[f + 1] & 255);
                const long long nrow0 = last ? row0 + gstride * RW : row0;
                if (last ? nrow0 < rows : nin != in) {
                    const float2* src = z.in + nin * z.in_stride + nrow0 * M;
                    float2* dst = wbase + (buf ^ 1) * WIN;
#pragma unroll
                    for (int u = 0; u < WIN / 64; ++u)
                        cp_async16z(dst + 2 * (lane + 32 * u), src + 2 * (lane + 32 * u), (inb >> u) & 1u);
                    have_next = true;
                }
            }
            cp_async_commit();
            const float2* colp = wbase + buf * WIN + r * M;
            float2 x[E];
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int k = p + P * i;
                float2 Xk = colp[k];
                float2 Xm = k ? colp[M - k] : make_float2(0.f, 0.f);
                if (g) {
                    const float k1 = kF * (float)k, k2 = kF * (float)(M - k);
                    Xk = cscale(Xk, g == 1 ? k1 : k1 * k1);
                    Xm = cscale(Xm, g == 1 ? k2 : k2 * k2);
                }
                if (cc == 1) {
                    Xk = cmul_i<+1>(Xk);
                    Xm = cmul_i<+1>(Xm);
                } else if (cc == 2) {
                    Xk = cmul_i<-1>(Xk);
                    Xm = cmul_i<-1>(Xm);
                }
                Xm = cconj(Xm);
                const float2 Ev = cadd(Xk, Xm);
                const float2 Ov = cmul(csub(Xk, Xm), twp[i * P + p]);
                x[i] = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);
            }
            fft_row<M, +1>(x, p, xrow, twl);              // x[i]: real cells 2n, 2n + 1, n = p + P i
            float2* dst = NT > 0 ? (args.store ? reinterpret_cast<float2*>(args.store) + slot * fstride2 : nullptr)
                                 : z.out + slot * z.out_stride;
            if (dst) {
#pragma unroll
                for (int i = 0; i < E; ++i) dst[row * M + p + P * i] = x[i];
            }
            cp_async_wait_all();
            __syncwarp();                                  // partner and next-input rows of every lane have landed
            if constexpr (NT > 0) {
                np = 0;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    if (t >= args.ntargets) break;
                    const PairTarget& T = args.t[t];
                    for (int q = 0; q < T.pcount[slot]; ++q) {
                        const float ca = T.pcoef_a[slot][q], cb = T.pcoef_b[slot][q];
                        const bool sq = T.pfield[slot][q] < 0;
                        const float2* pr = wpt + np * WIN + r * M;
#pragma unroll
                        for (int i = 0; i < E; ++i) {
                            const float2 gv = sq ? x[i] : pr[p + P * i];
                            const float2 fg = lmul(x[i], gv);
                            accA[t][i] = lfma(ca, fg, accA[t][i]);
                            accB[t][i] = lfma(cb, fg, accB[t][i]);
                        }
                        if (!sq) ++np;
                    }
                }
            }
        }
        if constexpr (NT > 0) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (t >= args.ntargets) break;
                const PairTarget& T = args.t[t];
                if (T.acc_in_a) {
                    const float2* ia = reinterpret_cast<const float2*>(T.acc_in_a) + row * M;
                    const float2* ib = reinterpret_cast<const float2*>(T.acc_in_b) + row * M;
#pragma unroll
                    for (int i = 0; i < E; ++i) {
                        const float2 va = ia[p + P * i], vb = ib[p + P * i];
                        accA[t][i] = cadd(accA[t][i], va);
                        accB[t][i] = cadd(accB[t][i], vb);
                    }
                }
                float2* oa = reinterpret_cast<float2*>(T.out_a) + row * M;
                float2* ob = reinterpret_cast<float2*>(T.out_b) + row * M;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    oa[p + P * i] = lfma(T.ca0, accA[t][i], cscale(accB[t][i], T.ca1));
                    ob[p + P * i] = lfma(T.cb0, accA[t][i], cscale(accB[t][i], T.cb1));
                }
            }
        }
    }
}

template <int N, int NT, bool BAND>
__global__ void __launch_bounds__(kRowWarps * 32, NT == 0 ? 3 : 2)
k_zrow(const __grid_constant__ ZPairArgs args, const float2* __restrict__ twg, float kF) {
    extern __shared__ __align__(16) float2 sm[];
    zrow_body<N, NT, BAND>(args, twg, kF, (long long)blockIdx.x * kRowWarps, (long long)gridDim.x * kRowWarps, sm);
}

// ------------------------------------------------- TMA-staged y expansion
// Same computation as k_yexp, but each input column tile (all N rows of TZ
// adjacent kz columns of one x plane) is copied into shared memory by the
// tensor-memory accelerator (cp.async.bulk.tensor, 4D map over kz, ky, x and
// field), completion tracked by an mbarrier, while the previous input's
// outputs are transformed. The tile being consumed is read into registers and
// then serves as the transform's exchange buffer. Every wait is bounded: on
// timeout the kernel sets *status and continues (results are then invalid and
// gridspt_check reports GRIDSPT_E_TIMEOUT); it never traps or spins forever.
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
                 "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(bar)), "r"(bytes) : "memory");
}
// true when the phase with the given parity has completed; bounded
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"((unsigned)__cvta_generic_to_shared(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// rows per TMA box: the largest divisor of N not above 256 (a box dimension is at most 256)
__host__ __device__ constexpr int tma_rows(int N) { return N <= 256 ? N : (N % 256 == 0 ? 256 : N / 2 <= 256 ? N / 2 : 192); }

template <int N, int TZ>
__global__ void __launch_bounds__(TZ * Cfg<N>::PC, (TZ * Cfg<N>::PC <= 512) ? 2 : 1)
k_yexp_tma(YZExpArgs args, const __grid_constant__ CUtensorMap tmap, const float2* __restrict__ twg, float kF,
           int* __restrict__ status) {
    constexpr int M = N / 2, E = fft_elems(N), P = N / E;
    constexpr int BR = tma_rows(N);
    static_assert(N % BR == 0 && BR <= 256, "TMA box rows must divide N");
    constexpr unsigned TILE_BYTES = (unsigned)N * TZ * sizeof(float2);
    extern __shared__ unsigned char smraw[];
    // tiles start on a 1024-byte boundary (TMA destinations need at least 128)
    const unsigned base_off = (1024u - ((unsigned)__cvta_generic_to_shared(smraw) & 1023u)) & 1023u;
    unsigned char* smb = smraw + base_off;
    float2* tile[2] = {reinterpret_cast<float2*>(smb), reinterpret_cast<float2*>(smb + TILE_BYTES)};
    float2* tw = reinterpret_cast<float2*>(smb + 2 * TILE_BYTES);
    __shared__ uint64_t bar[2];
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    const int kz0 = blockIdx.x * TZ;
    const int xr = blockIdx.y;
    load_table(tw, twg, N);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    auto issue = [&](int b, int in) {   // thread 0 only
        mbar_expect_tx(&bar[b], TILE_BYTES);
#pragma unroll
        for (int r = 0; r < N / BR; ++r) tma_load_4d(tile[b] + r * BR * TZ, &tmap, kz0, r * BR, xr, in, &bar[b]);
    };
    if (tid == 0) issue(0, args.codes[0] & 255);
    unsigned phase[2] = {0u, 0u};
    int pending[2] = {1, 0};
    int buf = 0, cur = -1;
    bool ok = true;
    constexpr long long estride = (long long)M;
    const long long colofs = (long long)xr * N * M + kz0 + c;
    float2 xin[E];
    for (int f = 0; f < args.nout; ++f) {
        const int code = args.codes[f];
        const int in = code & 255, pb = (code >> 8) & 3, slot = code >> 16;
        if (in != cur) {
            if (cur >= 0) buf ^= 1;
            ok = mbar_wait(&bar[buf], phase[buf]) && ok;
            phase[buf] ^= 1u;
            pending[buf] = 0;
#pragma unroll
            for (int i = 0; i < E; ++i) xin[i] = tile[buf][(p + P * i) * TZ + c];
            fence_proxy_async();     // generic-proxy use of the other tile ends before the TMA refills it
            __syncthreads();
            int nf = f + 1;
            while (nf < args.nout && (args.codes[nf] & 255) == in) ++nf;
            if (nf < args.nout) {
                if (tid == 0) issue(buf ^ 1, args.codes[nf] & 255);
                pending[buf ^ 1] = 1;
            }
            cur = in;
        }
        float2 y[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float ky = kF * (float)signed_idx(p + P * i, N);
            y[i] = pb == 0 ? xin[i] : cscale(xin[i], pb == 1 ? ky : ky * ky);
        }
        fft_column<N, +1, N>(y, p, tile[buf] + c, TZ, tw);
        float2* o = args.out + slot * args.out_stride + colofs;
#pragma unroll
        for (int i = 0; i < E; ++i) o[(p + P * i) * estride] = y[i];
    }
    // never leave with a copy in flight into this block's shared memory
    for (int b = 0; b < 2; ++b)
        if (pending[b]) ok = mbar_wait(&bar[b], phase[b]) && ok;
    if (!ok && tid == 0) atomicOr(status, kStatusWaitTma);
}

// ------------------------------------------- z pass fused with the shell sums
// Bispectrum estimator, one shell (Sec. III.B.1, Eq. bk_tree, FFT shell
// estimator): the three xy-fields I_a, I_b, J (nonzero only for kz < band)
// are transformed to real rows in shared memory; every thread then holds the
// same cells of all three rows, forms I_a^2 I_b and J^3 in FP32 and keeps
// Kahan-compensated FP32 sums (FP64 sums of the same terms, in the same order,
// with the FP64 accumulator choice, f64 = 1); the block writes FP64 partials
// (fixed order).
__device__ __forceinline__ void kahan_add2(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}
// a b c summed over the two cells of a float2, with explicit roundings (no
// contraction), so that every shell kernel forms bitwise the same terms (and
// a a b here is bitwise the a^2 b of the two-field estimator)
__device__ __forceinline__ float cell_mul3(float2 a, float2 b, float2 c) {
    return __fadd_rn(__fmul_rn(__fmul_rn(a.x, b.x), c.x), __fmul_rn(__fmul_rn(a.y, b.y), c.y));
}

// TRI: the data fields are I_a, I_b, I_c and the first sum is I_a I_b I_c
// (triple-product estimator, one-loop bispectrum); otherwise I_a, I_b and
// I_a^2 I_b. NF counts the data fields plus J when present.
template <int N, int TZ, int NF, bool TRI>
__global__ void __launch_bounds__(TZ * Cfg<N>::PZ, (TZ * Cfg<N>::PZ <= 512) ? 2 : 1)
k_zshell(const float2* __restrict__ in, long long in_stride, int band, const float2* __restrict__ twg,
         double* __restrict__ partial, int f64) {
    constexpr int M = N / 2, E = fft_elems(M), P = M / E, PITCH = Cfg<N>::PITCH, NT = TZ * P;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* t3 = sm + N;
    static_assert(NT % 32 == 0, "block of whole warps");
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    load_table(tw, twg, N);
    const long long rows = (long long)N * N;
    const long long row0 = (long long)blockIdx.x * TZ;
    const int B = band < M ? band : M;
    // kz < B of each field (asynchronous copies), zeros elsewhere
    for (int f = 0; f < NF; ++f) {
        const float2* src = in + f * in_stride;
        float2* tile = t3 + f * TZ * PITCH;
        for (int idx = tid; idx < TZ * M; idx += NT) {
            const int r = idx / M, j = idx - r * M;
            const long long row = row0 + r;
            if (j < B && row < rows)
                cp_async8(tile + r * PITCH + j, src + row * M + j, 8);
            else
                tile[r * PITCH + j] = make_float2(0.f, 0.f);
        }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    float2 x[NF][E];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const float2* colp = t3 + f * TZ * PITCH + c * PITCH;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int k = p + P * i;
            const float2 Xk = colp[k];
            const float2 Xm = k ? cconj(colp[M - k]) : make_float2(0.f, 0.f);
            const float2 Ev = cadd(Xk, Xm);
            const float2 Ov = cmul(csub(Xk, Xm), tw[k]);
            x[f][i] = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);
        }
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < NF; ++f) fft_column<M, +1, N>(x[f], p, t3 + f * TZ * PITCH + c * PITCH, 1, tw);
    constexpr int ND = TRI ? 3 : 2;                   // data fields; J follows when NF > ND
    // fixed-order reduction, grouped as in the warp-row kernel: 32 chains
    // (slot l = r P + p: rows c = r, r + 32/P, ... of the block in order, each
    // row's elements i in order) of Kahan FP32 sums, then one FP64 shuffle tree
    // over the 32 chains. The terms go through shared memory so that one warp
    // can run the chains.
    __syncthreads();                                   // tiles are no longer read
    float* T1 = reinterpret_cast<float*>(t3);          // [TZ][P][E] terms
    float* T2 = T1 + TZ * P * E;
    const bool live = row0 + c < rows;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        T1[(c * P + p) * E + i] = live ? cell_mul3(x[0][i], TRI ? x[1][i] : x[0][i], x[TRI ? 2 : 1][i]) : 0.f;
        if constexpr (NF > ND) T2[(c * P + p) * E + i] = live ? cell_mul3(x[NF - 1][i], x[NF - 1][i], x[NF - 1][i]) : 0.f;
    }
    __syncthreads();
    if (tid < 32) {
        float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
        double d1 = 0.0, d2 = 0.0;                     // FP64 accumulator choice (f64)
        auto chain = [&](int cc, int pp) {
            if (f64) {
                for (int i = 0; i < E; ++i) {
                    d1 += (double)T1[(cc * P + pp) * E + i];
                    if constexpr (NF > ND) d2 += (double)T2[(cc * P + pp) * E + i];
                }
                return;
            }
#pragma unroll
            for (int i = 0; i < E; ++i) {
                kahan_add2(s1, c1, T1[(cc * P + pp) * E + i]);
                if constexpr (NF > ND) kahan_add2(s2, c2, T2[(cc * P + pp) * E + i]);
            }
        };
        if constexpr (P <= 32) {
            constexpr int RWS = 32 / P;
            for (int cc = tid / P; cc < TZ; cc += RWS) chain(cc, tid % P);
        } else {                                       // rows longer than a warp (P = 64)
            for (int cc = 0; cc < TZ; ++cc)
                for (int pp = tid; pp < P; pp += 32) chain(cc, pp);
        }
        double a = f64 ? d1 : (double)s1 - (double)c1, b = f64 ? d2 : (double)s2 - (double)c2;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, off);
            b += __shfl_down_sync(0xffffffffu, b, off);
        }
        if (tid == 0) {
            partial[2 * blockIdx.x] = a;
            partial[2 * blockIdx.x + 1] = b;
        }
    }
}

// Warp-row form of k_zshell: one z row per P lanes, the band-limited inputs
// (kz < band) read straight into registers by coalesced loads, the transform
// exchanged through a per-warp buffer. Each warp sums a group of G = TZZ0
// consecutive rows (G is the tile kernel's block height): every lane keeps one
// Kahan FP32 sum over its rows of the group (in row order), then one FP64
// shuffle tree over the 32 lanes gives the group's partial pair. The FP64
// pipe (a small fraction of the FP32 rate on this GPU) sees one tree per
// group instead of one per row. Terms, chains and tree are those of the tile
// kernel, so the partials are bitwise equal.
template <int N, int NF, bool TRI>
__global__ void __launch_bounds__(kRowWarps * 32, 2)
k_zrow_shell(const float2* __restrict__ in, long long in_stride, int band, const float2* __restrict__ twg,
             double* __restrict__ partial, int f64) {
    using C = RowCfg<N>;
    constexpr int M = C::M, E = C::E, P = C::P, RW = C::RW;
    constexpr int G = Cfg<N>::TZZ0;
    static_assert(C::ok && G % RW == 0, "warp-row shell pass: whole rows per warp and per group");
    extern __shared__ __align__(16) float2 sm[];
    float2* twl = sm;
    float2* twp = twl + C::NTW * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane / P, p = lane - r * P;
    zrow_tables<N>(twl, twp, twg);
    float2* xrow = sm + C::HDR + (warp * RW + r) * C::XROW;
    const int B = band < M ? band : M;
    const long long groups = (long long)N * N / G;
    for (long long grp = (long long)blockIdx.x * kRowWarps + warp; grp < groups;
         grp += (long long)gridDim.x * kRowWarps) {
        float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;   // this lane's chains over its rows
        double d1 = 0.0, d2 = 0.0;                      // FP64 accumulator choice (f64)
        for (int rr = 0; rr < G; rr += RW) {
            const long long row = grp * G + rr + r;
            // one band-limited row of field f, packed and transformed to real cells
            auto real_row = [&](int f, float2 (&x)[E]) {
                const float2* src = in + f * in_stride + row * M;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int k = p + P * i;
                    const float2 Xk = k < B ? __ldg(src + k) : make_float2(0.f, 0.f);
                    const float2 Xm = k ? cconj(M - k < B ? __ldg(src + M - k) : make_float2(0.f, 0.f))
                                        : make_float2(0.f, 0.f);
                    const float2 Ev = cadd(Xk, Xm);
                    const float2 Ov = cmul(csub(Xk, Xm), twp[i * P + p]);
                    x[i] = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);
                }
                fft_row<M, +1>(x, p, xrow, twl);
            };
            constexpr int ND = TRI ? 3 : 2;               // data fields; J follows when NF > ND
            {
                float2 x[ND][E];
#pragma unroll
                for (int f = 0; f < ND; ++f) real_row(f, x[f]);
                if (f64) {
#pragma unroll
                    for (int i = 0; i < E; ++i) d1 += (double)cell_mul3(x[0][i], x[TRI ? 1 : 0][i], x[ND - 1][i]);
                } else {
#pragma unroll
                    for (int i = 0; i < E; ++i)
                        kahan_add2(s1, c1, cell_mul3(x[0][i], x[TRI ? 1 : 0][i], x[ND - 1][i]));
                }
            }
            if constexpr (NF > ND) {                      // J after the data fields: fewer live registers
                float2 xj[E];
                real_row(NF - 1, xj);
                if (f64) {
#pragma unroll
                    for (int i = 0; i < E; ++i) d2 += (double)cell_mul3(xj[i], xj[i], xj[i]);
                } else {
#pragma unroll
                    for (int i = 0; i < E; ++i) kahan_add2(s2, c2, cell_mul3(xj[i], xj[i], xj[i]));
                }
            }
        }
        double a = f64 ? d1 : (double)s1 - (double)c1, b = f64 ? d2 : (double)s2 - (double)c2;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, off);
            b += __shfl_down_sync(0xffffffffu, b, off);
        }
        if (lane == 0) {
            partial[2 * grp] = a;
            partial[2 * grp + 1] = b;
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kRowWarps * 32, 3)
k_zrow_r2c(const float2* in, float2* out, long long fstride, int count, const float2* __restrict__ twg,
           float scale, int band) {
    using C = RowCfg<N>;
    constexpr int M = C::M, E = C::E, P = C::P, RW = C::RW;
    static_assert(C::ok, "warp-row z pass needs P <= 32, 32 % P == 0 and a power-of-two row");
    extern __shared__ __align__(16) float2 sm[];
    float2* twl = sm;
    float2* twp = twl + C::NTW * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane / P, p = lane - r * P;
    zrow_tables<N>(twl, twp, twg);
    float2* xrow = sm + C::HDR + (warp * RW + r) * C::XROW;
    const long long per = (long long)N * N / RW;        // row groups per field
    const long long groups = per * count;
    const float half = 0.5f * scale;
    for (long long grp = (long long)blockIdx.x * kRowWarps + warp; grp < groups;
         grp += (long long)gridDim.x * kRowWarps) {
        const long long fld = grp / per, row = (grp - fld * per) * RW + r;
        const float2* src = in + fld * fstride + row * M;
        float2* dst = out + fld * fstride + row * M;
        float2 x[E];
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = src[p + P * i];
        fft_row<M, -1>(x, p, xrow, twl);
#pragma unroll
        for (int i = 0; i < E; ++i) xrow[xpad(p + P * i)] = x[i];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int k = p + P * i;
            const float2 Z = xrow[xpad(k)];
            const float2 Zr = cconj(xrow[xpad(k ? M - k : 0)]);
            const float2 S = cadd(Z, Zr);                            // 2 E[k]
            const float2 t = cmul(cconj(twp[i * P + p]), csub(Z, Zr));  // e^{-2 pi i k/N} 2i O[k]
            if (band <= 0 || k < band) dst[k] = make_float2(half * (S.x + t.y), half * (S.y - t.x));
        }
        __syncwarp();                                    // exchange buffer free for the next row
    }
}

// ------------------------------------------------------------- launchers
// cuTensorMapEncodeTiled through the runtime's driver entry point (k_tma_host.cpp)
cudaError_t encode_tensor_map(CUtensorMap* map, void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                              const cuuint32_t* box, const cuuint32_t* elem_strides);

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

template <int N, int TZC, int TZZ>
struct Launch {
    static constexpr int M = N / 2;
    static constexpr int PC = Cfg<N>::PC, PZ = Cfg<N>::PZ, PITCH = Cfg<N>::PITCH;
    static cudaError_t colpass(const Geo& g, float2* d, long long fs, int count, int axis, int fin,
                               long long s2_nl, int band, cudaStream_t s) {
        const int B = axis == 1 && band > 0 && band < M ? band : 0;
        dim3 grid(((B ? B : M) + TZC - 1) / TZC, N, count);
        const size_t smem = colpass_smem<N, TZC>();
        cudaError_t e;
#define GRIDSPT_COL(AX_, FIN_)                                                        \
    e = set_smem(k_colpass<N, TZC, AX_, FIN_>, smem);                                 \
    if (e != cudaSuccess) return e;                                                   \
    k_colpass<N, TZC, AX_, FIN_><<<grid, TZC * PC, smem, s>>>(d, fs, g.tw, s2_nl, fin == 2, B); \
    return cudaGetLastError();
        if (axis == 0) {
            if (fin) { GRIDSPT_COL(0, true) }
            GRIDSPT_COL(0, false)
        }
        GRIDSPT_COL(1, false)
#undef GRIDSPT_COL
    }
    static cudaError_t zrow_r2c(const Geo& g, const float2* in, float2* out, long long fs, int count, float scale,
                                int band, cudaStream_t s) {
        using C = RowCfg<N>;
        if constexpr (!C::ok) {
            return cudaErrorNotSupported;
        } else {
            const size_t smem = sizeof(float2) * (C::HDR + (size_t)kRowWarps * C::RW * C::XROW);
            cudaError_t e = set_smem(k_zrow_r2c<N>, smem);
            if (e != cudaSuccess) return e;
            int dev = 0, sms = 0, per = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zrow_r2c<N>, kRowWarps * 32, smem)) !=
                cudaSuccess)
                return e;
            const long long groups = (long long)N * N / C::RW * count;
            const long long need = (groups + kRowWarps - 1) / kRowWarps;
            const long long resident = (long long)(per > 0 ? per : 1) * sms;
            k_zrow_r2c<N><<<(unsigned)(need < resident ? need : resident), kRowWarps * 32, smem, s>>>(
                in, out, fs, count, g.tw, scale, band > 0 && band < M ? band : 0);
            return cudaGetLastError();
        }
    }
    static cudaError_t zr2c(const Geo& g, const float2* in, float2* out, long long fs, int count,
                            float scale, int band, cudaStream_t s) {
        const long long rows = (long long)N * N;
        dim3 grid((unsigned)((rows + TZZ - 1) / TZZ), count);
        const size_t smem = sizeof(float2) * (N + (size_t)TZZ * PITCH);
        cudaError_t e = set_smem(k_zr2c<N, TZZ>, smem);
        if (e != cudaSuccess) return e;
        k_zr2c<N, TZZ><<<grid, TZZ * PZ, smem, s>>>(in, out, fs, g.tw, scale, band > 0 && band < M ? band : 0);
        return cudaGetLastError();
    }
    template <bool PAIR = false>
    static cudaError_t xexp(const Geo& g, const XExpArgs& a, cudaStream_t s) {
        if constexpr (!ColSm<N, TZC, PAIR ? 2 : 1>::fits) return cudaErrorNotSupported;
        else return xexp_fit<PAIR>(g, a, s);
    }
    template <bool PAIR>
    static cudaError_t xexp_fit(const Geo& g, const XExpArgs& a, cudaStream_t s) {
        const int B = a.band > 0 && a.band < M ? a.band : 0;
        dim3 grid(((B ? B : M) + TZC - 1) / TZC, B ? 2 * B - 1 : N);
        const size_t smem = ColSm<N, TZC, PAIR ? 2 : 1>::bytes;
        const float kF = kDerivUnit, ikF2 = 1.0f / (kDerivUnit * kDerivUnit);
        cudaError_t e;
        if (a.fwd_first && a.div_in) {
            e = set_smem(k_xexp<N, TZC, 2, false>, ColSm<N, TZC>::bytes);
            if (e != cudaSuccess) return e;
            k_xexp<N, TZC, 2, false><<<grid, TZC * PC, ColSm<N, TZC>::bytes, s>>>(a, g.tw, kF, ikF2);
        } else if (a.fwd_first) {
            e = set_smem(k_xexp<N, TZC, 1, PAIR>, smem);
            if (e != cudaSuccess) return e;
            k_xexp<N, TZC, 1, PAIR><<<grid, TZC * PC, smem, s>>>(a, g.tw, kF, ikF2);
        } else {
            e = set_smem(k_xexp<N, TZC, 0, PAIR>, smem);
            if (e != cudaSuccess) return e;
            k_xexp<N, TZC, 0, PAIR><<<grid, TZC * PC, smem, s>>>(a, g.tw, kF, ikF2);
        }
        return cudaGetLastError();
    }
    static cudaError_t yexp2(const Geo& g, const YZExpArgs& a, cudaStream_t s) {
        const int B = a.band > 0 && a.band < M ? a.band : 0;
        dim3 grid(((B ? B : M) + TZC - 1) / TZC, N);
        const size_t smem = sizeof(float2) * (N + (N & 1) + (size_t)N * TZC);
        cudaError_t e = set_smem(k_yexp2<N, TZC>, smem);
        if (e != cudaSuccess) return e;
        k_yexp2<N, TZC><<<grid, TZC / 2 * PC, smem, s>>>(a, g.tw, kDerivUnit);
        return cudaGetLastError();
    }
    template <bool PF = false, bool PAIR = false>
    static cudaError_t yexp(const Geo& g, const YZExpArgs& a, cudaStream_t s) {
        static_assert(!(PF && PAIR), "prefetching and paired outputs are separate variants");
        if constexpr (!ColSm<N, TZC, PAIR ? 2 : 1, PF ? N * TZC : 0>::fits) return cudaErrorNotSupported;
        else return yexp_fit<PF, PAIR>(g, a, s);
    }
    template <bool PF, bool PAIR>
    static cudaError_t yexp_fit(const Geo& g, const YZExpArgs& a, cudaStream_t s) {
        const int B = a.band > 0 && a.band < M ? a.band : 0;
        dim3 grid(((B ? B : M) + TZC - 1) / TZC, N);
        const size_t smem = ColSm<N, TZC, PAIR ? 2 : 1, PF ? N * TZC : 0>::bytes;
        cudaError_t e = set_smem(k_yexp<N, TZC, PF, PAIR>, smem);
        if (e != cudaSuccess) return e;
        k_yexp<N, TZC, PF, PAIR><<<grid, TZC * PC, smem, s>>>(a, g.tw, kDerivUnit);
        return cudaGetLastError();
    }
    template <bool PF>
    static cudaError_t zexp(const Geo& g, const YZExpArgs& a, cudaStream_t s) {
        const long long rows = (long long)N * N;
        dim3 grid((unsigned)((rows + TZZ - 1) / TZZ));
        const size_t smem = sizeof(float2) * (N + (PF ? 3 : 2) * (size_t)TZZ * PITCH);
        cudaError_t e = set_smem(k_zexp<N, TZZ, PF>, smem);
        if (e != cudaSuccess) return e;
        k_zexp<N, TZZ, PF><<<grid, TZZ * PZ, smem, s>>>(a, g.tw, kDerivUnit);
        return cudaGetLastError();
    }
    // TMA-staged y expansion: 8-column tiles, two tile buffers per block
    static cudaError_t yexp_tma(const Geo& g, const YZExpArgs& a, cudaStream_t s) {
        constexpr int TZ = 8;
        constexpr int BR = tma_rows(N);
        if (N < 128 || M % TZ != 0) return cudaErrorNotSupported;
        int nin = 0;
        for (int f = 0; f < a.nout; ++f) nin = (a.codes[f] & 255) + 1 > nin ? (a.codes[f] & 255) + 1 : nin;
        CUtensorMap map;
        // dims: kz (M), ky (N), x (N), field (nin); element = 8 bytes (one float2)
        const cuuint64_t dims[4] = {(cuuint64_t)M, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)nin};
        const cuuint64_t strides[3] = {(cuuint64_t)M * 8, (cuuint64_t)N * M * 8, (cuuint64_t)a.in_stride * 8};
        const cuuint32_t box[4] = {(cuuint32_t)TZ, (cuuint32_t)BR, 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        // host-side checks of the TMA rules: 16-byte aligned base and strides, inner box
        // extent a multiple of 16 bytes, box rows <= 256; every kz offset used is a
        // multiple of TZ = 8 columns (64 bytes)
        if ((reinterpret_cast<uintptr_t>(a.in) & 15) || (strides[2] & 15) || (TZ * 8) % 16 || BR > 256)
            return cudaErrorInvalidValue;
        cudaError_t e = encode_tensor_map(&map, const_cast<float2*>(a.in), dims, strides, box, estr);
        if (e != cudaSuccess) return e;
        const size_t smem = 2 * (size_t)N * TZ * sizeof(float2) + sizeof(float2) * N + 1024;   // + alignment slack
        if ((e = set_smem(k_yexp_tma<N, TZ>, smem)) != cudaSuccess) return e;
        dim3 grid(M / TZ, N);
        k_yexp_tma<N, TZ><<<grid, TZ * PC, smem, s>>>(a, map, g.tw, kDerivUnit, g.status);
        return cudaGetLastError();
    }
    static cudaError_t zexp_pairs(const Geo& g, const ZPairArgs& a, cudaStream_t s) {
        const long long rows = (long long)N * N;
        dim3 grid((unsigned)((rows + TZZ - 1) / TZZ));
        const size_t smem = sizeof(float2) * (N + 5 * (size_t)TZZ * PITCH);   // input, output, 3 partner tiles
        cudaError_t e;
        if (a.ntargets <= 1) {
            if ((e = set_smem(k_zexp_pairs<N, TZZ, 1>, smem)) != cudaSuccess) return e;
            k_zexp_pairs<N, TZZ, 1><<<grid, TZZ * PZ, smem, s>>>(a, g.tw, kDerivUnit);
        } else {
            if ((e = set_smem(k_zexp_pairs<N, TZZ, 2>, smem)) != cudaSuccess) return e;
            k_zexp_pairs<N, TZZ, 2><<<grid, TZZ * PZ, smem, s>>>(a, g.tw, kDerivUnit);
        }
        return cudaGetLastError();
    }
    // warp-row z pass (store only for NT = 0); persistent grid of resident blocks
    template <int NT>
    static cudaError_t zrow(const Geo& g, const ZPairArgs& a, cudaStream_t s) {
        return a.z.band > 0 ? zrow_k<NT, true>(g, a, s) : zrow_k<NT, false>(g, a, s);
    }
    template <int NT, bool BAND>
    static cudaError_t zrow_k(const Geo& g, const ZPairArgs& a, cudaStream_t s) {
        using C = RowCfg<N>;
        if constexpr (!C::ok) {
            return cudaErrorNotSupported;
        } else {
            const size_t smem = C::smem(NT);
            cudaError_t e = set_smem(k_zrow<N, NT, BAND>, smem);
            if (e != cudaSuccess) return e;
            int dev = 0, sms = 0, per = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zrow<N, NT, BAND>, kRowWarps * 32,
                                                                     smem)) != cudaSuccess)
                return e;
            const long long groups = (long long)N * N / C::RW;
            const long long need = (groups + kRowWarps - 1) / kRowWarps;
            const long long resident = (long long)(per > 0 ? per : 1) * sms;
            k_zrow<N, NT, BAND><<<(unsigned)(need < resident ? need : resident), kRowWarps * 32, smem, s>>>(
                a, g.tw, kDerivUnit);
            return cudaGetLastError();
        }
    }
    static int shell_blocks() { return (int)(((long long)N * N + TZZ - 1) / TZZ); }
    template <int NF, bool TRI>
    static cudaError_t zrow_shell(const Geo& g, const float2* in, long long st, int band, double* partial,
                                  cudaStream_t s) {
        using C = RowCfg<N>;
        if constexpr (!C::ok) {
            return cudaErrorNotSupported;
        } else {
            const size_t smem = sizeof(float2) * (C::HDR + (size_t)kRowWarps * C::RW * C::XROW);
            cudaError_t e = set_smem(k_zrow_shell<N, NF, TRI>, smem);
            if (e != cudaSuccess) return e;
            int dev = 0, sms = 0, per = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_zrow_shell<N, NF, TRI>, kRowWarps * 32,
                                                                     smem)) != cudaSuccess)
                return e;
            const long long groups = (long long)N * N / Cfg<N>::TZZ0;
            const long long need = (groups + kRowWarps - 1) / kRowWarps;
            const long long resident = (long long)(per > 0 ? per : 1) * sms;
            k_zrow_shell<N, NF, TRI><<<(unsigned)(need < resident ? need : resident), kRowWarps * 32, smem, s>>>(
                in, st, band, g.tw, partial, g.accum == kAccumFp64);
            return cudaGetLastError();
        }
    }
    template <int NF, bool TRI>
    static cudaError_t zshell_tile(const Geo& g, const float2* in, long long st, int band, double* partial,
                                   cudaStream_t s) {
        const size_t smem = sizeof(float2) * (N + (size_t)NF * TZZ * PITCH);
        cudaError_t e = set_smem(k_zshell<N, TZZ, NF, TRI>, smem);
        if (e != cudaSuccess) return e;
        k_zshell<N, TZZ, NF, TRI><<<shell_blocks(), TZZ * PZ, smem, s>>>(in, st, band, g.tw, partial,
                                                                          g.accum == kAccumFp64);
        return cudaGetLastError();
    }
    // nf: data fields (2: a, b; 3 with tri: a, b, c) plus J when present
    static cudaError_t zshell(const Geo& g, const float2* in, long long st, int band, int nf, int tri,
                              double* partial, cudaStream_t s) {
        if (g.var[TV_ZEXP] == 2 && RowCfg<N>::ok && TZZ == Cfg<N>::TZZ0) {
            if (tri) return nf == 4 ? zrow_shell<4, true>(g, in, st, band, partial, s)
                                    : zrow_shell<3, true>(g, in, st, band, partial, s);
            return nf == 3 ? zrow_shell<3, false>(g, in, st, band, partial, s)
                           : zrow_shell<2, false>(g, in, st, band, partial, s);
        }
        if (tri) return nf == 4 ? zshell_tile<4, true>(g, in, st, band, partial, s)
                                : zshell_tile<3, true>(g, in, st, band, partial, s);
        return nf == 3 ? zshell_tile<3, false>(g, in, st, band, partial, s)
                       : zshell_tile<2, false>(g, in, st, band, partial, s);
    }
};

// Per-size entry points (defined in the k_transform_*.cu units). The pass
// variant v selects tile widths: v = 0 default, v = 1 alternative.
#define GRIDSPT_TRANSFORM_SIZE(N)                                                                          \
    cudaError_t transform_colpass_##N(const Geo& g, float2* d, long long fs, int count, int axis, int fin, \
                                      long long s2, int band, int v, cudaStream_t s) {                     \
        return v ? Launch<N, Cfg<N>::TZC1, Cfg<N>::TZZ0>::colpass(g, d, fs, count, axis, fin, s2, band, s) \
                 : Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::colpass(g, d, fs, count, axis, fin, s2, band, s); \
    }                                                                                                      \
    cudaError_t transform_zr2c_##N(const Geo& g, const float2* in, float2* out, long long fs, int count,   \
                                   float scale, int band, int v, cudaStream_t s) {                         \
        if (v == 2 && RowCfg<N>::ok)                                                                       \
            return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::zrow_r2c(g, in, out, fs, count, scale, band, s);  \
        return v ? Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ1>::zr2c(g, in, out, fs, count, scale, band, s)      \
                 : Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::zr2c(g, in, out, fs, count, scale, band, s);     \
    }                                                                                                      \
    cudaError_t transform_xexp_##N(const Geo& g, const XExpArgs& a, int v, cudaStream_t s) {               \
        if (a.fwd_first && a.div_in) /* four input columns in registers: the narrower tile */              \
            return Launch<N, Cfg<N>::TZC1, Cfg<N>::TZZ0>::template xexp<false>(g, a, s);                   \
        if (v == 2) return Launch<N, Cfg<N>::TZC1, Cfg<N>::TZZ0>::template xexp<true>(g, a, s);            \
        if (v == 3) return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template xexp<true>(g, a, s);            \
        return v ? Launch<N, Cfg<N>::TZC1, Cfg<N>::TZZ0>::template xexp<false>(g, a, s)                    \
                 : Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template xexp<false>(g, a, s);                   \
    }                                                                                                      \
    cudaError_t transform_yexp_##N(const Geo& g, const YZExpArgs& a, int v, cudaStream_t s) {              \
        if (v == 2 && N >= 128 && a.band <= 0) return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::yexp_tma(g, a, s); \
        if (v == 3) return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::yexp2(g, a, s);                          \
        if (v == 4) return Launch<N, Cfg<N>::TZC1, Cfg<N>::TZZ0>::template yexp<true, false>(g, a, s);      \
        if (v == 5) return Launch<N, Cfg<N>::TZC1, Cfg<N>::TZZ0>::template yexp<false, true>(g, a, s);      \
        if (v == 6) return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template yexp<false, true>(g, a, s);      \
        return v == 1 ? Launch<N, Cfg<N>::TZC1, Cfg<N>::TZZ0>::template yexp<false, false>(g, a, s)        \
                      : Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template yexp<false, false>(g, a, s);       \
    }                                                                                                      \
    cudaError_t transform_zexp_##N(const Geo& g, const YZExpArgs& a, int v, cudaStream_t s) {              \
        if (a.band & 1) return cudaErrorInvalidValue; /* row copies move kz pairs */                       \
        if (v == 2 && RowCfg<N>::ok) {                                                                    \
            ZPairArgs za{};                                                                                \
            za.z = a;                                                                                      \
            return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template zrow<0>(g, za, s);                      \
        }                                                                                                  \
        return v == 1 ? Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template zexp<true>(g, a, s)                \
                      : Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template zexp<false>(g, a, s);              \
    }                                                                                                      \
    int transform_shell_blocks_##N() { return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::shell_blocks(); }     \
    cudaError_t transform_zexp_pairs_##N(const Geo& g, const ZPairArgs& a, cudaStream_t s) {               \
        if (a.z.band & 1) return cudaErrorInvalidValue; /* row copies move kz pairs */                     \
        if (g.var[TV_ZEXP] == 2 && RowCfg<N>::ok)                                                          \
            return a.ntargets <= 1 ? Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template zrow<1>(g, a, s)        \
                                   : Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::template zrow<2>(g, a, s);       \
        return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZP>::zexp_pairs(g, a, s);                                 \
    }                                                                                                      \
    cudaError_t transform_zshell_##N(const Geo& g, const float2* in, long long st, int band, int nf,       \
                                     int tri, double* partial, cudaStream_t s) {                           \
        return Launch<N, Cfg<N>::TZC0, Cfg<N>::TZZ0>::zshell(g, in, st, band, nf, tri, partial, s);        \
    }

}  // namespace gridspt
