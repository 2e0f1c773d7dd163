// Register-resident Stockham FFT used by every transform pass of the library.
//
// A batch of independent length-L transforms ("columns") is processed by one
// thread block. Thread p (0 <= p < P = L / E) of a column holds the E elements
// n = p + P * i (i = 0..E-1) in registers. Each radix-R stage does E / R
// butterflies per thread entirely in registers; between stages the outputs go
// through a shared-memory exchange buffer (Stockham autosort ordering), and
// after the last stage the thread again holds n = p + P * i in natural order,
// so a forward transform can feed an inverse transform without touching
// shared memory (used by the fused spectral-derivative pass).
//
// Sign convention: DIR = +1 computes y[n] = sum_t x[t] e^{+2 pi i n t / L}
// (the backward/synthesis sum of the paper's transform pair, Sec. II.C),
// DIR = -1 the analysis sum with e^{-...}; neither is normalised.
//
// Twiddle factors are read from a table of the N-th roots of unity
// e^{+2 pi i j / N} (FP64 on the host, rounded to FP32) held in shared memory;
// a length-L transform (L divides N) uses every (N / L)-th entry.
#pragma once
#include <cuda_runtime.h>

namespace gridspt {

// ----------------------------------------------------------- complex helpers
// The real and imaginary parts are combined with the packed two-lane FP32
// instructions of sm_100 and later (add/sub/mul/fma .rn .f32x2): each lane is
// rounded exactly as the scalar instruction would round it, so the results are
// those of the scalar forms below, with half the arithmetic instructions.
#ifndef GRIDSPT_PACKED_F32X2
#define GRIDSPT_PACKED_F32X2 1
#endif
#if GRIDSPT_PACKED_F32X2
__device__ __forceinline__ unsigned long long f2u(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 u2f(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(make_float2(s, s))));
    return u2f(r);
}
// (a.x b.x - a.y b.y, a.x b.y + a.y b.x): t = (a.y b.y, a.y b.x) rounded, then
// fma((a.x, a.x), (b.x, b.y), (-t.x, t.y)), as the scalar form
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    unsigned long long t, r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(f2u(make_float2(a.y, a.y))), "l"(f2u(make_float2(b.y, b.x))));
    const float2 tf = u2f(t);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r)
        : "l"(f2u(make_float2(a.x, a.x))), "l"(f2u(b)), "l"(f2u(make_float2(-tf.x, tf.y))));
    return u2f(r);
}
#else
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
#endif
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Lane-wise forms used by the pair products of real fields stored as float2
// pairs of cells: (a.x b.x, a.y b.y) and (fma(s, v.x, c.x), fma(s, v.y, c.y)),
// rounded as the scalar instructions.
#if GRIDSPT_PACKED_F32X2
__device__ __forceinline__ float2 lmul(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 lfma(float s, float2 v, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2u(make_float2(s, s))), "l"(f2u(v)), "l"(f2u(c)));
    return u2f(r);
}
#else
__device__ __forceinline__ float2 lmul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 lfma(float s, float2 v, float2 c) {
    return make_float2(fmaf(s, v.x, c.x), fmaf(s, v.y, c.y));
}
#endif
// multiply by DIR * i
template <int DIR>
__device__ __forceinline__ float2 cmul_i(float2 a) {
    return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------- radix schedule (L)
// Power-of-two lengths use E = 8 elements per thread: radix-8 stages and one
// final radix-2 or radix-4 stage. Lengths 3 * 2^a use E = 12 (E = 6 for L = 6):
// one radix-3 stage, then radix-4 stages and possibly one radix-2 stage.
__host__ __device__ constexpr bool fft_has3(int L) { return L % 3 == 0; }
__host__ __device__ constexpr int fft_pow2_part(int L) { return fft_has3(L) ? L / 3 : L; }
__host__ __device__ constexpr int fft_base(int L) { return fft_has3(L) ? 4 : 8; }
__host__ __device__ constexpr int fft_fullb(int m, int b) { return m >= b ? 1 + fft_fullb(m / b, b) : 0; }
__host__ __device__ constexpr int fft_remb(int m, int b) { return m >= b ? fft_remb(m / b, b) : m; }
__host__ __device__ constexpr int fft_nstages(int L) {
    return (fft_has3(L) ? 1 : 0) + fft_fullb(fft_pow2_part(L), fft_base(L)) +
           (fft_remb(fft_pow2_part(L), fft_base(L)) > 1 ? 1 : 0);
}
__host__ __device__ constexpr int fft_radix_p2(int m, int s, int b) {
    return s < fft_fullb(m, b) ? b : fft_remb(m, b);
}
__host__ __device__ constexpr int fft_radix(int L, int s) {
    return fft_has3(L) ? (s == 0 ? 3 : fft_radix_p2(fft_pow2_part(L), s - 1, 4))
                       : fft_radix_p2(L, s, 8);
}
__host__ __device__ constexpr int fft_ls(int L, int s) {  // product of radices before stage s
    return s == 0 ? 1 : fft_ls(L, s - 1) * fft_radix(L, s - 1);
}
__host__ __device__ constexpr int fft_elems(int L) {
    return fft_has3(L) ? (L >= 12 ? 12 : L) : (L >= 8 ? 8 : L);
}

// ------------------------------------------------------------ small DFTs
template <int R, int DIR>
__device__ __forceinline__ void dft_small(float2* v) {
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const float h = 0.86602540378443864676f;  // sqrt(3) / 2
        float2 s = cadd(v[1], v[2]);
        float2 d = csub(v[1], v[2]);
        float2 m = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
        float2 r = cscale(cmul_i<DIR>(d), h);
        v[0] = cadd(v[0], s);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    } else if constexpr (R == 4) {
        float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        float2 b0 = cadd(v[1], v[3]), b1 = cmul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(a0, b0);
        v[2] = csub(a0, b0);
        v[1] = cadd(a1, b1);
        v[3] = csub(a1, b1);
    } else if constexpr (R == 8) {
        const float r2 = 0.70710678118654752440f;  // 1 / sqrt(2)
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        dft_small<4, DIR>(e);
        dft_small<4, DIR>(o);
        // o[t] *= w8^t, w8 = (1 + DIR i) / sqrt(2)
        o[1] = cscale(cadd(o[1], cmul_i<DIR>(o[1])), r2);
        o[2] = cmul_i<DIR>(o[2]);
        o[3] = cscale(csub(cmul_i<DIR>(o[3]), o[3]), r2);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v[t] = cadd(e[t], o[t]);
            v[t + 4] = csub(e[t], o[t]);
        }
    }
}

// ------------------------------------------------------------- one stage
// Shared-memory exchange buffer of one column: element n at col[n * SN].
template <int L, int S, int DIR, int N>
__device__ __forceinline__ void fft_stage(float2 (&x)[fft_elems(L)], int p, float2* col, int SN,
                                          const float2* __restrict__ tw) {
    constexpr int E = fft_elems(L);
    constexpr int P = L / E;
    constexpr int R = fft_radix(L, S);
    constexpr int Ls = fft_ls(L, S);
    constexpr int Q = E / R;              // butterflies per thread
    constexpr int NS = fft_nstages(L);
    constexpr bool last = (S == NS - 1);
    constexpr int TWS = N / (Ls * R);     // table stride for angle t * k / (Ls * R)
    float2 y[E];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 v[R];
        const int b = p + q * P;          // butterfly index
        const int k = (Ls == 1) ? 0 : (b % Ls);
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = x[q + t * Q];
        if constexpr (Ls > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w = tw[t * k * TWS];  // t * k < Ls * R, so the index is < N
                if (DIR < 0) w.y = -w.y;
                v[t] = cmul(v[t], w);
            }
        }
        dft_small<R, DIR>(v);
        if constexpr (last) {
#pragma unroll
            for (int t = 0; t < R; ++t) y[q + t * Q] = v[t];
        } else {
            const int base = (b / Ls) * Ls * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t) col[(base + t * Ls) * SN] = v[t];
        }
    }
    if constexpr (last) {
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = y[i];
    } else {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = col[(p + P * i) * SN];
        __syncthreads();
    }
}

template <int L, int S, int DIR, int N>
__device__ __forceinline__ void fft_stages(float2 (&x)[fft_elems(L)], int p, float2* col, int SN,
                                           const float2* __restrict__ tw) {
    if constexpr (S < fft_nstages(L)) {
        fft_stage<L, S, DIR, N>(x, p, col, SN, tw);
        fft_stages<L, S + 1, DIR, N>(x, p, col, SN, tw);
    }
}

// Full length-L transform of the column whose exchange buffer is `col`
// (stride SN float2). Every thread of the block must call it the same number
// of times (it contains __syncthreads). tw: shared table of N-th roots.
template <int L, int DIR, int N>
__device__ __forceinline__ void fft_column(float2 (&x)[fft_elems(L)], int p, float2* col, int SN,
                                           const float2* __restrict__ tw) {
    fft_stages<L, 0, DIR, N>(x, p, col, SN, tw);
}


// ------------------------------------------------------- warp-row variant
// The same transform with the P threads of one length-L row on P consecutive
// lanes of one warp (P <= 32 and 32 % P == 0, so a warp holds 32 / P rows):
// the stage exchanges go through a per-warp buffer, ordered by __syncwarp, so
// rows never wait on a block-wide barrier. Stage arithmetic and twiddle values
// are those of fft_stage, so results are bitwise equal.
//
// Exchange buffer: element n of a row at xpad(n) = n + n / 16 (one float2 of
// padding per 16). With it every stage's scatter writes and gather reads of a
// warp take the minimum two shared-memory wavefronts for power-of-two L.
//
// Stage twiddles are read from a lane-major table twl[j][p] (conflict-free,
// identical for every row): j enumerates (stage S >= 1, butterfly q, t >= 1).
__device__ __forceinline__ int xpad(int n) { return n + (n >> 4); }

template <int L>
__host__ __device__ constexpr int fft_row_tw_count(int S) {   // stage twiddles of stages < S
    return S <= 0 ? 0
                  : fft_row_tw_count<L>(S - 1) +
                        (fft_ls(L, S - 1) > 1 ? (fft_elems(L) / fft_radix(L, S - 1)) * (fft_radix(L, S - 1) - 1) : 0);
}
template <int L>
__host__ __device__ constexpr int fft_row_tw_total() { return fft_row_tw_count<L>(fft_nstages(L)); }

// Fill twl[j * P + p] for p < P from the shared table of N-th roots tw.
template <int L, int N, int S = 0>
__device__ __forceinline__ void fft_row_twiddles(float2* twl, const float2* tw, int p) {
    if constexpr (S < fft_nstages(L)) {
        constexpr int E = fft_elems(L), P = L / E, R = fft_radix(L, S), Ls = fft_ls(L, S), Q = E / R;
        constexpr int TWS = N / (Ls * R);
        if constexpr (Ls > 1) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int k = (p + q * P) % Ls;
#pragma unroll
                for (int t = 1; t < R; ++t)
                    twl[(fft_row_tw_count<L>(S) + q * (R - 1) + (t - 1)) * P + p] = tw[t * k * TWS];
            }
        }
        fft_row_twiddles<L, N, S + 1>(twl, tw, p);
    }
}

template <int L, int S, int DIR>
__device__ __forceinline__ void fft_row_stage(float2 (&x)[fft_elems(L)], int p, float2* row,
                                              const float2* __restrict__ twl) {
    constexpr int E = fft_elems(L);
    constexpr int P = L / E;
    constexpr int R = fft_radix(L, S);
    constexpr int Ls = fft_ls(L, S);
    constexpr int Q = E / R;
    constexpr bool last = (S == fft_nstages(L) - 1);
    constexpr int J0 = fft_row_tw_count<L>(S);
    float2 y[E];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 v[R];
        const int b = p + q * P;
        const int k = (Ls == 1) ? 0 : (b % Ls);
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = x[q + t * Q];
        if constexpr (Ls > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w = twl[(J0 + q * (R - 1) + (t - 1)) * P + p];
                if (DIR < 0) w.y = -w.y;
                v[t] = cmul(v[t], w);
            }
        }
        dft_small<R, DIR>(v);
        if constexpr (last) {
#pragma unroll
            for (int t = 0; t < R; ++t) y[q + t * Q] = v[t];
        } else {
            const int base = (b / Ls) * Ls * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t) row[xpad(base + t * Ls)] = v[t];
        }
    }
    if constexpr (last) {
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = y[i];
    } else {
        __syncwarp();
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = row[xpad(p + P * i)];
        __syncwarp();
    }
}

template <int L, int S, int DIR>
__device__ __forceinline__ void fft_row_stages(float2 (&x)[fft_elems(L)], int p, float2* row,
                                               const float2* __restrict__ twl) {
    if constexpr (S < fft_nstages(L)) {
        fft_row_stage<L, S, DIR>(x, p, row, twl);
        fft_row_stages<L, S + 1, DIR>(x, p, row, twl);
    }
}

// Full length-L transform of one row held by P lanes (exchange buffer `row`,
// padded layout). Every lane of the warp must call it the same number of times.
template <int L, int DIR>
__device__ __forceinline__ void fft_row(float2 (&x)[fft_elems(L)], int p, float2* row,
                                        const float2* __restrict__ twl) {
    fft_row_stages<L, 0, DIR>(x, p, row, twl);
}


// ------------------------------------------------------ column-pair variant
// The same transform for two adjacent columns held by one thread (x[0], x[1]):
// each butterfly of fft_stage is done for both columns with one twiddle load,
// and the exchange moves both columns' elements in one 16-byte access (the
// buffer holds the two columns interleaved, i.e. the float2 layout of
// fft_column with columns 2c, 2c + 1). Per column the arithmetic is that of
// fft_stage, so results are bitwise equal.
template <int L, int S, int DIR, int N>
__device__ __forceinline__ void fft_stage_pair(float2 (&x)[2][fft_elems(L)], int p, float4* col, int SN,
                                               const float2* __restrict__ tw) {
    constexpr int E = fft_elems(L);
    constexpr int P = L / E;
    constexpr int R = fft_radix(L, S);
    constexpr int Ls = fft_ls(L, S);
    constexpr int Q = E / R;
    constexpr bool last = (S == fft_nstages(L) - 1);
    constexpr int TWS = N / (Ls * R);
    float2 y[2][E];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 v0[R], v1[R];
        const int b = p + q * P;
        const int k = (Ls == 1) ? 0 : (b % Ls);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            v0[t] = x[0][q + t * Q];
            v1[t] = x[1][q + t * Q];
        }
        if constexpr (Ls > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w = tw[t * k * TWS];
                if (DIR < 0) w.y = -w.y;
                v0[t] = cmul(v0[t], w);
                v1[t] = cmul(v1[t], w);
            }
        }
        dft_small<R, DIR>(v0);
        dft_small<R, DIR>(v1);
        if constexpr (last) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                y[0][q + t * Q] = v0[t];
                y[1][q + t * Q] = v1[t];
            }
        } else {
            const int base = (b / Ls) * Ls * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t) col[(base + t * Ls) * SN] = make_float4(v0[t].x, v0[t].y, v1[t].x, v1[t].y);
        }
    }
    if constexpr (last) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            x[0][i] = y[0][i];
            x[1][i] = y[1][i];
        }
    } else {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float4 u = col[(p + P * i) * SN];
            x[0][i] = make_float2(u.x, u.y);
            x[1][i] = make_float2(u.z, u.w);
        }
        __syncthreads();
    }
}

template <int L, int S, int DIR, int N>
__device__ __forceinline__ void fft_stages_pair(float2 (&x)[2][fft_elems(L)], int p, float4* col, int SN,
                                                const float2* __restrict__ tw) {
    if constexpr (S < fft_nstages(L)) {
        fft_stage_pair<L, S, DIR, N>(x, p, col, SN, tw);
        fft_stages_pair<L, S + 1, DIR, N>(x, p, col, SN, tw);
    }
}

template <int L, int DIR, int N>
__device__ __forceinline__ void fft_column_pair(float2 (&x)[2][fft_elems(L)], int p, float4* col, int SN,
                                                const float2* __restrict__ tw) {
    fft_stages_pair<L, 0, DIR, N>(x, p, col, SN, tw);
}


// ------------------------------------------------ column-pass variant (fft_col)
// The column transform of the column passes (colpass, x and y expansion), with
//  * NB = 2 exchange buffers used in turn (stage S writes buffer S % 2): a
//    buffer is rewritten only after a later block barrier that every reader of
//    its previous contents has passed, so each exchange takes one barrier
//    instead of two. A transform with an odd number of exchanges ends with a
//    barrier, so back-to-back transforms keep the alternation safe. NB = 1:
//    one buffer and two barriers per exchange, as fft_column.
//  * a padded exchange layout: element n of a column at col_row(n) * SN, one
//    padding row per 8 rows. The scatter of a radix-8 stage by a warp that
//    spans several butterflies of a narrow tile then hits distinct banks.
//  * the lane-major stage-twiddle table of fft_row, twl[j * P + p] (filled by
//    col_twiddles): the P-indexed twiddle loads of a warp read consecutive
//    entries instead of entries t * k * TWS apart.
// Butterfly arithmetic and twiddle values are those of fft_stage, so results
// are bitwise equal to fft_column.
__host__ __device__ constexpr int col_rows(int L) { return L + L / 8; }
__device__ __forceinline__ int col_row(int n) { return n + (n >> 3); }

// Fill the lane-major stage-twiddle table of a length-L column transform from
// the table of N-th roots (global or shared); threads p < P of the block each
// fill their own entries. The caller orders the table before its first use by
// a block barrier (the first exchange of fft_col has one before any stage
// that reads twiddles).
template <int L, int N>
__device__ __forceinline__ void col_twiddles(float2* twl, const float2* tw) {
    constexpr int P = L / fft_elems(L);
    if (threadIdx.x < P) fft_row_twiddles<L, N>(twl, tw, threadIdx.x);
}

template <int L, int S, int DIR, int NB>
__device__ __forceinline__ void fft_col_stage(float2 (&x)[fft_elems(L)], int p, float2* colA, float2* colB, int SN,
                                              const float2* __restrict__ twl) {
    constexpr int E = fft_elems(L);
    constexpr int P = L / E;
    constexpr int R = fft_radix(L, S);
    constexpr int Ls = fft_ls(L, S);
    constexpr int Q = E / R;
    constexpr bool last = (S == fft_nstages(L) - 1);
    constexpr int J0 = fft_row_tw_count<L>(S);
    float2* col = (NB == 2 && (S & 1)) ? colB : colA;
    float2 y[E];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 v[R];
        const int b = p + q * P;
        const int k = (Ls == 1) ? 0 : (b % Ls);
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = x[q + t * Q];
        if constexpr (Ls > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w = twl[(J0 + q * (R - 1) + (t - 1)) * P + p];
                if (DIR < 0) w.y = -w.y;
                v[t] = cmul(v[t], w);
            }
        }
        dft_small<R, DIR>(v);
        if constexpr (last) {
#pragma unroll
            for (int t = 0; t < R; ++t) y[q + t * Q] = v[t];
        } else {
            const int base = (b / Ls) * Ls * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t) col[col_row(base + t * Ls) * SN] = v[t];
        }
    }
    if constexpr (last) {
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = y[i];
    } else {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = col[col_row(p + P * i) * SN];
        if constexpr (NB == 1) __syncthreads();
    }
}

template <int L, int S, int DIR, int NB>
__device__ __forceinline__ void fft_col_stages(float2 (&x)[fft_elems(L)], int p, float2* colA, float2* colB, int SN,
                                               const float2* __restrict__ twl) {
    if constexpr (S < fft_nstages(L)) {
        fft_col_stage<L, S, DIR, NB>(x, p, colA, colB, SN, twl);
        fft_col_stages<L, S + 1, DIR, NB>(x, p, colA, colB, SN, twl);
    }
}

// Every thread of the block must call it the same number of times.
template <int L, int DIR, int NB>
__device__ __forceinline__ void fft_col(float2 (&x)[fft_elems(L)], int p, float2* colA, float2* colB, int SN,
                                        const float2* __restrict__ twl) {
    fft_col_stages<L, 0, DIR, NB>(x, p, colA, colB, SN, twl);
    if constexpr (NB == 2 && (fft_nstages(L) - 1) % 2 == 1) __syncthreads();
}

// Two columns per thread (the layout of fft_column_pair: 16-byte elements),
// same buffers, barriers and twiddle table as fft_col.
template <int L, int S, int DIR, int NB>
__device__ __forceinline__ void fft_col_pair_stage(float2 (&x)[2][fft_elems(L)], int p, float4* colA, float4* colB,
                                                   int SN, const float2* __restrict__ twl) {
    constexpr int E = fft_elems(L);
    constexpr int P = L / E;
    constexpr int R = fft_radix(L, S);
    constexpr int Ls = fft_ls(L, S);
    constexpr int Q = E / R;
    constexpr bool last = (S == fft_nstages(L) - 1);
    constexpr int J0 = fft_row_tw_count<L>(S);
    float4* col = (NB == 2 && (S & 1)) ? colB : colA;
    float2 y[2][E];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 v0[R], v1[R];
        const int b = p + q * P;
        const int k = (Ls == 1) ? 0 : (b % Ls);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            v0[t] = x[0][q + t * Q];
            v1[t] = x[1][q + t * Q];
        }
        if constexpr (Ls > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w = twl[(J0 + q * (R - 1) + (t - 1)) * P + p];
                if (DIR < 0) w.y = -w.y;
                v0[t] = cmul(v0[t], w);
                v1[t] = cmul(v1[t], w);
            }
        }
        dft_small<R, DIR>(v0);
        dft_small<R, DIR>(v1);
        if constexpr (last) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                y[0][q + t * Q] = v0[t];
                y[1][q + t * Q] = v1[t];
            }
        } else {
            const int base = (b / Ls) * Ls * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t)
                col[col_row(base + t * Ls) * SN] = make_float4(v0[t].x, v0[t].y, v1[t].x, v1[t].y);
        }
    }
    if constexpr (last) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            x[0][i] = y[0][i];
            x[1][i] = y[1][i];
        }
    } else {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float4 u = col[col_row(p + P * i) * SN];
            x[0][i] = make_float2(u.x, u.y);
            x[1][i] = make_float2(u.z, u.w);
        }
        if constexpr (NB == 1) __syncthreads();
    }
}

template <int L, int S, int DIR, int NB>
__device__ __forceinline__ void fft_col_pair_stages(float2 (&x)[2][fft_elems(L)], int p, float4* colA, float4* colB,
                                                    int SN, const float2* __restrict__ twl) {
    if constexpr (S < fft_nstages(L)) {
        fft_col_pair_stage<L, S, DIR, NB>(x, p, colA, colB, SN, twl);
        fft_col_pair_stages<L, S + 1, DIR, NB>(x, p, colA, colB, SN, twl);
    }
}

template <int L, int DIR, int NB>
__device__ __forceinline__ void fft_col_pair(float2 (&x)[2][fft_elems(L)], int p, float4* colA, float4* colB,
                                             int SN, const float2* __restrict__ twl) {
    fft_col_pair_stages<L, 0, DIR, NB>(x, p, colA, colB, SN, twl);
    if constexpr (NB == 2 && (fft_nstages(L) - 1) % 2 == 1) __syncthreads();
}

}  // namespace gridspt
