// 3D real<->half-complex transforms of the GridSPT path, as three axis passes.
//
// Layouts (every array is 4 N^3 bytes, no padding):
//   half spectrum / mixed data: float2[N][N][M], M = N / 2, index [x|kx][y|ky][kz]
//   real field:                 float[N][N][N]
// Backward (Sec. II.C synthesis sum a(x) = sum_k a(k) e^{i k.x}):
//   x pass (columns along the slowest axis, stride N*M)  -> k_derive or k_colpass
//   y pass (columns along the middle axis, stride M)     -> k_colpass
//   z pass (contiguous rows, half-complex -> real)       -> k_zc2r
// Forward (analysis sum, N^-3 folded into the producer): k_zr2c, then y, then x.
//
// Column passes stage a tile of TZ adjacent kz columns (TZ * 8 contiguous bytes
// per row of the column) and keep each column in registers (fft_core.cuh).
// The contiguous-axis passes use the half-length complex transform of the
// packed sequence z[m] = x[2m] + i x[2m+1]; the Nyquist coefficient X[N/2] is
// zero in every spectrum of this library and is not stored.
#include "fft_core.cuh"
#include "gridspt_internal.h"

namespace gridspt {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int N>
struct Cfg {
    static constexpr int M = N / 2;
    // column passes (length N)
    static constexpr int EC = fft_elems(N);
    static constexpr int PC = N / EC;
    static constexpr int TZC = cmin(16, 1024 / PC);
    static constexpr int TZD = cmin(16, 1024 / PC);  // fused derive pass
    // contiguous-axis passes (length M)
    static constexpr int EZ = fft_elems(M);
    static constexpr int PZ = M / EZ;
    // 16 rows or more per block: a warp then spans 16 rows of the odd-pitch
    // tile, so column accesses of a warp hit 16 distinct 8-byte bank pairs
    static constexpr int TZZ = cmin(cmin(64, cmax(16, 256 / PZ)), 1024 / PZ);
    static constexpr int PITCH = M + 1;
};

__device__ __forceinline__ int signed_idx(int n, int N) { return n < N / 2 ? n : n - N; }

__device__ __forceinline__ void load_table(float2* tw, const float2* __restrict__ twg, int N) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
}

// Copy TZ contiguous rows of M float2 between global memory and a shared tile
// of odd pitch PITCH. Consecutive threads move consecutive float2 of a row
// (coalesced, conflict-free); all loads are issued before the shared stores,
// so each thread has TZ * M / NTHR requests in flight.
template <int M, int TZ, int PITCH, int NTHR>
__device__ __forceinline__ void tile_load(float2* tile, const float2* src, long long row0, long long rows) {
    constexpr int NV = TZ * M;
    constexpr int PER = (NV + NTHR - 1) / NTHR;
    float2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NTHR;
        const int r = idx / M, j = idx - r * M;
        const long long row = row0 + r;
        v[u] = (idx < NV && row < rows) ? src[row * M + j] : make_float2(0.f, 0.f);
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

// ------------------------------------------------------------ column pass
template <int N, int DIR, int AXIS, bool FIN>
__global__ void __launch_bounds__(Cfg<N>::TZC * Cfg<N>::PC)
k_colpass(float2* __restrict__ data, long long fstride, const float2* __restrict__ twg,
          long long s2_nl) {
    constexpr int M = N / 2, E = fft_elems(N), P = N / E, TZ = Cfg<N>::TZC;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    load_table(tw, twg, N);
    const int kz = blockIdx.x * TZ + c;
    const int a = blockIdx.y;
    const bool act = kz < M;
    constexpr long long estride = AXIS == 0 ? (long long)N * M : (long long)M;
    constexpr long long astride = AXIS == 0 ? (long long)M : (long long)N * M;
    float2* col = data + blockIdx.z * fstride + a * astride + kz;
    float2 x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = act ? col[(p + P * i) * estride] : make_float2(0.f, 0.f);
    __syncthreads();
    fft_column<N, DIR, N>(x, p, buf + c, TZ, tw);
    if constexpr (FIN) {
        const int sy = signed_idx(a, N), sz = kz;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n = p + P * i;
            const int sx = signed_idx(n, N);
            const long long s2 = (long long)sx * sx + (long long)sy * sy + (long long)sz * sz;
            if (n == N / 2 || a == N / 2 || (s2_nl >= 0 && s2 > s2_nl)) x[i] = make_float2(0.f, 0.f);
        }
    }
    if (act) {
#pragma unroll
        for (int i = 0; i < E; ++i) col[(p + P * i) * estride] = x[i];
    }
}

// ------------------------------------------------ contiguous axis: C2R
template <int N>
__global__ void __launch_bounds__(Cfg<N>::TZZ * Cfg<N>::PZ)
k_zc2r(const float2* in, float2* out, long long fstride,
       const float2* __restrict__ twg) {
    constexpr int M = N / 2, E = fft_elems(M), P = M / E, TZ = Cfg<N>::TZZ, PITCH = Cfg<N>::PITCH;
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
    for (int i = 0; i < E; ++i) {
        const int k = p + P * i;
        const float2 Xk = colp[k];
        const float2 Xm = k ? cconj(colp[M - k]) : make_float2(0.f, 0.f);  // X[k + M]
        const float2 Ev = cadd(Xk, Xm);
        const float2 Ov = cmul(csub(Xk, Xm), tw[k]);                       // e^{+2 pi i k / N}
        x[i] = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);                      // E + i O
    }
    __syncthreads();
    fft_column<M, +1, N>(x, p, colp, 1, tw);
#pragma unroll
    for (int i = 0; i < E; ++i) colp[p + P * i] = x[i];
    __syncthreads();
    tile_store<M, TZ, PITCH, TZ * P>(dst, tile, row0, rows);
}

// ------------------------------------------------ contiguous axis: R2C
template <int N>
__global__ void __launch_bounds__(Cfg<N>::TZZ * Cfg<N>::PZ)
k_zr2c(const float2* in, float2* out, long long fstride,
       const float2* __restrict__ twg, float scale) {
    constexpr int M = N / 2, E = fft_elems(M), P = M / E, TZ = Cfg<N>::TZZ, PITCH = Cfg<N>::PITCH;
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
        if (idx >= NV || row >= rows) continue;
        const float2 Z = tile[r * PITCH + k];
        const float2 Zr = cconj(tile[r * PITCH + (k ? M - k : 0)]);
        const float2 S = cadd(Z, Zr);                      // 2 E[k]
        const float2 t = cmul(cconj(tw[k]), csub(Z, Zr));  // e^{-2 pi i k/N} 2i O[k]
        // X = E + e^{-2 pi i k / N} O = (S - i t) / 2
        dst[row * M + k] = make_float2(half * (S.x + t.y), half * (S.y - t.x));
    }
}

// --------------------------------------- fused spectral derivative + x pass
// Each output f: out_f(k) = mult_f(k) * src(k) (Sec. II.C steps (2)/(5)),
// transformed backward along x. With FWD, the inputs are first transformed
// forward along x and finalised (completing delta_n(k), theta_n(k), which are
// stored back in place) so that the spectrum is read from HBM only once.
template <int N, bool FWD>
__global__ void __launch_bounds__(Cfg<N>::TZD * Cfg<N>::PC)
k_derive(DeriveArgs args, const float2* __restrict__ twg, float kF, float inv_kF) {
    constexpr int M = N / 2, E = fft_elems(N), P = N / E, TZ = Cfg<N>::TZD;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* buf = sm + N;
    const int tid = threadIdx.x, c = tid % TZ, p = tid / TZ;
    load_table(tw, twg, N);
    const int kz = blockIdx.x * TZ + c;
    const int ky = blockIdx.y;
    const bool act = kz < M;
    constexpr long long estride = (long long)N * M;
    const long long colofs = (long long)ky * M + kz;
    const bool two = args.src1 != args.src0;
    float2 xd[E], xt[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        xd[i] = act ? args.src0[colofs + (p + P * i) * estride] : make_float2(0.f, 0.f);
        xt[i] = (act && two) ? args.src1[colofs + (p + P * i) * estride] : xd[i];
    }
    __syncthreads();
    const int sy = signed_idx(ky, N), sz = kz;
    if constexpr (FWD) {
        fft_column<N, -1, N>(xd, p, buf + c, TZ, tw);
        if (two) fft_column<N, -1, N>(xt, p, buf + c, TZ, tw);
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n = p + P * i;
            const int sx = signed_idx(n, N);
            const long long s2 = (long long)sx * sx + (long long)sy * sy + (long long)sz * sz;
            if (n == N / 2 || ky == N / 2 || (args.s2_nl >= 0 && s2 > args.s2_nl)) {
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
    for (int f = 0; f < args.nout; ++f) {
        const int code = args.codes[f];
        const int kind = code & 15, ca = (code >> 4) & 3, cb = (code >> 6) & 3, src = (code >> 8) & 3;
        float2 y[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n = p + P * i;
            const int sx = signed_idx(n, N);
            const int sa = ca == 0 ? sx : (ca == 1 ? sy : sz);
            const int sb = cb == 0 ? sx : (cb == 1 ? sy : sz);
            const int s2 = sx * sx + sy * sy + sz * sz;
            const float2 v = src == 0 ? xd[i] : (src == 1 ? xt[i] : make_float2(1.f, 0.f));
            float2 r;
            if (kind == DK_ONE) {
                r = v;
            } else if (kind == DK_IK) {
                const float ka = kF * (float)sa;
                r = make_float2(-ka * v.y, ka * v.x);
            } else if (kind == DK_NEG_IK_K2) {
                const float g = s2 ? inv_kF * (float)sa / (float)s2 : 0.f;
                r = make_float2(g * v.y, -g * v.x);
            } else if (kind == DK_KK_K2) {
                const float g = s2 ? (float)(sa * sb) / (float)s2 : 0.f;
                r = make_float2(g * v.x, g * v.y);
            } else {  // DK_SHELL
                const bool in = s2 > 0 && (long long)s2 >= args.shell_lo && (long long)s2 < args.shell_hi;
                r = in ? v : make_float2(0.f, 0.f);
            }
            y[i] = r;
        }
        fft_column<N, +1, N>(y, p, buf + c, TZ, tw);
        if (act) {
            float2* o = args.out + f * args.out_stride + colofs;
#pragma unroll
            for (int i = 0; i < E; ++i) o[(p + P * i) * estride] = y[i];
        }
    }
}

// ------------------------------------------------------------- launchers
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

template <int N>
struct Launch {
    static cudaError_t colpass(const Geo& g, float2* d, long long fs, int count, int axis, int dir,
                               int fin, long long s2_nl, cudaStream_t s) {
        using C = Cfg<N>;
        dim3 grid((C::M + C::TZC - 1) / C::TZC, N, count);
        const int thr = C::TZC * C::PC;
        const size_t smem = sizeof(float2) * (N + (size_t)N * C::TZC);
        cudaError_t e;
#define GRIDSPT_COL(DIR_, AX_, FIN_)                                                  \
    e = set_smem(k_colpass<N, DIR_, AX_, FIN_>, smem);                               \
    if (e != cudaSuccess) return e;                                                   \
    k_colpass<N, DIR_, AX_, FIN_><<<grid, thr, smem, s>>>(d, fs, g.tw, s2_nl);        \
    return cudaGetLastError();
        if (axis == 0) {
            if (dir > 0) { GRIDSPT_COL(+1, 0, false) }
            if (fin) { GRIDSPT_COL(-1, 0, true) }
            GRIDSPT_COL(-1, 0, false)
        } else {
            if (dir > 0) { GRIDSPT_COL(+1, 1, false) }
            GRIDSPT_COL(-1, 1, false)
        }
#undef GRIDSPT_COL
    }
    static cudaError_t zc2r(const Geo& g, const float2* in, float2* out, long long fs, int count,
                            cudaStream_t s) {
        using C = Cfg<N>;
        const long long rows = (long long)N * N;
        dim3 grid((unsigned)((rows + C::TZZ - 1) / C::TZZ), count);
        const size_t smem = sizeof(float2) * (N + (size_t)C::TZZ * C::PITCH);
        cudaError_t e = set_smem(k_zc2r<N>, smem);
        if (e != cudaSuccess) return e;
        k_zc2r<N><<<grid, C::TZZ * C::PZ, smem, s>>>(in, out, fs, g.tw);
        return cudaGetLastError();
    }
    static cudaError_t zr2c(const Geo& g, const float2* in, float2* out, long long fs, int count,
                            float scale, cudaStream_t s) {
        using C = Cfg<N>;
        const long long rows = (long long)N * N;
        dim3 grid((unsigned)((rows + C::TZZ - 1) / C::TZZ), count);
        const size_t smem = sizeof(float2) * (N + (size_t)C::TZZ * C::PITCH);
        cudaError_t e = set_smem(k_zr2c<N>, smem);
        if (e != cudaSuccess) return e;
        k_zr2c<N><<<grid, C::TZZ * C::PZ, smem, s>>>(in, out, fs, g.tw, scale);
        return cudaGetLastError();
    }
    static cudaError_t derive(const Geo& g, const DeriveArgs& a, cudaStream_t s) {
        using C = Cfg<N>;
        dim3 grid((C::M + C::TZD - 1) / C::TZD, N);
        const int thr = C::TZD * C::PC;
        const size_t smem = sizeof(float2) * (N + (size_t)N * C::TZD);
        const float kF = (float)g.kF, ikF = (float)(1.0 / g.kF);
        cudaError_t e;
        if (a.fwd_first) {
            e = set_smem(k_derive<N, true>, smem);
            if (e != cudaSuccess) return e;
            k_derive<N, true><<<grid, thr, smem, s>>>(a, g.tw, kF, ikF);
        } else {
            e = set_smem(k_derive<N, false>, smem);
            if (e != cudaSuccess) return e;
            k_derive<N, false><<<grid, thr, smem, s>>>(a, g.tw, kF, ikF);
        }
        return cudaGetLastError();
    }
};

#define GRIDSPT_FOR_EACH_N(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) \
    X(256) X(384) X(512) X(768) X(1024)

bool supported_n(int N) {
    switch (N) {
#define GRIDSPT_CASE(n) case n:
        GRIDSPT_FOR_EACH_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        return true;
        default: return false;
    }
}

cudaError_t launch_colpass(const Geo& g, float2* data, long long fstride, int count, int axis,
                           int dir, int finalize, long long s2_nl, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return Launch<n>::colpass(g, data, fstride, count, axis, dir, finalize, s2_nl, s);
        GRIDSPT_FOR_EACH_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zc2r(const Geo& g, const float2* in, float2* out, long long fstride, int count,
                        cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return Launch<n>::zc2r(g, in, out, fstride, count, s);
        GRIDSPT_FOR_EACH_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zr2c(const Geo& g, const float2* in, float2* out, long long fstride, int count,
                        float scale, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return Launch<n>::zr2c(g, in, out, fstride, count, scale, s);
        GRIDSPT_FOR_EACH_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_derive(const Geo& g, const DeriveArgs& a, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return Launch<n>::derive(g, a, s);
        GRIDSPT_FOR_EACH_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gridspt
