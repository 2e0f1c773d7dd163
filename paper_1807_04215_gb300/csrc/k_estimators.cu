// Shell estimators (Sec. III.B.1).
//
// Power (Eqs. pk_lin, pk_1loop, pk_2loop): P_ab(i) = L^3 / N_i sum_{k in bin i}
// Re[a(k) b*(k)] over the full grid. The half spectrum stores kz >= 0; modes
// with kz > 0 stand for themselves and their conjugate partners (weight 2),
// the kz = 0 plane holds both members of each pair (weight 1). Bins are
// integer ranges of |s|^2 precomputed on the host from the FP64 edges, so
// the bin decision equals the FP64 test edges[i] <= k_F sqrt(|s|^2).
//
// Determinism: one warp per (kx, ky) row, chunks of 32 consecutive kz (two
// chunks per step, scanned side by side). Along a row the bin index is
// non-decreasing in kz, so lanes with equal bins are contiguous: a segmented
// shuffle scan sums each run and its last lane adds the run to the warp's FP64
// accumulator (one writer per bin per chunk, chunks in kz order). Warps
// and blocks are then summed in a fixed order: results are bitwise repeatable.
// The scan runs in FP32 with each addition's rounding error carried exactly
// (Knuth's two-sum) and added at the tail, so a run's sum is good to about
// FP32^2 while the FP64 pipe (a small fraction of the FP32 rate here) sees
// one addition per run; the mode counts are exact in FP32. With the FP64
// accumulator choice (Geo::accum = kAccumFp64) every product is formed and
// scanned in FP64 instead (the FP32 inputs' products are exact in FP64).
// The final kernels flag a NaN or infinite result in the plan's status word
// (kStatusNonFinite), which gridspt_check reports as GRIDSPT_E_NUMERIC.
//
// Bispectrum (Eq. bk_tree, FFT shell estimator): the per-shell sums are formed
// in k_zshell (k_transform.cuh); the final fixed-order reduction is here.
#include "gridspt_internal.h"

namespace gridspt {

constexpr int kPowWarps = 8;

int power_blocks(const Geo& g) {
    const long long rows = (long long)g.N * g.N;
    long long b = (rows + kPowWarps - 1) / kPowWarps;
    return (int)(b < kPowerMaxBlocks ? b : kPowerMaxBlocks);
}

// Segmented inclusive scan over runs of equal bin within a warp; T = float
// (two-sum compensated, error carried in e) or double (plain FP64 adds, e
// unused). The scan's shuffles and the run boundaries are the same for both.
template <typename T>
__device__ __forceinline__ void seg_scan(T (&v)[2], T (&e)[2], float (&c)[2], const int (&bin)[2], int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T ov = __shfl_up_sync(0xffffffffu, v[h], off);
            T oe = T(0);
            if constexpr (sizeof(T) == 4) oe = __shfl_up_sync(0xffffffffu, e[h], off);
            const float oc = __shfl_up_sync(0xffffffffu, c[h], off);
            const int ob = __shfl_up_sync(0xffffffffu, bin[h], off);
            if (lane >= off && ob == bin[h]) {
                if constexpr (sizeof(T) == 4) {
                    const float t = __fadd_rn(v[h], ov);         // two-sum: t + r = v + ov exactly
                    const float bv = __fsub_rn(t, v[h]);
                    const float r = __fadd_rn(__fsub_rn(v[h], __fsub_rn(t, bv)), __fsub_rn(ov, bv));
                    v[h] = t;
                    e[h] = __fadd_rn(__fadd_rn(e[h], oe), r);
                } else {
                    v[h] = v[h] + ov;
                }
                c[h] += oc;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kPowWarps * 32)
k_power(const float2* __restrict__ a, const float2* __restrict__ b, BinSpec bins, int N, int M,
        double* __restrict__ partial) {
    __shared__ double acc[kPowWarps][2 * kMaxBins];
    __shared__ int thr[kMaxBins + 1];
    const int nb = bins.nbins;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kPowWarps * 2 * kMaxBins; i += blockDim.x) (&acc[0][0])[i] = 0.0;
    for (int i = threadIdx.x; i <= nb; i += blockDim.x) thr[i] = bins.thr[i];
    __syncthreads();
    const int top = thr[nb];
    const long long rows = (long long)N * N;
    for (long long row = (long long)blockIdx.x * kPowWarps + w; row < rows;
         row += (long long)gridDim.x * kPowWarps) {
        const int kx = (int)(row / N), ky = (int)(row % N);
        const int sx = kx < N / 2 ? kx : kx - N;
        const int sy = ky < N / 2 ? ky : ky - N;
        const int sxy = sx * sx + sy * sy;
        if (sxy >= top) continue;
        const float2* ar = a + row * M;
        const float2* br = b + row * M;
        // two chunks of 32 kz per step: their scans are independent chains
        // (latency hiding); their sums reach acc in chunk order, as one at a time
        for (int kz0 = 0; kz0 < M; kz0 += 64) {
            if (sxy + kz0 * kz0 >= top) break;
            T v[2], e[2];                        // sum, carried rounding error (FP32 only)
            float c[2];                          // weight (mode count)
            int bin[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kz = kz0 + 32 * h + lane;
                const int s2 = sxy + kz * kz;
                if (kz >= M || s2 >= top) {
                    bin[h] = nb;                 // above every bin
                } else if (s2 == 0 || s2 < thr[0]) {
                    bin[h] = -1;                 // k = 0 or below the first edge
                } else {
                    int lo = 0, hi = nb;         // thr[lo] <= s2 < thr[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (thr[mid] <= s2) lo = mid; else hi = mid;
                    }
                    bin[h] = lo;
                }
                v[h] = T(0);
                e[h] = T(0);
                c[h] = 0.f;
                if (bin[h] >= 0 && bin[h] < nb) {
                    const float2 x = ar[kz], y = br[kz];
                    const float wgt = kz == 0 ? 1.f : 2.f;
                    if constexpr (sizeof(T) == 4)
                        v[h] = wgt * fmaf(x.x, y.x, x.y * y.y);
                    else
                        v[h] = (double)wgt * ((double)x.x * (double)y.x + (double)x.y * (double)y.y);
                    c[h] = wgt;
                }
            }
            seg_scan<T>(v, e, c, bin, lane);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int nxt = __shfl_down_sync(0xffffffffu, bin[h], 1);
                const bool tail = (lane == 31) || (nxt != bin[h]);
                if (tail && bin[h] >= 0 && bin[h] < nb) {
                    acc[w][bin[h]] += (double)v[h] + (double)e[h];
                    acc[w][kMaxBins + bin[h]] += (double)c[h];
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        double s = 0.0, c = 0.0;
        for (int ww = 0; ww < kPowWarps; ++ww) {
            s += acc[ww][t];
            c += acc[ww][kMaxBins + t];
        }
        partial[(long long)blockIdx.x * 2 * nb + t] = s;
        partial[(long long)blockIdx.x * 2 * nb + nb + t] = c;
    }
}

// One block per bin: thread t sums partials t, t + 256, ... in order, then a
// fixed shared-memory tree; bitwise repeatable.
__global__ void __launch_bounds__(256)
k_power_final(const double* __restrict__ partial, int G, int nb, double vol,
              double* __restrict__ p_out, int64_t* __restrict__ nk_out, int* __restrict__ status) {
    __shared__ double rs[256], rc[256];
    const int t = blockIdx.x;
    double s = 0.0, c = 0.0;
    for (int g = threadIdx.x; g < G; g += 256) {
        s += partial[(long long)g * 2 * nb + t];
        c += partial[(long long)g * 2 * nb + nb + t];
    }
    rs[threadIdx.x] = s;
    rc[threadIdx.x] = c;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            rs[threadIdx.x] += rs[threadIdx.x + h];
            rc[threadIdx.x] += rc[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double pv = rc[0] > 0.0 ? vol * rs[0] / rc[0] : 0.0;
        p_out[t] = pv;
        if (nk_out) nk_out[t] = (int64_t)(rc[0] + 0.5);
        if (!isfinite(pv)) atomicOr(status, kStatusNonFinite);
    }
}

cudaError_t launch_power(const Geo& g, const float2* a, const float2* b, const BinSpec& bins,
                         double* partial, double* p_out, int64_t* nk_out, double volume,
                         cudaStream_t s) {
    const int G = power_blocks(g);
    if (g.accum == kAccumFp64)
        k_power<double><<<G, kPowWarps * 32, 0, s>>>(a, b, bins, g.N, g.M, partial);
    else
        k_power<float><<<G, kPowWarps * 32, 0, s>>>(a, b, bins, g.N, g.M, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_power_final<<<bins.nbins, 256, 0, s>>>(partial, G, bins.nbins, volume, p_out, nk_out, g.status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ bispectrum
// Final reduction of the per-block partials written by k_zshell (one shell):
// E = L^6 sum I_a^2 I_b / sum J^3, N_tri = sum J^3 / N^3; one block, fixed order.
__global__ void __launch_bounds__(256)
k_bispec_final(const double* __restrict__ partial, int G, int nfields, double* __restrict__ j3_cache, double vol2,
               double cells, double* __restrict__ e_out, double* __restrict__ ntri_out, int* __restrict__ status) {
    __shared__ double r1[256], r2[256];
    double s1 = 0.0, s2 = 0.0;
    for (int g = threadIdx.x; g < G; g += 256) {
        s1 += partial[2 * g];
        s2 += partial[2 * g + 1];
    }
    r1[threadIdx.x] = s1;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            r1[threadIdx.x] += r1[threadIdx.x + h];
            r2[threadIdx.x] += r2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double j3 = r2[0];
        if (nfields == 3) *j3_cache = j3;
        else j3 = *j3_cache;
        const double nt = j3 / cells;
        const double ev = nt > 0.5 ? vol2 * r1[0] / j3 : 0.0;
        *ntri_out = nt;
        *e_out = ev;
        if (!isfinite(ev) || !isfinite(nt) || !isfinite(r1[0])) atomicOr(status, kStatusNonFinite);
    }
}

cudaError_t launch_bispec_final(const Geo& g, const double* partial, int blocks, int nfields, double* j3_cache,
                                double* e_out, double* ntri_out, double vol2, cudaStream_t s) {
    k_bispec_final<<<1, 256, 0, s>>>(partial, blocks, nfields, j3_cache, vol2, (double)g.N * g.N * g.N, e_out,
                                     ntri_out, g.status);
    return cudaGetLastError();
}

// Sub-grid copy for the bispectrum: every shell field is band limited (each
// component |s_a| < B), so the sums over cells of a product of three shell
// fields only see the wavevector sums s_1 + s_2 + s_3 = 0 on any grid of size
// S > 3 (B - 1) (no other sum is a multiple of S), and the shells can be
// evaluated on that smaller grid. Two modes (one 16-byte vector) per thread;
// blockIdx.y selects the field.
struct SubgridArgs {
    const float2* in[3];
    float2* out;
    long long out_stride;
    int N, S;
};

__global__ void __launch_bounds__(256) k_subgrid(SubgridArgs a) {
    const int S = a.S, MS = S / 2, N = a.N, MN = N / 2;
    const long long pairs = (long long)S * S * (MS / 2);
    const long long i2 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i2 >= pairs) return;
    const long long m0 = 2 * i2;                  // even kz, kz + 1 < S / 2
    const int kz = (int)(m0 % MS);
    const long long xy = m0 / MS;
    const int iy = (int)(xy % S), ix = (int)(xy / S);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ix != S / 2 && iy != S / 2) {
        const int bx = ix < S / 2 ? ix : ix - S + N;
        const int by = iy < S / 2 ? iy : iy - S + N;
        v = __ldg(reinterpret_cast<const float4*>(a.in[blockIdx.y] + ((long long)bx * N + by) * MN + kz));
    }
    reinterpret_cast<float4*>(a.out + blockIdx.y * a.out_stride)[i2] = v;
}

cudaError_t launch_subgrid(int N, int S, const float2* const* in, int nin, float2* out, long long out_stride,
                           cudaStream_t s) {
    if (nin < 1 || nin > 3 || S > N || S < 8 || (S / 2) % 2) return cudaErrorInvalidValue;
    SubgridArgs a{};
    for (int f = 0; f < nin; ++f) a.in[f] = in[f];
    a.out = out;
    a.out_stride = out_stride;
    a.N = N;
    a.S = S;
    const long long pairs = (long long)S * S * (S / 4);
    k_subgrid<<<dim3((unsigned)((pairs + 255) / 256), (unsigned)nin), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gridspt
