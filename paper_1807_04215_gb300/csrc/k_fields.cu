// Field-level products of the recursion (Sec. III.A and Sec. III.B):
//
// * delta_SPT(k) = W(k R) sum_{i=1}^{n} D_+^i delta_i(k), W(x) = exp(-x^2 / 2):
//   the summed density field the paper smooths with a Gaussian filter before
//   comparing fields. Elementwise over the half spectrum, two modes (one
//   16-byte vector) per thread; the powers D_+^i arrive from the host (FP64,
//   rounded to FP32), W in FP32.
// * the cross-correlation coefficient r = P_ab / sqrt(P_aa P_bb) per bin
//   (Eqs. r_corr_nthPT, r_corr_sum_nth) from three shell power spectra (the
//   volume and N_k factors cancel), FP64.
// * zeros outside the band columns of band-limited spectra (run_orders).
#include "gridspt_internal.h"

namespace gridspt {

namespace {

__global__ void __launch_bounds__(256) k_sum_orders(SumOrdersArgs a) {
    const long long half = (long long)a.N * a.N * (a.N / 2);   // modes of the half spectrum
    const long long i2 = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // pair of modes
    if (2 * i2 >= half) return;
    const int M = a.N / 2;
    const long long m0 = 2 * i2;
    const int kz = (int)(m0 % M);                  // even; kz + 1 < M
    const long long xy = m0 / M;
    const int ky = (int)(xy % a.N), kx = (int)(xy / a.N);
    const int sx = kx < a.N / 2 ? kx : kx - a.N, sy = ky < a.N / 2 ? ky : ky - a.N;
    const float syx = (float)(sx * sx + sy * sy);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < a.n; ++i) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(a.field[i]) + i2);
        const float c = a.coef[i];
        acc.x = fmaf(c, v.x, acc.x);
        acc.y = fmaf(c, v.y, acc.y);
        acc.z = fmaf(c, v.z, acc.z);
        acc.w = fmaf(c, v.w, acc.w);
    }
    if (a.r2kf2 > 0.f) {
        const float w0 = expf(-0.5f * a.r2kf2 * (syx + (float)(kz * kz)));
        const float w1 = expf(-0.5f * a.r2kf2 * (syx + (float)((kz + 1) * (kz + 1))));
        acc.x *= w0;
        acc.y *= w0;
        acc.z *= w1;
        acc.w *= w1;
    }
    reinterpret_cast<float4*>(a.out)[i2] = acc;
}

// Spectra of order n >= 2 formed from band-limited lower orders are zero
// outside the band columns; the x pass that finalises them moves only those
// columns, and this kernel writes the zeros of the others. One 16-byte vector
// (two kz modes) per thread, blockIdx.y selects the field.
__global__ void __launch_bounds__(256) k_zero_outside_band(float2* f0, float2* f1, int N, int band) {
    const int H = N / 4;                           // 16-byte pairs per row
    const int pairs = N * N * H;                   // < 2^31 for N <= 1024
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (i2 >= pairs) return;
    const int row = i2 / H;
    const int kz = 2 * (i2 - row * H);             // even: the pair lies on one side of the even band edge
    const int ky = row % N;
    if (kz < band && (ky < band || ky > N - band)) return;
    reinterpret_cast<float4*>(blockIdx.y ? f1 : f0)[i2] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_rcorr(const double* __restrict__ pab, const double* __restrict__ paa,
                        const double* __restrict__ pbb, int nbins, double* __restrict__ r) {
    const int i = threadIdx.x;
    if (i >= nbins) return;
    const double d = paa[i] * pbb[i];
    r[i] = d > 0.0 ? pab[i] / sqrt(d) : 0.0;
}

}  // namespace

cudaError_t launch_sum_orders(const SumOrdersArgs& a, cudaStream_t s) {
    const long long pairs = (long long)a.N * a.N * (a.N / 2) / 2;
    k_sum_orders<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_zero_outside_band(float2* f0, float2* f1, int N, int band, cudaStream_t s) {
    if (band <= 0 || (band & 1) || 2 * band >= N) return cudaErrorInvalidValue;
    const long long pairs = (long long)N * N * (N / 4);
    k_zero_outside_band<<<dim3((unsigned)((pairs + 255) / 256), 2), 256, 0, s>>>(f0, f1, N, band);
    return cudaGetLastError();
}

cudaError_t launch_rcorr(const double* pab, const double* paa, const double* pbb, int nbins, double* r,
                         cudaStream_t s) {
    k_rcorr<<<1, 64, 0, s>>>(pab, paa, pbb, nbins, r);
    return cudaGetLastError();
}

}  // namespace gridspt
