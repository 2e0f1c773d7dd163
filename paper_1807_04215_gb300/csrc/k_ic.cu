// Gaussian initial field delta_1(k) (Sec. II.C step (1); Eq. recursion_n=1).
//
// One thread per stored mode of the half spectrum float2[N][N][M]. Only modes
// with 0 < |s|^2 <= s2_cut and no Nyquist component draw random numbers; the
// rest are written as zero. The draw is keyed by the canonical member c of the
// pair {s, -s} (c_z > 0, or c_z = 0 and c_y > 0, or c_z = c_y = 0 and c_x > 0),
// so the two members of a pair on the kz = 0 plane get conjugate values.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), written
// from its published definition: 10 rounds of two 32x32->64-bit multiplies
// with constants 0xD2511F53 and 0xCD9E8D57 and a key bumped by the Weyl
// constants 0x9E3779B9, 0xBB67AE85. Key = seed; counter = (packed c low word,
// packed c high word, 0, 0) with c packed as three 21-bit two's-complement
// fields (x bits 0-20, y 21-41, z 42-62).
//
// Spectrum: P(k) = A k^{n_s} T(k / Gamma)^2 with the BBKS transfer function
// T(q) = ln(1 + 2.34 q)/(2.34 q) [1 + 3.89 q + (16.1 q)^2 + (5.46 q)^3 + (6.71 q)^4]^{-1/4}.
// delta(c) = sqrt(P / L^3) (g1 + i g2) / sqrt(2), g1 + i g2 = sqrt(-2 ln u1) e^{2 pi i u2},
// all in FP64, stored as FP32.
#include <cstdint>

#include "gridspt_internal.h"

namespace gridspt {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double bbks_t(double q) {
    if (q <= 0.0) return 1.0;
    const double a = 16.1 * q, b = 5.46 * q, c = 6.71 * q;
    const double poly = 1.0 + 3.89 * q + a * a + b * b * b + (c * c) * (c * c);
    return log1p(2.34 * q) / (2.34 * q) * pow(poly, -0.25);
}

__global__ void k_ic(IcArgs a, int N, int M, double kF) {
    const long long total = (long long)N * N * M;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const int kz = (int)(idx % M);
        const int ky = (int)((idx / M) % N);
        const int kx = (int)(idx / ((long long)M * N));
        const int sx = kx < N / 2 ? kx : kx - N;
        const int sy = ky < N / 2 ? ky : ky - N;
        const int sz = kz;
        float2 out = make_float2(0.f, 0.f);
        const long long s2 = (long long)sx * sx + (long long)sy * sy + (long long)sz * sz;
        if (sx != -N / 2 && sy != -N / 2 && s2 > 0 && s2 <= a.s2_cut) {
            const bool canon = sz > 0 || (sz == 0 && sy > 0) || (sz == 0 && sy == 0 && sx > 0);
            const long long cx = canon ? sx : -sx, cy = canon ? sy : -sy, cz = canon ? sz : -sz;
            const unsigned long long packed = ((unsigned long long)cx & 0x1FFFFFull) |
                                              (((unsigned long long)cy & 0x1FFFFFull) << 21) |
                                              (((unsigned long long)cz & 0x1FFFFFull) << 42);
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)packed, (uint32_t)(packed >> 32), 0u, 0u),
                make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32)));
            const double u1 = ((double)r.x + 0.5) * 0x1p-32;
            const double u2 = ((double)r.y + 0.5) * 0x1p-32;
            const double rad = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);
            const double sd = a.table[s2];
            const double re = sd * rad * cs;
            const double im = sd * rad * sn;
            out = make_float2((float)re, (float)(canon ? im : -im));
        }
        a.out[idx] = out;
    }
}

// sqrt(P(k) / L^3) / sqrt(2) with P(k) = A k^n_s T_BBKS(k / Gamma)^2 at
// k = k_F sqrt(s2), one thread per integer s2 (FP64).
__global__ void k_ic_table(IcArgs a) {
    const long long s2 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s2 > a.s2_cut) return;
    double sd = 0.0;
    if (s2 > 0) {
        const double k = a.kF * sqrt((double)s2);
        const double t = bbks_t(k / a.gamma);
        const double pk = a.amp * pow(k, a.n_s) * t * t;
        sd = sqrt(pk * a.inv_vol) * 0.70710678118654752440;
    }
    a.table[s2] = sd;
}

cudaError_t launch_ic_table(const IcArgs& a, cudaStream_t s) {
    k_ic_table<<<(unsigned)((a.s2_cut + 1 + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ic(const Geo& g, const IcArgs& a, cudaStream_t s) {
    const long long total = (long long)g.N * g.N * g.M;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_ic<<<(unsigned)blocks, 256, 0, s>>>(a, g.N, g.M, g.kF);
    return cudaGetLastError();
}

}  // namespace gridspt
