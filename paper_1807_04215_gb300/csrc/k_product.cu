// Real-space source terms and recursion of Eq. recursion_formula (Sec. II.B),
// steps (3)/(6) of the Sec. II.C recipe, for one order n:
//
//   A_n = sum_{m=1}^{n-1} grad delta_m . u_{n-m} + delta_m theta_{n-m}
//   B_n = sum_{m=1}^{n-1} d_j(u_m)_k d_k(u_{n-m})_j + u_m . grad theta_{n-m}
//   (delta_n, theta_n) = 2/((2n+3)(n-1)) [[n + 1/2, 1], [3/2, n]] (A_n, B_n)
//
// The ordered pairs (m, n-m) and (n-m, m) are taken together so that every
// field of every lower order is read from HBM exactly once per order n: the
// fields of the higher order of the pair are held in registers and those of
// the lower order are streamed past them. d_a u_b = d_a d_b nabla^-2 theta is
// symmetric, so 6 components are stored and the off-diagonal products carry
// weight 2 in the contraction.
//
// Field slots of an order (17): delta, theta, grad delta (3), grad theta (3),
// u (3), d_a u_b (xx, yy, zz, xy, xz, yz). Order 1 stores 13 fields (theta_1 =
// delta_1): delta, grad delta (3), u (3), d_a u_b (6).
//
// Four adjacent cells per thread (16-byte loads and stores). The output is
// scaled by N^-3 so that the following forward transform is unnormalised.
// With diag_only = m only the pair (m, m) of order n = 2m is formed (used by the
// accumulate-ahead schedule, where the other pairs are summed in the z pass).
#include "gridspt_internal.h"

namespace gridspt {

namespace {

struct Held {
    float4 v[17];
};

__device__ __forceinline__ void fma4(float4& acc, float4 a, float4 b, float w) {
    acc.x = fmaf(w * a.x, b.x, acc.x);
    acc.y = fmaf(w * a.y, b.y, acc.y);
    acc.z = fmaf(w * a.z, b.z, acc.z);
    acc.w = fmaf(w * a.w, b.w, acc.w);
}

__device__ __forceinline__ void load_order(Held& H, const float4* __restrict__ base, long long fs, int m) {
    if (m == 1) {
        H.v[0] = __ldg(base);
        H.v[1] = H.v[0];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            H.v[2 + a] = __ldg(base + (1 + a) * fs);
            H.v[5 + a] = H.v[2 + a];
            H.v[8 + a] = __ldg(base + (4 + a) * fs);
        }
#pragma unroll
        for (int t = 0; t < 6; ++t) H.v[11 + t] = __ldg(base + (7 + t) * fs);
    } else {
#pragma unroll
        for (int j = 0; j < 17; ++j) H.v[j] = __ldg(base + j * fs);
    }
}

// Contribution of one streamed slot s (value v, lower order) against the held
// higher order H, for both ordered pairs.
__device__ __forceinline__ void stream_slot(int s, float4 v, const Held& H, float4& A, float4& B) {
    if (s == 0) {                      // delta_m theta_{m'}
        fma4(A, v, H.v[1], 1.f);
    } else if (s == 1) {               // delta_{m'} theta_m
        fma4(A, v, H.v[0], 1.f);
    } else if (s <= 4) {               // grad delta_m . u_{m'}
        fma4(A, v, H.v[8 + (s - 2)], 1.f);
    } else if (s <= 7) {               // u_{m'} . grad theta_m
        fma4(B, v, H.v[8 + (s - 5)], 1.f);
    } else if (s <= 10) {              // grad delta_{m'} . u_m  and  u_m . grad theta_{m'}
        fma4(A, v, H.v[2 + (s - 8)], 1.f);
        fma4(B, v, H.v[5 + (s - 8)], 1.f);
    } else if (s <= 13) {              // diagonal tensor terms, both orders
        fma4(B, v, H.v[s], 2.f);
    } else {                           // off-diagonal: symmetric pair x both orders
        fma4(B, v, H.v[s], 4.f);
    }
}

__device__ __forceinline__ void stream_order(const float4* __restrict__ base, long long fs, int m,
                                             const Held& H, float4& A, float4& B) {
    if (m == 1) {
        const float4 d = __ldg(base);
        stream_slot(0, d, H, A, B);
        stream_slot(1, d, H, A, B);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float4 g = __ldg(base + (1 + a) * fs);
            stream_slot(2 + a, g, H, A, B);
            stream_slot(5 + a, g, H, A, B);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) stream_slot(8 + a, __ldg(base + (4 + a) * fs), H, A, B);
#pragma unroll
        for (int t = 0; t < 6; ++t) stream_slot(11 + t, __ldg(base + (7 + t) * fs), H, A, B);
    } else {
#pragma unroll
        for (int j = 0; j < 17; ++j) stream_slot(j, __ldg(base + j * fs), H, A, B);
    }
}

// m = m' (n even): the single ordered pair (n/2, n/2).
__device__ __forceinline__ void diagonal(const Held& H, float4& A, float4& B) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        fma4(A, H.v[2 + a], H.v[8 + a], 1.f);
        fma4(B, H.v[8 + a], H.v[5 + a], 1.f);
    }
    fma4(A, H.v[0], H.v[1], 1.f);
#pragma unroll
    for (int t = 11; t < 14; ++t) fma4(B, H.v[t], H.v[t], 1.f);
#pragma unroll
    for (int t = 14; t < 17; ++t) fma4(B, H.v[t], H.v[t], 2.f);
}

}  // namespace

__global__ void __launch_bounds__(256) k_product(ProductArgs a) {
    const long long n4 = a.cells / 4;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const float4* ws = reinterpret_cast<const float4*>(a.ws);
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
    const int n = a.n;
    for (int m = a.diag_only > 0 ? a.diag_only : 1; 2 * m <= n; ++m) {
        const int mh = n - m;   // held (higher) order
        Held H;
        load_order(H, ws + (long long)a.base[mh] * n4 + i, n4, mh);
        if (mh == m)
            diagonal(H, A, B);
        else
            stream_order(ws + (long long)a.base[m] * n4 + i, n4, m, H, A, B);
        if (a.diag_only > 0) break;
    }
    float4 d, t;
    d.x = fmaf(a.cdA, A.x, a.cdB * B.x);
    d.y = fmaf(a.cdA, A.y, a.cdB * B.y);
    d.z = fmaf(a.cdA, A.z, a.cdB * B.z);
    d.w = fmaf(a.cdA, A.w, a.cdB * B.w);
    t.x = fmaf(a.ctA, A.x, a.ctB * B.x);
    t.y = fmaf(a.ctA, A.y, a.ctB * B.y);
    t.z = fmaf(a.ctA, A.z, a.ctB * B.z);
    t.w = fmaf(a.ctA, A.w, a.ctB * B.w);
    reinterpret_cast<float4*>(a.out_delta)[i] = d;
    reinterpret_cast<float4*>(a.out_theta)[i] = t;
}

// Divergence-form sources (Eq. recursion_formula with grad delta . u + delta
// theta = div(delta u) and the u-tensor terms = (1/2) lap(u . u), u curl free):
// V_n = sum_m delta_m u_{n-m}, S_n = sum_m u_m . u_{n-m}. The ordered pairs (m,
// n-m) and (n-m, m) are taken together (the higher order held in registers,
// the lower streamed), so each stored field is read once; four cells per thread.
__global__ void __launch_bounds__(256) k_product_div(ProductDivArgs a) {
    const long long n4 = a.cells / 4;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const float4* ws = reinterpret_cast<const float4*>(a.ws);
    float4 V[3], S = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 3; ++q) V[q] = S;
    for (int m = 1; 2 * m <= a.n; ++m) {
        const int r = a.n - m;   // held (higher) order
        const float4* hb = ws + 4LL * (r - 1) * n4 + i;
        const float4 dr = __ldg(hb);
        float4 ur[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) ur[q] = __ldg(hb + (1 + q) * n4);
        if (r == m) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                fma4(V[q], dr, ur[q], 1.f);
                fma4(S, ur[q], ur[q], 1.f);
            }
        } else {
            const float4* sb = ws + 4LL * (m - 1) * n4 + i;
            const float4 dm = __ldg(sb);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 um = __ldg(sb + (1 + q) * n4);
                fma4(V[q], dm, ur[q], 1.f);
                fma4(V[q], dr, um, 1.f);
                fma4(S, um, ur[q], 2.f);
            }
        }
    }
    float4* out = reinterpret_cast<float4*>(a.out);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        out[q * n4 + i] = make_float4(a.scale * V[q].x, a.scale * V[q].y, a.scale * V[q].z, a.scale * V[q].w);
    out[3 * n4 + i] = make_float4(a.scale * S.x, a.scale * S.y, a.scale * S.z, a.scale * S.w);
}

cudaError_t launch_product_div(const Geo& g, const ProductDivArgs& a, cudaStream_t s) {
    const long long n4 = a.cells / 4;
    k_product_div<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_product(const Geo& g, const ProductArgs& a, cudaStream_t s) {
    const long long n4 = a.cells / 4;
    k_product<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gridspt
