// Pair products of Eq. recursion_formula, cell by cell (shared by the product
// kernel and the persistent work-queue kernel). The loader LD reads one float4
// of a stored field: __ldg in a kernel that only reads the fields, a plain
// (coherent) load where they were written earlier in the same launch.
#pragma once
#include "gridspt_internal.h"

namespace gridspt {

struct LdgLoad {
    __device__ __forceinline__ float4 operator()(const float4* p) const { return __ldg(p); }
};
struct PlainLoad {
    __device__ __forceinline__ float4 operator()(const float4* p) const { return *p; }
};

namespace prod {

struct Held {
    float4 v[17];
};

__device__ __forceinline__ void fma4(float4& acc, float4 a, float4 b, float w) {
    acc.x = fmaf(w * a.x, b.x, acc.x);
    acc.y = fmaf(w * a.y, b.y, acc.y);
    acc.z = fmaf(w * a.z, b.z, acc.z);
    acc.w = fmaf(w * a.w, b.w, acc.w);
}

template <class LD>
__device__ __forceinline__ void load_order(Held& H, const float4* __restrict__ base, long long fs, int m, LD ld) {
    if (m == 1) {
        H.v[0] = ld(base);
        H.v[1] = H.v[0];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            H.v[2 + a] = ld(base + (1 + a) * fs);
            H.v[5 + a] = H.v[2 + a];
            H.v[8 + a] = ld(base + (4 + a) * fs);
        }
#pragma unroll
        for (int t = 0; t < 6; ++t) H.v[11 + t] = ld(base + (7 + t) * fs);
    } else {
#pragma unroll
        for (int j = 0; j < 17; ++j) H.v[j] = ld(base + j * fs);
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

template <class LD>
__device__ __forceinline__ void stream_order(const float4* __restrict__ base, long long fs, int m,
                                             const Held& H, float4& A, float4& B, LD ld) {
    if (m == 1) {
        const float4 d = ld(base);
        stream_slot(0, d, H, A, B);
        stream_slot(1, d, H, A, B);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float4 g = ld(base + (1 + a) * fs);
            stream_slot(2 + a, g, H, A, B);
            stream_slot(5 + a, g, H, A, B);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) stream_slot(8 + a, ld(base + (4 + a) * fs), H, A, B);
#pragma unroll
        for (int t = 0; t < 6; ++t) stream_slot(11 + t, ld(base + (7 + t) * fs), H, A, B);
    } else {
#pragma unroll
        for (int j = 0; j < 17; ++j) stream_slot(j, ld(base + j * fs), H, A, B);
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

}  // namespace prod

// Four adjacent cells i (float4 index) of order n's sources and outputs.
template <class LD>
__device__ __forceinline__ void product_cells(const ProductArgs& a, long long i, LD ld) {
    using namespace prod;
    const long long n4 = a.cells / 4;
    const float4* ws = reinterpret_cast<const float4*>(a.ws);
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
    const int n = a.n;
    for (int m = a.diag_only > 0 ? a.diag_only : 1; 2 * m <= n; ++m) {
        const int mh = n - m;   // held (higher) order
        Held H;
        load_order(H, ws + (long long)a.base[mh] * n4 + i, n4, mh, ld);
        if (mh == m)
            diagonal(H, A, B);
        else
            stream_order(ws + (long long)a.base[m] * n4 + i, n4, m, H, A, B, ld);
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

}  // namespace gridspt
