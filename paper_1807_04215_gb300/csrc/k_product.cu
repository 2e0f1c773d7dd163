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
#include "product_core.cuh"

namespace gridspt {

using prod::fma4;

__global__ void __launch_bounds__(256) k_product(ProductArgs a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.cells / 4) return;
    product_cells(a, i, LdgLoad{});
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
