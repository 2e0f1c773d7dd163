// Multilayer-perceptron emulator kernels (not part of the GridSPT paper: the
// emulator maps linear-spectrum parameters to binned P-terms).
//
// Network: I -> H -> H -> O, SiLU(z) = z / (1 + e^{-z}) after the two hidden
// layers, linear output. Parameter vector (row-major [in][out] weights):
// W1[I][H], b1[H], W2[H][H], b2[H], W3[H][O], b3[O]. Storage type T of the
// weights and of the saved activations is float or bfloat16; every product is
// accumulated in FP32. Activations saved for the backward pass, per row:
// z1[H], a1[H], z2[H], a2[H] as FP32 (a1, a2 hold T-rounded values).
//
// At these sizes (B <= 4096 rows, 128 hidden units) the network is latency
// bound (about 0.3 GFLOP per forward at B = 4096), so the layers are plain
// shared-memory tiled FP32 FMA loops.
#include <cuda_bf16.h>

#include "gridspt_internal.h"

namespace gridspt {

namespace {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename T> __device__ __forceinline__ float round_t(float v) { return to_f<T>(from_f<T>(v)); }

__device__ __forceinline__ float silu(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.f / (1.f + expf(-z));
    return s * (1.f + z * (1.f - s));
}

constexpr int kFwdRows = 32;
constexpr int kBwdRows = 16;
constexpr int kThreads = 256;

// out[r][c] = sum_k in[r][k] W[k][c] + b[c] for r < R, c < C; in, out in
// shared memory (row pitch K and C); W, b global (T). One thread per (c, row
// group of 16 rows); the W element is loaded once per k and reused 16 times.
template <typename T, int R>
__device__ void dense(const float* __restrict__ in, int K, const T* __restrict__ W, const T* __restrict__ b,
                      int C, float* __restrict__ out) {
    constexpr int RG = R / 16;
    for (int w = threadIdx.x; w < C * RG; w += blockDim.x) {
        const int c = w % C, g = w / C;
        float acc[16];
        const float bc = to_f<T>(b[c]);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = bc;
        for (int k = 0; k < K; ++k) {
            const float wk = to_f<T>(W[(long long)k * C + c]);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = fmaf(in[(g * 16 + j) * K + k], wk, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) out[(g * 16 + j) * C + c] = acc[j];
    }
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mlp_forward(const float* __restrict__ x, int B, int I, int H, int O, const T* __restrict__ theta,
              float* __restrict__ y, float* __restrict__ act) {
    extern __shared__ float sm[];
    float* xs = sm;                      // R x I
    float* h1 = xs + kFwdRows * I;       // R x H
    float* h2 = h1 + kFwdRows * H;       // R x H
    float* ys = h2 + kFwdRows * H;       // R x O
    const T* W1 = theta;
    const T* b1 = W1 + I * H;
    const T* W2 = b1 + H;
    const T* b2 = W2 + H * H;
    const T* W3 = b2 + H;
    const T* b3 = W3 + H * O;
    const int r0 = blockIdx.x * kFwdRows;
    for (int i = threadIdx.x; i < kFwdRows * I; i += blockDim.x) {
        const int r = i / I;
        xs[i] = r0 + r < B ? x[(long long)(r0 + r) * I + (i % I)] : 0.f;
    }
    __syncthreads();
    dense<T, kFwdRows>(xs, I, W1, b1, H, h1);
    __syncthreads();
    for (int i = threadIdx.x; i < kFwdRows * H; i += blockDim.x) {
        const int r = i / H, c = i % H;
        const float z = h1[i];
        const float a = round_t<T>(silu(z));
        if (act && r0 + r < B) {
            act[(long long)(r0 + r) * 4 * H + c] = z;
            act[(long long)(r0 + r) * 4 * H + H + c] = a;
        }
        h1[i] = a;
    }
    __syncthreads();
    dense<T, kFwdRows>(h1, H, W2, b2, H, h2);
    __syncthreads();
    for (int i = threadIdx.x; i < kFwdRows * H; i += blockDim.x) {
        const int r = i / H, c = i % H;
        const float z = h2[i];
        const float a = round_t<T>(silu(z));
        if (act && r0 + r < B) {
            act[(long long)(r0 + r) * 4 * H + 2 * H + c] = z;
            act[(long long)(r0 + r) * 4 * H + 3 * H + c] = a;
        }
        h2[i] = a;
    }
    __syncthreads();
    dense<T, kFwdRows>(h2, H, W3, b3, O, ys);
    __syncthreads();
    for (int i = threadIdx.x; i < kFwdRows * O; i += blockDim.x) {
        const int r = i / O;
        if (r0 + r < B) y[(long long)(r0 + r) * O + (i % O)] = ys[i];
    }
}

// Backward of sum(dy * y) for one tile of kBwdRows rows: writes this block's
// partial gradient (parameter layout) to part + blockIdx.x * n_params.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mlp_backward(const float* __restrict__ x, int B, int I, int H, int O, const T* __restrict__ theta,
               const float* __restrict__ act, const float* __restrict__ dy, float* __restrict__ part) {
    constexpr int R = kBwdRows;
    extern __shared__ float sm[];
    float* xs = sm;              // R x I
    float* z1 = xs + R * I;      // R x H
    float* a1 = z1 + R * H;
    float* z2 = a1 + R * H;
    float* a2 = z2 + R * H;
    float* d3 = a2 + R * H;      // R x O
    float* d2 = d3 + R * O;      // R x H
    float* d1 = d2 + R * H;      // R x H
    const T* W1 = theta;
    const T* b1 = W1 + I * H;
    const T* W2 = b1 + H;
    const T* b2 = W2 + H * H;
    const T* W3 = b2 + H;
    (void)b2;
    const long long np = (long long)I * H + H + (long long)H * H + H + (long long)H * O + O;
    float* g = part + blockIdx.x * np;
    float* gW1 = g;
    float* gb1 = gW1 + I * H;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + H * O;
    const int r0 = blockIdx.x * R;
    for (int i = threadIdx.x; i < R * I; i += blockDim.x) {
        const int r = i / I;
        xs[i] = r0 + r < B ? x[(long long)(r0 + r) * I + (i % I)] : 0.f;
    }
    for (int i = threadIdx.x; i < R * H; i += blockDim.x) {
        const int r = i / H, c = i % H;
        const bool ok = r0 + r < B;
        const float* ar = act + (long long)(r0 + r) * 4 * H;
        z1[i] = ok ? ar[c] : 0.f;
        a1[i] = ok ? ar[H + c] : 0.f;
        z2[i] = ok ? ar[2 * H + c] : 0.f;
        a2[i] = ok ? ar[3 * H + c] : 0.f;
    }
    for (int i = threadIdx.x; i < R * O; i += blockDim.x) {
        const int r = i / O;
        d3[i] = r0 + r < B ? dy[(long long)(r0 + r) * O + (i % O)] : 0.f;
    }
    __syncthreads();
    // output layer
    for (int w = threadIdx.x; w < H * O; w += blockDim.x) {
        const int h = w / O, o = w % O;
        float s = 0.f;
        for (int r = 0; r < R; ++r) s = fmaf(a2[r * H + h], d3[r * O + o], s);
        gW3[w] = s;
    }
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < R; ++r) s += d3[r * O + o];
        gb3[o] = s;
    }
    for (int w = threadIdx.x; w < R * H; w += blockDim.x) {
        const int r = w / H, h = w % H;
        float s = 0.f;
        for (int o = 0; o < O; ++o) s = fmaf(d3[r * O + o], to_f<T>(W3[(long long)h * O + o]), s);
        d2[w] = s * silu_grad(z2[w]);
    }
    __syncthreads();
    // second hidden layer
    for (int w = threadIdx.x; w < H * H; w += blockDim.x) {
        const int k = w / H, h = w % H;
        float s = 0.f;
        for (int r = 0; r < R; ++r) s = fmaf(a1[r * H + k], d2[r * H + h], s);
        gW2[w] = s;
    }
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < R; ++r) s += d2[r * H + h];
        gb2[h] = s;
    }
    for (int w = threadIdx.x; w < R * H; w += blockDim.x) {
        const int r = w / H, k = w % H;
        float s = 0.f;
        for (int h = 0; h < H; ++h) s = fmaf(d2[r * H + h], to_f<T>(W2[(long long)k * H + h]), s);
        d1[w] = s * silu_grad(z1[w]);
    }
    __syncthreads();
    // first layer
    for (int w = threadIdx.x; w < I * H; w += blockDim.x) {
        const int i = w / H, h = w % H;
        float s = 0.f;
        for (int r = 0; r < R; ++r) s = fmaf(xs[r * I + i], d1[r * H + h], s);
        gW1[w] = s;
    }
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < R; ++r) s += d1[r * H + h];
        gb1[h] = s;
    }
    (void)W1;
}

// grad[i] = sum over blocks (in order) of part[b][i]
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblocks, long long np, float* __restrict__ grad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblocks; ++b) s += part[b * np + i];
        grad[i] = s;
    }
}

// Masked mean-squared error: dy = 2 mask (y - t) / sum(mask); loss = sum(mask (y - t)^2) / sum(mask).
// One block, fixed-order reduction.
__global__ void __launch_bounds__(1024)
k_mlp_mse(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ mask, long long n,
          float* __restrict__ dy, float* __restrict__ loss) {
    __shared__ float rs[1024], rc[1024];
    float s = 0.f, c = 0.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = (y[i] - t[i]) * mask[i];
        s = fmaf(d, d, s);
        c += mask[i];
    }
    rs[threadIdx.x] = s;
    rc[threadIdx.x] = c;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            rs[threadIdx.x] += rs[threadIdx.x + h];
            rc[threadIdx.x] += rc[threadIdx.x + h];
        }
        __syncthreads();
    }
    const float cnt = rc[0] > 0.f ? rc[0] : 1.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) dy[i] = 2.f * (y[i] - t[i]) * mask[i] / cnt;
    if (threadIdx.x == 0 && loss) *loss = rs[0] / cnt;
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters; the step count lives
// in device memory (incremented by thread 0 of block 0 after use via a second
// kernel) so that a captured training step can be replayed.
template <typename T>
__global__ void k_mlp_adam(float* __restrict__ master, T* __restrict__ lowp, const float* __restrict__ grad,
                           float* __restrict__ m, float* __restrict__ v, const int* __restrict__ step, long long n,
                           float lr, float b1, float b2, float eps) {
    const int t = *step;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float p = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        master[i] = p;
        if (lowp) lowp[i] = from_f<T>(p);
    }
}

__global__ void k_step_inc(int* step) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

template <typename T>
__global__ void k_convert(const float* __restrict__ src, T* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = from_f<T>(src[i]);
}

// ---------------------------------------------------------------- launchers
long long mlp_params(int I, int H, int O) { return (long long)I * H + H + (long long)H * H + H + (long long)H * O + O; }
int mlp_bwd_blocks(int B) { return (B + kBwdRows - 1) / kBwdRows; }

static size_t fwd_smem(int I, int H, int O) { return sizeof(float) * (size_t)kFwdRows * (I + 2 * H + O); }
static size_t bwd_smem(int I, int H, int O) { return sizeof(float) * (size_t)kBwdRows * (I + 6 * H + O); }

template <typename K>
static cudaError_t smem_attr(K k, size_t bytes) {
    return bytes > 48 * 1024 ? cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
                             : cudaSuccess;
}

cudaError_t launch_mlp_forward(const float* x, int B, int I, int H, int O, const void* theta, int bf16, float* y,
                               float* act, cudaStream_t s) {
    const size_t sm = fwd_smem(I, H, O);
    const unsigned g = (unsigned)((B + kFwdRows - 1) / kFwdRows);
    cudaError_t e;
    if (bf16) {
        if ((e = smem_attr(k_mlp_forward<__nv_bfloat16>, sm)) != cudaSuccess) return e;
        k_mlp_forward<__nv_bfloat16><<<g, kThreads, sm, s>>>(x, B, I, H, O, (const __nv_bfloat16*)theta, y, act);
    } else {
        if ((e = smem_attr(k_mlp_forward<float>, sm)) != cudaSuccess) return e;
        k_mlp_forward<float><<<g, kThreads, sm, s>>>(x, B, I, H, O, (const float*)theta, y, act);
    }
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float* x, int B, int I, int H, int O, const void* theta, int bf16,
                                const float* act, const float* dy, float* part, float* grad, cudaStream_t s) {
    const size_t sm = bwd_smem(I, H, O);
    const int nb = mlp_bwd_blocks(B);
    cudaError_t e;
    if (bf16) {
        if ((e = smem_attr(k_mlp_backward<__nv_bfloat16>, sm)) != cudaSuccess) return e;
        k_mlp_backward<__nv_bfloat16><<<nb, kThreads, sm, s>>>(x, B, I, H, O, (const __nv_bfloat16*)theta, act, dy,
                                                               part);
    } else {
        if ((e = smem_attr(k_mlp_backward<float>, sm)) != cudaSuccess) return e;
        k_mlp_backward<float><<<nb, kThreads, sm, s>>>(x, B, I, H, O, (const float*)theta, act, dy, part);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long np = mlp_params(I, H, O);
    k_mlp_reduce<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(part, nb, np, grad);
    return cudaGetLastError();
}

cudaError_t launch_mlp_mse(const float* y, const float* t, const float* mask, long long n, float* dy, float* loss,
                           cudaStream_t s) {
    k_mlp_mse<<<1, 1024, 0, s>>>(y, t, mask, n, dy, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* master, void* lowp, int bf16, const float* grad, float* m, float* v, int* step,
                            long long n, float lr, float b1, float b2, float eps, cudaStream_t s) {
    k_step_inc<<<1, 32, 0, s>>>(step);
    const unsigned g = (unsigned)((n + 255) / 256);
    if (bf16)
        k_mlp_adam<__nv_bfloat16><<<g, 256, 0, s>>>(master, (__nv_bfloat16*)lowp, grad, m, v, step, n, lr, b1, b2, eps);
    else
        k_mlp_adam<float><<<g, 256, 0, s>>>(master, (float*)lowp, grad, m, v, step, n, lr, b1, b2, eps);
    return cudaGetLastError();
}

cudaError_t launch_mlp_convert(const float* src, void* dst, int bf16, long long n, cudaStream_t s) {
    const unsigned g = (unsigned)((n + 255) / 256);
    if (bf16)
        k_convert<__nv_bfloat16><<<g, 256, 0, s>>>(src, (__nv_bfloat16*)dst, n);
    else
        k_convert<float><<<g, 256, 0, s>>>(src, (float*)dst, n);
    return cudaGetLastError();
}

}  // namespace gridspt
