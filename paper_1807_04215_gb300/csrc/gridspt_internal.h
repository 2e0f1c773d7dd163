// Internal launcher interface between the host runtime (api.cpp) and the CUDA
// kernels. Host-only C++: no CUDA device code here.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace gridspt {

constexpr int kMaxBins = 64;
constexpr int kMaxOrder = 8;
constexpr int kMaxDeriveOut = 17;

// Grid geometry shared by every launch. Half spectra are float2[N][N][M],
// M = N / 2 (kz = 0..M-1); real fields float[N][N][N]; both 4 N^3 bytes.
struct Geo {
    int N;
    int M;
    double kF;              // 2 pi / L
    const float2* tw;       // device table e^{+2 pi i j / N}, j < N (FP32 from FP64)
};

// Multiplier codes of the fused spectral-derivative pass (Sec. II.C steps (2)
// and (5)): out(k) = mult(k) * src(k), then the inverse transform along x.
enum DeriveKind : int {
    DK_ONE = 0,        // 1
    DK_IK = 1,         // i k_a                  (gradient)
    DK_NEG_IK_K2 = 2,  // -i k_a / k^2           (u = grad nabla^-2 theta)
    DK_KK_K2 = 3,      // k_a k_b / k^2          (d_a u_b)
    DK_SHELL = 4       // 1 inside the shell [s2_lo, s2_hi), else 0
};
// code = kind | a << 4 | b << 6 | src << 8 ; src 0 = first input, 1 = second, 2 = constant 1
constexpr int derive_code(int kind, int a, int b, int src) { return kind | (a << 4) | (b << 6) | (src << 8); }

struct DeriveArgs {
    float2* src0;          // first input spectrum (x-column layout [n][ky][kz])
    float2* src1;          // second input (may equal src0)
    float2* out;           // output field f at out + f * out_stride
    long long out_stride;  // float2 elements between output fields
    int nout;
    int codes[kMaxDeriveOut];
    int fwd_first;         // 1: inputs hold [x][ky][kz] data; transform forward along x,
                           //    finalise (zero Nyquist, optional cut) and store back in place
    long long s2_nl;       // finalise: zero modes with |s|^2 > s2_nl (< 0: no cut)
    long long shell_lo;    // DK_SHELL: lo <= |s|^2 < hi
    long long shell_hi;
};

struct IcArgs {
    float2* out;           // one realisation
    uint64_t seed;
    double amp;            // A of P(k) = A k^ns T^2
    double n_s;
    double gamma;
    double inv_vol;        // 1 / L^3
    long long s2_cut;      // keep 0 < |s|^2 <= s2_cut
};

struct ProductArgs {
    const float* ws;       // derived fields; order m field j at ws + (base[m] + j) * cells
    long long cells;       // N^3
    int base[kMaxOrder + 1];
    int n;                 // order being formed
    float* out_delta;      // real field written (4 N^3 bytes)
    float* out_theta;
    float cdA, cdB, ctA, ctB;  // recursion coefficients times N^-3
};

struct BinSpec {
    int nbins;
    int thr[kMaxBins + 1]; // bin i holds thr[i] <= |s|^2 < thr[i+1]
};

cudaError_t launch_ic(const Geo& g, const IcArgs& a, cudaStream_t s);
cudaError_t launch_derive(const Geo& g, const DeriveArgs& a, cudaStream_t s);
// Column transform along x (axis 0) or y (axis 1) of `count` fields, in place.
// dir = +1 backward, -1 forward. finalize (x axis, forward only): zero Nyquist
// modes and |s|^2 > s2_nl (s2_nl < 0: no cut).
cudaError_t launch_colpass(const Geo& g, float2* data, long long fstride, int count, int axis,
                           int dir, int finalize, long long s2_nl, cudaStream_t s);
// Contiguous-axis complex-to-real (in [x][y][kz] -> out real [x][y][z]).
cudaError_t launch_zc2r(const Geo& g, const float2* in, float2* out, long long fstride, int count,
                        cudaStream_t s);
// Contiguous-axis real-to-complex with output scale.
cudaError_t launch_zr2c(const Geo& g, const float2* in, float2* out, long long fstride, int count,
                        float scale, cudaStream_t s);
cudaError_t launch_product(const Geo& g, const ProductArgs& a, cudaStream_t s);

// Power: per-block partial sums (2 * nbins doubles per block) then a fixed-order
// final reduction. blocks: number of partial-sum blocks (power_blocks()).
int power_blocks(const Geo& g);
cudaError_t launch_power(const Geo& g, const float2* a, const float2* b, const BinSpec& bins,
                         double* partial, double* p_out, int64_t* nk_out, double volume,
                         cudaStream_t s);
// Bispectrum reduction of three real fields (I_a, I_b, J) for one shell.
int bispec_blocks(const Geo& g);
cudaError_t launch_bispec_reduce(const Geo& g, const float* ia, const float* ib, const float* j,
                                 double* partial, double* e_out, double* ntri_out, double vol2,
                                 cudaStream_t s);

bool supported_n(int N);

// Library-owned scratch of the allocation-free power entry point
// (k_power_static.cu): device address of the static array on the current
// device (looked up once per device), its size, and whether a request fits.
cudaError_t power_static_scratch(double** out);
size_t power_static_scratch_bytes();
bool power_static_fits(const Geo& g, int nbins);

}  // namespace gridspt
