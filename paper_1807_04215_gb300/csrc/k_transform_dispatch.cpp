// Size and tile-variant dispatch of the transform passes (host code). The
// kernels are instantiated per grid size in k_transform_*.cu.
#include "gridspt_internal.h"

namespace gridspt {

#define GRIDSPT_ALL_N(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) \
    X(512) X(768) X(1024)

#define GRIDSPT_DECLARE(N)                                                                                 \
    cudaError_t transform_colpass_##N(const Geo&, float2*, long long, int, int, int, long long, int, int,  \
                                      cudaStream_t);                                                       \
    cudaError_t transform_zr2c_##N(const Geo&, const float2*, float2*, long long, int, float, int, int,    \
                                   cudaStream_t);                                                          \
    cudaError_t transform_xexp_##N(const Geo&, const XExpArgs&, int, cudaStream_t);                        \
    cudaError_t transform_yexp_##N(const Geo&, const YZExpArgs&, int, cudaStream_t);                       \
    cudaError_t transform_zexp_##N(const Geo&, const YZExpArgs&, int, cudaStream_t);                       \
    int transform_shell_blocks_##N();                                                                      \
    cudaError_t transform_zexp_pairs_##N(const Geo&, const ZPairArgs&, cudaStream_t);                      \
    cudaError_t transform_zshell_##N(const Geo&, const float2*, long long, int, int, int, double*, cudaStream_t);
GRIDSPT_ALL_N(GRIDSPT_DECLARE)
#undef GRIDSPT_DECLARE

bool supported_n(int N) {
    switch (N) {
#define GRIDSPT_CASE(n) case n:
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        return true;
        default: return false;
    }
}

cudaError_t launch_colpass_fwd(const Geo& g, float2* data, long long fstride, int count, int axis,
                               int finalize, long long s2_nl, int band, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n)                                                                                       \
    case n:                                                                                                   \
        return transform_colpass_##n(g, data, fstride, count, axis, finalize, s2_nl, band, g.var[TV_COLPASS], s);
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zr2c(const Geo& g, const float2* in, float2* out, long long fstride, int count, float scale,
                        int band, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) \
    case n: return transform_zr2c_##n(g, in, out, fstride, count, scale, band, g.var[TV_ZR2C], s);
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_xexp(const Geo& g, const XExpArgs& a, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return transform_xexp_##n(g, a, g.var[TV_XEXP], s);
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_yexp(const Geo& g, const YZExpArgs& a, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return transform_yexp_##n(g, a, g.var[TV_YEXP], s);
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zexp(const Geo& g, const YZExpArgs& a, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return transform_zexp_##n(g, a, g.var[TV_ZEXP], s);
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zexp_pairs(const Geo& g, const ZPairArgs& a, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return transform_zexp_pairs_##n(g, a, s);
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

int shell_blocks(const Geo& g) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return transform_shell_blocks_##n();
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return 0;
    }
}

cudaError_t launch_zshell(const Geo& g, const float2* in, long long in_stride, int band, int nfields, int triple,
                          double* partial, cudaStream_t s) {
    switch (g.N) {
#define GRIDSPT_CASE(n) case n: return transform_zshell_##n(g, in, in_stride, band, nfields, triple, partial, s);
        GRIDSPT_ALL_N(GRIDSPT_CASE)
#undef GRIDSPT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gridspt
