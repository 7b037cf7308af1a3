// pt_display.cu -- display resolve: progressive mean -> Khronos PBR Neutral tone map ->
// optional sRGB encoding -> 8-bit RGBA (Sec. 5.1.4).  The paper applies the tone mapper in the
// full-screen pass that draws the path tracer's texture; here it writes a device buffer.
//
// The steps are FP32 operations in a fixed order with explicit rounding intrinsics, so the
// compiler fuses nothing and the floats match a plain FP32 evaluation of the same formula.
#include <cmath>

#include "pt_internal.h"

namespace {

constexpr float F90 = 0.04f;                       // offset scale of the toe
constexpr float K_S = 0.8f - 0.04f;                // start of highlight compression
constexpr float K_D = 0.15f;                       // desaturation strength
constexpr float INV_GAMMA = (float)(1.0 / 2.4);    // sRGB exponent

__device__ __forceinline__ float3 pbr_neutral(float r, float g, float b) {
    const float x = fminf(r, fminf(g, b));
    // toe: x - x^2 / (4 F90) below 2 F90, then the constant F90
    const float f = x < __fmul_rn(2.0f, F90) ? __fsub_rn(x, __fdiv_rn(__fmul_rn(x, x), __fmul_rn(4.0f, F90))) : F90;
    r = __fsub_rn(r, f);
    g = __fsub_rn(g, f);
    b = __fsub_rn(b, f);
    const float p = fmaxf(r, fmaxf(g, b));
    if (p < K_S) return make_float3(r, g, b);
    const float d = __fsub_rn(1.0f, K_S);
    const float pn = __fsub_rn(1.0f, __fdiv_rn(__fmul_rn(d, d), __fsub_rn(__fadd_rn(p, d), K_S)));
    const float s = __fdiv_rn(pn, p);
    r = __fmul_rn(r, s);
    g = __fmul_rn(g, s);
    b = __fmul_rn(b, s);
    const float gm = __fsub_rn(1.0f, __fdiv_rn(1.0f, __fadd_rn(__fmul_rn(K_D, __fsub_rn(p, pn)), 1.0f)));
    const float keep = __fsub_rn(1.0f, gm), add = __fmul_rn(gm, pn);
    return make_float3(__fadd_rn(__fmul_rn(keep, r), add), __fadd_rn(__fmul_rn(keep, g), add),
                       __fadd_rn(__fmul_rn(keep, b), add));
}

__device__ __forceinline__ float srgb_encode(float v) {
    if (v <= 0.0031308f) return __fmul_rn(12.92f, v);
    return __fsub_rn(__fmul_rn(1.055f, powf(v, INV_GAMMA)), 0.055f);
}

__device__ __forceinline__ uint32_t quantise(float v) {
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    return (uint32_t)floorf(__fadd_rn(__fmul_rn(v, 255.0f), 0.5f));
}

__device__ __forceinline__ float clean(float m) {
    return m != m ? 0.0f : fminf(fmaxf(m, 0.0f), 1e30f);
}

// one thread per pixel: 12 bytes in, 4 bytes out
__global__ void k_tonemap(const float* __restrict__ sum, uint32_t npix, float inv_spp, float exposure, uint32_t srgb,
                          uchar4* __restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
        const float r = clean(__fmul_rn(__fmul_rn(sum[3u * i + 0], inv_spp), exposure));
        const float g = clean(__fmul_rn(__fmul_rn(sum[3u * i + 1], inv_spp), exposure));
        const float b = clean(__fmul_rn(__fmul_rn(sum[3u * i + 2], inv_spp), exposure));
        float3 c = pbr_neutral(r, g, b);
        c.x = fminf(fmaxf(c.x, 0.0f), 1.0f);
        c.y = fminf(fmaxf(c.y, 0.0f), 1.0f);
        c.z = fminf(fmaxf(c.z, 0.0f), 1.0f);
        if (srgb) {
            c.x = srgb_encode(c.x);
            c.y = srgb_encode(c.y);
            c.z = srgb_encode(c.z);
        }
        out[i] = make_uchar4((unsigned char)quantise(c.x), (unsigned char)quantise(c.y), (unsigned char)quantise(c.z), 255);
    }
}

}  // namespace

extern "C" pt_status pt_tonemap(const pt_accum* accum, float exposure, uint32_t flags, uint8_t* rgba_out,
                                void* cuda_stream) {
    PT_CHECK_ARG(accum && accum->sum && rgba_out, "NULL argument");
    PT_CHECK_ARG(accum->spp_done > 0, "the accumulator holds no samples (spp_done == 0)");
    PT_CHECK_ARG(std::isfinite(exposure) && exposure >= 0.0f, "exposure must be finite and >= 0");
    PT_CHECK_ARG(((uintptr_t)rgba_out & 3u) == 0, "rgba_out must be 4-byte aligned");
    PT_CHECK_ARG((flags & ~PT_TONEMAP_SRGB) == 0, "unknown flags");
    const uint64_t npix = (uint64_t)accum->width * accum->height;
    if (npix == 0) return PT_OK;
    PT_CHECK_ARG(npix < (1ull << 32), "image too large");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float inv_spp = (float)(1.0 / (double)accum->spp_done);
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((npix + 255) / 256, 16ull * pt_num_sms());
    PT_LAUNCH(k_tonemap, blocks, 256, 0, st, accum->sum, (uint32_t)npix, inv_spp, exposure, flags & PT_TONEMAP_SRGB,
              reinterpret_cast<uchar4*>(rgba_out));
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}
