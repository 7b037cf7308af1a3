// pt_denoise.cu -- regression denoiser: blockwise multi-order feature regression (BMFR,
// Koskela et al. 2019; the paper names denoising as future work, Sec. 6.3).
//
// pt_render_features: per pixel, the mean over the render's samples of the first hit's
// normal (towards the camera), position and albedo, and the fraction of samples that hit a
// scattering surface.  pt_denoise_bmfr: per square block, the least-squares fit of the
// albedo-demodulated colour on the columns 1, n, q, q^2 (q = position scaled to [-1, 1] over
// the block); near-constant features and columns that add no direction are left out.  One CTA
// per block holds the block's columns in shared memory and runs Householder QR in FP32 (the
// remaining norm of a column after the earlier reflections is exactly its part outside the
// span of the kept columns, which the drop rule tests), then back-substitution and the fit.
#include <algorithm>
#include <cmath>

#include "pt_device.cuh"
#include "pt_internal.h"

namespace {

// ------------------------------------------------------------------ primary-hit features
__global__ void k_features(DScene S, DCam cam, uint32_t x0, uint32_t y0, uint32_t cw, uint32_t ch, uint32_t s0,
                           uint32_t spp, uint64_t seed, float4* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cw * ch) return;
    const uint32_t px = x0 + i % cw, py = y0 + i / cw;
    const uint32_t p = py * cam.width + px;
    float3 n_sum = splat3(0.0f), x_sum = splat3(0.0f), a_sum = splat3(0.0f);
    float hits = 0.0f;
    for (uint32_t k = 0; k < spp; ++k) {
        float3 o, d;
        camera_ray_ps(cam, px, py, p, s0 + k, (uint32_t)seed, (uint32_t)(seed >> 32), o, d);
        HitRec h;
        trace_closest(S, o, d, __int_as_float(0x7f800000), h);
        if (h.tri == PT_NO_HIT) continue;
        const float4 ta = __ldg(S.tris + 3u * h.tri), tb = __ldg(S.tris + 3u * h.tri + 1),
                     tc = __ldg(S.tris + 3u * h.tri + 2);
        const uint32_t code = __float_as_uint(tb.w);
        if (code & PT_LIGHT_BIT) continue;
        const DMat& M = S.mats[code];
        const float3 ng = norm3(cross3(xyz(tb) - xyz(ta), xyz(tc) - xyz(ta)));
        n_sum = n_sum + (dot3(-d, ng) > 0.0f ? ng : -ng);
        x_sum = x_sum + (o + d * h.t);
        // reading: albedo = (m + (1-m)(1-t)) bw bc + (1-m) t tc
        a_sum = a_sum + M.base_color * ((M.metalness + (1.0f - M.metalness) * (1.0f - M.trans_weight)) * M.base_weight) +
                M.trans_color * ((1.0f - M.metalness) * M.trans_weight);
        hits += 1.0f;
    }
    const float inv = spp ? 1.0f / (float)spp : 0.0f;
    out[3u * i] = make_float4(n_sum.x * inv, n_sum.y * inv, n_sum.z * inv, hits * inv);
    out[3u * i + 1] = make_float4(x_sum.x * inv, x_sum.y * inv, x_sum.z * inv, 0.0f);
    out[3u * i + 2] = make_float4(a_sum.x * inv, a_sum.y * inv, a_sum.z * inv, 0.0f);
}

// ------------------------------------------------------------------ the regression
constexpr int BM_FEAT = 10;            // 1, n (3), q (3), q^2 (3)
constexpr int BM_COLS = BM_FEAT + 3;   // + the three demodulated colour channels
constexpr int BM_ROWS = 1024;          // pixels of the largest block (32 x 32)
constexpr int BM_THREADS = 256;
constexpr int BM_WARPS = BM_THREADS / 32;
constexpr float BM_ALBEDO_EPS = 1e-2f, BM_RANGE_TOL = 1e-4f, BM_DEP_TOL = 1e-3f;

struct BmfrSmem {
    float M[BM_COLS][BM_ROWS];     // working columns, reduced in place by the reflections
    float part[BM_WARPS][16];      // per-warp partial results of a block reduction
    float bc[16];                  // reduced values, broadcast to the block
    float lo[6], hi[6];            // block ranges of n and p
    float scale[6];                // 2 / (hi - lo), or 0 for a near-constant feature
    float norm0[BM_FEAT];          // norms of the feature columns
    float diag[BM_FEAT];           // R's diagonal, per kept column
    float z[3][BM_FEAT];           // coefficients per channel, per kept column
    int kept[BM_FEAT];
    int nk;
};

// sum over the block of N per-thread values; every thread receives the sums in out[]
template <int N>
__device__ __forceinline__ void block_sum(BmfrSmem& sm, float (&v)[N], float (&out)[N]) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        float x = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sm.part[warp][j] = x;
    }
    __syncthreads();
    if (threadIdx.x < (uint32_t)N) {
        float x = 0.0f;
#pragma unroll
        for (int w = 0; w < BM_WARPS; ++w) x += sm.part[w][threadIdx.x];
        sm.bc[threadIdx.x] = x;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < N; ++j) out[j] = sm.bc[j];
    __syncthreads();
}

// the ten feature columns of one taking-part pixel: 1, n, q, q^2 scaled over the block
__device__ __forceinline__ void bm_columns(const BmfrSmem& sm, float4 f0, float4 f1, float (&col)[BM_FEAT]) {
    const float v[6] = {f0.x, f0.y, f0.z, f1.x, f1.y, f1.z};
    col[0] = 1.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        col[1 + k] = sm.scale[k] != 0.0f ? (v[k] - sm.lo[k]) * sm.scale[k] - 1.0f : 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float qk = sm.scale[3 + k] != 0.0f ? (v[3 + k] - sm.lo[3 + k]) * sm.scale[3 + k] - 1.0f : 0.0f;
        col[4 + k] = qk;
        col[7 + k] = sm.scale[3 + k] != 0.0f ? qk * qk : 0.0f;
    }
}

__global__ void __launch_bounds__(BM_THREADS) k_bmfr(const float* color, const float4* feat, uint32_t W, uint32_t H,
                                                    uint32_t B, uint32_t ox, uint32_t oy, uint32_t nbx, float* out) {
    extern __shared__ __align__(16) unsigned char bm_raw[];
    BmfrSmem& sm = *reinterpret_cast<BmfrSmem*>(bm_raw);
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const int bx0 = (int)((blockIdx.x % nbx) * B) - (int)ox;
    const int by0 = (int)((blockIdx.x / nbx) * B) - (int)oy;
    const uint32_t nrows = B * B;
    auto pixel = [&](uint32_t r, int& x, int& y) {
        x = bx0 + (int)(r % B);
        y = by0 + (int)(r / B);
        return x >= 0 && y >= 0 && x < (int)W && y < (int)H;
    };

    // 1. ranges of n and p over the pixels that take part (all samples hit a scattering surface)
    float lo[6], hi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) { lo[k] = __int_as_float(0x7f800000); hi[k] = -lo[k]; }
    for (uint32_t r = t; r < nrows; r += BM_THREADS) {
        int x, y;
        if (!pixel(r, x, y)) continue;
        const size_t q = (size_t)y * W + (size_t)x;
        const float4 f0 = feat[3 * q], f1 = feat[3 * q + 1];
        if (!(f0.w >= 1.0f)) continue;
        const float v[6] = {f0.x, f0.y, f0.z, f1.x, f1.y, f1.z};
#pragma unroll
        for (int k = 0; k < 6; ++k) { lo[k] = fminf(lo[k], v[k]); hi[k] = fmaxf(hi[k], v[k]); }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float a = lo[k], b = hi[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { sm.part[warp][k] = a; sm.part[warp][6 + k] = b; }
    }
    __syncthreads();
    if (t < 6) {
        float a = sm.part[0][t], b = sm.part[0][6 + t];
        for (int w = 1; w < BM_WARPS; ++w) { a = fminf(a, sm.part[w][t]); b = fmaxf(b, sm.part[w][6 + t]); }
        sm.lo[t] = a;
        sm.hi[t] = b;
    }
    __syncthreads();
    const bool any = sm.lo[0] <= sm.hi[0];   // some pixel takes part
    // per feature: scale 2 / (hi - lo), or 0 if the feature is near-constant over the block
    if (t < 6) {
        const float a = sm.lo[t], b = sm.hi[t];
        const bool keep = any && (b - a) > BM_RANGE_TOL * fmaxf(fmaxf(fabsf(a), fabsf(b)), 1e-2f);
        sm.scale[t] = keep ? 2.0f / (b - a) : 0.0f;
    }
    __syncthreads();

    // 2. columns: 1, n, q, q^2, demodulated colour (rows of pixels that do not take part: 0)
    float nrm[BM_FEAT];
#pragma unroll
    for (int j = 0; j < BM_FEAT; ++j) nrm[j] = 0.0f;
    for (uint32_t r = t; r < nrows; r += BM_THREADS) {
        int x, y;
        float col[BM_COLS];
#pragma unroll
        for (int j = 0; j < BM_COLS; ++j) col[j] = 0.0f;
        if (any && pixel(r, x, y)) {
            const size_t q = (size_t)y * W + (size_t)x;
            const float4 f0 = feat[3 * q], f1 = feat[3 * q + 1], f2 = feat[3 * q + 2];
            if (f0.w >= 1.0f) {
                float fc[BM_FEAT];
                bm_columns(sm, f0, f1, fc);
#pragma unroll
                for (int j = 0; j < BM_FEAT; ++j) col[j] = fc[j];
                col[10] = color[3 * q] / (f2.x + BM_ALBEDO_EPS);
                col[11] = color[3 * q + 1] / (f2.y + BM_ALBEDO_EPS);
                col[12] = color[3 * q + 2] / (f2.z + BM_ALBEDO_EPS);
            }
        }
#pragma unroll
        for (int j = 0; j < BM_COLS; ++j) sm.M[j][r] = col[j];
#pragma unroll
        for (int j = 0; j < BM_FEAT; ++j) nrm[j] += col[j] * col[j];
    }
    float n2[BM_FEAT];
    block_sum<BM_FEAT>(sm, nrm, n2);   // (its barriers also publish the columns)
    if (t < BM_FEAT) sm.norm0[t] = sqrtf(n2[t]);
    if (t == 0) sm.nk = 0;
    __syncthreads();

    // 3. Householder QR over the feature columns in order, reflections applied to all later
    // columns (the colour columns included); a column whose remaining norm is at most
    // BM_DEP_TOL of its own norm adds no direction and is left out
    uint32_t rp = 0;   // pivot row = number of kept columns
    for (int k = 0; k < BM_FEAT && any; ++k) {
        if (!(sm.norm0[k] > 0.0f)) continue;
        float s2p[1] = {0.0f}, s2[1];
        for (uint32_t r = rp + t; r < nrows; r += BM_THREADS) s2p[0] += sm.M[k][r] * sm.M[k][r];
        block_sum<1>(sm, s2p, s2);
        const float sigma = sqrtf(s2[0]);
        if (!(sigma > BM_DEP_TOL * sm.norm0[k])) continue;
        const float x0 = sm.M[k][rp];
        const float alpha = x0 >= 0.0f ? -sigma : sigma;
        const float vnorm2 = s2[0] - x0 * x0 + (x0 - alpha) * (x0 - alpha);
        __syncthreads();
        if (t == 0) sm.M[k][rp] = x0 - alpha;
        __syncthreads();
        // dot products of v with the later columns
        float dp[BM_COLS - 1], dots[BM_COLS - 1];
#pragma unroll
        for (int j = 0; j < BM_COLS - 1; ++j) dp[j] = 0.0f;
        for (uint32_t r = rp + t; r < nrows; r += BM_THREADS) {
            const float v = sm.M[k][r];
#pragma unroll
            for (int j = 0; j < BM_COLS - 1; ++j)
                if (j + 1 > k) dp[j] += v * sm.M[j + 1][r];   // dp[j]: column j + 1
        }
        block_sum<BM_COLS - 1>(sm, dp, dots);
        for (uint32_t r = rp + t; r < nrows; r += BM_THREADS) {
            const float v = sm.M[k][r];
#pragma unroll
            for (int j = 0; j < BM_COLS - 1; ++j)
                if (j + 1 > k) sm.M[j + 1][r] -= (2.0f * dots[j] / vnorm2) * v;
        }
        if (t == 0) {
            sm.kept[sm.nk] = k;
            sm.diag[sm.nk] = alpha;
            sm.nk += 1;
        }
        __syncthreads();
        ++rp;
    }

    // 4. back-substitution R z = Q^T b, one thread per channel: R[a][b] = M[kept[b]][a]
    if (t < 3) {
        const int nk = sm.nk;
        for (int a = nk - 1; a >= 0; --a) {
            float s = sm.M[BM_FEAT + t][a];
            for (int b = a + 1; b < nk; ++b) s -= sm.M[sm.kept[b]][a] * sm.z[t][b];
            sm.z[t][a] = s / sm.diag[a];
        }
    }
    __syncthreads();

    // 5. fitted values, remodulated; pixels that do not take part keep their colour
    const int nk = sm.nk;
    for (uint32_t r = t; r < nrows; r += BM_THREADS) {
        int x, y;
        if (!pixel(r, x, y)) continue;
        const size_t q = (size_t)y * W + (size_t)x;
        const float4 f0 = feat[3 * q];
        float3 c = mk3(color[3 * q], color[3 * q + 1], color[3 * q + 2]);
        if (any && f0.w >= 1.0f) {
            const float4 f1 = feat[3 * q + 1], f2 = feat[3 * q + 2];
            float fc[BM_FEAT];
            bm_columns(sm, f0, f1, fc);
            float y3[3] = {0.0f, 0.0f, 0.0f};
            for (int a = 0; a < nk; ++a) {
                float fa = 0.0f;
#pragma unroll
                for (int j = 0; j < BM_FEAT; ++j)
                    if (j == sm.kept[a]) fa = fc[j];
                y3[0] += sm.z[0][a] * fa;
                y3[1] += sm.z[1][a] * fa;
                y3[2] += sm.z[2][a] * fa;
            }
            c = mk3(y3[0] * (f2.x + BM_ALBEDO_EPS), y3[1] * (f2.y + BM_ALBEDO_EPS), y3[2] * (f2.z + BM_ALBEDO_EPS));
        }
        out[3 * q] = c.x;
        out[3 * q + 1] = c.y;
        out[3 * q + 2] = c.z;
    }
}

}  // namespace

extern "C" pt_status pt_render_features(pt_scene* s, const pt_camera* camera, uint32_t crop_x0, uint32_t crop_y0,
                                        uint32_t width, uint32_t height, uint32_t s0, uint32_t spp, uint64_t seed,
                                        float* out, void* cuda_stream) {
    PT_CHECK_ARG(s && camera && out, "NULL argument");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    PT_CHECK_ARG(camera->width > 0 && camera->height > 0, "empty frame");
    PT_CHECK_ARG(camera->vfov_deg > 0.0f && camera->vfov_deg < 180.0f, "vfov outside (0, 180)");
    PT_CHECK_ARG(lens_ok(*camera), "lens_radius must be finite and >= 0, with focus_distance > 0 when it is > 0");
    PT_CHECK_ARG((uint64_t)crop_x0 + width <= camera->width && (uint64_t)crop_y0 + height <= camera->height,
                 "window outside the frame");
    PT_CHECK_ARG(((uintptr_t)out & 15u) == 0, "out must be 16-byte aligned");
    PT_CHECK_ARG((uint64_t)s0 + spp < (1ull << 32), "sample index overflows 32 bits");
    const uint64_t n = (uint64_t)width * height;
    if (n == 0) return PT_OK;
    PT_CHECK_ARG(n < (1ull << 31), "window too large");
    PT_LAUNCH(k_features, (uint32_t)((n + 127) / 128), 128, 0, (cudaStream_t)cuda_stream, s->view(), to_dcam(*camera),
              crop_x0, crop_y0, width, height, s0, spp, seed, reinterpret_cast<float4*>(out));
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

extern "C" pt_status pt_denoise_bmfr(const float* color, const float* features, uint32_t width, uint32_t height,
                                     uint32_t block, uint32_t offset_x, uint32_t offset_y, float* out,
                                     void* cuda_stream) {
    PT_CHECK_ARG(color && features && out, "NULL argument");
    PT_CHECK_ARG(block >= 4 && block <= 32, "block must be 4..32 pixels");
    PT_CHECK_ARG(offset_x < block && offset_y < block, "offsets must be below the block size");
    PT_CHECK_ARG(((uintptr_t)features & 15u) == 0, "features must be 16-byte aligned");
    const uint64_t n = (uint64_t)width * height;
    if (n == 0) return PT_OK;
    PT_CHECK_ARG(n < (1ull << 31), "image too large");
    const uint32_t nbx = (width + offset_x + block - 1) / block, nby = (height + offset_y + block - 1) / block;
    static bool attr_set = false;
    if (!attr_set) {
        PT_CUDA_TRY(cudaFuncSetAttribute(k_bmfr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BmfrSmem)));
        attr_set = true;
    }
    PT_LAUNCH(k_bmfr, nbx * nby, BM_THREADS, sizeof(BmfrSmem), (cudaStream_t)cuda_stream, color,
              reinterpret_cast<const float4*>(features), width, height, block, offset_x, offset_y, nbx, out);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}
