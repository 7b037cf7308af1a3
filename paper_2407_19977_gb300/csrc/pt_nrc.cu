// pt_nrc.cu -- neural radiance cache: multiresolution hash-grid encoding + 64-wide MLP
// (4 hidden ReLU layers, no biases), trained online with Adam on a relative L2 loss.
// The paper names neural radiance caching as future work to cut the samples per pixel
// (Sec. 6.1); the cache here is the one the path tracer queries at a path's second
// diffuse-ish vertex.
//
// Tensor cores: every layer is a [rows x 64] x [64 x 64] product on mma.sync m16n8k16
// (FP16 operands, FP32 accumulation).  A warp owns 16 rows; the FP32 accumulator fragment
// of one layer is exactly the FP16 A-operand fragment of the next, so activations stay in
// registers across layers (forward) and across the backward chain.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "pt_internal.h"

namespace {

constexpr int W = 64;          // layer width
constexpr int N_HIDDEN = 4;    // hidden layers
constexpr int OUT_PAD = 16;    // output rows padded to one mma n-pair
constexpr int SROW = 72;       // padded shared-memory row (halves): conflict-free B loads
constexpr uint32_t HASH_P1 = 2654435761u, HASH_P2 = 805459861u;
constexpr int QSTRIDE = 16;    // floats per query / sample record
constexpr int N_WEIGHTS = N_HIDDEN * W * W + OUT_PAD * W;

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_hh(__half lo, __half hi) {
    __half2 h = __halves2half2(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_h2(uint32_t v) {
    __half2 h = *reinterpret_cast<const __half2*>(&v);
    return __half22float2(h);
}

// row count of a launch: the host value, or the rows of a device counter past `off`
// (clamped to the capacity n) -- one batch of a list whose length only the device knows
struct RowCount {
    uint32_t n;              // host count, or capacity when `dev` is set
    const uint32_t* dev;     // optional device counter
    uint32_t off;            // first row of this batch in the counted list
    __device__ __forceinline__ uint32_t get() const {
        if (!dev) return n;
        const uint32_t c = *dev;
        return c > off ? min(c - off, n) : 0u;
    }
};

struct GridDesc {
    const __half* table;     // L x T x 2 (FP16 copy used by lookups)
    float* grad;             // L x T x 2 (FP32)
    const uint32_t* res;     // L resolutions
    uint32_t L, T;
    float3 lo, inv_ext;
};

// corner index of level l for integer cell coordinates (dense while (N+1)^3 <= T, else hashed)
__device__ __forceinline__ uint32_t corner_index(uint32_t cx, uint32_t cy, uint32_t cz, uint32_t res, uint32_t T) {
    const uint32_t n1 = res + 1;
    if ((uint64_t)n1 * n1 * n1 <= T) return cx + n1 * (cy + n1 * cz);
    const uint32_t h = cx ^ (cy * HASH_P1) ^ (cz * HASH_P2);
    return h & (T - 1u);
}

__device__ __forceinline__ float3 pos01(const GridDesc& G, const float* q) {
    return mk3(fminf(fmaxf((q[0] - G.lo.x) * G.inv_ext.x, 0.0f), 1.0f),
               fminf(fmaxf((q[1] - G.lo.y) * G.inv_ext.y, 0.0f), 1.0f),
               fminf(fmaxf((q[2] - G.lo.z) * G.inv_ext.z, 0.0f), 1.0f));
}

// cell and in-cell fraction of a coordinate u in [0, 1] on a grid of res cells.  The product
// u * res is carried as the unevaluated sum hi + lo (lo = fma(u, res, -hi) is its exact rounding
// error), so the cell and the fraction are those of the exact product, as FP64 has them,
// rather than off by up to half an FP32 ulp of u * res (3e-5 of a cell at res ~ 1000) -- an
// error that flips the FP16 rounding of fine-level features.
__device__ __forceinline__ void cell_frac(float u, uint32_t res, uint32_t& c, float& f) {
    const float r = (float)res;
    const float hi = u * r;
    const float lo = fmaf(u, r, -hi);
    int ci = (int)floorf(hi);
    float fr = (hi - (float)ci) + lo;        // hi - ci is exact
    if (fr < 0.0f) { ci -= 1; fr += 1.0f; }  // hi an integer and the exact product just below it
    if (ci > (int)res - 1) { ci = (int)res - 1; fr = 1.0f; }   // u = 1: the far face of the last cell
    if (ci < 0) { ci = 0; fr = 0.0f; }
    c = (uint32_t)ci;
    f = fr;
}

__device__ __forceinline__ void grid_cell(float3 p, uint32_t res, uint32_t& cx, uint32_t& cy, uint32_t& cz, float& rx,
                                          float& ry, float& rz) {
    cell_frac(p.x, res, cx, rx);
    cell_frac(p.y, res, cy, ry);
    cell_frac(p.z, res, cz, rz);
}

// one thread per (query, level): interpolated features of that level -> X[q][2l..2l+1];
// the same thread writes columns 32 + 2l, 33 + 2l of the non-grid part
__global__ void k_encode(GridDesc G, const float* __restrict__ queries, RowCount rc, __half* __restrict__ X) {
  const uint32_t n = rc.get();
  for (uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; gid < (uint64_t)n * G.L;
       gid += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q = (uint32_t)(gid / G.L), l = (uint32_t)(gid % G.L);
    const float* rec = queries + (size_t)QSTRIDE * q;
    const float3 p = pos01(G, rec);
    const uint32_t res = G.res[l];
    uint32_t cx, cy, cz;
    float rx, ry, rz;
    grid_cell(p, res, cx, cy, cz, rx, ry, rz);
    const __half2* tab = reinterpret_cast<const __half2*>(G.table) + (size_t)l * G.T;
    float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
        const float w = (ox ? rx : 1.0f - rx) * (oy ? ry : 1.0f - ry) * (oz ? rz : 1.0f - rz);
        const float2 v = __half22float2(tab[corner_index(cx + ox, cy + oy, cz + oz, res, G.T)]);
        f0 += w * v.x;
        f1 += w * v.y;
    }
    __half* row = X + (size_t)W * q;
    row[2 * l] = __float2half_rn(f0);
    row[2 * l + 1] = __float2half_rn(f1);
    // non-grid inputs: direction, normal, roughness, a constant 1, then zeros
    const uint32_t g0 = 2 * G.L;
    for (uint32_t c = g0 + 2 * l; c < g0 + 2 * l + 2 && c < (uint32_t)W; ++c) {
        const uint32_t k = c - g0;
        float v = 0.0f;
        if (k < 3) v = rec[3 + k];
        else if (k < 6) v = rec[6 + (k - 3)];
        else if (k == 6) v = rec[9];
        else if (k == 7) v = 1.0f;
        row[c] = __float2half_rn(v);
    }
    if (l == 0)
        for (uint32_t c = g0 + 2 * G.L; c < (uint32_t)W; ++c) row[c] = __float2half_rn(0.0f);
  }
}

// grid gradient: recompute the corners and scatter dL/dfeature (FP32 atomics, both features
// of an entry in one 8-byte vector atomic)
__global__ void k_grid_backward(GridDesc G, const float* __restrict__ samples, RowCount rc, const float* __restrict__ dX) {
  const uint32_t n = rc.get();
  const float scale = n ? 1.0f / (3.0f * (float)n) : 0.0f;
  for (uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; gid < (uint64_t)n * G.L;
       gid += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q = (uint32_t)(gid / G.L), l = (uint32_t)(gid % G.L);
    const float3 p = pos01(G, samples + (size_t)QSTRIDE * q);
    const uint32_t res = G.res[l];
    uint32_t cx, cy, cz;
    float rx, ry, rz;
    grid_cell(p, res, cx, cy, cz, rx, ry, rz);
    const float g0 = dX[(size_t)2 * G.L * q + 2 * l] * scale, g1 = dX[(size_t)2 * G.L * q + 2 * l + 1] * scale;
    float* gr = G.grad + (size_t)l * G.T * 2;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
        const float w = (ox ? rx : 1.0f - rx) * (oy ? ry : 1.0f - ry) * (oz ? rz : 1.0f - rz);
        const uint32_t idx = corner_index(cx + ox, cy + oy, cz + oz, res, G.T);
        atomicAdd(reinterpret_cast<float2*>(gr + 2 * idx), make_float2(w * g0, w * g1));
    }
  }
}

// ---- fused MLP forward: one warp per 16 rows, weights in padded shared memory ----
__device__ __forceinline__ void load_weights_smem(__half* sw, const __half* __restrict__ Wg) {
    // 16-byte chunks: 8 per 64-wide row
    for (int i = threadIdx.x; i < (N_HIDDEN * W + OUT_PAD) * (W / 8); i += blockDim.x) {
        const int r = i / (W / 8), c = 8 * (i % (W / 8));
        *reinterpret_cast<uint4*>(sw + r * SROW + c) = *reinterpret_cast<const uint4*>(Wg + (size_t)r * W + c);
    }
}

// A fragment of k-tile kt for rows r0+g, r0+g+8 of a row-major [n x 64] FP16 matrix
__device__ __forceinline__ void load_afrag(uint32_t (&a)[4], const __half* M, uint32_t n, uint32_t r0, int kt, int g, int t) {
    const uint32_t ra = r0 + g, rb = r0 + g + 8;
    const int c = 16 * kt + 2 * t;
    a[0] = ra < n ? *reinterpret_cast<const uint32_t*>(M + (size_t)W * ra + c) : 0u;
    a[1] = rb < n ? *reinterpret_cast<const uint32_t*>(M + (size_t)W * rb + c) : 0u;
    a[2] = ra < n ? *reinterpret_cast<const uint32_t*>(M + (size_t)W * ra + c + 8) : 0u;
    a[3] = rb < n ? *reinterpret_cast<const uint32_t*>(M + (size_t)W * rb + c + 8) : 0u;
}

// out[j] (n-tile j) = A (16 x 64) . W_l^T, W_l stored [out][in] (B column-major = W row-major)
template <int NT>
__device__ __forceinline__ void layer_fwd(float (&acc)[NT][4], const uint32_t (&a)[4][4], const __half* sw_l, int g, int t) {
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const __half* wr = sw_l + (8 * j + g) * SROW + 16 * kt + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 8);
            mma16816(acc[j], a[kt], b0, b1);
        }
    }
}

__device__ __forceinline__ void relu_to_a(uint32_t (&a)[4][4], const float (&acc)[8][4]) {
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        a[kt][0] = pack_h2(fmaxf(acc[2 * kt][0], 0.0f), fmaxf(acc[2 * kt][1], 0.0f));
        a[kt][1] = pack_h2(fmaxf(acc[2 * kt][2], 0.0f), fmaxf(acc[2 * kt][3], 0.0f));
        a[kt][2] = pack_h2(fmaxf(acc[2 * kt + 1][0], 0.0f), fmaxf(acc[2 * kt + 1][1], 0.0f));
        a[kt][3] = pack_h2(fmaxf(acc[2 * kt + 1][2], 0.0f), fmaxf(acc[2 * kt + 1][3], 0.0f));
    }
}

__device__ __forceinline__ void store_afrag(__half* M, uint32_t n, uint32_t r0, const uint32_t (&a)[4][4], int g, int t) {
    const uint32_t ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        const int c = 16 * kt + 2 * t;
        if (ra < n) {
            *reinterpret_cast<uint32_t*>(M + (size_t)W * ra + c) = a[kt][0];
            *reinterpret_cast<uint32_t*>(M + (size_t)W * ra + c + 8) = a[kt][2];
        }
        if (rb < n) {
            *reinterpret_cast<uint32_t*>(M + (size_t)W * rb + c) = a[kt][1];
            *reinterpret_cast<uint32_t*>(M + (size_t)W * rb + c + 8) = a[kt][3];
        }
    }
}

// X (n x 64 FP16) -> Y (n x 4 FP32, RGB + unused); acts (optional): A1..A4 (4 x n x 64)
__global__ void __launch_bounds__(128) k_mlp_forward(const __half* __restrict__ X, RowCount rc,
                                                     const __half* __restrict__ Wg, float* __restrict__ Y,
                                                     __half* __restrict__ acts) {
    __shared__ __align__(16) __half sw[(N_HIDDEN * W + OUT_PAD) * SROW];
    load_weights_smem(sw, Wg);
    __syncthreads();
    const uint32_t n = rc.get();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < n; tile += warps) {
        const uint32_t r0 = tile * 16;
        uint32_t a[4][4];
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) load_afrag(a[kt], X, n, r0, kt, g, t);
#pragma unroll
        for (int l = 0; l < N_HIDDEN; ++l) {
            float acc[8][4];
            layer_fwd<8>(acc, a, sw + l * W * SROW, g, t);
            relu_to_a(a, acc);
            if (acts) store_afrag(acts + (size_t)l * rc.n * W, n, r0, a, g, t);
        }
        float out[2][4];
        layer_fwd<2>(out, a, sw + N_HIDDEN * W * SROW, g, t);
        // output columns 0..2 live in n-tile 0: lane t holds columns 2t, 2t+1
        const uint32_t ra = r0 + g, rb = r0 + g + 8;
        if (t < 2) {
            if (ra < n) { Y[4 * ra + 2 * t] = out[0][0]; Y[4 * ra + 2 * t + 1] = out[0][1]; }
            if (rb < n) { Y[4 * rb + 2 * t] = out[0][2]; Y[4 * rb + 2 * t + 1] = out[0][3]; }
        }
    }
}

// ldmatrix without transpose: lane i names row i%8 of tile i/8; each lane receives, per tile,
// two consecutive columns of one row (the mma A-fragment layout)
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const __half* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// Fused cache inference: encoding and MLP of 16 queries per warp, the 64-wide input built in
// a shared-memory tile (never written to HBM).  Lane j encodes level j % 16 of queries
// 2r + j / 16 (r = 0..7): its level's resolution and table stay in registers and it issues
// its 64 corner gathers back to back.  The tile then feeds the same tensor-core layers as
// k_mlp_forward, with the A fragments read by ldmatrix.
// 512 threads share one copy of the weights in shared memory (the copy, not the registers,
// limited 128-thread blocks to 4 per SM); two blocks of sixteen warps fit per SM (64
// registers, no spills)
constexpr int INFER_THREADS = 512;
__global__ void __launch_bounds__(INFER_THREADS, 2) k_nrc_infer(GridDesc G, const float* __restrict__ queries,
                                                                RowCount rc, const __half* __restrict__ Wg,
                                                                float* __restrict__ Y) {
    __shared__ __align__(16) __half sw[(N_HIDDEN * W + OUT_PAD) * SROW];
    __shared__ __align__(16) __half sx[INFER_THREADS / 32][16 * SROW];
    load_weights_smem(sw, Wg);
    __syncthreads();
    const uint32_t n = rc.get();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    __half* X = sx[warp];
    const uint32_t l = lane & 15;
    const bool grid_lane = l < G.L;
    const uint32_t res = grid_lane ? G.res[l] : 1u;
    const __half2* tab = reinterpret_cast<const __half2*>(G.table) + (size_t)l * G.T;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < n; tile += warps) {
        const uint32_t r0 = tile * 16;
        // grid features: columns 2l, 2l + 1 of rows 2r + lane / 16
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint32_t row = 2 * r + (lane >> 4);
            const uint32_t q = r0 + row;
            float f0 = 0.0f, f1 = 0.0f;
            if (grid_lane && q < n) {
                const float3 p = pos01(G, queries + (size_t)QSTRIDE * q);
                uint32_t cx, cy, cz;
                float rx, ry, rz;
                grid_cell(p, res, cx, cy, cz, rx, ry, rz);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint32_t ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
                    const float w = (ox ? rx : 1.0f - rx) * (oy ? ry : 1.0f - ry) * (oz ? rz : 1.0f - rz);
                    const float2 v = __half22float2(tab[corner_index(cx + ox, cy + oy, cz + oz, res, G.T)]);
                    f0 += w * v.x;
                    f1 += w * v.y;
                }
            }
            if (grid_lane) *reinterpret_cast<__half2*>(X + row * SROW + 2 * l) = __floats2half2_rn(f0, f1);
        }
        // the other 64 - 2L columns: direction, normal, roughness, a constant 1, zeros
        for (uint32_t e = lane; e < 16u * (W - 2 * G.L); e += 32) {
            const uint32_t row = e / (W - 2 * G.L), k = e % (W - 2 * G.L);
            const uint32_t q = r0 + row;
            float v = 0.0f;
            if (q < n) {
                const float* rec = queries + (size_t)QSTRIDE * q;
                if (k < 3) v = rec[3 + k];
                else if (k < 6) v = rec[6 + (k - 3)];
                else if (k == 6) v = rec[9];
                else if (k == 7) v = 1.0f;
            }
            X[row * SROW + 2 * G.L + k] = __float2half_rn(v);
        }
        __syncwarp();
        uint32_t a[4][4];
        const int j4 = lane >> 3, r8 = lane & 7;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) ldsm_x4(a[kt], X + (r8 + ((j4 & 1) << 3)) * SROW + 16 * kt + ((j4 >> 1) << 3));
        __syncwarp();
#pragma unroll
        for (int ly = 0; ly < N_HIDDEN; ++ly) {
            float acc[8][4];
            layer_fwd<8>(acc, a, sw + ly * W * SROW, g, t);
            relu_to_a(a, acc);
        }
        float out[2][4];
        layer_fwd<2>(out, a, sw + N_HIDDEN * W * SROW, g, t);
        const uint32_t ra = r0 + g, rb = r0 + g + 8;
        if (t < 2) {
            if (ra < n) { Y[4 * ra + 2 * t] = out[0][0]; Y[4 * ra + 2 * t + 1] = out[0][1]; }
            if (rb < n) { Y[4 * rb + 2 * t] = out[0][2]; Y[4 * rb + 2 * t + 1] = out[0][3]; }
        }
    }
}

// ---- tcgen05 (5th-generation tensor cores, accumulators in tensor memory) ----------------
// Shared-memory operands use the canonical no-swizzle K-major layout: 8 x 8 FP16 core
// matrices of 128 contiguous bytes (8 rows of 16 bytes); core matrix (row group, k group)
// sits at ((row / 8) * 8 + k / 8) * 128 bytes, so the K-adjacent core matrix is 128 bytes
// on (leading byte offset) and the next 8-row group 1024 bytes on (stride byte offset) for
// a 64-wide K.
constexpr uint32_t TC_TILE = 128;          // rows per group tile (the MMA's M)
constexpr uint32_t TC_GROUPS = 1;          // independent groups of 4 warps per CTA (measured:
                                           // 4 CTAs of 1 group beat 2 CTAs of 4 groups)
constexpr uint32_t TC_THREADS = 128 * TC_GROUPS;
constexpr uint32_t TC_LBO = 128, TC_SBO = 1024;
constexpr uint32_t TC_W_HALVES = N_HIDDEN * W * W + OUT_PAD * W;
constexpr uint32_t TC_SMEM = 1024 + TC_W_HALVES * 2 + TC_GROUPS * TC_TILE * W * 2 + 16 * TC_GROUPS + 16;
constexpr uint32_t TC_TMEM_COLS = 64 * TC_GROUPS;
constexpr uint32_t TC_SPIN = 1u << 24;     // bounded mbarrier wait (iterations)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// element (r, k) of a K-major FP16 tile with 64 columns, in halves
__device__ __forceinline__ uint32_t tc_off(uint32_t r, uint32_t k) {
    return (((r >> 3) * 8u + (k >> 3)) << 6) + ((r & 7u) << 3) + (k & 7u);
}

// shared-memory matrix descriptor: start, leading / stride byte offsets (16-byte units),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(const __half* p) {
    uint64_t d = (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t m, uint32_t n) {
    return (1u << 4) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" :: "r"(mbar) : "memory");
}

// bounded wait for the mbarrier phase `parity`; false if it did not complete
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < TC_SPIN; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

#define TC_LD_REGS8(i) "=r"(v[i]), "=r"(v[i + 1]), "=r"(v[i + 2]), "=r"(v[i + 3]), "=r"(v[i + 4]), "=r"(v[i + 5]), "=r"(v[i + 6]), "=r"(v[i + 7])

// 32 lanes x 32 columns of FP32 from tensor memory: this thread's row, 32 columns from taddr
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : TC_LD_REGS8(0), TC_LD_REGS8(8), TC_LD_REGS8(16), TC_LD_REGS8(24)
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tc_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// named barrier of one 4-warp group (ids 1..4; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(uint32_t g) {
    asm volatile("bar.sync %0, 128;\n" :: "r"(1u + g) : "memory");
}
// the same barrier with an AND vote over the group's 128 threads
__device__ __forceinline__ bool group_and(uint32_t g, bool v) {
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %2, 0;\n bar.red.and.pred q, %1, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r) : "r"(1u + g), "r"(v ? 1u : 0u) : "memory");
    return r != 0;
}

// Cache inference on tcgen05.  A CTA holds the weights once and four independent groups of
// four warps; each group owns a 128-query tile at a time: the encoding is written straight
// into the group's K-major A tile in shared memory, then each of the five layers is four
// tcgen05.mma (K = 16 each, M = 128, N = 64 / 16) issued by one thread of the group into the
// group's 128 x 64 FP32 accumulator in tensor memory; the group's warps read their 32 rows
// back with tcgen05.ld, apply ReLU and store FP16 into the A tile for the next layer.  Groups
// synchronise on their own named barriers, so one group's encoding overlaps another's
// layers.  A wait that runs out sets err[0]; the group stops, and the CTA frees its tensor
// memory and returns.
__global__ void __launch_bounds__(TC_THREADS, 2) k_nrc_infer_tc(GridDesc G, const float* __restrict__ queries, RowCount rc,
                                                             const __half* __restrict__ Wg, float* __restrict__ Y,
                                                             uint32_t* __restrict__ err) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __half* sW = reinterpret_cast<__half*>(base);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t g = warp >> 2, wq = warp & 3u;       // group, quarter of the tile's rows
    __half* sA = sW + TC_W_HALVES + g * TC_TILE * W;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sW + TC_W_HALVES + TC_GROUPS * TC_TILE * W) + 2 * g;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(reinterpret_cast<uint64_t*>(sW + TC_W_HALVES + TC_GROUPS * TC_TILE * W) +
                                                  2 * TC_GROUPS);
    // weights: global row-major [out][in] -> K-major core matrices (16-byte chunks)
    for (uint32_t i = tid; i < (N_HIDDEN * W + OUT_PAD) * (W / 8); i += blockDim.x) {
        const uint32_t row = i / (W / 8), c = i % (W / 8);
        const uint32_t layer = min(row / W, (uint32_t)N_HIDDEN), r = row - layer * W;
        *reinterpret_cast<uint4*>(sW + layer * W * W + tc_off(r, 8 * c)) =
            *reinterpret_cast<const uint4*>(Wg + (size_t)row * W + 8 * c);
    }
    if ((tid & 127u) == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(tslot)), "r"(TC_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot + 64u * g;                 // the group's 64 columns
    const uint32_t my_lanes = tmem + ((32u * wq) << 16);     // this warp's 32 lanes
    const uint32_t n = rc.get();
    const uint32_t n_tiles = (n + TC_TILE - 1) / TC_TILE;
    const uint32_t l = lane & 15u;
    const bool grid_lane = l < G.L;
    const uint32_t res = grid_lane ? G.res[l] : 1u;
    const __half2* tab = reinterpret_cast<const __half2*>(G.table) + (size_t)l * G.T;
    const uint32_t ncols = W - 2 * G.L;
    const bool issuer = (tid & 127u) == 0;
    uint32_t phase = 0;
    for (uint32_t tile = blockIdx.x * TC_GROUPS + g; tile < n_tiles; tile += gridDim.x * TC_GROUPS) {
        const uint32_t t0 = tile * TC_TILE;
        // encoding of this warp's 32 rows: grid features of 8 rows at a time are gathered into
        // registers first and stored afterwards, so that their corner loads are all in flight
        // together, then the other columns
#pragma unroll
        for (uint32_t rb = 0; rb < 16; rb += 8) {
            __half2 f[8];
#pragma unroll
            for (uint32_t r = 0; r < 8; ++r) {
                const uint32_t q = t0 + 32u * wq + 2u * (rb + r) + (lane >> 4);
                float f0 = 0.0f, f1 = 0.0f;
                if (grid_lane && q < n) {
                    const float3 p = pos01(G, queries + (size_t)QSTRIDE * q);
                    uint32_t cx, cy, cz;
                    float rx, ry, rz;
                    grid_cell(p, res, cx, cy, cz, rx, ry, rz);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint32_t ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
                        const float w = (ox ? rx : 1.0f - rx) * (oy ? ry : 1.0f - ry) * (oz ? rz : 1.0f - rz);
                        const float2 v = __half22float2(__ldg(tab + corner_index(cx + ox, cy + oy, cz + oz, res, G.T)));
                        f0 += w * v.x;
                        f1 += w * v.y;
                    }
                }
                f[r] = __floats2half2_rn(f0, f1);
            }
            if (grid_lane) {
#pragma unroll
                for (uint32_t r = 0; r < 8; ++r)
                    *reinterpret_cast<__half2*>(sA + tc_off(32u * wq + 2u * (rb + r) + (lane >> 4), 2 * l)) = f[r];
            }
        }
        for (uint32_t e = lane; e < 32u * ncols; e += 32) {
            const uint32_t row = 32u * wq + e / ncols, k = e % ncols;
            const uint32_t q = t0 + row;
            float v = 0.0f;
            if (q < n) {
                const float* rec = queries + (size_t)QSTRIDE * q;
                if (k < 3) v = rec[3 + k];
                else if (k < 6) v = rec[6 + (k - 3)];
                else if (k == 6) v = rec[9];
                else if (k == 7) v = 1.0f;
            }
            sA[tc_off(row, 2 * G.L + k)] = __float2half_rn(v);
        }
        const uint32_t row = 32u * wq + lane;
        bool ok = true;
        for (int layer = 0; layer <= N_HIDDEN; ++layer) {
            // the A tile (written by every thread of the group) must be visible to the tensor core
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            group_sync(g);
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const bool out_layer = layer == N_HIDDEN;
            if (issuer) {
                const __half* wl = sW + layer * W * W;
                const uint32_t idesc = tc_idesc(TC_TILE, out_layer ? OUT_PAD : W);
#pragma unroll
                for (uint32_t kk = 0; kk < 4; ++kk)
                    tc_mma(tmem, tc_desc(sA + kk * 128), tc_desc(wl + kk * 128), idesc, kk > 0 ? 1u : 0u);
                tc_commit(smem_u32(mbar));
            }
            __syncwarp();
            const bool got = mbar_wait(smem_u32(mbar), phase);
            if (!got && lane == 0) atomicOr(err, 1u);
            // one decision for the whole group, so all its threads leave at the same barrier
            if (!group_and(g, got)) {
                ok = false;
                mbar_wait(smem_u32(mbar), phase);   // one more bounded wait for the MMA in flight
                break;
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!out_layer) {
                // two halves of 32 columns keep fewer registers live
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    uint32_t v[32];
                    tc_ld32(my_lanes + 32u * half, v);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint4 pk;
                        uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
                        for (int h = 0; h < 4; ++h)
                            pw[h] = pack_h2(fmaxf(__uint_as_float(v[8 * c + 2 * h]), 0.0f),
                                            fmaxf(__uint_as_float(v[8 * c + 2 * h + 1]), 0.0f));
                        *reinterpret_cast<uint4*>(sA + tc_off(row, 32 * half + 8 * c)) = pk;
                    }
                }
            } else {
                uint32_t v[4];
                tc_ld4(my_lanes, v);
                const uint32_t q = t0 + row;
                if (q < n)
                    *reinterpret_cast<float4*>(Y + 4ull * q) = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]),
                                                                           __uint_as_float(v[2]), __uint_as_float(v[3]));
            }
        }
        // the next tile's encoding overwrites the A tile and the accumulator is reused
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        group_sync(g);
        if (!ok) break;
    }
    // every group is done and each of its MMAs completed (waited for) unless a wait ran out
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(*tslot), "r"(TC_TMEM_COLS) : "memory");
}

// ---- fused training step on tcgen05 -----------------------------------------------------
// One persistent kernel computes a training batch's loss and every gradient: per 128-sample
// tile the hash-grid encoding, the five forward layers, the relative L2 loss, the backward
// chain, the weight gradients and the scatter of the grid gradient, with the activations and
// output gradients kept in shared memory and the accumulators in tensor memory.  Every product
// is a tcgen05.mma with M = 128 and FP16 operands (FP32 accumulation), issued by one thread.
//
// Shared-memory tiles are K-major FP16 (8 x 8 core matrices of 128 bytes) whose rows hold 16
// core matrices along K, so one tile stores two layers side by side: H01 = [h0 | h1], H23 =
// [h2 | h3] (h0 the encoded input, h_l the l-th hidden activation), DZ01 = [dz1 | dz2], DZ23 =
// [dz3 | dz4] (dz_l the gradient of the l-th pre-activation, in units of the loss sum).  A
// layer's product reads its half as a K-major A operand.  The weight gradients of a pair,
// dW_l = dz_(l+1)^T h_l (sum over the tile's rows), come from ONE product that reads the pair
// tiles themselves as MN-major operands: A = [dz_(l+1) | dz_(l+2)]^T (M = 128, K = rows),
// B = [h_l | h_(l+1)]^T (N = 128), whose diagonal 64 x 64 blocks are dW_l and dW_(l+1) (the
// off-diagonal blocks are never read); they accumulate in tensor memory over all the CTA's
// tiles and go out with one atomic add per weight at the end.  The backward products read the
// forward weight tiles as MN-major B operands (N = layer input, K = layer output).  The output
// layer's gradient uses A = DZ01 read from its first 16 columns (dy); its rows 16..127 hold
// stale data and produce accumulator rows that are never read.
//
// MN-major descriptors: SBO = the stride between core matrices along M/N, LBO = along K (the
// reverse of K-major).
//
// The encoding gathers 16 levels x 8 corners of table entries per sample: they are copied
// straight into a shared-memory staging area with cp.async (no registers held while in flight,
// so a tile's gathers are in flight together), 8 levels at a time, then interpolated.
constexpr uint32_t TR_TILE = 128;
constexpr uint32_t TR_W_BYTES = (N_HIDDEN * W * W + OUT_PAD * W) * 2;   // 34,816
constexpr uint32_t TR_PAIR_BYTES = TR_TILE * 2 * W * 2;                   // 32,768: 128 rows x 128 FP16
constexpr uint32_t TR_H4_BYTES = TR_TILE * W * 2;                         // 16,384
constexpr uint32_t TR_STAGE_BYTES = TR_TILE * 8 * 8 * 4;                  // 32,768: 8 levels x 8 corners
constexpr uint32_t TR_SMEM = 1024 + TR_W_BYTES + 4 * TR_PAIR_BYTES + TR_H4_BYTES + TR_STAGE_BYTES + 64;
constexpr uint32_t TR_TMEM_COLS = 512;   // 0..63 layer products, 64..191 dW01, 192..319 dW23, 320..383 dW4

// element (r, k) of a K-major FP16 tile whose rows hold kg core matrices along K, in halves
__device__ __forceinline__ uint32_t kmaj_off(uint32_t r, uint32_t k, uint32_t kg) {
    return (((r >> 3) * kg + (k >> 3)) << 6) + ((r & 7u) << 3) + (k & 7u);
}

// shared-memory matrix descriptor with explicit leading / stride byte offsets, no swizzle
__device__ __forceinline__ uint64_t tc_desc_ls(const void* p, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16 with the major-ness of A and B (1 = MN-major)
__host__ __device__ constexpr uint32_t tc_idesc_t(uint32_t m, uint32_t n, uint32_t a_mn, uint32_t b_mn) {
    return (1u << 4) | (a_mn << 15) | (b_mn << 16) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// every thread waits for the products committed to the barrier; false in every thread if the
// wait ran out (after one more bounded wait for what is in flight)
__device__ __forceinline__ bool tr_wait(uint32_t mbar, uint32_t& phase, uint32_t* err) {
    const bool got = mbar_wait(mbar, phase);
    if (!got && (threadIdx.x & 31u) == 0) atomicOr(err, 1u);
    if (!__syncthreads_and(got)) {
        mbar_wait(mbar, phase);
        return false;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    return true;
}

// the tiles written by every thread are visible to the tensor core, and every thread's
// tensor-memory loads are complete, before thread 0 issues the next products
__device__ __forceinline__ void tr_publish() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// 32 FP32 columns of this thread's row (tensor-memory address taddr): ReLU (recording its mask
// bits) or the recorded mask applied, to FP16 in row r of a K-major tile at column col0
template <bool FWD>
__device__ __forceinline__ void tr_row_out(uint32_t taddr, __half* tile, uint32_t kg, uint32_t r, uint32_t col0,
                                           uint32_t& mask) {
    uint32_t v[32];
    tc_ld32(taddr, v);
    uint32_t bits = FWD ? 0u : mask;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 pk;
        uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = 8 * c + 2 * h;
            float a = __uint_as_float(v[j]), b = __uint_as_float(v[j + 1]);
            if (FWD) {
                bits |= (a > 0.0f ? 1u : 0u) << j;
                bits |= (b > 0.0f ? 1u : 0u) << (j + 1);
                a = fmaxf(a, 0.0f);
                b = fmaxf(b, 0.0f);
            } else {
                a = ((bits >> j) & 1u) ? a : 0.0f;
                b = ((bits >> (j + 1)) & 1u) ? b : 0.0f;
            }
            pw[h] = pack_h2(a, b);
        }
        *reinterpret_cast<uint4*>(tile + kmaj_off(r, col0 + 8u * c, kg)) = pk;
    }
    if (FWD) mask = bits;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : TC_LD_REGS8(0), TC_LD_REGS8(8)
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// The CTA has 8 warps: warp w reaches tensor-memory lanes 32 (w % 4) .. + 31 (one row of the
// tile per thread) and takes the column half w / 4 of each 64-wide layer output, so two warps
// share a row quarter.
constexpr uint32_t TR_THREADS = 256;

__global__ void __launch_bounds__(TR_THREADS, 1) k_nrc_train_tc(GridDesc G, const float* __restrict__ samples, RowCount rc,
                                                             const __half* __restrict__ Wg, float* __restrict__ dW,
                                                             float* __restrict__ loss_sum, uint32_t* __restrict__ err) {
    extern __shared__ unsigned char tr_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)tr_raw + 1023) & ~(uintptr_t)1023);
    __half* sW = reinterpret_cast<__half*>(base);
    __half* H01 = reinterpret_cast<__half*>(base + TR_W_BYTES);
    __half* H23 = reinterpret_cast<__half*>(base + TR_W_BYTES + TR_PAIR_BYTES);
    __half* DZ01 = reinterpret_cast<__half*>(base + TR_W_BYTES + 2 * TR_PAIR_BYTES);
    __half* DZ23 = reinterpret_cast<__half*>(base + TR_W_BYTES + 3 * TR_PAIR_BYTES);
    __half* H4 = reinterpret_cast<__half*>(base + TR_W_BYTES + 4 * TR_PAIR_BYTES);
    __half2* stage = reinterpret_cast<__half2*>(base + TR_W_BYTES + 4 * TR_PAIR_BYTES + TR_H4_BYTES);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(base + TR_W_BYTES + 4 * TR_PAIR_BYTES + TR_H4_BYTES + TR_STAGE_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t quarter = warp & 3u, hf = warp >> 2;
    // weights: global row-major [out][in] -> K-major tiles of 8 core matrices per row, 16-byte
    // asynchronous copies
    for (uint32_t i = tid; i < (N_HIDDEN * W + OUT_PAD) * (W / 8); i += blockDim.x) {
        const uint32_t row = i / (W / 8), c = i % (W / 8);
        const uint32_t layer = min(row / W, (uint32_t)N_HIDDEN), r = row - layer * W;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n"
                     :: "r"(smem_u32(sW + layer * W * W + kmaj_off(r, 8 * c, 8))), "l"(Wg + (size_t)row * W + 8 * c)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(tslot)), "r"(TR_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t lanes = (32u * quarter) << 16;          // this warp's 32 tensor-memory lanes
    const uint32_t c32 = 32u * hf;                           // this warp's 32 columns of a layer output
    const uint32_t t_main = tbase, t_w01 = tbase + 64u, t_w23 = tbase + 192u, t_w4 = tbase + 320u;
    const uint32_t n = rc.get();
    const uint32_t n_tiles = (n + TR_TILE - 1) / TR_TILE;
    const float scale = n ? 1.0f / (3.0f * (float)n) : 0.0f;
    const uint32_t mb = smem_u32(mbar);
    const uint32_t ncols = W - 2 * G.L;
    const uint32_t r = 32u * quarter + lane;                // this thread's row of the tile
    const uint32_t idesc_f64 = tc_idesc_t(TR_TILE, W, 0, 0), idesc_f16 = tc_idesc_t(TR_TILE, OUT_PAD, 0, 0);
    const uint32_t idesc_b = tc_idesc_t(TR_TILE, W, 0, 1);
    const uint32_t idesc_w128 = tc_idesc_t(TR_TILE, 2 * W, 1, 1), idesc_w64 = tc_idesc_t(TR_TILE, W, 1, 1);
    uint32_t phase = 0;
    bool first = true, ok = true;
    float loss_acc = 0.0f;
    for (uint32_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const uint32_t t0 = tile * TR_TILE;
        // ---- encoding into H01 columns 0..63 (h0): thread pair (2 rows' worth of threads per
        // row) row = tid / 2 takes levels 4 sub .. 4 sub + 3 of each 8-level pass (sub = tid % 2);
        // a row past n reads the last row's record and is written as zeros
        {
            const uint32_t row = tid >> 1, sub = tid & 1u;
            const uint32_t q = t0 + row;
            const bool valid = q < n;
            const float* rec = samples + (size_t)QSTRIDE * min(q, n - 1u);
            const float3 p = pos01(G, rec);
            for (uint32_t pass = 0; pass < 2; ++pass) {
                float3 fr[4];
#pragma unroll
                for (uint32_t j = 0; j < 4; ++j) {
                    const uint32_t l = 8u * pass + 4u * sub + j;
                    fr[j] = make_float3(0.0f, 0.0f, 0.0f);
                    if (l < G.L) {
                        const uint32_t res = G.res[l];
                        uint32_t cx, cy, cz;
                        grid_cell(p, res, cx, cy, cz, fr[j].x, fr[j].y, fr[j].z);
                        const __half2* tl = reinterpret_cast<const __half2*>(G.table) + (size_t)l * G.T;
                        __half2* dst = stage + (row * 8u + 4u * sub + j) * 8u;
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const uint32_t ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
                            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n"
                                         :: "r"(smem_u32(dst + c)),
                                            "l"(tl + corner_index(cx + ox, cy + oy, cz + oz, res, G.T))
                                         : "memory");
                        }
                    }
                }
                asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
#pragma unroll
                for (uint32_t j = 0; j < 4; ++j) {
                    const uint32_t l = 8u * pass + 4u * sub + j;
                    if (l >= G.L) continue;
                    const __half2* src = stage + (row * 8u + 4u * sub + j) * 8u;
                    float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint32_t ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
                        const float w = (ox ? fr[j].x : 1.0f - fr[j].x) * (oy ? fr[j].y : 1.0f - fr[j].y) *
                                        (oz ? fr[j].z : 1.0f - fr[j].z);
                        const float2 v = __half22float2(src[c]);
                        f0 += w * v.x;
                        f1 += w * v.y;
                    }
                    *reinterpret_cast<__half2*>(H01 + kmaj_off(row, 2 * l, 16)) =
                        valid ? __floats2half2_rn(f0, f1) : __floats2half2_rn(0.0f, 0.0f);
                }
            }
            // the other columns: direction, normal, roughness, a constant 1, zeros (each
            // thread of the pair half of them)
            for (uint32_t k = sub; k < ncols; k += 2) {
                float v = 0.0f;
                if (valid) {
                    if (k < 3) v = rec[3 + k];
                    else if (k < 6) v = rec[6 + (k - 3)];
                    else if (k == 6) v = rec[9];
                    else if (k == 7) v = 1.0f;
                }
                H01[kmaj_off(row, 2 * G.L + k, 16)] = __float2half_rn(v);
            }
        }
        // ---- forward: four hidden layers, then the output layer
        uint32_t mask[4];
        __half* const in_tile[4] = {H01, H01 + 512, H23, H23 + 512};   // 512 halves = 8 core matrices on
        __half* const out_tile[4] = {H01, H23, H23, H4};
        const uint32_t out_col[4] = {64, 0, 64, 0};
        const uint32_t out_kg[4] = {16, 16, 16, 8};
        for (int l = 0; l < N_HIDDEN && ok; ++l) {
            tr_publish();
            if (tid == 0) {
#pragma unroll
                for (uint32_t kk = 0; kk < 4; ++kk)
                    tc_mma(t_main, tc_desc_ls(in_tile[l] + kk * 128, 128, 2048), tc_desc_ls(sW + l * W * W + kk * 128, 128, 1024),
                           idesc_f64, kk > 0 ? 1u : 0u);
                tc_commit(mb);
            }
            __syncwarp();
            if (!(ok = tr_wait(mb, phase, err))) break;
            tr_row_out<true>(t_main + lanes + c32, out_tile[l], out_kg[l], r, out_col[l] + c32, mask[l]);
        }
        if (!ok) break;
        tr_publish();
        if (tid == 0) {
#pragma unroll
            for (uint32_t kk = 0; kk < 4; ++kk)
                tc_mma(t_main, tc_desc_ls(H4 + kk * 128, 128, 1024), tc_desc_ls(sW + N_HIDDEN * W * W + kk * 128, 128, 1024),
                       idesc_f16, kk > 0 ? 1u : 0u);
            tc_commit(mb);
        }
        __syncwarp();
        if (!(ok = tr_wait(mb, phase, err))) break;
        // ---- relative L2 loss; dy (times 3n) into DZ01 columns 0..15 (warps 0-3)
        if (hf == 0) {
            uint32_t v[4];
            tc_ld4(t_main + lanes, v);
            const uint32_t q = t0 + r;
            float d[3] = {0.0f, 0.0f, 0.0f};
            if (q < n) {
                const float* tg = samples + (size_t)QSTRIDE * q + 10;
                for (int c = 0; c < 3; ++c) {
                    const float y = __uint_as_float(v[c]);
                    const float den = y * y + 0.01f;
                    const float diff = y - tg[c];
                    loss_acc += diff * diff / den;
                    d[c] = 2.0f * diff / den;
                }
            }
            uint4 lo, hi = make_uint4(0u, 0u, 0u, 0u);
            lo.x = pack_h2(d[0], d[1]);
            lo.y = pack_h2(d[2], 0.0f);
            lo.z = 0u;
            lo.w = 0u;
            *reinterpret_cast<uint4*>(DZ01 + kmaj_off(r, 0, 16)) = lo;
            *reinterpret_cast<uint4*>(DZ01 + kmaj_off(r, 8, 16)) = hi;
        }
        // ---- backward: dh4 = dy W4 and the output layer's weight gradient
        tr_publish();
        if (tid == 0) {
            tc_mma(t_main, tc_desc_ls(DZ01, 128, 2048), tc_desc_ls(sW + N_HIDDEN * W * W, 1024, 128), idesc_b, 0u);
#pragma unroll
            for (uint32_t kr = 0; kr < TR_TILE / 16; ++kr)
                tc_mma(t_w4, tc_desc_ls(DZ01 + kr * 2048, 2048, 128), tc_desc_ls(H4 + kr * 1024, 1024, 128), idesc_w64,
                       (first && kr == 0) ? 0u : 1u);
            tc_commit(mb);
        }
        __syncwarp();
        if (!(ok = tr_wait(mb, phase, err))) break;
        tr_row_out<false>(t_main + lanes + c32, DZ23, 16, r, 64 + c32, mask[3]);          // dz4
        // dh3 = dz4 W3
        tr_publish();
        if (tid == 0) {
#pragma unroll
            for (uint32_t kk = 0; kk < 4; ++kk)
                tc_mma(t_main, tc_desc_ls(DZ23 + 512 + kk * 128, 128, 2048), tc_desc_ls(sW + 3 * W * W + kk * 1024, 1024, 128),
                       idesc_b, kk > 0 ? 1u : 0u);
            tc_commit(mb);
        }
        __syncwarp();
        if (!(ok = tr_wait(mb, phase, err))) break;
        tr_row_out<false>(t_main + lanes + c32, DZ23, 16, r, c32, mask[2]);               // dz3
        // dW2, dW3 from [dz3 | dz4]^T [h2 | h3]; dh2 = dz3 W2
        tr_publish();
        if (tid == 0) {
#pragma unroll
            for (uint32_t kr = 0; kr < TR_TILE / 16; ++kr)
                tc_mma(t_w23, tc_desc_ls(DZ23 + kr * 2048, 2048, 128), tc_desc_ls(H23 + kr * 2048, 2048, 128), idesc_w128,
                       (first && kr == 0) ? 0u : 1u);
#pragma unroll
            for (uint32_t kk = 0; kk < 4; ++kk)
                tc_mma(t_main, tc_desc_ls(DZ23 + kk * 128, 128, 2048), tc_desc_ls(sW + 2 * W * W + kk * 1024, 1024, 128),
                       idesc_b, kk > 0 ? 1u : 0u);
            tc_commit(mb);
        }
        __syncwarp();
        if (!(ok = tr_wait(mb, phase, err))) break;
        tr_row_out<false>(t_main + lanes + c32, DZ01, 16, r, 64 + c32, mask[1]);          // dz2
        // dh1 = dz2 W1
        tr_publish();
        if (tid == 0) {
#pragma unroll
            for (uint32_t kk = 0; kk < 4; ++kk)
                tc_mma(t_main, tc_desc_ls(DZ01 + 512 + kk * 128, 128, 2048), tc_desc_ls(sW + 1 * W * W + kk * 1024, 1024, 128),
                       idesc_b, kk > 0 ? 1u : 0u);
            tc_commit(mb);
        }
        __syncwarp();
        if (!(ok = tr_wait(mb, phase, err))) break;
        tr_row_out<false>(t_main + lanes + c32, DZ01, 16, r, c32, mask[0]);               // dz1
        // dW0, dW1 from [dz1 | dz2]^T [h0 | h1]; dx = dz1 W0
        tr_publish();
        if (tid == 0) {
#pragma unroll
            for (uint32_t kr = 0; kr < TR_TILE / 16; ++kr)
                tc_mma(t_w01, tc_desc_ls(DZ01 + kr * 2048, 2048, 128), tc_desc_ls(H01 + kr * 2048, 2048, 128), idesc_w128,
                       (first && kr == 0) ? 0u : 1u);
#pragma unroll
            for (uint32_t kk = 0; kk < 4; ++kk)
                tc_mma(t_main, tc_desc_ls(DZ01 + kk * 128, 128, 2048), tc_desc_ls(sW + kk * 1024, 1024, 128), idesc_b,
                       kk > 0 ? 1u : 0u);
            tc_commit(mb);
        }
        __syncwarp();
        if (!(ok = tr_wait(mb, phase, err))) break;
        first = false;
        // ---- grid gradient: dx of the grid columns (levels 8 hf .. 8 hf + 7 in this warp),
        // scattered onto the corners with FP32 vector atomics
        {
            uint32_t v[16];
            tc_ld16(t_main + lanes + 16u * hf, v);
            const uint32_t q = t0 + r;
            if (q < n) {
                const float3 p = pos01(G, samples + (size_t)QSTRIDE * q);
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) {
                    const uint32_t l = 8u * hf + j;
                    if (l >= G.L) break;
                    const uint32_t res = G.res[l];
                    uint32_t cx, cy, cz;
                    float rx, ry, rz;
                    grid_cell(p, res, cx, cy, cz, rx, ry, rz);
                    const float g0 = __uint_as_float(v[2 * j]) * scale, g1 = __uint_as_float(v[2 * j + 1]) * scale;
                    float* gr = G.grad + (size_t)l * G.T * 2;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint32_t ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
                        const float w = (ox ? rx : 1.0f - rx) * (oy ? ry : 1.0f - ry) * (oz ? rz : 1.0f - rz);
                        const uint32_t idx = corner_index(cx + ox, cy + oy, cz + oz, res, G.T);
                        atomicAdd(reinterpret_cast<float2*>(gr + 2 * idx), make_float2(w * g0, w * g1));
                    }
                }
            }
        }
        // the next tile's encoding and dy rewrite tiles the finished products have read
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
    }
    // loss of the CTA's rows
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
    if (lane == 0 && loss_acc != 0.0f) atomicAdd(loss_sum, loss_acc);
    if (blockIdx.x == 0 && tid == 0 && n) atomicAdd(loss_sum + 1, (float)n);
    // weight gradients: one vector atomic add per 4 weights (the rows of the diagonal blocks),
    // scaled by 1/(3n); this warp takes 32 of the row's 64 columns
    if (ok && !first) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t lo = (r < 64 ? 0u : 64u) + c32;   // this row's layer block, this warp's half
        for (int pr = 0; pr < 2; ++pr) {
            uint32_t v[32];
            tc_ld32((pr == 0 ? t_w01 : t_w23) + lanes + lo, v);
            float* dst = dW + (size_t)(2 * pr + (r < 64 ? 0 : 1)) * W * W + (size_t)(r & 63u) * W + c32;
#pragma unroll
            for (int c = 0; c < 32; c += 4)
                atomicAdd(reinterpret_cast<float4*>(dst + c),
                          make_float4(__uint_as_float(v[c]) * scale, __uint_as_float(v[c + 1]) * scale,
                                      __uint_as_float(v[c + 2]) * scale, __uint_as_float(v[c + 3]) * scale));
        }
        uint32_t v[32];
        tc_ld32(t_w4 + lanes + c32, v);
        if (r < OUT_PAD) {
            float* dst = dW + (size_t)N_HIDDEN * W * W + (size_t)r * W + c32;
#pragma unroll
            for (int c = 0; c < 32; c += 4)
                atomicAdd(reinterpret_cast<float4*>(dst + c),
                          make_float4(__uint_as_float(v[c]) * scale, __uint_as_float(v[c + 1]) * scale,
                                      __uint_as_float(v[c + 2]) * scale, __uint_as_float(v[c + 3]) * scale));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(TR_TMEM_COLS) : "memory");
}

// relative L2 loss: dL/dy * (3n) (the 1/(3n) of the mean is applied to the gradients later
// so that FP16 keeps them in its normal range); adds the loss sum and the row count to
// loss_sum[0..1], which the caller zeroes once per training call (all its batches)
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ samples, RowCount rc, __half* __restrict__ dY,
                       float* __restrict__ loss_sum) {
  const uint32_t n = rc.get();
  if (blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd(loss_sum + 1, (float)n);
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const uint32_t q = base + threadIdx.x;
    float l = 0.0f;
    if (q < n) {
        const float* tg = samples + (size_t)QSTRIDE * q + 10;
        __half* d = dY + (size_t)OUT_PAD * q;
        for (int c = 0; c < 3; ++c) {
            const float y = Y[4 * q + c];
            const float den = y * y + 0.01f;
            const float diff = y - tg[c];
            l += diff * diff / den;
            d[c] = __float2half_rn(2.0f * diff / den);
        }
        for (int c = 3; c < OUT_PAD; ++c) d[c] = __float2half_rn(0.0f);
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, l);
  }
}

// B fragment of W_l read transposed: B[k][n] = W_l[k][n] (k = layer output, n = layer input)
__device__ __forceinline__ void bfrag_t(uint32_t& b0, uint32_t& b1, const __half* sw_l, int kt, int j, int g, int t) {
    const __half* c0 = sw_l + (16 * kt + 2 * t) * SROW + 8 * j + g;
    b0 = pack_hh(c0[0], c0[SROW]);
    b1 = pack_hh(c0[8 * SROW], c0[9 * SROW]);
}

// backward chain per 16-row tile: dZ4 = (dY W4) * [A4 > 0], ..., dZ1 = (dZ2 W1) * [A1 > 0],
// dX = dZ1 W0 (grid columns only).  Stores dZ1..dZ4 (FP16) for the weight gradients.
__global__ void __launch_bounds__(128) k_mlp_backward(const __half* __restrict__ dY, RowCount rc,
                                                      const __half* __restrict__ Wg, const __half* __restrict__ acts,
                                                      __half* __restrict__ dZ, float* __restrict__ dX, uint32_t n_grid_cols) {
    __shared__ __align__(16) __half sw[(N_HIDDEN * W + OUT_PAD) * SROW];
    load_weights_smem(sw, Wg);
    __syncthreads();
    const uint32_t n = rc.get();
    const size_t cap = rc.n;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < n; tile += warps) {
        const uint32_t r0 = tile * 16, ra = r0 + g, rb = r0 + g + 8;
        // dY as a 16 x 16 A fragment (one k-tile)
        uint32_t a1[4];
        a1[0] = ra < n ? *reinterpret_cast<const uint32_t*>(dY + (size_t)OUT_PAD * ra + 2 * t) : 0u;
        a1[1] = rb < n ? *reinterpret_cast<const uint32_t*>(dY + (size_t)OUT_PAD * rb + 2 * t) : 0u;
        a1[2] = ra < n ? *reinterpret_cast<const uint32_t*>(dY + (size_t)OUT_PAD * ra + 2 * t + 8) : 0u;
        a1[3] = rb < n ? *reinterpret_cast<const uint32_t*>(dY + (size_t)OUT_PAD * rb + 2 * t + 8) : 0u;
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
            uint32_t b0, b1;
            bfrag_t(b0, b1, sw + N_HIDDEN * W * SROW, 0, j, g, t);
            mma16816(acc[j], a1, b0, b1);
        }
        uint32_t a[4][4];
        for (int l = N_HIDDEN - 1; l >= 0; --l) {
            // mask with A_{l+1} > 0 (A index l holds the output of hidden layer l)
            const __half* A = acts + (size_t)l * cap * W;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = 8 * j + 2 * t;
                const float2 ma = ra < n ? unpack_h2(*reinterpret_cast<const uint32_t*>(A + (size_t)W * ra + c)) : make_float2(0, 0);
                const float2 mb = rb < n ? unpack_h2(*reinterpret_cast<const uint32_t*>(A + (size_t)W * rb + c)) : make_float2(0, 0);
                acc[j][0] = ma.x > 0.0f ? acc[j][0] : 0.0f;
                acc[j][1] = ma.y > 0.0f ? acc[j][1] : 0.0f;
                acc[j][2] = mb.x > 0.0f ? acc[j][2] : 0.0f;
                acc[j][3] = mb.y > 0.0f ? acc[j][3] : 0.0f;
            }
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                a[kt][0] = pack_h2(acc[2 * kt][0], acc[2 * kt][1]);
                a[kt][1] = pack_h2(acc[2 * kt][2], acc[2 * kt][3]);
                a[kt][2] = pack_h2(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
                a[kt][3] = pack_h2(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
            }
            store_afrag(dZ + (size_t)l * cap * W, n, r0, a, g, t);
            // propagate through W_l: next acc = dZ_l . W_l
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint32_t b0, b1;
                    bfrag_t(b0, b1, sw + l * W * SROW, kt, j, g, t);
                    mma16816(acc[j], a[kt], b0, b1);
                }
            }
        }
        // acc holds dX (16 x 64); keep the grid columns
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t c = 8 * j + 2 * t;
            if (c < n_grid_cols) {
                if (ra < n) { dX[(size_t)n_grid_cols * ra + c] = acc[j][0]; dX[(size_t)n_grid_cols * ra + c + 1] = acc[j][1]; }
                if (rb < n) { dX[(size_t)n_grid_cols * rb + c] = acc[j][2]; dX[(size_t)n_grid_cols * rb + c + 1] = acc[j][3]; }
            }
        }
    }
}

// ldmatrix with transpose: four 8x8 FP16 tiles of shared memory, lane i naming row i%8 of
// tile i/8; each lane receives, per tile, two consecutive rows of one column
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const __half* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// Weight gradients of all layers in one launch: dW_l[o][i] = sum_r G_l[r][o] * A_l[r][i] with
// G_l the layer's output gradient (dZ_l, or dY for the output layer) and A_l its input.
// blockIdx.y = layer, blockIdx.x = a chunk of DW_ROWS rows (split-K; the partial 64 x 64 sums
// go to `part` and k_reduce_grad adds them in a fixed order, so the result is deterministic).
// Row tiles of G and A are staged in shared memory with 16-byte loads; ldmatrix.trans turns
// them into the transposed mma operands (A operand = G^T, B operand = A_l).  Warp w owns
// outputs 16w..16w+15 and all 64 inputs.
constexpr int DW_ROWS = 256;
constexpr int DW_KT = 64;
struct DwArgs {
    const __half* G[N_HIDDEN + 1];
    const __half* A[N_HIDDEN + 1];
    uint32_t g_stride[N_HIDDEN + 1];
    uint32_t n_out[N_HIDDEN + 1];
};

__global__ void __launch_bounds__(128) k_weight_grad(const __grid_constant__ DwArgs D, RowCount rc, float* __restrict__ part) {
    __shared__ __align__(16) __half sG[DW_KT * SROW];
    __shared__ __align__(16) __half sA[DW_KT * SROW];
    const uint32_t n = rc.get();
    const int layer = blockIdx.y;
    const __half* __restrict__ G = D.G[layer];
    const __half* __restrict__ A = D.A[layer];
    const uint32_t gs = D.g_stride[layer], n_out = D.n_out[layer];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int m0 = 16 * warp;
    const bool active = m0 < (int)n_out;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    const uint32_t rbeg = blockIdx.x * DW_ROWS, rend = min(rbeg + DW_ROWS, n);
    for (uint32_t s0 = rbeg; s0 < rend; s0 += DW_KT) {
        for (int c = threadIdx.x; c < DW_KT * 8; c += blockDim.x) {
            const int r = c >> 3, q = c & 7;   // staged row, 16-byte chunk of it
            const uint32_t row = s0 + r;
            uint4 va = make_uint4(0u, 0u, 0u, 0u), vg = make_uint4(0u, 0u, 0u, 0u);
            if (row < rend) {
                va = *reinterpret_cast<const uint4*>(A + (size_t)W * row + 8 * q);
                if (8 * q < (int)n_out) vg = *reinterpret_cast<const uint4*>(G + (size_t)gs * row + 8 * q);
            }
            *reinterpret_cast<uint4*>(sA + r * SROW + 8 * q) = va;
            *reinterpret_cast<uint4*>(sG + r * SROW + 8 * q) = vg;
        }
        __syncthreads();
        if (active) {
            const int j4 = lane >> 3, r8 = lane & 7;
#pragma unroll
            for (int kk = 0; kk < DW_KT; kk += 16) {
                uint32_t a[4];
                // tiles (rows kk, cols m0), (kk, m0+8), (kk+8, m0), (kk+8, m0+8) of G
                ldsm_x4_trans(a, sG + (kk + r8 + ((j4 >> 1) << 3)) * SROW + m0 + ((j4 & 1) << 3));
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    uint32_t b[4];
                    // tiles (kk, 16pp), (kk+8, 16pp), (kk, 16pp+8), (kk+8, 16pp+8) of A_l
                    ldsm_x4_trans(b, sA + (kk + r8 + ((j4 & 1) << 3)) * SROW + 16 * pp + ((j4 >> 1) << 3));
                    mma16816(acc[2 * pp], a, b[0], b[1]);
                    mma16816(acc[2 * pp + 1], a, b[2], b[3]);
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    float* out = part + ((size_t)layer * gridDim.x + blockIdx.x) * W * W;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        *reinterpret_cast<float2*>(out + (m0 + g) * W + c) = make_float2(acc[j][0], acc[j][1]);
        *reinterpret_cast<float2*>(out + (m0 + g + 8) * W + c) = make_float2(acc[j][2], acc[j][3]);
    }
}

// dW = (1 / 3n) * sum over the row chunks, every layer, in chunk order
__global__ void k_reduce_grad(const float* __restrict__ part, uint32_t nparts, float* __restrict__ dw, RowCount rc) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint32_t)N_WEIGHTS) return;
    const uint32_t layer = i / (W * W), e = i % (W * W);
    const uint32_t n = rc.get();
    const float scale = n ? 1.0f / (3.0f * (float)n) : 0.0f;
    const float* src = part + (size_t)layer * nparts * W * W + e;
    float s = 0.0f;
    for (uint32_t p = 0; p < nparts; ++p) s += src[(size_t)p * W * W];
    dw[i] = s * scale;
}

// the step counter of Adam lives on the device: a batch that the device finds empty is no
// step, and a captured graph replays with the current count
__global__ void k_adam_step(uint32_t* step, RowCount rc) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && rc.get() > 0) *step += 1u;
}

// bias corrections 1 - b^t of step t
__device__ __forceinline__ void adam_corrections(const uint32_t* step, float b1, float b2, float& c1, float& c2) {
    const float t = (float)*step;
    c1 = 1.0f - powf(b1, t);
    c2 = 1.0f - powf(b2, t);
}

// Adam (Kingma & Ba): master FP32 parameters, FP16 copy for the kernels, gradient zeroed
__global__ void k_adam(float* __restrict__ p, float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                       __half* __restrict__ copy, uint64_t n, float lr, float b1, float b2, float eps,
                       const uint32_t* __restrict__ step, RowCount rc) {
    if (rc.get() == 0) return;   // an empty batch is no step
    float c1, c2;
    adam_corrections(step, b1, b2, c1, c2);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gr;
        const float vi = b2 * v[i] + (1.0f - b2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        const float np = p[i] - lr * mh / (sqrtf(vh) + eps);
        p[i] = np;
        copy[i] = __float2half_rn(np);
        grad[i] = 0.0f;
    }
}

// lazy Adam for the grid table: an entry whose gradient is exactly zero keeps its value and
// moments.  Four entries per thread: the gradient group is read first, and a group with any
// non-zero entry moves its parameters and moments as float4 (untouched lanes write back what
// they read)
__device__ __forceinline__ float adam_lane(float gr, float& pm, float& mm, float& vm, float lr, float b1, float b2,
                                           float eps, float c1, float c2) {
    if (gr == 0.0f) return pm;
    mm = b1 * mm + (1.0f - b1) * gr;
    vm = b2 * vm + (1.0f - b2) * gr * gr;
    pm = pm - lr * (mm / c1) / (sqrtf(vm / c2) + eps);
    return pm;
}

__global__ void k_adam_lazy(float* __restrict__ p, float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                            __half* __restrict__ copy, uint64_t n4, float lr, float b1, float b2, float eps,
                            const uint32_t* __restrict__ step, RowCount rc) {
    if (rc.get() == 0) return;
    float c1, c2;
    adam_corrections(step, b1, b2, c1, c2);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 g4 = reinterpret_cast<const float4*>(grad)[i];
        if (g4.x == 0.0f && g4.y == 0.0f && g4.z == 0.0f && g4.w == 0.0f) continue;
        float4 p4 = reinterpret_cast<const float4*>(p)[i];
        float4 m4 = reinterpret_cast<const float4*>(m)[i];
        float4 v4 = reinterpret_cast<const float4*>(v)[i];
        adam_lane(g4.x, p4.x, m4.x, v4.x, lr, b1, b2, eps, c1, c2);
        adam_lane(g4.y, p4.y, m4.y, v4.y, lr, b1, b2, eps, c1, c2);
        adam_lane(g4.z, p4.z, m4.z, v4.z, lr, b1, b2, eps, c1, c2);
        adam_lane(g4.w, p4.w, m4.w, v4.w, lr, b1, b2, eps, c1, c2);
        reinterpret_cast<float4*>(p)[i] = p4;
        reinterpret_cast<float4*>(m)[i] = m4;
        reinterpret_cast<float4*>(v)[i] = v4;
        const __half2 h01 = __floats2half2_rn(p4.x, p4.y), h23 = __floats2half2_rn(p4.z, p4.w);
        uint2 hv;
        hv.x = *reinterpret_cast<const uint32_t*>(&h01);
        hv.y = *reinterpret_cast<const uint32_t*>(&h23);
        reinterpret_cast<uint2*>(copy)[i] = hv;
        reinterpret_cast<float4*>(grad)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

__global__ void k_to_half(const float* __restrict__ src, __half* __restrict__ dst, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}

// initial parameters from a counter-based stream: Xavier-uniform weights, small uniform grid
__global__ void k_init(float* w, uint64_t nw, float* grid, uint64_t ng, uint64_t seed) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nw + ng; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x4e5243u, 0u), (uint32_t)seed,
                                      (uint32_t)(seed >> 32));
        const float u = u24(r.x) * 2.0f - 1.0f;
        if (i < nw) {
            const uint64_t layer = i / (W * W);
            const uint64_t row = (i % (W * W)) / W;
            float bound = sqrtf(6.0f / (W + W));
            if (layer >= N_HIDDEN) bound = row < 3 ? sqrtf(6.0f / (W + 3)) : 0.0f;
            w[i] = u * bound;
        } else {
            grid[i - nw] = u * 1e-4f;
        }
    }
}

}  // namespace

struct pt_nrc {
    uint64_t serial = 0;    // pt_next_serial() at creation
    pt_nrc_opts o;
    uint32_t L = 16, T = 1u << 19, grid_cols = 32;
    uint32_t* d_res = nullptr;
    float* d_w = nullptr;  __half* d_wh = nullptr;  float *d_wm = nullptr, *d_wv = nullptr, *d_wg = nullptr;
    float* d_grid = nullptr;  __half* d_gh = nullptr;  float *d_gm = nullptr, *d_gv = nullptr, *d_gg = nullptr;
    uint64_t n_grid = 0;
    uint32_t step = 0;
    // training buffers
    uint32_t cap = 0;
    __half *X = nullptr, *acts = nullptr, *dY = nullptr, *dZ = nullptr;
    float *Y = nullptr, *dX = nullptr, *part = nullptr, *d_loss = nullptr;
    uint32_t* d_step = nullptr;   // Adam's step count (device)
    uint32_t* d_err = nullptr;     // device error word (1: a tensor-core wait ran out)
    // inference buffers
    uint32_t icap = 0;
    __half* iX = nullptr;
    float* iY = nullptr;
    float3 lo, inv_ext;
    uint64_t launches = 0;
};

static GridDesc grid_desc(pt_nrc* N) {
    GridDesc G;
    G.table = N->d_gh;
    G.grad = N->d_gg;
    G.res = N->d_res;
    G.L = N->L;
    G.T = N->T;
    G.lo = N->lo;
    G.inv_ext = N->inv_ext;
    return G;
}

static pt_status ensure_train(pt_nrc* N, uint32_t n) {
    if (N->cap >= n) return PT_OK;
    void* ps[] = {N->X, N->acts, N->dY, N->dZ, N->Y, N->dX, N->part};
    for (void* p : ps)
        if (p) cudaFree(p);
    const size_t c = n;
    PT_CUDA_TRY(cudaMalloc(&N->X, c * W * sizeof(__half)));
    PT_CUDA_TRY(cudaMalloc(&N->acts, c * W * N_HIDDEN * sizeof(__half)));
    PT_CUDA_TRY(cudaMalloc(&N->dY, c * OUT_PAD * sizeof(__half)));
    PT_CUDA_TRY(cudaMalloc(&N->dZ, c * W * N_HIDDEN * sizeof(__half)));
    PT_CUDA_TRY(cudaMalloc(&N->Y, c * 4 * sizeof(float)));
    PT_CUDA_TRY(cudaMalloc(&N->dX, c * N->grid_cols * sizeof(float)));
    PT_CUDA_TRY(cudaMalloc(&N->part, (N_HIDDEN + 1) * ((c + DW_ROWS - 1) / DW_ROWS) * W * W * sizeof(float)));
    N->cap = n;
    return PT_OK;
}

static int g_mlp_blocks = 0;
static uint32_t mlp_grid(uint32_t n) {
    if (g_mlp_blocks == 0) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mlp_forward, 128, 0);
        g_mlp_blocks = std::max(b, 1) * pt_num_sms();
    }
    const uint32_t tiles = (n + 15) / 16;
    return std::max(1u, std::min((uint32_t)g_mlp_blocks, (tiles + 3) / 4));
}

extern "C" pt_status pt_nrc_create(const pt_nrc_opts* opts, void* cuda_stream, pt_nrc** out) {
    PT_CHECK_ARG(opts && out, "NULL argument");
    *out = nullptr;
    pt_nrc_opts o = *opts;
    if (!o.n_levels) o.n_levels = 16;
    if (!o.log2_table) o.log2_table = 19;
    if (!o.base_resolution) o.base_resolution = 16;
    if (!o.n_hidden) o.n_hidden = N_HIDDEN;
    if (o.learning_rate <= 0.0f) o.learning_rate = 1e-2f;
    if (!o.batch) o.batch = 1u << 13;
    if (!o.frame_samples) o.frame_samples = 1u << 15;
    PT_CHECK_ARG(o.frame_samples >= 2 && o.frame_samples <= (1u << 22), "frame_samples must be 2..2^22");
    PT_CHECK_ARG(o.n_hidden == N_HIDDEN, "n_hidden must be 4");
    PT_CHECK_ARG(o.n_levels >= 1 && o.n_levels <= 16, "n_levels must be 1..16 (2 features each fill 32 inputs)");
    PT_CHECK_ARG(o.log2_table >= 8 && o.log2_table <= 24, "log2_table must be 8..24");
    PT_CHECK_ARG(o.base_resolution >= 2, "base_resolution must be >= 2");
    PT_CHECK_ARG(o.train_kernels <= 1, "train_kernels must be 0 (fused) or 1 (separate kernels)");
    for (int a = 0; a < 3; ++a)
        PT_CHECK_ARG(o.scene_max[a] > o.scene_min[a], "empty normalisation box");
    pt_nrc* N = new pt_nrc();
    N->serial = pt_next_serial();
    N->o = o;
    N->L = o.n_levels;
    N->T = 1u << o.log2_table;
    N->grid_cols = 2 * N->L;
    N->lo = make_float3(o.scene_min[0], o.scene_min[1], o.scene_min[2]);
    N->inv_ext = make_float3(1.0f / (o.scene_max[0] - o.scene_min[0]), 1.0f / (o.scene_max[1] - o.scene_min[1]),
                             1.0f / (o.scene_max[2] - o.scene_min[2]));
    // level resolutions: floor(N_min * b^l), b from the per-level scale or a 2048 finest level
    std::vector<uint32_t> res(N->L);
    const double b = o.per_level_scale > 0.0f ? o.per_level_scale
                                              : std::exp((std::log(2048.0) - std::log((double)o.base_resolution)) /
                                                         std::max<int>((int)N->L - 1, 1));
    for (uint32_t l = 0; l < N->L; ++l) res[l] = (uint32_t)std::floor(o.base_resolution * std::pow(b, (double)l));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    N->n_grid = (uint64_t)N->L * N->T * 2;
    auto fail = [&](pt_status s) { pt_nrc_destroy(N); return s; };
#define NTRY(call)                                                                      \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            pt_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));           \
            return fail(e_ == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA);    \
        }                                                                               \
    } while (0)
    NTRY(cudaMalloc(&N->d_res, N->L * sizeof(uint32_t)));
    NTRY(cudaMemcpyAsync(N->d_res, res.data(), N->L * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    float** f32[] = {&N->d_w, &N->d_wm, &N->d_wv, &N->d_wg};
    for (float** p : f32) NTRY(cudaMalloc(p, N_WEIGHTS * sizeof(float)));
    NTRY(cudaMalloc(&N->d_wh, N_WEIGHTS * sizeof(__half)));
    float** g32[] = {&N->d_grid, &N->d_gm, &N->d_gv, &N->d_gg};
    for (float** p : g32) NTRY(cudaMalloc(p, N->n_grid * sizeof(float)));
    NTRY(cudaMalloc(&N->d_gh, N->n_grid * sizeof(__half)));
    NTRY(cudaMalloc(&N->d_loss, 4 * sizeof(float)));
    NTRY(cudaMalloc(&N->d_err, sizeof(uint32_t)));
    NTRY(cudaMemsetAsync(N->d_err, 0, sizeof(uint32_t), st));
    NTRY(cudaMalloc(&N->d_step, sizeof(uint32_t)));
    NTRY(cudaMemsetAsync(N->d_step, 0, sizeof(uint32_t), st));
    for (float* p : {N->d_wm, N->d_wv, N->d_wg}) NTRY(cudaMemsetAsync(p, 0, N_WEIGHTS * sizeof(float), st));
    for (float* p : {N->d_gm, N->d_gv, N->d_gg}) NTRY(cudaMemsetAsync(p, 0, N->n_grid * sizeof(float), st));
    NTRY(cudaMemsetAsync(N->d_loss, 0, 4 * sizeof(float), st));
    PT_LAUNCH(k_init, 4 * pt_num_sms(), 256, 0, st, N->d_w, (uint64_t)N_WEIGHTS, N->d_grid, N->n_grid, o.seed);
    PT_LAUNCH(k_to_half, 4 * pt_num_sms(), 256, 0, st, N->d_w, N->d_wh, (uint64_t)N_WEIGHTS);
    PT_LAUNCH(k_to_half, 4 * pt_num_sms(), 256, 0, st, N->d_grid, N->d_gh, N->n_grid);
    NTRY(cudaGetLastError());
    NTRY(cudaStreamSynchronize(st));
#undef NTRY
    *out = N;
    return PT_OK;
}

extern "C" void pt_nrc_destroy(pt_nrc* N) {
    if (!N) return;
    cudaDeviceSynchronize();
    void* ps[] = {N->d_res, N->d_w, N->d_wh, N->d_wm, N->d_wv, N->d_wg, N->d_grid, N->d_gh, N->d_gm, N->d_gv, N->d_gg,
                  N->X, N->acts, N->dY, N->dZ, N->Y, N->dX, N->part, N->d_loss, N->iX, N->iY, N->d_err,
                  N->d_step};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete N;
}

static uint32_t encode_grid(uint32_t cap, uint32_t L) {
    const uint64_t threads = (uint64_t)cap * L;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((threads + 255) / 256, 32ull * pt_num_sms()));
}

// forward (+ optional activations) of rc rows already resident on the device
static int g_infer_blocks = 0, g_infer_tc_blocks = 0;

static pt_status nrc_forward(pt_nrc* N, const float* q, RowCount rc, __half* X, float* Y, __half* acts, cudaStream_t st) {
    const GridDesc G = grid_desc(N);
    if (!acts && N->o.tcgen05) {
        // inference on the tcgen05 tensor cores (TMEM accumulators), persistent over
        // 128-row tiles
        if (g_infer_tc_blocks == 0) {
            PT_CUDA_TRY(cudaFuncSetAttribute(k_nrc_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
            // the largest shared-memory carveout, so that 4 CTAs (4 x 52 KB) fit on an SM
            PT_CUDA_TRY(cudaFuncSetAttribute(k_nrc_infer_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared));
            // 4 CTAs per SM: 4 x 52 KB of shared memory and 4 x 64 of the 512 tensor-memory
            // columns (the occupancy query does not account for the latter)
            g_infer_tc_blocks = 4 * pt_num_sms();
        }
        const uint32_t tiles = (rc.n + TC_TILE - 1) / TC_TILE;
        const uint32_t blocks = std::max(1u, std::min((uint32_t)g_infer_tc_blocks, (tiles + TC_GROUPS - 1) / TC_GROUPS));
        PT_LAUNCH(k_nrc_infer_tc, blocks, TC_THREADS, TC_SMEM, st, G, q, rc, N->d_wh, Y, N->d_err);
        N->launches += 1;
        PT_CUDA_TRY(cudaGetLastError());
        return PT_OK;
    }
    if (!acts) {
        // inference: encoding and MLP in one kernel on mma.sync, persistent over 16-row tiles
        if (g_infer_blocks == 0) {
            int b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_nrc_infer, INFER_THREADS, 0);
            g_infer_blocks = std::max(b, 1) * pt_num_sms();
        }
        const uint32_t tiles = (rc.n + 15) / 16;
        const uint32_t per_block = INFER_THREADS / 32;
        const uint32_t blocks = std::max(1u, std::min((uint32_t)g_infer_blocks, (tiles + per_block - 1) / per_block));
        PT_LAUNCH(k_nrc_infer, blocks, INFER_THREADS, 0, st, G, q, rc, N->d_wh, Y);
        N->launches += 1;
        PT_CUDA_TRY(cudaGetLastError());
        return PT_OK;
    }
    PT_LAUNCH(k_encode, encode_grid(rc.n, N->L), 256, 0, st, G, q, rc, X);
    PT_LAUNCH(k_mlp_forward, mlp_grid(rc.n), 128, 0, st, X, rc, N->d_wh, Y, acts);
    N->launches += 2;
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

// loss and gradients of one batch into d_wg / d_gg (accumulated; caller zeroes via Adam).
// rc.n is the capacity the buffers are laid out with; rc.dev (optional) the row count.
static int g_train_tc_blocks = 0;

static pt_status nrc_gradients(pt_nrc* N, const float* samples, RowCount rc, cudaStream_t st) {
    if (N->o.train_kernels == 0) {
        // one fused tcgen05 kernel, persistent over the batch's 128-sample tiles (one CTA per SM:
        // its shared memory and all 512 tensor-memory columns)
        if (g_train_tc_blocks == 0) {
            PT_CUDA_TRY(cudaFuncSetAttribute(k_nrc_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM));
            g_train_tc_blocks = pt_num_sms();
        }
        const uint32_t tiles = (rc.n + TR_TILE - 1) / TR_TILE;
        const uint32_t blocks = std::max(1u, std::min((uint32_t)g_train_tc_blocks, tiles));
        PT_LAUNCH(k_nrc_train_tc, blocks, TR_THREADS, TR_SMEM, st, grid_desc(N), samples, rc, N->d_wh, N->d_wg,
                  N->d_loss, N->d_err);
        N->launches += 1;
        PT_CUDA_TRY(cudaGetLastError());
        return PT_OK;
    }
    pt_status r = ensure_train(N, rc.n);
    if (r != PT_OK) return r;
    // every training buffer is addressed with the row stride rc.n (<= the allocation)
    const RowCount rb = rc;
    r = nrc_forward(N, samples, rb, N->X, N->Y, N->acts, st);
    if (r != PT_OK) return r;
    const uint32_t gl = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((rb.n + 255) / 256, 8ull * pt_num_sms()));
    PT_LAUNCH(k_loss, gl, 256, 0, st, N->Y, samples, rb, N->dY, N->d_loss);
    PT_LAUNCH(k_mlp_backward, mlp_grid(rb.n), 128, 0, st, N->dY, rb, N->d_wh, N->acts, N->dZ, N->dX, N->grid_cols);
    const uint32_t nparts = (rb.n + DW_ROWS - 1) / DW_ROWS;
    // layer l's weight gradient pairs dZ_l (its output gradient) with its input
    DwArgs D;
    for (int l = 0; l <= N_HIDDEN; ++l) {
        D.G[l] = l < N_HIDDEN ? N->dZ + (size_t)l * rb.n * W : N->dY;
        D.g_stride[l] = l < N_HIDDEN ? W : OUT_PAD;
        D.n_out[l] = l < N_HIDDEN ? W : OUT_PAD;
        D.A[l] = l == 0 ? N->X : N->acts + (size_t)(l - 1) * rb.n * W;
    }
    PT_LAUNCH(k_weight_grad, dim3(nparts, N_HIDDEN + 1), 128, 0, st, D, rb, N->part);
    PT_LAUNCH(k_reduce_grad, (N_WEIGHTS + 255) / 256, 256, 0, st, N->part, nparts, N->d_wg, rb);
    PT_LAUNCH(k_grid_backward, encode_grid(rb.n, N->L), 256, 0, st, grid_desc(N), samples, rb, N->dX);
    N->launches += 6;
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

static pt_status nrc_adam(pt_nrc* N, RowCount rc, cudaStream_t st) {
    N->step++;
    const float b1 = 0.9f, b2 = 0.99f, eps = 1e-15f;
    const float lr = N->o.learning_rate;
    PT_LAUNCH(k_adam_step, 1, 32, 0, st, N->d_step, rc);
    PT_LAUNCH(k_adam, 2 * pt_num_sms(), 256, 0, st, N->d_w, N->d_wg, N->d_wm, N->d_wv, N->d_wh, (uint64_t)N_WEIGHTS, lr,
              b1, b2, eps, N->d_step, rc);
    // one thread per float4 group: every group's loads are in flight at once
    const uint64_t groups = N->n_grid / 4;
    const uint32_t ablocks = (uint32_t)std::min<uint64_t>((groups + 255) / 256, 1u << 20);
    PT_LAUNCH(k_adam_lazy, ablocks, 256, 0, st, N->d_grid, N->d_gg, N->d_gm, N->d_gv, N->d_gh, groups,
              lr, b1, b2, eps, N->d_step, rc);
    N->launches += 3;
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

extern "C" pt_status pt_nrc_train(pt_nrc* N, const float* samples, uint32_t n, void* cuda_stream) {
    PT_CHECK_ARG(N && samples, "NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    PT_CUDA_TRY(cudaMemsetAsync(N->d_loss, 0, 2 * sizeof(float), st));
    for (uint32_t b = 0; b < n; b += N->o.batch) {
        const uint32_t m = std::min(N->o.batch, n - b);
        pt_status r = nrc_gradients(N, samples + (size_t)QSTRIDE * b, RowCount{m, nullptr, 0}, st);
        if (r != PT_OK) return r;
        r = nrc_adam(N, RowCount{m, nullptr, 0}, st);
        if (r != PT_OK) return r;
    }
    return PT_OK;
}

extern "C" pt_status pt_nrc_gradients(pt_nrc* N, const float* samples, uint32_t n, float* dw_out, float* dgrid_out,
                                      void* cuda_stream) {
    PT_CHECK_ARG(N && samples, "NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    PT_CUDA_TRY(cudaMemsetAsync(N->d_loss, 0, 2 * sizeof(float), st));
    PT_CUDA_TRY(cudaMemsetAsync(N->d_wg, 0, N_WEIGHTS * sizeof(float), st));
    PT_CUDA_TRY(cudaMemsetAsync(N->d_gg, 0, N->n_grid * sizeof(float), st));
    pt_status r = nrc_gradients(N, samples, RowCount{n, nullptr, 0}, st);
    if (r != PT_OK) return r;
    if (dw_out) PT_CUDA_TRY(cudaMemcpyAsync(dw_out, N->d_wg, N_WEIGHTS * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (dgrid_out) PT_CUDA_TRY(cudaMemcpyAsync(dgrid_out, N->d_gg, N->n_grid * sizeof(float), cudaMemcpyDeviceToDevice, st));
    PT_CUDA_TRY(cudaMemsetAsync(N->d_wg, 0, N_WEIGHTS * sizeof(float), st));
    PT_CUDA_TRY(cudaMemsetAsync(N->d_gg, 0, N->n_grid * sizeof(float), st));
    return PT_OK;
}

extern "C" pt_status pt_nrc_infer(pt_nrc* N, const float* queries, uint32_t n, float* out_rgb, void* cuda_stream) {
    PT_CHECK_ARG(N && queries && out_rgb, "NULL argument");
    if (n == 0) return PT_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (N->icap < n) {
        if (N->iX) cudaFree(N->iX);
        N->iX = nullptr;
        PT_CUDA_TRY(cudaMalloc(&N->iX, (size_t)n * W * sizeof(__half)));
        N->icap = n;
    }
    // the MLP writes 4 floats per row; out_rgb is the caller's n x 4 buffer
    return nrc_forward(N, queries, RowCount{n, nullptr, 0}, N->iX, out_rgb, nullptr, st);
}

extern "C" pt_status pt_nrc_params(pt_nrc* N, int which, float** ptr, uint64_t* count) {
    PT_CHECK_ARG(N && ptr && count, "NULL argument");
    PT_CHECK_ARG(which == 0 || which == 1, "which must be 0 (MLP) or 1 (grid)");
    *ptr = which == 0 ? N->d_w : N->d_grid;
    *count = which == 0 ? (uint64_t)N_WEIGHTS : N->n_grid;
    return PT_OK;
}

extern "C" pt_status pt_nrc_commit(pt_nrc* N, void* cuda_stream) {
    PT_CHECK_ARG(N != nullptr, "NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    PT_LAUNCH(k_to_half, 4 * pt_num_sms(), 256, 0, st, N->d_w, N->d_wh, (uint64_t)N_WEIGHTS);
    PT_LAUNCH(k_to_half, 8 * pt_num_sms(), 256, 0, st, N->d_grid, N->d_gh, N->n_grid);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

extern "C" pt_status pt_nrc_last_loss(pt_nrc* N, float* loss) {
    PT_CHECK_ARG(N && loss, "NULL argument");
    PT_CUDA_TRY(cudaDeviceSynchronize());
    float s[2] = {0.0f, 0.0f};
    PT_CUDA_TRY(cudaMemcpy(s, N->d_loss, 2 * sizeof(float), cudaMemcpyDeviceToHost));
    uint32_t e = 0;
    PT_CUDA_TRY(cudaMemcpy(&e, N->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (e) {
        pt_set_error("a tensor-core completion wait of the cache ran out of its spin budget");
        return PT_ERR_TIMEOUT;
    }
    *loss = s[1] > 0.0f ? s[0] / (3.0f * s[1]) : 0.0f;
    return PT_OK;
}

// ---- hooks used by the renderer: the row counts stay on the device (no host round trip) ----
static pt_status ensure_infer(pt_nrc* N, uint32_t cap) {
    if (N->icap >= cap) return PT_OK;
    if (N->iX) cudaFree(N->iX);
    N->iX = nullptr;
    PT_CUDA_TRY(cudaMalloc(&N->iX, (size_t)cap * W * sizeof(__half)));
    N->icap = cap;
    return PT_OK;
}

// scratch for a renderer's calls, allocated before a graph capture (none happens inside one)
pt_status pt_nrc_render_prepare(pt_nrc* N, uint32_t infer_cap, uint32_t train_cap) {
    pt_status r = ensure_infer(N, infer_cap);
    if (r != PT_OK) return r;
    if (N->o.train_kernels == 0) return PT_OK;   // the fused training kernel needs no scratch
    return ensure_train(N, std::min(N->o.batch, std::max(train_cap, 1u)));
}

pt_status pt_nrc_render_infer_dev(pt_nrc* N, const float* queries, const uint32_t* n_dev, uint32_t cap, float* out4,
                                  cudaStream_t st) {
    pt_status r = ensure_infer(N, cap);
    if (r != PT_OK) return r;
    return nrc_forward(N, queries, RowCount{cap, n_dev, 0}, N->iX, out4, nullptr, st);
}

uint32_t pt_nrc_frame_samples(const pt_nrc* N) { return N->o.frame_samples; }

// one Adam step per `batch` samples of the frame's training list (its length is on the device;
// a batch past the end of the list is no step)
pt_status pt_nrc_render_train_dev(pt_nrc* N, const float* samples, const uint32_t* n_dev, uint32_t cap, cudaStream_t st) {
    const uint32_t batch = std::min(N->o.batch, cap);
    pt_status r = N->o.train_kernels == 0 ? PT_OK : ensure_train(N, batch);
    if (r != PT_OK) return r;
    PT_CUDA_TRY(cudaMemsetAsync(N->d_loss, 0, 2 * sizeof(float), st));
    for (uint32_t b0 = 0; b0 < cap; b0 += batch) {
        const RowCount rc{std::min(batch, cap - b0), n_dev, b0};
        r = nrc_gradients(N, samples + (size_t)QSTRIDE * b0, rc, st);
        if (r != PT_OK) return r;
        r = nrc_adam(N, rc, st);
        if (r != PT_OK) return r;
    }
    return PT_OK;
}

uint64_t pt_nrc_serial(const pt_nrc* N) { return N ? N->serial : 0u; }
