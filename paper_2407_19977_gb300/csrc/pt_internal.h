// pt_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <vector>
#include <cstdint>
#include <string>

#include "pt.h"
#include "pt_device.cuh"

// ---- error reporting -------------------------------------------------------------------
void pt_set_error(const std::string& msg);

#define PT_CUDA_TRY(call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            pt_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
            return e_ == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA;              \
        }                                                                                   \
    } while (0)

#define PT_CHECK_ARG(cond, msg)                                                             \
    do {                                                                                    \
        if (!(cond)) {                                                                      \
            pt_set_error(msg);                                                              \
            return PT_ERR_INVALID_ARG;                                                      \
        }                                                                                   \
    } while (0)

// ---- launch accounting -----------------------------------------------------------------
extern std::atomic<uint64_t> g_pt_launches;
inline void pt_count_launch(uint64_t n = 1) { g_pt_launches.fetch_add(n, std::memory_order_relaxed); }
#define PT_LAUNCH(kernel, grid, block, smem, stream, ...)                                   \
    do {                                                                                    \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                         \
        pt_count_launch();                                                                  \
    } while (0)

int pt_num_sms();

// ---- device statistics slots -----------------------------------------------------------
enum { ST_EXT = 0, ST_SHADOW = 1, ST_PATHS = 2, ST_NAN = 3, ST_RR = 4, ST_NRC = 5, ST_NODES = 6, ST_TRIS = 7,
       ST_SH_NODES = 8, ST_SH_TRIS = 9, ST_TAIL_EXT = 10, ST_TAIL_SH = 11, ST_TAIL_NODES = 12, ST_TAIL_TRIS = 13,
       ST_TAIL_SH_NODES = 14, ST_TAIL_SH_TRIS = 15, ST_BOXES = 16, ST_SH_BOXES = 17, ST_TAIL_BOXES = 18,
       ST_TAIL_SH_BOXES = 19, ST_COUNT = 20 };

// ---- wavefront workspace ---------------------------------------------------------------
struct WaveBuffers {
    uint32_t capacity = 0;       // paths per wave
    float4* ray_o[2] = {nullptr, nullptr};   // queue entries: origin (w unused)
    float4* ray_d[2] = {nullptr, nullptr};   // direction, w = path id bits
    float4* hit = nullptr;       // t, u, v, tri bits (per queue slot)
    float4* beta = nullptr;      // per path: beta.xyz, prev_pdf
    float4* radiance = nullptr;  // per path: L.xyz
    float4* sh_o = nullptr;      // shadow queue: origin, tmax
    float4* sh_d = nullptr;      // direction, path id bits
    float4* sh_c = nullptr;      // contribution
    uint32_t* perm = nullptr;    // material-sorted order of the queue slots
    uint32_t* keys = nullptr;    // per slot sort key
    uint32_t* counters = nullptr;  // [0..1] queue sizes, [2] shadow size, [3..6] heads, [8..] buckets
    size_t bytes = 0;
    // radiance-cache buffers (allocated on the first cache render)
    uint32_t nrc_capacity = 0, train_slots = 0, rec_per_path = 0, sample_cap = 0;
    uint32_t* aux = nullptr;
    float* nrc_q = nullptr;
    float* nrc_out = nullptr;
    uint32_t* nrc_counters = nullptr;
    float* train_rec = nullptr;
    uint32_t* train_nv = nullptr;
    uint32_t* train_id = nullptr;
    float* train_samples = nullptr;
    // ReSTIR DI buffers (allocated on the first ReSTIR render): per path the primary surface
    // (x, depth), (wo, triangle), (normal), and the initial and final reservoirs (2 float4 each)
    uint32_t restir_capacity = 0;
    float4* rs_g0 = nullptr;
    float4* rs_g1 = nullptr;
    float4* rs_gn = nullptr;
    float4* rs_i = nullptr;
    float4* rs_f = nullptr;
};

// A number no other scene or cache of this process has had: graph caches key on it, since a
// destroyed object's host address can come back for a new one.
uint64_t pt_next_serial();

struct pt_scene {
    int device = 0;
    uint64_t serial = 0;                 // pt_next_serial() at creation
    uint32_t n_vertices = 0, n_mesh_tris = 0, n_tris = 0, n_mats = 0, n_quads = 0;
    float* d_vertices = nullptr;
    uint32_t* d_indices = nullptr;
    uint32_t* d_matids = nullptr;
    float4* d_tris_raw = nullptr;   // triangle records in input order (mesh, then lights)
    float4* d_tris = nullptr;       // leaf order
    uint4* d_nodes = nullptr;
    uint32_t n_nodes = 0, depth = 0;
    DMat* d_mats = nullptr;
    float* d_fuzz = nullptr;         // FUZZ_FLOATS per material: the fuzz lobe's series
    bool has_fuzz = false;           // some material has fuzz_weight > 0
    DQuad* d_quads = nullptr;
    float* d_quads_raw = nullptr;
    float* d_env = nullptr;
    float* d_env_marg = nullptr;
    float* d_env_cond = nullptr;
    float* d_env_wtex = nullptr;
    float* d_env_total = nullptr;
    int* d_env_guide = nullptr;      // search guides of the marginal and conditional CDFs
    int env_gm = 0, env_gc = 0;
    float env_total = 0.0f;
    int env_w = 0, env_h = 0;
    float eps = 0.0f;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    uint32_t* d_err = nullptr;
    unsigned long long* d_stats = nullptr;
    uint32_t* d_head = nullptr;      // persistent work-queue heads (scratch)
    bool built = false;
    WaveBuffers wave;
    cudaStream_t last_stream = nullptr;
    uint64_t launches = 0;
    // captured wavefront call (pt_render_opts.use_graph): the graph, what it was captured for,
    // the kernels it launches, the stream it was captured on, calls that replayed it
    cudaGraphExec_t wf_graph = nullptr;
    std::vector<unsigned char> wf_key;
    uint64_t wf_graph_launches = 0;
    cudaStream_t cap_stream = nullptr;
    uint64_t graph_replays = 0;
    uint32_t leaf_size = 4;          // of the current BVH
    uint32_t builder = PT_BVH_PLOC;  // of the current BVH
    uint32_t collapse = PT_COLLAPSE_OPTIMAL;
    float tri_cost = 0.0f;           // 0: the default
    float box_cost = 0.0f;           // as passed (0: the default)
    uint32_t max_width = 8;          // most children per wide node of the current BVH
    // schedule chosen by pt_autotune for frames of tuned_w x tuned_h (used by PT_MODE_AUTO)
    bool tuned = false;
    uint32_t tuned_w = 0, tuned_h = 0;
    pt_render_opts tuned_opts{};

    DScene view() const {
        DScene s;
        s.tris = d_tris;
        s.nodes = d_nodes;
        s.mats = d_mats;
        s.fuzz = d_fuzz;
        s.quads = d_quads;
        s.env = d_env;
        s.env_marg = d_env_marg;
        s.env_cond = d_env_cond;
        s.env_wtex = d_env_wtex;
        s.env_guide = d_env_guide;
        s.env_gm = env_gm;
        s.env_gc = env_gc;
        s.err = d_err;
        s.env_total = env_total;
        s.eps = eps;
        s.env_w = env_w;
        s.env_h = env_h;
        s.n_quads = (int)n_quads;
        s.n_nodes = (int)n_nodes;
        s.n_tris = (int)n_tris;
        s.pad = 0;
        return s;
    }
};

// implemented in pt_bvh.cu
pt_status pt_build_bvh_impl(pt_scene* s, uint32_t leaf_size, uint32_t builder, uint32_t collapse, float tri_cost,
                            float box_cost, uint32_t max_width, cudaStream_t st);
pt_status pt_build_env_impl(pt_scene* s, cudaStream_t st);

// implemented in pt_render.cu
pt_status pt_free_wave(WaveBuffers& w);
// paths the wavefront tail kernel holds resident (its automatic limit)
pt_status pt_wavefront_tail_limit(int* out);

// implemented in pt_nrc.cu: cache forward pass / one training step for the renderer; the
// row count is read from device memory (n_dev), cap bounds it and sizes the launches
pt_status pt_nrc_render_infer_dev(pt_nrc* N, const float* queries, const uint32_t* n_dev, uint32_t cap, float* out4,
                                  cudaStream_t st);
uint32_t pt_nrc_frame_samples(const pt_nrc* N);
uint64_t pt_nrc_serial(const pt_nrc* N);
pt_status pt_nrc_render_prepare(pt_nrc* N, uint32_t infer_cap, uint32_t train_cap);
// Series of the fuzz lobe (FUZZ_FLOATS per row) for n raw material rows of PT_OPENPBR_FLOATS
// floats on the device; rows without fuzz get zeros (pt_fuzz.cu).
pt_status pt_fuzz_series(const float* raw_materials, uint32_t n, float* out, cudaStream_t st);
pt_status pt_nrc_render_train_dev(pt_nrc* N, const float* samples, const uint32_t* n_dev, uint32_t cap, cudaStream_t st);

// the lens of a camera: radius finite and >= 0; an open lens needs a finite focus distance > 0
inline bool lens_ok(const pt_camera& c) {
    return std::isfinite(c.lens_radius) && c.lens_radius >= 0.0f &&
           (c.lens_radius == 0.0f || (std::isfinite(c.focus_distance) && c.focus_distance > 0.0f));
}

inline DCam to_dcam(const pt_camera& c) {
    DCam d;
    d.origin = make_float3(c.origin[0], c.origin[1], c.origin[2]);
    d.target = make_float3(c.target[0], c.target[1], c.target[2]);
    d.up = make_float3(c.up[0], c.up[1], c.up[2]);
    d.vfov_deg = c.vfov_deg;
    d.width = c.width;
    d.height = c.height;
    d.lens_radius = c.lens_radius;
    d.focus_distance = c.focus_distance;
    return d;
}

// device-side material repack (runs the conversion in a kernel)
struct RawMat { float v[PT_OPENPBR_FLOATS]; };
