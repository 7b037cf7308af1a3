// pt_api.cu -- C-ABI entry points: scene setup and teardown, diagnostics, statistics.
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "pt_internal.h"

uint64_t pt_next_serial() {
    static std::atomic<uint64_t> next{1};
    return next.fetch_add(1);
}

std::atomic<uint64_t> g_pt_launches{0};
static thread_local std::string t_last_error;

void pt_set_error(const std::string& msg) { t_last_error = msg; }

int pt_num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ------------------------------------------------------------------ ordered float atomics
__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ------------------------------------------------------------------ setup kernels
__global__ void k_validate(const float* v, uint32_t nv, const uint32_t* idx, uint32_t nt,
                           const uint32_t* mid, uint32_t nm, uint32_t* bad) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv * 3u && !isfinite(v[i])) atomicOr(bad, 1u);
    if (i < nt * 3u && idx[i] >= nv) atomicOr(bad, 2u);
    if (i < nt && mid[i] >= nm) atomicOr(bad, 4u);
}

__global__ void k_validate_env(const float* env, uint32_t n, uint32_t* bad) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (!isfinite(env[i]) || env[i] < 0.0f)) atomicOr(bad, 8u);
}

// Triangle records (three float4) for the mesh triangles followed by two per quad light.
__global__ void k_make_tris(const float* v, const uint32_t* idx, const uint32_t* mid, uint32_t n_mesh,
                            const float* quads, uint32_t n_quads, float4* out, uint32_t* bounds) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = n_mesh + 2u * n_quads;
    float3 p[3];
    uint32_t code = 0;
    if (i < n_mesh) {
        for (int k = 0; k < 3; ++k) {
            const uint32_t j = idx[3u * i + k];
            p[k] = mk3(v[3u * j], v[3u * j + 1], v[3u * j + 2]);
        }
        code = mid[i];
    } else if (i < n) {
        const uint32_t l = (i - n_mesh) >> 1, second = (i - n_mesh) & 1u;
        const float* q = quads + 13u * l;
        const float3 p0 = mk3(q[0], q[1], q[2]), e1 = mk3(q[3], q[4], q[5]), e2 = mk3(q[6], q[7], q[8]);
        const float3 p2 = (p0 + e1) + e2;
        p[0] = p0;
        p[1] = second ? p2 : p0 + e1;
        p[2] = second ? p0 + e2 : p2;
        code = PT_LIGHT_BIT | l;
    } else {
        return;
    }
    out[3u * i + 0] = make_float4(p[0].x, p[0].y, p[0].z, __uint_as_float(i));
    out[3u * i + 1] = make_float4(p[1].x, p[1].y, p[1].z, __uint_as_float(code));
    out[3u * i + 2] = make_float4(p[2].x, p[2].y, p[2].z, 0.0f);
    for (int a = 0; a < 3; ++a) {
        const float lo = fminf(comp3(p[0], a), fminf(comp3(p[1], a), comp3(p[2], a)));
        const float hi = fmaxf(comp3(p[0], a), fmaxf(comp3(p[1], a), comp3(p[2], a)));
        atomicMin(&bounds[a], f2ord(lo));
        atomicMax(&bounds[3 + a], f2ord(hi));
    }
}

// spawn offset = 1e-4 * diagonal of the scene box
__global__ void k_finish_bounds(const uint32_t* bounds, float* out) {
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = ord2f(bounds[a]); hi[a] = ord2f(bounds[3 + a]); }
    const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    out[0] = 1e-4f * sqrtf(dx * dx + dy * dy + dz * dz);
    for (int a = 0; a < 3; ++a) { out[1 + a] = lo[a]; out[4 + a] = hi[a]; }
}

__device__ __forceinline__ DMat pack_material(const float* v) {
    DMat m;
    m.base_weight = v[0];
    m.base_color = mk3(v[1], v[2], v[3]);
    m.metalness = v[4];
    m.diffuse_rough = v[5];
    m.thin_walled = v[26];
    m.spec_aniso = v[27];
    m.spec_rot = v[28];
    m.fuzz_weight = v[29];
    m.pad0 = m.pad1 = m.pad2 = 0.0f;
    m.spec_weight = v[6];
    m.spec_color = mk3(v[7], v[8], v[9]);
    m.spec_rough = v[10];
    m.spec_ior = v[11];
    m.trans_weight = v[12];
    m.trans_color = mk3(v[13], v[14], v[15]);
    m.coat_weight = v[16];
    m.coat_color = mk3(v[17], v[18], v[19]);
    m.coat_rough = v[20];
    m.coat_ior = v[21];
    m.emission = mk3(v[23], v[24], v[25]) * v[22];
    return m;
}

__global__ void k_pack_mats(const float* raw, uint32_t n, DMat* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = pack_material(raw + (uint32_t)PT_OPENPBR_FLOATS * i);
}

__global__ void k_prepare_quads(const float* raw, uint32_t n, DQuad* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* q = raw + 13u * i;
    DQuad d;
    d.p0 = mk3(q[0], q[1], q[2]);
    d.e1 = mk3(q[3], q[4], q[5]);
    d.e2 = mk3(q[6], q[7], q[8]);
    d.L = mk3(q[9], q[10], q[11]);
    d.two_sided = q[12] != 0.0f;
    const float3 c = cross3(d.e1, d.e2);
    d.area = len3(c);
    d.n = norm3(c);
    d.pad0 = d.pad1 = d.pad2 = 0.0f;
    out[i] = d;
}

static bool material_ok(const pt_openpbr& m, std::string& why) {
    const float* v = reinterpret_cast<const float*>(&m);
    for (int i = 0; i < PT_OPENPBR_FLOATS; ++i)
        if (!std::isfinite(v[i])) { why = "non-finite material parameter"; return false; }
    if (v[26] != 0.0f && v[26] != 1.0f) { why = "geometry_thin_walled must be 0 or 1"; return false; }
    auto unit = [](float x) { return x >= 0.0f && x <= 1.0f; };
    const int unit_idx[] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 13, 14, 15, 16, 17, 18, 19, 20, 23, 24, 25, 27, 28,
                             29, 30, 31, 32, 33};
    for (int i : unit_idx)
        if (!unit(v[i])) { why = "material parameter " + std::to_string(i) + " outside [0,1]"; return false; }
    if (!(v[11] > 1.0f && v[11] <= 3.0f)) { why = "specular_ior outside (1,3]"; return false; }
    if (!(v[21] > 1.0f && v[21] <= 3.0f)) { why = "coat_ior outside (1,3]"; return false; }
    if (v[22] < 0.0f) { why = "negative emission"; return false; }
    return true;
}

static void free_scene(pt_scene* s) {
    if (!s) return;
    void* ptrs[] = {s->d_vertices, s->d_indices, s->d_matids, s->d_tris_raw, s->d_tris, s->d_nodes,
                    s->d_mats, s->d_fuzz, s->d_quads, s->d_quads_raw, s->d_env, s->d_env_marg, s->d_env_cond,
                    s->d_env_wtex, s->d_env_total, s->d_env_guide, s->d_err, s->d_stats, s->d_head};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    pt_free_wave(s->wave);
    if (s->wf_graph) cudaGraphExecDestroy(s->wf_graph);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
}

extern "C" pt_status pt_scene_create(const float* vertices, uint32_t n_vertices, const uint32_t* indices,
                                     uint32_t n_triangles, const uint32_t* material_ids,
                                     const pt_openpbr* materials, uint32_t n_materials,
                                     const pt_quad_light* lights, uint32_t n_lights, const float* env_rgb,
                                     uint32_t env_w, uint32_t env_h, int inputs_on_device,
                                     void* cuda_stream, pt_scene** out) {
    PT_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    PT_CHECK_ARG(n_triangles + n_lights > 0, "scene has no triangles and no lights");
    PT_CHECK_ARG(n_triangles == 0 || (vertices && indices && material_ids && n_vertices > 0),
                 "triangle arrays missing");
    PT_CHECK_ARG(n_materials > 0 || n_triangles == 0, "no materials");
    PT_CHECK_ARG(n_materials == 0 || materials != nullptr, "materials is NULL");
    PT_CHECK_ARG(n_lights == 0 || lights != nullptr, "lights is NULL");
    PT_CHECK_ARG(env_rgb == nullptr || (env_w > 0 && env_h > 0), "env size is zero");
    PT_CHECK_ARG((uint64_t)n_triangles + 2ull * n_lights < (1ull << 31), "too many triangles");
    PT_CHECK_ARG((uint64_t)n_vertices * 3ull < (1ull << 32), "too many vertices");
    std::string why;
    for (uint32_t i = 0; i < n_materials; ++i)
        PT_CHECK_ARG(material_ok(materials[i], why), "material " + std::to_string(i) + ": " + why);
    for (uint32_t l = 0; l < n_lights; ++l) {
        const float* q = reinterpret_cast<const float*>(&lights[l]);
        for (int i = 0; i < 12; ++i) PT_CHECK_ARG(std::isfinite(q[i]), "non-finite light parameter");
        for (int i = 9; i < 12; ++i) PT_CHECK_ARG(q[i] >= 0.0f, "negative light radiance");
        const double cx = (double)q[4] * q[8] - (double)q[5] * q[7];
        const double cy = (double)q[5] * q[6] - (double)q[3] * q[8];
        const double cz = (double)q[3] * q[7] - (double)q[4] * q[6];
        PT_CHECK_ARG(cx * cx + cy * cy + cz * cz > 0.0, "degenerate quad light");
    }
    if (!inputs_on_device) {
        for (uint64_t i = 0; i < (uint64_t)n_vertices * 3; ++i)
            PT_CHECK_ARG(std::isfinite(vertices[i]), "non-finite vertex");
        for (uint64_t i = 0; i < (uint64_t)n_triangles * 3; ++i)
            PT_CHECK_ARG(indices[i] < n_vertices, "vertex index out of range");
        for (uint64_t i = 0; i < n_triangles; ++i)
            PT_CHECK_ARG(material_ids[i] < n_materials, "material id out of range");
        if (env_rgb)
            for (uint64_t i = 0; i < (uint64_t)env_w * env_h * 3; ++i)
                PT_CHECK_ARG(std::isfinite(env_rgb[i]) && env_rgb[i] >= 0.0f, "bad env texel");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    pt_scene* s = new pt_scene();
    s->serial = pt_next_serial();
    cudaGetDevice(&s->device);
    s->n_vertices = n_vertices;
    s->n_mesh_tris = n_triangles;
    s->n_quads = n_lights;
    s->n_tris = n_triangles + 2 * n_lights;
    s->n_mats = n_materials;
    for (uint32_t i = 0; i < n_materials; ++i) s->has_fuzz |= materials[i].fuzz_weight > 0.0f;
    s->last_stream = st;
    const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    auto fail = [&](pt_status code) { free_scene(s); return code; };
#define TRY(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            pt_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                \
            return fail(e_ == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA);         \
        }                                                                                    \
    } while (0)
    const size_t nv3 = (size_t)std::max<uint32_t>(n_vertices, 1) * 3;
    const size_t nt3 = (size_t)std::max<uint32_t>(n_triangles, 1) * 3;
    TRY(cudaMalloc(&s->d_vertices, nv3 * sizeof(float)));
    TRY(cudaMalloc(&s->d_indices, nt3 * sizeof(uint32_t)));
    TRY(cudaMalloc(&s->d_matids, (nt3 / 3) * sizeof(uint32_t)));
    TRY(cudaMalloc(&s->d_tris_raw, (size_t)s->n_tris * 3 * sizeof(float4)));
    TRY(cudaMalloc(&s->d_mats, std::max<uint32_t>(n_materials, 1) * sizeof(DMat)));
    TRY(cudaMalloc(&s->d_fuzz, (size_t)std::max<uint32_t>(n_materials, 1) * FUZZ_FLOATS * sizeof(float)));
    TRY(cudaMalloc(&s->d_quads, std::max<uint32_t>(n_lights, 1) * sizeof(DQuad)));
    TRY(cudaMalloc(&s->d_quads_raw, std::max<uint32_t>(n_lights, 1) * 13 * sizeof(float)));
    TRY(cudaMalloc(&s->d_err, 16 * sizeof(uint32_t)));
    TRY(cudaMalloc(&s->d_stats, ST_COUNT * sizeof(unsigned long long)));
    TRY(cudaMalloc(&s->d_head, 64 * sizeof(uint32_t)));
    TRY(cudaMemsetAsync(s->d_err, 0, 16 * sizeof(uint32_t), st));
    TRY(cudaMemsetAsync(s->d_stats, 0, ST_COUNT * sizeof(unsigned long long), st));
    if (n_triangles > 0) {
        TRY(cudaMemcpyAsync(s->d_vertices, vertices, (size_t)n_vertices * 3 * sizeof(float), kind, st));
        TRY(cudaMemcpyAsync(s->d_indices, indices, (size_t)n_triangles * 3 * sizeof(uint32_t), kind, st));
        TRY(cudaMemcpyAsync(s->d_matids, material_ids, (size_t)n_triangles * sizeof(uint32_t), kind, st));
    }
    // host parameter tables go through a staging buffer that lives until the stream syncs
    std::vector<float> mat_raw((size_t)std::max<uint32_t>(n_materials, 1) * PT_OPENPBR_FLOATS, 0.0f);
    if (n_materials) std::memcpy(mat_raw.data(), materials, (size_t)n_materials * PT_OPENPBR_FLOATS * sizeof(float));
    std::vector<float> quad_raw((size_t)std::max<uint32_t>(n_lights, 1) * 13, 0.0f);
    for (uint32_t l = 0; l < n_lights; ++l) {
        std::memcpy(&quad_raw[13 * l], &lights[l], 12 * sizeof(float));
        quad_raw[13 * l + 12] = lights[l].two_sided ? 1.0f : 0.0f;
    }
    float* d_mat_raw = nullptr;
    TRY(cudaMalloc(&d_mat_raw, mat_raw.size() * sizeof(float)));
    TRY(cudaMemcpyAsync(d_mat_raw, mat_raw.data(), mat_raw.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(s->d_quads_raw, quad_raw.data(), quad_raw.size() * sizeof(float),
                        cudaMemcpyHostToDevice, st));
    // scratch words: [0..5] ordered-int bounds, [8] validation flags, [10..16] eps + box
    constexpr int kScratchWords = 32;
    uint32_t* d_scratch = nullptr;
    TRY(cudaMalloc(&d_scratch, kScratchWords * sizeof(uint32_t)));
    TRY(cudaMemsetAsync(d_scratch, 0, kScratchWords * sizeof(uint32_t), st));
    if (inputs_on_device && n_triangles > 0) {
        const uint64_t m = std::max<uint64_t>((uint64_t)n_vertices * 3, (uint64_t)n_triangles * 3);
        PT_LAUNCH(k_validate, (uint32_t)((m + 255) / 256), 256, 0, st, s->d_vertices, n_vertices, s->d_indices,
                  n_triangles, s->d_matids, n_materials, d_scratch + 8);
    }
    if (n_materials) PT_LAUNCH(k_pack_mats, (n_materials + 127) / 128, 128, 0, st, d_mat_raw, n_materials, s->d_mats);
    {
        pt_status fr = pt_fuzz_series(d_mat_raw, n_materials, s->d_fuzz, st);
        if (fr != PT_OK) return fail(fr);
    }
    if (n_lights) PT_LAUNCH(k_prepare_quads, (n_lights + 127) / 128, 128, 0, st, s->d_quads_raw, n_lights, s->d_quads);
    // bounds accumulate in ordered-int form: mins start at max, maxs at 0
    std::vector<uint32_t> binit = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    TRY(cudaMemcpyAsync(d_scratch, binit.data(), 6 * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    uint32_t bad = 0;
    {
        const uint32_t n = s->n_tris;
        PT_LAUNCH(k_make_tris, (n + 255) / 256, 256, 0, st, s->d_vertices, s->d_indices, s->d_matids,
                  n_triangles, s->d_quads_raw, n_lights, s->d_tris_raw, d_scratch);
        float* d_fin = reinterpret_cast<float*>(d_scratch + 10);
        PT_LAUNCH(k_finish_bounds, 1, 1, 0, st, d_scratch, d_fin);
        float fin[7];
        TRY(cudaMemcpyAsync(&bad, d_scratch + 8, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(fin, d_fin, 7 * sizeof(float), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        s->eps = fin[0];
        for (int a = 0; a < 3; ++a) { s->lo[a] = fin[1 + a]; s->hi[a] = fin[4 + a]; }
    }
    if (env_rgb) {
        const size_t ne = (size_t)env_w * env_h * 3;
        TRY(cudaMalloc(&s->d_env, ne * sizeof(float)));
        TRY(cudaMemcpyAsync(s->d_env, env_rgb, ne * sizeof(float), kind, st));
        if (inputs_on_device) {
            TRY(cudaMemsetAsync(d_scratch + 8, 0, sizeof(uint32_t), st));
            PT_LAUNCH(k_validate_env, (uint32_t)((ne + 255) / 256), 256, 0, st, s->d_env, (uint32_t)ne, d_scratch + 8);
            uint32_t bad_env = 0;
            TRY(cudaMemcpyAsync(&bad_env, d_scratch + 8, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            TRY(cudaStreamSynchronize(st));
            bad |= bad_env;
        }
        s->env_w = (int)env_w;
        s->env_h = (int)env_h;
    }
    TRY(cudaStreamSynchronize(st));
    cudaFree(d_mat_raw);
    cudaFree(d_scratch);
#undef TRY
    if (bad) {
        pt_set_error(bad & 1 ? "non-finite vertex" : bad & 2 ? "vertex index out of range"
                     : bad & 4 ? "material id out of range" : "bad env texel");
        free_scene(s);
        return PT_ERR_INVALID_ARG;
    }
    *out = s;
    return PT_OK;
}

extern "C" pt_status pt_bvh_build(pt_scene* s, const pt_bvh_opts* opts, void* cuda_stream) {
    PT_CHECK_ARG(s != nullptr, "scene is NULL");
    uint32_t leaf = opts && opts->leaf_size ? opts->leaf_size : 4;
    PT_CHECK_ARG(leaf >= 1 && leaf <= 4, "leaf_size must be 1..4");
    uint32_t builder = opts && opts->builder ? opts->builder : (uint32_t)PT_BVH_PLOC;
    PT_CHECK_ARG(builder == PT_BVH_LBVH || builder == PT_BVH_PLOC, "builder must be PT_BVH_LBVH or PT_BVH_PLOC");
    uint32_t collapse = opts && opts->collapse ? opts->collapse : (uint32_t)PT_COLLAPSE_OPTIMAL;
    PT_CHECK_ARG(collapse == PT_COLLAPSE_OPTIMAL || collapse == PT_COLLAPSE_GREEDY,
                 "collapse must be PT_COLLAPSE_OPTIMAL or PT_COLLAPSE_GREEDY");
    const float tri_cost = opts && opts->tri_cost != 0.0f ? opts->tri_cost : 0.8f;
    PT_CHECK_ARG(tri_cost > 0.0f && tri_cost < 1e6f, "tri_cost must be positive and finite");
    float box_cost = opts && opts->box_cost != 0.0f ? opts->box_cost : 0.0f;
    PT_CHECK_ARG(box_cost < 1e6f && box_cost == box_cost, "box_cost must be finite");
    if (box_cost < 0.0f) box_cost = 0.0f;
    const uint32_t width = opts && opts->max_width ? opts->max_width : 8u;
    PT_CHECK_ARG(width >= 2 && width <= 8, "max_width must be 2..8");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->last_stream = st;
    pt_status r = pt_build_bvh_impl(s, leaf, builder, collapse, tri_cost, box_cost, width, st);
    if (r == PT_OK) {
        s->max_width = width;
        s->leaf_size = leaf;
        s->builder = builder;
        s->collapse = collapse;
        s->tri_cost = tri_cost;
        s->box_cost = opts ? opts->box_cost : 0.0f;
    }
    if (r != PT_OK) return r;
    r = pt_build_env_impl(s, st);
    if (r != PT_OK) return r;
    s->built = true;
    return PT_OK;
}

extern "C" void pt_scene_destroy(pt_scene* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    free_scene(s);
}

extern "C" pt_status pt_scene_sync(pt_scene* s) {
    PT_CHECK_ARG(s != nullptr, "scene is NULL");
    PT_CUDA_TRY(cudaStreamSynchronize(s->last_stream));
    uint32_t err = 0;
    PT_CUDA_TRY(cudaMemcpy(&err, s->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (err & 2u) { pt_set_error("device wait ran out of its spin budget"); return PT_ERR_TIMEOUT; }
    if (err & 1u) { pt_set_error("traversal stack or work queue overflow"); return PT_ERR_QUEUE_OVERFLOW; }
    if (err & 4u) { pt_set_error("BVH traversal exceeded its node budget (malformed tree)"); return PT_ERR_CUDA; }
    return PT_OK;
}

extern "C" pt_status pt_get_stats(pt_scene* s, pt_stats* out) {
    PT_CHECK_ARG(s != nullptr && out != nullptr, "NULL argument");
    PT_CUDA_TRY(cudaStreamSynchronize(s->last_stream));
    unsigned long long st[ST_COUNT];
    uint32_t err = 0;
    PT_CUDA_TRY(cudaMemcpy(st, s->d_stats, sizeof(st), cudaMemcpyDeviceToHost));
    PT_CUDA_TRY(cudaMemcpy(&err, s->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->ext_rays = st[ST_EXT];
    out->shadow_rays = st[ST_SHADOW];
    out->paths = st[ST_PATHS];
    out->nan_dropped = st[ST_NAN];
    out->rr_terminated = st[ST_RR];
    out->nrc_queries = st[ST_NRC];
    out->kernel_launches = s->launches;
    out->bvh_nodes = s->n_nodes;
    out->bvh_depth = s->depth;
    out->bvh_width = s->built ? s->max_width : 0u;
    out->n_triangles = s->n_tris;
    out->trace_nodes = st[ST_NODES];
    out->trace_tris = st[ST_TRIS];
    out->shadow_nodes = st[ST_SH_NODES];
    out->shadow_tris = st[ST_SH_TRIS];
    out->tail_ext_rays = st[ST_TAIL_EXT];
    out->tail_shadow_rays = st[ST_TAIL_SH];
    out->tail_trace_nodes = st[ST_TAIL_NODES];
    out->tail_trace_tris = st[ST_TAIL_TRIS];
    out->tail_shadow_nodes = st[ST_TAIL_SH_NODES];
    out->tail_shadow_tris = st[ST_TAIL_SH_TRIS];
    out->graph_replays = s->graph_replays;
    out->error_flags = err;
    out->trace_boxes = st[ST_BOXES];
    out->shadow_boxes = st[ST_SH_BOXES];
    out->tail_trace_boxes = st[ST_TAIL_BOXES];
    out->tail_shadow_boxes = st[ST_TAIL_SH_BOXES];
    if (err & 2u) { pt_set_error("device wait ran out of its spin budget"); return PT_ERR_TIMEOUT; }
    if (err & 1u) { pt_set_error("traversal stack or work queue overflow"); return PT_ERR_QUEUE_OVERFLOW; }
    if (err & 4u) { pt_set_error("BVH traversal exceeded its node budget (malformed tree)"); return PT_ERR_CUDA; }
    return PT_OK;
}

extern "C" uint64_t pt_launch_count(void) { return g_pt_launches.load(); }

extern "C" const char* pt_status_string(pt_status s) {
    switch (s) {
        case PT_OK: return "PT_OK";
        case PT_ERR_INVALID_ARG: return "PT_ERR_INVALID_ARG";
        case PT_ERR_OOM: return "PT_ERR_OOM";
        case PT_ERR_CUDA: return "PT_ERR_CUDA";
        case PT_ERR_NOT_BUILT: return "PT_ERR_NOT_BUILT";
        case PT_ERR_TIMEOUT: return "PT_ERR_TIMEOUT";
        case PT_ERR_QUEUE_OVERFLOW: return "PT_ERR_QUEUE_OVERFLOW";
        case PT_ERR_UNSUPPORTED: return "PT_ERR_UNSUPPORTED";
    }
    return "PT_UNKNOWN";
}

extern "C" const char* pt_last_error(void) { return t_last_error.c_str(); }

// ------------------------------------------------------------------ diagnostics
__global__ void k_trace(DScene S, const float* rays, uint32_t n, int flags, uint32_t* tri, float* t, float* uv) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* r = rays + 8u * i;
    const float3 o = mk3(r[0], r[1], r[2]), d = mk3(r[3], r[4], r[5]);
    const float tmax = r[6];
    TravCount tc = {0, 0, 0};
    if (flags & PT_TRACE_ANY) {
        const bool occ = (flags & PT_TRACE_COUNT) ? trace_any_t<true>(S, o, d, tmax, tc) : trace_any(S, o, d, tmax);
        tri[i] = occ ? 0u : PT_NO_HIT;
        if (t) t[i] = 0.0f;
        if (uv && (flags & PT_TRACE_COUNT)) { uv[2 * i] = (float)tc.nodes; uv[2 * i + 1] = (float)tc.tris; }
        return;
    }
    HitRec h;
    if (flags & PT_TRACE_COUNT) trace_closest_t<true>(S, o, d, tmax, h, tc);
    else trace_closest(S, o, d, tmax, h);
    if (h.tri == PT_NO_HIT) {
        tri[i] = PT_NO_HIT;
        if (t) t[i] = __int_as_float(0x7f800000);
    } else {
        tri[i] = __float_as_uint(S.tris[3u * h.tri].w);
        if (t) t[i] = h.t;
    }
    if (uv) {
        if (flags & PT_TRACE_COUNT) { uv[2 * i] = (float)tc.nodes; uv[2 * i + 1] = (float)tc.tris; }
        else if (h.tri == PT_NO_HIT) { uv[2 * i] = 0.0f; uv[2 * i + 1] = 0.0f; }
        else { uv[2 * i] = h.u; uv[2 * i + 1] = h.v; }
    }
}

// the same with the cooperative traversal: ray i is carried by the 8 lanes of group i
__global__ void __launch_bounds__(128) k_trace_coop(DScene S, const float* rays, uint32_t n, int flags, uint32_t* tri,
                                                    float* t, float* uv) {
    __shared__ CoopShared gsh[128 / COOP_W];
    const uint32_t lane = threadIdx.x & 31u, gl = lane & (COOP_W - 1u), gbase = lane & ~(COOP_W - 1u);
    const uint32_t gm = 0xffu << gbase;
    const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) / COOP_W;
    if (i >= n) return;   // whole groups leave together
    CoopShared& sh = gsh[threadIdx.x / COOP_W];
    const float* r = rays + 8u * i;
    const float3 o = mk3(r[0], r[1], r[2]), d = mk3(r[3], r[4], r[5]);
    const float tmax = r[6];
    const bool count = (flags & PT_TRACE_COUNT) != 0;
    TravCount tc = {0, 0, 0};
    if (flags & PT_TRACE_ANY) {
        CoopAny st;
        coop_any_init(S, o, d, tmax, st);
        if (count) while (!coop_any_step<true>(S, st, sh, gl, gm, gbase, tc)) {}
        else while (!coop_any_step<false>(S, st, sh, gl, gm, gbase, tc)) {}
        if (gl == 0) {
            tri[i] = st.hit ? 0u : PT_NO_HIT;
            if (t) t[i] = 0.0f;
            if (uv && count) { uv[2 * i] = (float)tc.nodes; uv[2 * i + 1] = (float)tc.tris; }
        }
        return;
    }
    CoopClosest st;
    coop_closest_init(S, o, d, tmax, st);
    if (count) while (!coop_closest_step<true>(S, st, sh, gl, gm, gbase, tc)) {}
    else while (!coop_closest_step<false>(S, st, sh, gl, gm, gbase, tc)) {}
    HitRec h;
    const bool mine = coop_closest_finish(st, gl, gm, gbase, h);
    // the counts live in lane 0 of the group, the hit in the lane that found it
    const uint32_t cn = __shfl_sync(gm, tc.nodes, 0, COOP_W), ct = __shfl_sync(gm, tc.tris, 0, COOP_W);
    if (!mine) return;
    if (h.tri == PT_NO_HIT) {
        tri[i] = PT_NO_HIT;
        if (t) t[i] = __int_as_float(0x7f800000);
    } else {
        tri[i] = __float_as_uint(S.tris[3u * h.tri].w);
        if (t) t[i] = h.t;
    }
    if (uv) {
        if (count) { uv[2 * i] = (float)cn; uv[2 * i + 1] = (float)ct; }
        else if (h.tri == PT_NO_HIT) { uv[2 * i] = 0.0f; uv[2 * i + 1] = 0.0f; }
        else { uv[2 * i] = h.u; uv[2 * i + 1] = h.v; }
    }
}

extern "C" pt_status pt_trace(pt_scene* s, const float* rays, uint32_t n, int flags, uint32_t* hit_tri,
                              float* hit_t, float* hit_uv, void* cuda_stream) {
    PT_CHECK_ARG(s && rays && hit_tri, "NULL argument");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    if (n == 0) return PT_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->last_stream = st;
    PT_CHECK_ARG((flags & ~(PT_TRACE_ANY | PT_TRACE_COUNT | PT_TRACE_COOP)) == 0, "unknown trace flags");
    if (flags & PT_TRACE_COOP) {
        const uint64_t threads = (uint64_t)n * COOP_W;
        PT_LAUNCH(k_trace_coop, (uint32_t)((threads + 127) / 128), 128, 0, st, s->view(), rays, n, flags, hit_tri,
                  hit_t, hit_uv);
    } else {
        PT_LAUNCH(k_trace, (n + 127) / 128, 128, 0, st, s->view(), rays, n, flags, hit_tri, hit_t, hit_uv);
    }
    s->launches++;
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

__global__ void k_bsdf_eval(const float* mats, const float* fuzz, const int32_t* front, const float* wo,
                            const float* wi, uint32_t n, float* f_out, float* pdf_out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DMat M = pack_material(mats + (uint32_t)PT_OPENPBR_FLOATS * i);
    const float3 o = mk3(wo[3 * i], wo[3 * i + 1], wo[3 * i + 2]);
    const float3 w = mk3(wi[3 * i], wi[3 * i + 1], wi[3 * i + 2]);
    Closure C;
    closure_setup(C, M, front[i] != 0, o.z, fuzz + (size_t)FUZZ_FLOATS * i);
    float3 f;
    float pdf;
    closure_eval(C, o, w, f, pdf);
    f_out[3 * i] = f.x;
    f_out[3 * i + 1] = f.y;
    f_out[3 * i + 2] = f.z;
    pdf_out[i] = pdf;
}

__global__ void k_bsdf_sample(const float* mats, const float* fuzz, const int32_t* front, const float* wo,
                              const float* u, uint32_t n, float* wi_out, float* w_out, float* pdf_out,
                              uint32_t* flags) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DMat M = pack_material(mats + (uint32_t)PT_OPENPBR_FLOATS * i);
    const float3 o = mk3(wo[3 * i], wo[3 * i + 1], wo[3 * i + 2]);
    Closure C;
    closure_setup(C, M, front[i] != 0, o.z, fuzz + (size_t)FUZZ_FLOATS * i);
    BsdfSample bs;
    const bool ok = closure_sample(C, o, u[4 * i], u[4 * i + 1], u[4 * i + 2], u[4 * i + 3], bs);
    if (!ok) {
        bs.wi = splat3(0.0f);
        bs.weight = splat3(0.0f);
        bs.pdf = 0.0f;
        bs.delta = false;
    }
    wi_out[3 * i] = bs.wi.x; wi_out[3 * i + 1] = bs.wi.y; wi_out[3 * i + 2] = bs.wi.z;
    w_out[3 * i] = bs.weight.x; w_out[3 * i + 1] = bs.weight.y; w_out[3 * i + 2] = bs.weight.z;
    pdf_out[i] = bs.pdf;
    flags[i] = (ok ? 1u : 0u) | (bs.delta ? 2u : 0u);
}

extern "C" pt_status pt_bsdf_eval(const pt_openpbr* materials, const int32_t* front, const float* wo,
                                  const float* wi, uint32_t n, float* f_out, float* pdf_out, void* cuda_stream) {
    PT_CHECK_ARG(materials && front && wo && wi && f_out && pdf_out, "NULL argument");
    if (n == 0) return PT_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float* raw = reinterpret_cast<const float*>(materials);
    float* fuzz = nullptr;   // the rows' fuzz series, stream-ordered scratch
    PT_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&fuzz), (size_t)n * FUZZ_FLOATS * sizeof(float), st));
    pt_status r = pt_fuzz_series(raw, n, fuzz, st);
    if (r == PT_OK) {
        PT_LAUNCH(k_bsdf_eval, (n + 127) / 128, 128, 0, st, raw, fuzz, front, wo, wi, n, f_out, pdf_out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            pt_set_error(std::string("k_bsdf_eval: ") + cudaGetErrorString(e));
            r = PT_ERR_CUDA;
        }
    }
    cudaFreeAsync(fuzz, st);
    return r;
}

extern "C" pt_status pt_bsdf_sample(const pt_openpbr* materials, const int32_t* front, const float* wo,
                                    const float* u, uint32_t n, float* wi_out, float* weight_out,
                                    float* pdf_out, uint32_t* flags_out, void* cuda_stream) {
    PT_CHECK_ARG(materials && front && wo && u && wi_out && weight_out && pdf_out && flags_out, "NULL argument");
    if (n == 0) return PT_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float* raw = reinterpret_cast<const float*>(materials);
    float* fuzz = nullptr;   // the rows' fuzz series, stream-ordered scratch
    PT_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&fuzz), (size_t)n * FUZZ_FLOATS * sizeof(float), st));
    pt_status r = pt_fuzz_series(raw, n, fuzz, st);
    if (r == PT_OK) {
        PT_LAUNCH(k_bsdf_sample, (n + 127) / 128, 128, 0, st, raw, fuzz, front, wo, u, n, wi_out, weight_out,
                  pdf_out, flags_out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            pt_set_error(std::string("k_bsdf_sample: ") + cudaGetErrorString(e));
            r = PT_ERR_CUDA;
        }
    }
    cudaFreeAsync(fuzz, st);
    return r;
}

__global__ void k_camera_rays(DCam cam, uint64_t seed, const uint32_t* pix, uint32_t n, float* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t x = pix[3 * i], y = pix[3 * i + 1], s = pix[3 * i + 2];
    const uint32_t p = y * cam.width + x;
    float3 o, d;
    camera_ray_ps(cam, x, y, p, s, (uint32_t)seed, (uint32_t)(seed >> 32), o, d);
    float* r = out + 6 * i;
    r[0] = o.x; r[1] = o.y; r[2] = o.z; r[3] = d.x; r[4] = d.y; r[5] = d.z;
}

extern "C" pt_status pt_camera_rays(const pt_camera* camera, uint64_t seed, const uint32_t* pixels, uint32_t n,
                                    float* out, void* cuda_stream) {
    PT_CHECK_ARG(camera && pixels && out, "NULL argument");
    PT_CHECK_ARG(camera->width > 0 && camera->height > 0, "empty frame");
    PT_CHECK_ARG(lens_ok(*camera), "lens_radius must be finite and >= 0, with focus_distance > 0 when it is > 0");
    if (n == 0) return PT_OK;
    PT_LAUNCH(k_camera_rays, (n + 127) / 128, 128, 0, (cudaStream_t)cuda_stream, to_dcam(*camera), seed, pixels, n, out);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

__global__ void k_uniforms(uint64_t seed, const uint32_t* keys, uint32_t n, float* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = uniform_at(keys[4 * i], keys[4 * i + 1], keys[4 * i + 2], keys[4 * i + 3], seed);
}

extern "C" pt_status pt_uniforms(uint64_t seed, const uint32_t* keys, uint32_t n, float* out, void* cuda_stream) {
    PT_CHECK_ARG(keys && out, "NULL argument");
    if (n == 0) return PT_OK;
    PT_LAUNCH(k_uniforms, (n + 255) / 256, 256, 0, (cudaStream_t)cuda_stream, seed, keys, n, out);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

__global__ void k_env_sample(DScene S, const float* u, uint32_t n, float* dir, float* pdf) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 d = splat3(0.0f), L;
    float p = 0.0f;
    if (!env_sample(S, u[2 * i], u[2 * i + 1], d, p, L)) p = 0.0f;
    dir[3 * i] = d.x; dir[3 * i + 1] = d.y; dir[3 * i + 2] = d.z;
    pdf[i] = p;
}

__global__ void k_env_pdf(DScene S, const float* dirs, uint32_t n, float* pdf) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pdf[i] = env_pdf(S, mk3(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]));
}

extern "C" pt_status pt_env_sample(pt_scene* s, const float* u, uint32_t n, float* dir_out, float* pdf_out,
                                   void* cuda_stream) {
    PT_CHECK_ARG(s && u && dir_out && pdf_out, "NULL argument");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    PT_CHECK_ARG(s->env_w > 0, "scene has no environment map");
    if (n == 0) return PT_OK;
    PT_LAUNCH(k_env_sample, (n + 127) / 128, 128, 0, (cudaStream_t)cuda_stream, s->view(), u, n, dir_out, pdf_out);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

extern "C" pt_status pt_env_pdf(pt_scene* s, const float* dirs, uint32_t n, float* pdf_out, void* cuda_stream) {
    PT_CHECK_ARG(s && dirs && pdf_out, "NULL argument");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    PT_CHECK_ARG(s->env_w > 0, "scene has no environment map");
    if (n == 0) return PT_OK;
    PT_LAUNCH(k_env_pdf, (n + 127) / 128, 128, 0, (cudaStream_t)cuda_stream, s->view(), dirs, n, pdf_out);
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

extern "C" pt_status pt_bvh_export(pt_scene* s, uint32_t* nodes_out, float* tris_out, uint32_t* n_nodes,
                                   uint32_t* n_tris, void* cuda_stream) {
    PT_CHECK_ARG(s != nullptr, "scene is NULL");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n_nodes) *n_nodes = s->n_nodes;
    if (n_tris) *n_tris = s->n_tris;
    if (nodes_out)
        PT_CUDA_TRY(cudaMemcpyAsync(nodes_out, s->d_nodes, (size_t)s->n_nodes * 5 * sizeof(uint4),
                                    cudaMemcpyDeviceToHost, st));
    if (tris_out)
        PT_CUDA_TRY(cudaMemcpyAsync(tris_out, s->d_tris, (size_t)s->n_tris * 3 * sizeof(float4),
                                    cudaMemcpyDeviceToHost, st));
    PT_CUDA_TRY(cudaStreamSynchronize(st));
    return PT_OK;
}
