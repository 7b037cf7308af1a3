/*
 * pt.h -- C-ABI of the GB300 path tracer (CUDA, sm_103a).
 *
 * The library computes the Monte Carlo estimate of the rendering equation
 *   I(x, x') = g(x, x') [ eps(x, x') + int_S p(x, x', x'') I(x', x'') dx'' ]
 * ("Physically-based Path Tracer using WebGPU and OpenPBR", Sec. 1.1) by backward path
 * tracing from a perspective camera with per-sample jitter (Sec. 5.1.2), closest-hit
 * search through a BVH over triangle meshes (Sec. 5.1.1), OpenPBR shading with importance
 * sampling and Russian roulette at every hit (Sec. 4, Sec. 5.1.3), and progressive
 * per-pixel averaging (Sec. 5.1.3, Sec. 5.1.4).  Scene setup happens once, sampling runs
 * repeatedly on the GPU (Sec. 5.1, Fig. "path tracer pipeline").
 *
 * Conventions for every call:
 *  - Returns a pt_status; nothing throws or aborts across the ABI.  pt_last_error() gives
 *    a human-readable detail for the calling thread's most recent failure.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously on that stream; device-side failures (for example an
 *    exhausted spin budget) are reported by the next call that synchronises
 *    (pt_get_stats, pt_scene_sync) as PT_ERR_TIMEOUT / PT_ERR_QUEUE_OVERFLOW.
 *  - Pointers documented as "device" must be device memory of the current CUDA device;
 *    "host" pointers are ordinary host memory.  The library copies every scene input at
 *    create time: the caller may free its arrays when pt_scene_create returns.
 *  - Caller-owned output buffers (accumulators, hit arrays, NRC buffers) stay owned by
 *    the caller and must outlive the enqueued work.
 *  - Coordinates are right-handed, +y up; triangles wind counter-clockwise seen from their
 *    front side; the geometric normal is normalize((v1 - v0) x (v2 - v0)).
 */
#ifndef PT_H_
#define PT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PT_OK = 0,
    PT_ERR_INVALID_ARG = 1,     /* bad pointer, size, index, NaN/Inf or parameter range */
    PT_ERR_OOM = 2,             /* device or host allocation failed */
    PT_ERR_CUDA = 3,            /* a CUDA runtime call failed (detail in pt_last_error) */
    PT_ERR_NOT_BUILT = 4,       /* pt_render before pt_bvh_build */
    PT_ERR_TIMEOUT = 5,         /* a bounded device-side wait ran out of budget */
    PT_ERR_QUEUE_OVERFLOW = 6,  /* a device work queue or traversal stack overflowed */
    PT_ERR_UNSUPPORTED = 7      /* option value not supported by this build */
} pt_status;

typedef struct pt_scene pt_scene;   /* opaque, library-owned */
typedef struct pt_nrc pt_nrc;       /* opaque, library-owned */

/* OpenPBR surface parameters (Sec. 4; the paper's material model).  PT_OPENPBR_FLOATS (34)
 * floats, in this order; the Python generators and the oracle use the same order.
 * Valid ranges (checked by pt_scene_create): weights, colors, roughnesses, metalness,
 * anisotropy and rotation in [0, 1]; specular_ior and coat_ior in (1, 3];
 * emission_luminance >= 0; geometry_thin_walled 0 or 1.
 * base_diffuse_roughness sigma scales the diffuse base by the qualitative Oren-Nayar factor
 * (1 + sigma s/t) / (1 + c sigma), c = 1/2 - 2/(3 pi), s = wi.wo - cos_i cos_o,
 * t = max(cos_i, cos_o) if s > 0 else 1 (0 = Lambertian). */
typedef struct {
    float base_weight;
    float base_color[3];
    float base_metalness;
    float base_diffuse_roughness;
    float specular_weight;
    float specular_color[3];
    float specular_roughness;
    float specular_ior;
    float transmission_weight;
    float transmission_color[3];
    float coat_weight;
    float coat_color[3];
    float coat_roughness;
    float coat_ior;
    float emission_luminance;
    float emission_color[3];
    float geometry_thin_walled; /* 0 or 1: an infinitely thin sheet.  Both sides are alike
                                   (eta = specular_ior from either side) and transmission
                                   does not refract: its lobe is the specular reflection lobe
                                   mirrored through the surface plane (straight through when
                                   smooth), weighted transmission_color * (1 - specular_weight
                                   * F), without the 1/eta^2 radiance scaling */
    float specular_roughness_anisotropy; /* a: the specular GGX lobe (metal, dielectric,
                                   transmission) gets widths ax = r^2 sqrt(2/(1+(1-a)^2))
                                   along the tangent and ay = (1-a) ax along the bitangent
                                   (r = specular_roughness; 0 = isotropic).  Without vertex
                                   tangents the tangent is the triangle's first edge
                                   (v1 - v0) projected into the surface plane */
    float specular_rotation;    /* turns of the tangent about the normal (0..1) */
    float fuzz_weight;          /* fw: a layer of fibres over the coat.  Its lobe is the
                                   Charlie sheen distribution (Estevez & Kulla 2017)
                                   D = (2 + 1/a) sin(theta_h)^(1/a) / (2 pi) with its exact
                                   Smith masking (projected area A(mu) by quadrature),
                                   a = max(fuzz_roughness, 0.2)^2; the layers below are
                                   scaled by (1 - fw) + fw (1 - E(|cos_i|)) (1 - E(cos_o)),
                                   E the lobe's directional albedo */
    float fuzz_color[3];
    float fuzz_roughness;
} pt_openpbr;
enum { PT_OPENPBR_FLOATS = 34 };

/* Parallelogram area light p0 + a e1 + b e2, (a, b) in [0,1]^2, radiance L emitted on the
 * side of e1 x e2 (both sides if two_sided).  The library also makes it geometry: two
 * black triangles appended after the mesh's triangles, light l -> triangle ids
 * n_triangles + 2l and n_triangles + 2l + 1. */
typedef struct {
    float p0[3];
    float e1[3];
    float e2[3];
    float radiance[3];
    int32_t two_sided;
} pt_quad_light;

/* Perspective camera: vertical field of view vfov_deg; the full frame is width x height
 * pixels, pixel (x, y) with y growing downwards; pixel id p = y * width + x keys the
 * random numbers (Sec. 5.1.2: adjacent pixels run concurrently, each sample jittered).
 * lens_radius = 0 is a pinhole.  lens_radius > 0 is a thin lens (depth of field, named as
 * future work in Sec. 6.3): rays start on a disk of that radius around `origin` in the
 * camera's (right, up) plane and pass through the point where the pinhole ray of the same
 * jitter meets the plane of focus, focus_distance along the view direction
 * (focus_distance > 0 is then required).  The lens point uses dimensions 12-13 of the first
 * vertex. */
typedef struct {
    float origin[3];
    float target[3];
    float up[3];
    float vfov_deg;
    uint32_t width;
    uint32_t height;
    float lens_radius;
    float focus_distance;
} pt_camera;

/* Progressive accumulator (Sec. 5.1.4), caller-owned DEVICE buffers of width*height*3
 * floats each, row-major RGB over the rendered window (the whole frame or a crop).
 * sum/comp are a Kahan-compensated running sum of the sample radiance; the estimate is
 * sum / spp_done.  pt_render adds samples spp_done .. spp_done+spp-1 and advances
 * spp_done, so calling it repeatedly equals one long call (same random numbers). */
typedef struct {
    float* sum;
    float* comp;
    uint64_t spp_done;
    uint32_t width;
    uint32_t height;
} pt_accum;

enum {
    PT_FLAG_NO_NEE = 1u,        /* BSDF sampling only; every emission hit gets weight 1 */
    PT_FLAG_NO_RR = 2u,         /* no Russian roulette */
    PT_FLAG_COUNT = 4u          /* wavefront: count BVH node visits and triangle tests (slower) */
};

/* wavefront kernel kinds, indices of pt_render_opts.kernel_ms */
enum { PT_K_RAYGEN = 0, PT_K_TRACE = 1, PT_K_SORT = 2, PT_K_SHADE = 3, PT_K_SHADOW = 4, PT_K_ACCUM = 5,
       PT_K_TAIL = 6, PT_K_RESTIR = 7, PT_K_KINDS = 8 };

/* ReSTIR DI at the primary vertex (the paper names reservoir resampling for many-light
 * scenes as future work, Sec. 2 and Sec. 6.3; the algorithm is Bitterli et al. 2020).  Per
 * pixel and sample: `candidates` light samples from the next-event light sampler are
 * resampled into a one-sample reservoir with the cheap target lum(L_e) G |cos| on the side
 * the surface scatters to; one spatial pass then resamples, with the full target (the
 * luminance of the unshadowed contribution f L_e |cos| G), this pixel's and the reservoirs of up to
 * `spatial_neighbors` pixels of the same sample (offsets uniform in [-R, R]^2, R =
 * `spatial_radius`, inside the window; neighbours with normal cosine < 0.9 or depth
 * differing by > 10 % are skipped) with the unbiased 1/Z weights (Z counts the reservoirs
 * whose cheap target is positive at the chosen sample).  Vertex 0 shades the
 * result with one shadow ray in place of next-event estimation, and a BSDF-sampled light
 * hit at vertex 1 then counts with weight 0.  Each wave holds whole samples of the window.
 * Random numbers: candidate i uses (pixel, sample, 0xFFFF0001, dims 4i..4i+3), neighbour j
 * (pixel, sample, 0xFFFF0002, dims 4j..4j+2).  Wavefront mode only (PT_MODE_MEGAKERNEL and
 * the radiance cache give PT_ERR_UNSUPPORTED); not with PT_FLAG_NO_NEE. */
typedef struct {
    uint32_t candidates;        /* M >= 1 (at most 4096) */
    uint32_t spatial_neighbors; /* K, 0..64 (0 = no spatial pass) */
    uint32_t spatial_radius;    /* R >= 1 pixels (at most 4096) */
    uint32_t later_candidates;  /* L, 0..4096: at every later vertex, next-event estimation
                                   resamples L light candidates with the cheap target (no
                                   reuse; candidate i of vertex k: (pixel, sample,
                                   0xFFFF0100 + k, dims 4i..4i+3)) and a BSDF-sampled light
                                   hit after it counts with weight 0; 0 = next-event
                                   estimation with MIS there */
} pt_restir_opts;

enum {
    PT_MODE_AUTO = 0,           /* pick per the autotuned table (pt_autotune) */
    PT_MODE_WAVEFRONT = 1,      /* queue-driven kernels per bounce (raygen/trace/sort/shade/shadow) */
    PT_MODE_MEGAKERNEL = 2      /* persistent kernel, one path per thread, work-queue fetch */
};

typedef struct {
    uint32_t crop_x0, crop_y0;  /* window origin in the full frame; size = accum->width/height */
    uint32_t flags;             /* PT_FLAG_* */
    uint32_t mode;              /* PT_MODE_* */
    uint32_t wave_paths;        /* wavefront: paths per wave (0 = automatic) */
    int32_t sort_by_material;   /* wavefront: -1 automatic, 0 off, 1 on */
    uint32_t block_size;        /* threads per block (0 = automatic) */
    float* sample_out;          /* optional DEVICE buffer, height*width*spp*3 floats: the
                                   radiance of each sample (pixel-major, then sample) */
    pt_nrc* nrc;                /* optional neural radiance cache: paths end at their 2nd
                                   diffuse-ish vertex and add beta * cache(vertex) */
    uint32_t nrc_train;         /* with nrc: collect training suffixes and train this frame */
    float* kernel_ms;           /* optional HOST float[PT_K_KINDS]: wavefront mode adds the
                                   CUDA-event time of each kernel kind (synchronises the
                                   stream at the end of the call) */
    uint32_t* kernel_launches;  /* optional HOST uint32[PT_K_KINDS]: launches per kind */
    int32_t tail_paths;         /* wavefront: once the paths left to trace at a bounce number at
                                   most this many, one launch carries each of them to its end
                                   (closest hit, shade, shadow ray per thread) instead of one
                                   launch per stage and bounce; same per-vertex code and random
                                   numbers, so the image is the same.  -1 off, 0 automatic
                                   (the paths the tail kernel holds resident on the GPU) */
    uint32_t use_graph;         /* wavefront: 1 = capture the call's launch sequence into a CUDA
                                   graph once and replay it while the call looks the same (scene,
                                   camera, window, accumulator, spp, depth, options); the first
                                   sample index and the seed are written to device memory before
                                   each replay, so progressive calls reuse one graph.  The capture
                                   runs on a stream of the scene; replays run on cuda_stream.  With
                                   nrc the cache's inference and training are in the graph too
                                   (Adam's step count lives on the device); not with kernel_ms
                                   (that call launches directly). */
    const pt_restir_opts* restir; /* optional: ReSTIR DI at the primary vertex (NULL = next-event
                                   estimation) */
    uint32_t traversal;         /* wavefront closest-hit and shadow passes: PT_TRAVERSAL_* (the
                                   hits, and the node and triangle counts, are the same) */
    uint32_t tail_bounce;       /* wavefront with a tail limit (tail_paths >= 0): 0 = the
                                   per-bounce launches are issued for every bounce up to
                                   max_depth (after the tail kernel has taken over they find
                                   nothing to do); k > 0 = at bounce k the tail kernel takes every
                                   path still running, however many, and no launch is issued for
                                   the later bounces.  The samples are the same. */
} pt_render_opts;

enum {
    PT_TRAVERSAL_AUTO = 0,      /* one ray per lane */
    PT_TRAVERSAL_PER_LANE = 1,  /* one ray per lane, its 8 child boxes tested in a loop */
    PT_TRAVERSAL_COOP = 2       /* one ray per group of 8 lanes: a lane per child box, a node's
                                   leaf triangles spread over the group (more lanes busy, but
                                   more instructions per ray: slower on the CAD frames) */
};

/* Binary tree that the wide BVH is collapsed from (Sec. 5.1.1 builds an AABB hierarchy on
 * the CPU; here both builders run on the device over the same 63-bit Morton order):
 *  PT_BVH_LBVH  Karras' radix tree over the Morton codes (fastest build, splits at the
 *               codes' highest differing bit whatever the triangles' sizes);
 *  PT_BVH_PLOC  parallel locally-ordered clustering (Meister & Bittner 2018): rounds in which
 *               each cluster merges with its mutual nearest neighbour by surface area within
 *               16 positions in the Morton order (a tree close to a full SAH build; the
 *               default). */
enum { PT_BVH_DEFAULT = 0, PT_BVH_LBVH = 1, PT_BVH_PLOC = 2 };

/* How the binary tree is folded into wide nodes (at most max_width children each):
 *  PT_COLLAPSE_OPTIMAL  the least surface-area cost (a wide node visit costs 1 plus box_cost
 *                       per child slot, a triangle test tri_cost, each weighted by area / root
 *                       area), found per binary node by a dynamic programme over the number of
 *                       slots its subtree fills (Ylitie, Karras, Laine, HPG 2017); the default;
 *  PT_COLLAPSE_GREEDY   open the child of largest area until max_width slots are used. */
enum { PT_COLLAPSE_DEFAULT = 0, PT_COLLAPSE_OPTIMAL = 1, PT_COLLAPSE_GREEDY = 2 };

typedef struct {
    uint32_t leaf_size;         /* max triangles per leaf, 1..4 (0 = 4) */
    uint32_t builder;           /* PT_BVH_* (0 = PT_BVH_PLOC) */
    uint32_t collapse;          /* PT_COLLAPSE_* (0 = PT_COLLAPSE_OPTIMAL) */
    float tri_cost;             /* cost of a triangle test against a wide node visit, > 0 and
                                   finite (0 = 0.8: measured best of 0.15 .. 1.5 on the CAD
                                   frames); used by PT_COLLAPSE_OPTIMAL */
    float box_cost;             /* cost of each child slot of a visited wide node, >= 0 and
                                   finite (0 = 0, negative = exactly 0); PT_COLLAPSE_OPTIMAL */
    uint32_t max_width;         /* BVH width: most children a node may have, 2..8 (0 = 8).  The
                                   node format keeps 8 slots; a narrower tree leaves the rest
                                   empty (more, smaller nodes, fewer box tests per node).  Both
                                   collapse rules honour it; pt_autotune with PT_TUNE_BVH and
                                   pt_autotune_batch with PT_TUNE_BVH choose it. */
} pt_bvh_opts;

typedef struct {
    uint64_t ext_rays;          /* extension rays traced (camera + BSDF-sampled) */
    uint64_t shadow_rays;       /* shadow rays traced */
    uint64_t paths;             /* paths started */
    uint64_t nan_dropped;       /* samples with NaN/Inf radiance, discarded */
    uint64_t rr_terminated;     /* paths ended by Russian roulette */
    uint64_t nrc_queries;       /* paths ended by the radiance cache */
    uint64_t kernel_launches;   /* kernels this library launched for this scene */
    uint64_t bvh_nodes;         /* wide BVH nodes */
    uint64_t bvh_depth;         /* wide BVH depth */
    uint64_t n_triangles;       /* mesh + light triangles */
    uint64_t trace_nodes;       /* PT_FLAG_COUNT: wide nodes visited by closest-hit rays */
    uint64_t trace_tris;        /* PT_FLAG_COUNT: triangle tests of closest-hit rays */
    uint64_t shadow_nodes;      /* PT_FLAG_COUNT: wide nodes visited by shadow rays */
    uint64_t shadow_tris;       /* PT_FLAG_COUNT: triangle tests of shadow rays */
    /* the wavefront tail kernel (pt_render_opts.tail_paths): rays it traced (also counted in
       ext_rays / shadow_rays) and, with PT_FLAG_COUNT, its node visits and triangle tests
       (not counted in trace_* / shadow_* above, which cover the per-bounce kernels only) */
    uint64_t tail_ext_rays;
    uint64_t tail_shadow_rays;
    uint64_t tail_trace_nodes;
    uint64_t tail_trace_tris;
    uint64_t tail_shadow_nodes;
    uint64_t tail_shadow_tris;
    uint64_t graph_replays;     /* wavefront calls served by replaying a captured CUDA graph */
    uint32_t error_flags;       /* sticky device error bits (1 = stack overflow, 2 = timeout) */
    uint32_t bvh_width;         /* most children a node of the current BVH may have
                                   (pt_bvh_opts.max_width as built; 0 before the first build) */
    /* PT_FLAG_COUNT: child box tests (filled child slots of the nodes visited) of closest-hit
       and shadow rays in the per-bounce kernels, and in the tail kernel */
    uint64_t trace_boxes;
    uint64_t shadow_boxes;
    uint64_t tail_trace_boxes;
    uint64_t tail_shadow_boxes;
} pt_stats;

/* Scene setup (Sec. 5.1.1 "CPU setup": load geometry and materials).
 *  vertices      float[n_vertices*3]      positions
 *  indices       uint32[n_triangles*3]    vertex indices, each < n_vertices
 *  material_ids  uint32[n_triangles]      each < n_materials
 *  materials     pt_openpbr[n_materials]  (host memory always)
 *  lights        pt_quad_light[n_lights]  (host memory always; may be NULL if 0)
 *  env_rgb       float[env_h*env_w*3]     lat-long radiance, row 0 looks along +y;
 *                u = 0.5 + atan2(dx, -dz)/(2 pi), v = acos(dy)/pi; NULL = black
 *  inputs_on_device: 1 if vertices/indices/material_ids/env_rgb are device pointers.
 * Errors: PT_ERR_INVALID_ARG (out-of-range index or parameter, NaN/Inf vertex or env,
 * zero-sized arrays with non-NULL requirements), PT_ERR_OOM, PT_ERR_CUDA. */
pt_status pt_scene_create(const float* vertices, uint32_t n_vertices, const uint32_t* indices,
                          uint32_t n_triangles, const uint32_t* material_ids,
                          const pt_openpbr* materials, uint32_t n_materials,
                          const pt_quad_light* lights, uint32_t n_lights, const float* env_rgb,
                          uint32_t env_w, uint32_t env_h, int inputs_on_device,
                          void* cuda_stream, pt_scene** out);

/* Device BVH build (Sec. 5.1.1: AABB hierarchy, O(log n) intersection): 64-bit Morton codes,
 * radix sort, linear BVH, collapse to a compressed wide BVH (80-byte nodes of 8 child slots,
 * at most pt_bvh_opts.max_width of them used) with 8-bit child boxes.
 * Enqueued on cuda_stream; synchronises that stream once per wide-tree level.  Also
 * builds the environment sampling tables. */
pt_status pt_bvh_build(pt_scene* scene, const pt_bvh_opts* opts, void* cuda_stream);

/* Render spp samples per pixel of the window accum->width x accum->height at
 * (opts->crop_x0, opts->crop_y0) of the camera's frame (Sec. 5.1.2-5.1.4): camera ray,
 * closest hit, emission with MIS, next-event estimation to quads and the environment,
 * OpenPBR BSDF sample, Russian roulette, max_depth BSDF bounces, Kahan accumulation.
 * seed keys the Philox4x32-10 counter (pixel, sample, bounce, dim/4).
 * Errors: PT_ERR_NOT_BUILT, PT_ERR_INVALID_ARG (window outside the frame, NULL accum),
 * PT_ERR_OOM (work buffers), PT_ERR_CUDA. */
pt_status pt_render(pt_scene* scene, const pt_camera* camera, uint32_t spp, uint32_t max_depth,
                    uint64_t seed, pt_accum* accum, const pt_render_opts* opts,
                    void* cuda_stream);

/* pt_render for callers that cannot allocate device memory (no counterpart in the paper).
 * Some host programs are not allowed to call cudaMalloc: they run under a device-memory
 * budget fixed at start-up, inside a host application that owns every allocation, or in a
 * real-time loop that must not enter the allocator.  This call renders what pt_render
 * renders in PT_MODE_WAVEFRONT: the same per-bounce kernels and random numbers, so the
 * accumulators are bit-identical to pt_render's (pt_render may finish small queues in its
 * tail kernel, which gives the same bits; this call never launches it).  Its work queues live
 * in one fixed array compiled into the library (16,384 paths, about 2.7 MB, held on every GPU
 * that loads the library until the process exits) and it calls no allocating routine.
 * Limits and rules:
 *  - the window (accum->width * accum->height) holds at most 16,384 pixels; larger images
 *    are rendered tile by tile (crop_x0, crop_y0); larger windows return PT_ERR_INVALID_ARG;
 *  - opts->nrc, opts->restir and opts->kernel_ms / kernel_launches must be NULL, and
 *    opts->flags may hold PT_FLAG_NO_NEE and PT_FLAG_NO_RR only (PT_ERR_INVALID_ARG);
 *    mode, wave_paths, tail_paths, tail_bounce, traversal and use_graph are ignored (waves
 *    of the array's size, one ray per lane, no tail kernel, direct launches: the same bits);
 *  - every call shares the one array and leaves its contents behind; the kernels reset every
 *    counter they read before reading it.  Calls that overlap on the GPU (different streams,
 *    or threads without ordering) race on the array and corrupt each other's work;
 *  - each call looks the array's device address up in the current context with
 *    cudaGetSymbolAddress (no allocation once the library's device code is loaded there); the
 *    first call on a device loads that code, so make it before any stream capture.
 * Inputs, outputs and errors otherwise as pt_render. */
pt_status pt_render_noalloc(pt_scene* scene, const pt_camera* camera, uint32_t spp,
                            uint32_t max_depth, uint64_t seed, pt_accum* accum,
                            const pt_render_opts* opts, void* cuda_stream);

/* One job of a batched launch: a built scene, its camera, its accumulator (whole frame). */
typedef struct {
    pt_scene* scene;
    pt_camera camera;
    uint32_t spp;
    uint32_t max_depth;
    uint64_t seed;
    pt_accum* accum;
} pt_job;

typedef struct {
    uint32_t mode;              /* PT_MODE_MEGAKERNEL (or AUTO = 0): every job in ONE persistent
                                   launch that pops (job, pixel tile) items from a shared queue;
                                   PT_MODE_WAVEFRONT: each job rendered by the wavefront path
                                   (graph-replayed launches), the jobs spread over `streams`
                                   concurrent streams forked from and joined back to the
                                   caller's stream (jobs of one scene stay on one stream) */
    uint32_t streams;           /* wavefront mode: concurrent streams (0 = 4, at most 16) */
    uint32_t tile_pixels;       /* megakernel: pixels per work item, a multiple of 32 (0 = 64); a
                                   warp owns an item and traces all samples of its pixels in order */
    uint32_t blocks_per_sm;     /* megakernel: resident blocks per SM (0 = auto) */
    uint32_t use_graph;         /* megakernel, 1: the launch (job-table copy from a library-owned pinned
                                   buffer, queue reset, persistent kernel) is captured once per
                                   job count and work-item layout and replayed; the table is
                                   rewritten before each replay, so seeds, sample indices and
                                   cameras may change between calls.  The call then waits for the
                                   previous graph batch to finish before rewriting the table.
                                   Merged wavefront mode: the same for its launch sequence. */
    uint32_t merged;            /* wavefront mode, 1: ONE wavefront for all jobs -- the paths of
                                   every job share each wave's queues and launches (a wave holds
                                   pixel ranges of several jobs, a job split only along pixels,
                                   so each pixel's samples are accumulated in sample order); the
                                   kernels find a path's scene, camera, depth and seed through
                                   its wave segment; hits are sorted by (job, material) while the
                                   keys fit (at most 1024).  With use_graph the whole launch
                                   sequence is one graph.  The batch's rays and paths are counted
                                   in the first job's scene (pt_get_stats).  0: each job's own
                                   wavefront on `streams` streams */
    uint32_t wave_paths;        /* merged mode: paths per wave (0 = 2^22) */
} pt_batch_opts;

/* Batched rendering of many scenes of uneven size in ONE persistent launch: blocks pop
 * (job, tile, sample-chunk) items from a shared work queue in device memory until it is
 * empty.  Each job's image equals rendering it alone with pt_render.  */
pt_status pt_render_batch(const pt_job* jobs, uint32_t n_jobs, const pt_batch_opts* opts,
                          void* cuda_stream);

/* Autotuner of the execution schedule (beyond the paper).  Renders `frames` frames (after one
 * warm-up frame) of `spp` samples per candidate into a scratch accumulator of camera->width x
 * height and times them with CUDA events on the stream; candidates: wavefront with material
 * sort off/on x tail limit (off, automatic, a quarter, four times) x wave size (2^20 .. 2^23
 * paths, as far as the call needs them), graph replay on; megakernel with 32, 64, 128 pixels
 * per work item; then the winner's traversal passes one ray per lane or per 8-lane group, and a
 * wavefront winner with a tail limit with tail_bounce 3, 4, 5 and 6.  With
 * PT_TUNE_BVH it first rebuilds the BVH with both builders and leaf sizes 1..4 at width 8, then
 * the fastest of those at widths 4 and 6 (pt_bvh_opts.max_width), and keeps the fastest tree.  The winner goes to *best (and ms per frame to
 * *best_ms) and is stored in the scene: pt_render with PT_MODE_AUTO then uses it for frames
 * of that size (not with nrc; with kernel_ms the launches are direct, not replayed).  No candidate changes the image: they render the
 * same samples; the tuning renders do count in pt_get_stats.  Synchronises the stream.
 * Errors: PT_ERR_NOT_BUILT, PT_ERR_INVALID_ARG, PT_ERR_OOM (scratch), PT_ERR_CUDA. */
#define PT_TUNE_BVH 1u
pt_status pt_autotune(pt_scene* scene, const pt_camera* camera, uint32_t spp, uint32_t max_depth,
                      uint32_t frames, uint32_t tune_flags, pt_render_opts* best, float* best_ms,
                      void* cuda_stream);
/* The same for a batch: each job rendered into scratch accumulators (the jobs' own are not
 * touched); candidates: megakernel with tile_pixels 32..256 x blocks_per_sm (automatic, 2, 4),
 * wavefront with 1, 2, 4, 8 streams, merged wavefront with 2^22, 2^23, 2^24 paths per wave.
 * With PT_TUNE_BVH it first rebuilds every scene of the jobs at BVH widths 8, 6 and 4 (each
 * scene keeps its builder, leaf size and collapse rule), times one merged wavefront of 2^23
 * paths per wave on each, and leaves the scenes built at the fastest width, which goes to
 * the schedule sweep; the scenes' trees change, their images do not. */
pt_status pt_autotune_batch(const pt_job* jobs, uint32_t n_jobs, uint32_t frames, uint32_t tune_flags,
                            pt_batch_opts* best, float* best_ms, void* cuda_stream);

/* Closest hit of n rays through the scene's BVH (Sec. 5.1.3 "checks for intersections using
 * the BVH").  rays: DEVICE float[n*8] = origin[3], dir[3], tmax, unused.  Outputs (DEVICE):
 * hit_tri uint32[n] triangle id (mesh ids, then light triangles; 0xFFFFFFFF on a miss),
 * hit_t float[n], hit_uv float[n*2] barycentric weights of v1 and v2.  Ties at equal t go
 * to the lower triangle id.  flags bit 0 (PT_TRACE_ANY): occlusion only (hit_tri = 0 or ~0);
 * bit 1 (PT_TRACE_COUNT): hit_uv receives the ray's wide-node visits and triangle tests;
 * bit 2 (PT_TRACE_COOP): the cooperative traversal of the wavefront passes (a group of 8
 * lanes per ray) instead of one ray per thread -- the same results and counts.
 * Asynchronous on the stream. */
enum { PT_TRACE_ANY = 1, PT_TRACE_COUNT = 2, PT_TRACE_COOP = 4 };
pt_status pt_trace(pt_scene* scene, const float* rays, uint32_t n, int flags,
                   uint32_t* hit_tri, float* hit_t, float* hit_uv, void* cuda_stream);

/* OpenPBR BSDF in the local shading frame (normal = +z, wo.z > 0) for n tuples (Sec. 4,
 * Sec. 5.1.3 importance sampling).  All arrays DEVICE.  materials pt_openpbr[n],
 * front int32[n] (1 = the side the winding faces), wo/wi float[n*3].
 * eval: f_out float[n*3] (non-delta lobes), pdf_out float[n] (mixture sampling pdf).
 * sample: u float[n*4] = (lobe, dir1, dir2, refract) uniforms; outputs wi float[n*3],
 * weight float[n*3] = f|cos|/pdf, pdf float[n], flags uint32[n] (1 = valid, 2 = delta). */
pt_status pt_bsdf_eval(const pt_openpbr* materials, const int32_t* front, const float* wo,
                       const float* wi, uint32_t n, float* f_out, float* pdf_out,
                       void* cuda_stream);
pt_status pt_bsdf_sample(const pt_openpbr* materials, const int32_t* front, const float* wo,
                         const float* u, uint32_t n, float* wi_out, float* weight_out,
                         float* pdf_out, uint32_t* flags_out, void* cuda_stream);

/* Camera rays of n (pixel x, pixel y, sample) triples (Sec. 5.1.2).  pixels: DEVICE
 * uint32[n*3]; out: DEVICE float[n*6] = origin[3], dir[3]. */
pt_status pt_camera_rays(const pt_camera* camera, uint64_t seed, const uint32_t* pixels,
                         uint32_t n, float* out, void* cuda_stream);

/* Philox4x32-10 uniforms for n (pixel, sample, bounce, dim) keys: keys DEVICE uint32[n*4],
 * out DEVICE float[n]. */
pt_status pt_uniforms(uint64_t seed, const uint32_t* keys, uint32_t n, float* out,
                      void* cuda_stream);

/* Environment sampling table queries (DEVICE arrays): sample n directions from uniforms
 * u float[n*2] -> dir float[n*3], pdf float[n] (solid angle); or evaluate the pdf of
 * n directions. */
pt_status pt_env_sample(pt_scene* scene, const float* u, uint32_t n, float* dir_out,
                        float* pdf_out, void* cuda_stream);
pt_status pt_env_pdf(pt_scene* scene, const float* dirs, uint32_t n, float* pdf_out,
                     void* cuda_stream);

/* Copy the built BVH to HOST memory for inspection (Sec. 5.1.1 structure checks): nodes
 * uint32[5*4*n_nodes] in the 80-byte node layout, triangles float[12*n_tris] in leaf order
 * (w of the first float4 = original triangle id bits, of the second = material code).
 * Pass NULL buffers to query n_nodes / n_tris only.  Synchronises the stream. */
pt_status pt_bvh_export(pt_scene* scene, uint32_t* nodes_out, float* tris_out, uint32_t* n_nodes,
                        uint32_t* n_tris, void* cuda_stream);

/* Display resolve (Sec. 5.1.4: the accumulated texture is shown through a full-screen pass
 * that applies the Khronos PBR Neutral tone mapper).  Per pixel: mean = sum / spp_done,
 * times `exposure`; NaN becomes 0 and the mean is clamped to [0, 1e30]; PBR Neutral
 * (offset toe with F90 = 0.04, highlight compression from 0.76, desaturation 0.15); clamp
 * to [0, 1]; with PT_TONEMAP_SRGB the sRGB transfer function (IEC 61966-2-1); then
 * floor(255 v + 0.5) into R, G, B and 255 into A.  Every step is an FP32 operation in that
 * order (no fused multiply-adds), as the tone mapper runs in the paper's shader.
 *  accum     the accumulator (DEVICE sum, height*width*3 floats; comp is not read)
 *  rgba_out  DEVICE uint8[height*width*4], 4-byte aligned, row-major RGBA
 * Errors: PT_ERR_INVALID_ARG (NULL pointers, spp_done == 0, exposure negative or not
 * finite, misaligned output).  Asynchronous on the stream. */
#define PT_TONEMAP_SRGB 1u
pt_status pt_tonemap(const pt_accum* accum, float exposure, uint32_t flags, uint8_t* rgba_out,
                     void* cuda_stream);

/* Primary-hit features for the regression denoiser (the paper names denoising as future
 * work, Sec. 6.3; BMFR, Koskela et al. 2019, takes these inputs).  For every pixel of the
 * window (crop_x0, crop_y0, width, height) of the frame, the mean over samples
 * s0 .. s0+spp-1 -- the same camera rays as pt_render's samples with that seed -- of the
 * first hit's shading normal (turned towards the camera), hit position and albedo
 * ((m + (1-m)(1-t)) base_weight base_color + (1-m) t transmission_color), and the fraction
 * of the samples whose first hit is a scattering surface (misses and light quads add
 * nothing to the means).
 *  out  DEVICE float[height*width*12], 16-byte aligned, row-major: normal[3], fraction,
 *       position[3], 0, albedo[3], 0
 * Errors: PT_ERR_INVALID_ARG (NULL, window outside the frame, misaligned out, bad camera),
 * PT_ERR_NOT_BUILT.  Asynchronous on the stream. */
pt_status pt_render_features(pt_scene* scene, const pt_camera* camera, uint32_t crop_x0, uint32_t crop_y0,
                             uint32_t width, uint32_t height, uint32_t s0, uint32_t spp, uint64_t seed,
                             float* out, void* cuda_stream);

/* Blockwise multi-order feature regression (BMFR): per square block of `block` pixels
 * (block (i, j) covers x in [i*block - offset_x, (i+1)*block - offset_x), likewise y, clipped
 * to the image), the least-squares fit of the demodulated colour c / (albedo + 0.01) on the
 * columns 1, n[3], q[3], q[3]^2 over the block's pixels whose feature fraction is 1 (q = the
 * position scaled to [-1, 1] over the block; n scaled likewise); a feature whose block range
 * is at most 1e-4 * max(|lo|, |hi|, 0.01) is left out, then, in that column order, a column
 * whose part outside the span of the kept earlier ones is at most 1e-3 of its norm.  The
 * output is the fitted value times (albedo + 0.01); other pixels keep their colour.  FP32
 * Householder QR per block in shared memory.
 *  color     DEVICE float[height*width*3], mean radiance (e.g. sum / spp of an accumulator)
 *  features  DEVICE float[height*width*12] from pt_render_features, 16-byte aligned
 *  block     4..32; offset_x, offset_y < block
 *  out       DEVICE float[height*width*3]; may be `color` itself
 * Errors: PT_ERR_INVALID_ARG.  Asynchronous on the stream. */
pt_status pt_denoise_bmfr(const float* color, const float* features, uint32_t width, uint32_t height,
                          uint32_t block, uint32_t offset_x, uint32_t offset_y, float* out, void* cuda_stream);

/* Statistics and sticky device error bits; synchronises the scene's last stream. */
pt_status pt_get_stats(pt_scene* scene, pt_stats* out);
pt_status pt_scene_sync(pt_scene* scene);
void pt_scene_destroy(pt_scene* scene);

/* Kernels launched by this library in this process (all scenes). */
uint64_t pt_launch_count(void);

/* ---------------- Neural radiance cache (the paper's future work, Sec. 6.1) ----------------
 * Multiresolution hash-grid encoding of the vertex position (levels x features per entry,
 * 2^log2_table entries per level) concatenated with direction, normal and roughness, fed
 * to a 64-wide MLP with n_hidden hidden layers (ReLU), output RGB.  Weights and grid are
 * trained online with Adam on a relative L2 loss by the library's own forward/backward
 * kernels; the MLP runs on the tensor cores (FP16 operands, FP32 accumulation). */
typedef struct {
    uint32_t n_levels;          /* hash-grid levels (16) */
    uint32_t log2_table;        /* log2 entries per level (19) */
    uint32_t base_resolution;   /* coarsest grid resolution (16) */
    float per_level_scale;      /* resolution growth per level (0 = from 2048 finest) */
    uint32_t n_hidden;          /* hidden layers (4) */
    float learning_rate;        /* Adam step size (1e-2 grid and MLP) */
    uint32_t batch;             /* training samples per Adam step (8192); a rendered frame
                                   with nrc_train takes one step per batch of its samples */
    uint64_t seed;              /* weight initialisation seed */
    float scene_min[3];         /* position normalisation box */
    float scene_max[3];
    uint32_t frame_samples;     /* training samples a rendered frame collects (32768), from
                                   frame_samples / 2 training paths */
    uint32_t tcgen05;           /* 1: inference MLP on the tcgen05 tensor cores (128-row tiles,
                                   accumulators in tensor memory); 0: on mma.sync, 16-row tiles
                                   per warp, which measures faster here because inference is
                                   bound by the hash-grid gathers, not by the MLP */
    uint32_t train_kernels;     /* 0: each training batch's loss and gradients in ONE fused
                                   tcgen05 kernel (encoding, forward, loss, backward, weight and
                                   grid gradients per 128-sample tile); 1: the same steps as
                                   separate mma.sync kernels.  Adam runs after either. */
} pt_nrc_opts;

/* Query layout for pt_nrc_infer / training samples (DEVICE arrays of float[n*16]):
 * pos[3] (world space, normalised by the opts box), dir[3], normal[3], roughness,
 * target_rgb[3] (training only), pad[3].
 * pt_nrc_train: one Adam step per `batch` samples.  pt_nrc_infer: out_rgb is DEVICE
 * float[n*4] (RGB + one unused column).  pt_nrc_gradients: loss gradients of one batch
 * without an update, into DEVICE buffers (MLP: same layout as pt_nrc_params(0); grid:
 * same layout as pt_nrc_params(1); either may be NULL). */
pt_status pt_nrc_create(const pt_nrc_opts* opts, void* cuda_stream, pt_nrc** out);
pt_status pt_nrc_train(pt_nrc* nrc, const float* samples, uint32_t n, void* cuda_stream);
pt_status pt_nrc_infer(pt_nrc* nrc, const float* queries, uint32_t n, float* out_rgb,
                       void* cuda_stream);
pt_status pt_nrc_gradients(pt_nrc* nrc, const float* samples, uint32_t n, float* dw_out,
                           float* dgrid_out, void* cuda_stream);
/* Parameter access for tests and checkpoints: FP32 master copies (DEVICE float arrays).
 * which = 0: MLP weights (4 hidden layers [64][64] then the output layer padded to
 * [16][64], each [out][in]), 1: hash-grid table [levels][2^log2_table][2].  After writing
 * through the pointer call pt_nrc_commit to refresh the FP16 copies the kernels read. */
pt_status pt_nrc_params(pt_nrc* nrc, int which, float** ptr, uint64_t* count);
pt_status pt_nrc_commit(pt_nrc* nrc, void* cuda_stream);
/* Training loss of the most recent training call (pt_nrc_train, pt_nrc_gradients or a
 * rendered frame with nrc_train): mean relative L2 over all its samples, evaluated before
 * each batch's update; synchronises. */
pt_status pt_nrc_last_loss(pt_nrc* nrc, float* loss);
void pt_nrc_destroy(pt_nrc* nrc);

const char* pt_status_string(pt_status status);
const char* pt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PT_H_ */
