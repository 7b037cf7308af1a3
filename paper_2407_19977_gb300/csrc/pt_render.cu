// pt_render.cu -- path tracing kernels (Sec. 5.1.2 ray generator, Sec. 5.1.3 path tracer,
// Sec. 5.1.4 progressive averaging).
//
// Two executions of the same per-vertex code (shade_vertex in pt_device.cuh):
//  * megakernel: a persistent grid; warps pop (job, pixel tile) items from a work queue in
//    device memory, each lane traces its pixel's samples in order and Kahan-accumulates.
//    One launch also serves a batch of many scenes (pt_render_batch).
//  * wavefront: one kernel per stage and bounce over queues in HBM: raygen -> closest hit
//    (persistent, queue-fetching) -> optional sort of the queue by material -> shade
//    (appends next rays and shadow rays with warp-aggregated atomics) -> shadow any-hit
//    -> per-pixel Kahan accumulation in sample order.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "pt_internal.h"

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ------------------------------------------------------------------ megakernel
struct DJob {
    DScene S;
    DCam cam;
    uint32_t x0, y0, cw, ch;      // window in the full frame
    uint32_t s0, spp, max_depth, flags;
    uint64_t seed;
    float* sum;
    float* comp;
    float* sample_out;
    unsigned long long* stats;
    uint32_t tile_begin;          // first work item of this job
    uint32_t n_tiles;
    uint32_t n_mats;              // materials of the scene
    uint32_t key_base;            // merged batch waves: first material-sort key of this job
};

struct PixelCounters {
    unsigned long long ext, shadow, nan, rr, paths;
};

__device__ __forceinline__ void render_pixel(const DJob& J, uint32_t lp, PixelCounters& cnt) {
    const uint32_t px = J.x0 + lp % J.cw, py = J.y0 + lp / J.cw;
    const uint32_t p = py * J.cam.width + px;
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    float* sp = J.sum + 3ull * lp;
    float* cp = J.comp + 3ull * lp;
    float s0 = sp[0], s1 = sp[1], s2 = sp[2], c0 = cp[0], c1 = cp[1], c2 = cp[2];
    for (uint32_t i = 0; i < J.spp; ++i) {
        const uint32_t s = J.s0 + i;
        float3 o, d;
        camera_ray_ps(J.cam, px, py, p, s, k0, k1, o, d);
        PathState ps;
        ps.beta = splat3(1.0f);
        ps.L = splat3(0.0f);
        ps.prev_pdf = -1.0f;
        for (uint32_t k = 0;; ++k) {
            HitRec h;
            trace_closest(J.S, o, d, __int_as_float(0x7f800000), h);
            cnt.ext++;
            VertexRng rng;
            rng.p = p; rng.s = s; rng.k = k; rng.k0 = k0; rng.k1 = k1;
            ShadeOut so;
            const int r = shade_vertex(J.S, h, o, d, k, J.max_depth, J.flags, rng, ps, so);
            if (so.has_shadow) {
                cnt.shadow++;
                if (!trace_any(J.S, so.sh.o, so.sh.d, so.sh.tmax)) ps.L = ps.L + so.sh.contrib;
            }
            if (r == SHADE_END) {
                if (so.rr_end) cnt.rr++;
                break;
            }
            o = so.next_o;
            d = so.next_d;
        }
        cnt.paths++;
        float3 L = ps.L;
        if (!isfinite(L.x) || !isfinite(L.y) || !isfinite(L.z)) {
            cnt.nan++;
            L = splat3(0.0f);
        }
        if (J.sample_out) {
            float* o3 = J.sample_out + 3ull * ((uint64_t)lp * J.spp + i);
            o3[0] = L.x; o3[1] = L.y; o3[2] = L.z;
        }
        kahan_add(s0, c0, L.x);
        kahan_add(s1, c1, L.y);
        kahan_add(s2, c2, L.z);
    }
    sp[0] = s0; sp[1] = s1; sp[2] = s2;
    cp[0] = c0; cp[1] = c1; cp[2] = c2;
}

__device__ __forceinline__ void megakernel_item(const DJob& J, uint32_t item, uint32_t tile_pixels) {
    const uint32_t lane = lane_id();
    const uint32_t npix = J.cw * J.ch;
    const uint32_t pb = (item - J.tile_begin) * tile_pixels;
    const uint32_t pe = min(pb + tile_pixels, npix);
    PixelCounters cnt = {0, 0, 0, 0, 0};
    for (uint32_t lp = pb + lane; lp < pe; lp += 32) render_pixel(J, lp, cnt);
    const unsigned long long e = warp_sum_u64(cnt.ext), sh = warp_sum_u64(cnt.shadow),
                             nn = warp_sum_u64(cnt.nan), rr = warp_sum_u64(cnt.rr), pa = warp_sum_u64(cnt.paths);
    if (lane == 0) {
        atomicAdd(&J.stats[ST_EXT], e);
        atomicAdd(&J.stats[ST_SHADOW], sh);
        if (nn) atomicAdd(&J.stats[ST_NAN], nn);
        if (rr) atomicAdd(&J.stats[ST_RR], rr);
        atomicAdd(&J.stats[ST_PATHS], pa);
    }
}

// warps pop work items until the queue is empty; an item is a tile of pixels of one job
__device__ __forceinline__ uint32_t pop_item(uint32_t* head) {
    uint32_t item = 0;
    if (lane_id() == 0) item = atomicAdd(head, 1u);
    return __shfl_sync(0xffffffffu, item, 0);
}

__global__ void __launch_bounds__(128) k_megakernel(const DJob* __restrict__ jobs, uint32_t n_jobs,
                                                    uint32_t total_items, uint32_t tile_pixels, uint32_t* head) {
    for (;;) {
        const uint32_t item = pop_item(head);
        if (item >= total_items) break;
        uint32_t lo = 0, hi = n_jobs - 1;
        while (lo < hi) {  // last job with tile_begin <= item
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (jobs[mid].tile_begin <= item) lo = mid; else hi = mid - 1;
        }
        megakernel_item(jobs[lo], item, tile_pixels);
    }
}

__global__ void __launch_bounds__(128) k_megakernel_one(const __grid_constant__ DJob job, uint32_t total_items,
                                                        uint32_t tile_pixels, uint32_t* head) {
    for (;;) {
        const uint32_t item = pop_item(head);
        if (item >= total_items) break;
        megakernel_item(job, item, tile_pixels);
    }
}

static int g_mk_blocks_per_sm = 0;

static uint32_t megakernel_grid(uint32_t total_items, uint32_t blocks_per_sm) {
    if (g_mk_blocks_per_sm == 0) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_megakernel, 128, 0);
        g_mk_blocks_per_sm = std::max(b, 1);
    }
    const uint32_t bps = blocks_per_sm ? blocks_per_sm : (uint32_t)g_mk_blocks_per_sm;
    uint32_t grid = (uint32_t)pt_num_sms() * bps;
    grid = std::min(grid, (total_items + 3) / 4);   // 4 warps per block, one item per warp at a time
    return std::max(grid, 1u);
}

// one job: the job travels as a kernel parameter, nothing is staged in device memory
static pt_status launch_megakernel_one(DJob job, uint32_t tile_pixels, uint32_t blocks_per_sm, cudaStream_t st,
                                       uint32_t* d_head, uint64_t* launches) {
    job.tile_begin = 0;
    job.n_tiles = (job.cw * job.ch + tile_pixels - 1) / tile_pixels;
    if (job.n_tiles == 0) return PT_OK;
    PT_CUDA_TRY(cudaMemsetAsync(d_head, 0, sizeof(uint32_t), st));
    PT_LAUNCH(k_megakernel_one, megakernel_grid(job.n_tiles, blocks_per_sm), 128, 0, st, job, job.n_tiles,
              tile_pixels, d_head);
    (*launches)++;
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

// many jobs: the job table goes to a device buffer owned by the caller of this function
static pt_status launch_megakernel(const std::vector<DJob>& jobs_in, uint32_t tile_pixels, uint32_t blocks_per_sm,
                                   cudaStream_t st, uint32_t* d_head, DJob* d_jobs, uint64_t* launches) {
    std::vector<DJob> jobs = jobs_in;
    uint32_t total = 0;
    for (auto& j : jobs) {
        j.tile_begin = total;
        j.n_tiles = (j.cw * j.ch + tile_pixels - 1) / tile_pixels;
        total += j.n_tiles;
    }
    if (total == 0) return PT_OK;
    PT_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(DJob), cudaMemcpyHostToDevice, st));
    PT_CUDA_TRY(cudaMemsetAsync(d_head, 0, sizeof(uint32_t), st));
    PT_LAUNCH(k_megakernel, megakernel_grid(total, blocks_per_sm), 128, 0, st, d_jobs, (uint32_t)jobs.size(), total,
              tile_pixels, d_head);
    (*launches)++;
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

// Batch as a replayed graph: {copy of the job table from a pinned host buffer, reset of the
// queue head, persistent kernel}.  Everything that changes between calls (cameras, seeds,
// first sample indices) is table data, so the graph depends only on the job count and the
// work-item layout.  One cached graph per process; the pinned table is rewritten only after
// the previous replay has finished.
struct BatchGraph {
    int device = -1;
    uint32_t n_jobs = 0, total = 0, tile = 0, grid = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t done = nullptr;
    DJob* h_jobs = nullptr;      // pinned
    DJob* d_jobs = nullptr;
    uint32_t* d_head = nullptr;
    void release() {
        if (done) cudaEventSynchronize(done);
        if (exec) cudaGraphExecDestroy(exec);
        if (h_jobs) cudaFreeHost(h_jobs);
        if (d_jobs) cudaFree(d_jobs);
        if (d_head) cudaFree(d_head);
        if (done) cudaEventDestroy(done);
        if (cap) cudaStreamDestroy(cap);
        *this = BatchGraph();
    }
};
static std::mutex g_batch_mutex;
static BatchGraph g_batch_graph;

static pt_status launch_megakernel_graph(const std::vector<DJob>& jobs_in, uint32_t tile_pixels, uint32_t blocks_per_sm,
                                         cudaStream_t st, uint64_t* launches) {
    std::vector<DJob> jobs = jobs_in;
    uint32_t total = 0;
    for (auto& j : jobs) {
        j.tile_begin = total;
        j.n_tiles = (j.cw * j.ch + tile_pixels - 1) / tile_pixels;
        total += j.n_tiles;
    }
    if (total == 0) return PT_OK;
    const uint32_t grid = megakernel_grid(total, blocks_per_sm);
    int dev = 0;
    PT_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    BatchGraph& g = g_batch_graph;
    if (!(g.exec && g.device == dev && g.n_jobs == jobs.size() && g.total == total && g.tile == tile_pixels &&
          g.grid == grid)) {
        g.release();
        g.device = dev;
        g.n_jobs = (uint32_t)jobs.size();
        g.total = total;
        g.tile = tile_pixels;
        g.grid = grid;
        const size_t bytes = jobs.size() * sizeof(DJob);
        if (cudaMallocHost((void**)&g.h_jobs, bytes) != cudaSuccess || cudaMalloc((void**)&g.d_jobs, bytes) != cudaSuccess ||
            cudaMalloc((void**)&g.d_head, sizeof(uint32_t)) != cudaSuccess) {
            g.release();
            pt_set_error("batch graph buffers: out of memory");
            return PT_ERR_OOM;
        }
        PT_CUDA_TRY(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
        PT_CUDA_TRY(cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking));
        PT_CUDA_TRY(cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = g_pt_launches.load();
        cudaMemcpyAsync(g.d_jobs, g.h_jobs, bytes, cudaMemcpyHostToDevice, g.cap);
        cudaMemsetAsync(g.d_head, 0, sizeof(uint32_t), g.cap);
        PT_LAUNCH(k_megakernel, grid, 128, 0, g.cap, g.d_jobs, (uint32_t)jobs.size(), total, tile_pixels, g.d_head);
        g_pt_launches.fetch_sub(g_pt_launches.load() - before);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(g.cap, &graph);
        if (ce != cudaSuccess) {
            g.release();
            pt_set_error(std::string("batch graph capture: ") + cudaGetErrorString(ce));
            return PT_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            g.release();
            pt_set_error(std::string("batch graph instantiate: ") + cudaGetErrorString(ie));
            return PT_ERR_CUDA;
        }
    } else {
        // the previous replay may still read the pinned table
        PT_CUDA_TRY(cudaEventSynchronize(g.done));
    }
    std::memcpy(g.h_jobs, jobs.data(), jobs.size() * sizeof(DJob));
    PT_CUDA_TRY(cudaGraphLaunch(g.exec, st));
    PT_CUDA_TRY(cudaEventRecord(g.done, st));
    pt_count_launch(1);
    (*launches)++;
    return PT_OK;
}

// ------------------------------------------------------------------ wavefront
// counters: queue sizes, fetch heads, C_TAIL = 1 once the tail kernel has taken the wave's
// remaining paths (the per-bounce kernels then have nothing to do), C_FRAME.. the values that
// change from one call to the next (first sample index, seed: written by k_wf_frame, so the
// launch sequence of a call is the same every call and can be replayed as a CUDA graph),
// sort buckets
enum { C_Q0 = 0, C_Q1 = 1, C_SH = 2, C_HEAD_TRACE = 3, C_HEAD_SHADOW = 4, C_TAIL = 5, C_FRAME = 8,
       C_BUCKETS = 16 };
constexpr uint32_t MAX_SORT_KEYS = 1024;

struct WfParams {
    DScene S;
    DCam cam;
    uint32_t x0, y0, cw;           // window origin and width
    uint32_t pb, npix;             // pixel range of this wave (window-local linear index)
    uint32_t i0, nsamp;            // samples of this wave: call-relative first, count
    uint32_t spp_call;             // samples in the call
    uint32_t max_depth, flags;
    uint32_t n_keys;               // material sort buckets (0 = no sort)
    uint32_t tail_bounce;          // host: bounce at which the tail kernel takes every path (0: none)
    uint32_t tiled;                // 1: the first queue holds each sample's pixels in 8 x 4 tiles
    float4* ray_o[2];
    float4* ray_d[2];
    float4* hit;
    float4* beta;
    float4* radiance;
    float4* sh_o;
    float4* sh_d;
    float4* sh_c;
    uint32_t* perm;
    uint32_t* keys;
    uint32_t* counters;
    float* sum;
    float* comp;
    float* sample_out;
    unsigned long long* stats;
    // radiance cache (wavefront only)
    int nrc_on;
    uint32_t rec_per_path, max_train, sample_cap;
    float train_prob;
    uint32_t* aux;            // per path: diffuse-ish vertex count | (training slot + 1) << 8
    float* nrc_q;             // cache query records (16 floats)
    float* nrc_out;           // cache outputs (4 floats per query)
    uint32_t* nrc_counters;   // [0] queries, [1] training paths, [2] training samples
    float* train_rec;         // training slots x rec_per_path x 16 floats
    uint32_t* train_nv;       // vertices recorded per training path
    uint32_t* train_id;       // path id of each training path
    // ReSTIR DI at the primary vertex (whole windows per wave)
    int restir_on;
    uint32_t restir_M, restir_K, restir_R, restir_L;
    float4* rs_g0;            // per path: primary hit point, depth
    float4* rs_g1;            // per path: direction towards the camera, triangle bits (PT_NO_HIT: none)
    float4* rs_gn;            // per path: shading normal
    float4* rs_i;             // per path: initial reservoir (2 float4)
    float4* rs_f;             // per path: final reservoir (2 float4)
    float* train_samples;     // training sample records (16 floats)
    // merged batch waves (pt_render_batch): paths of several jobs share a wave
    const DJob* jobs;
    const struct WfmSeg* segs;  // this wave's segments
    uint32_t n_segs;
};

// A segment of a merged batch wave: samples i0 .. i0 + ns - 1 (relative to the job's first
// sample of the call) of the job's window pixels pb .. pb + npix - 1; its paths are path0 + i *
// npix + j (sample-major, as in a single-scene wave) and its pixels pix0 .. pix0 + npix - 1 of
// the wave's accumulation pass.  A job is split into segments only along pixels, so each
// pixel's samples stay in sample order from wave to wave.
struct WfmSeg {
    uint32_t job, pb, npix, i0, ns, path0, pix0, pad;
};

// the segment that holds path id (the last one whose first path is <= id)
__device__ __forceinline__ uint32_t wfm_seg_of(const WfParams& P, uint32_t id) {
    uint32_t lo = 0, hi = P.n_segs;
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (P.segs[mid].path0 <= id) lo = mid;
        else hi = mid;
    }
    return lo;
}

// scene, depth, flags and random-number keys of path id of a merged batch wave, from its
// segment (whose wave-local index the path carries in the w word of its radiance)
__device__ __forceinline__ void wfm_context(const WfParams& P, uint32_t seg, uint32_t id, DScene& S, VertexRng& rng,
                                            uint32_t& max_depth, uint32_t& flags, uint32_t& job) {
    const WfmSeg g = P.segs[seg];
    const DJob& J = P.jobs[g.job];
    S = J.S;
    const uint32_t local = id - g.path0;
    const uint32_t lp = g.pb + local % g.npix;
    rng.p = (J.y0 + lp / J.cw) * J.cam.width + (J.x0 + lp % J.cw);
    rng.s = J.s0 + g.i0 + local / g.npix;
    rng.k0 = (uint32_t)J.seed;
    rng.k1 = (uint32_t)(J.seed >> 32);
    max_depth = J.max_depth;
    flags = J.flags;
    job = g.job;
}

constexpr uint32_t NRC_DIM_TRAIN = 10;   // uniform dimension of the training-path choice
constexpr uint32_t NRC_TRAIN_END = 4;     // diffuse-ish vertex at which training paths end into the cache
constexpr bool NRC_FACTOR_ALBEDO = true;   // the cache learns radiance / (albedo + 0.01)

// albedo of a vertex for the factorisation: (m + (1-m)(1-t)) bw bc + (1-m) t tc + sw 0.04 sc
__device__ __forceinline__ float3 nrc_albedo(const DMat& M) {
    return M.base_color * ((M.metalness + (1.0f - M.metalness) * (1.0f - M.trans_weight)) * M.base_weight) +
           M.trans_color * ((1.0f - M.metalness) * M.trans_weight) + M.spec_color * (0.04f * M.spec_weight);
}

// first sample index of this wave and the seed, from the per-call words of the counters
__device__ __forceinline__ uint32_t wf_sample_base(const WfParams& P) { return P.counters[C_FRAME] + P.i0; }
__device__ __forceinline__ uint64_t wf_seed(const WfParams& P) {
    return *reinterpret_cast<const unsigned long long*>(P.counters + C_FRAME + 2);
}

__global__ void k_wf_frame(uint32_t* counters, uint32_t first_sample, uint64_t seed) {
    if (threadIdx.x == 0) {
        counters[C_FRAME] = first_sample;
        *reinterpret_cast<unsigned long long*>(counters + C_FRAME + 2) = seed;
    }
}

// Queue slot t of the first bounce holds path id = t unless the wave is tiled: then within
// each sample's block of npix slots, slot j holds the pixel of the 8 x 4 tile order (tiles
// left to right along each group of 4 rows), so that a warp's 32 camera rays cover a compact
// 8 x 4 footprint instead of 32 pixels of one row.  Only the order of the queue changes: the
// path id (pixel-major, as everywhere else) rides with the ray.
__device__ __forceinline__ uint32_t tiled_path(const WfParams& P, uint32_t t) {
    const uint32_t s = t / P.npix, j = t % P.npix, w4 = 4u * P.cw;
    const uint32_t g = j / w4, w = j % w4, k = w & 31u;
    return s * P.npix + (4u * g + (k >> 3)) * P.cw + (w >> 5) * 8u + (k & 7u);
}

__global__ void k_wf_raygen(WfParams P) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = P.npix * P.nsamp;
    if (t == 0) {
        P.counters[C_Q0] = n;
        P.counters[C_TAIL] = 0;
        atomicAdd(&P.stats[ST_PATHS], (unsigned long long)n);
    }
    if (t >= n) return;
    const uint32_t id = P.tiled ? tiled_path(P, t) : t;
    const uint32_t lp = P.pb + id % P.npix;
    const uint32_t s = wf_sample_base(P) + id / P.npix;
    const uint64_t seed = wf_seed(P);
    const uint32_t px = P.x0 + lp % P.cw, py = P.y0 + lp / P.cw;
    const uint32_t p = py * P.cam.width + px;
    float3 o, d;
    camera_ray_ps(P.cam, px, py, p, s, (uint32_t)seed, (uint32_t)(seed >> 32), o, d);
    P.ray_o[0][t] = make_float4(o.x, o.y, o.z, 0.0f);
    P.ray_d[0][t] = make_float4(d.x, d.y, d.z, __uint_as_float(id));
    P.beta[id] = make_float4(1.0f, 1.0f, 1.0f, -1.0f);
    P.radiance[id] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (P.nrc_on) {
        uint32_t aux = 0;
        if (P.max_train && u24(philox4x32_10(make_uint4(p, s, 0u, NRC_DIM_TRAIN >> 2), (uint32_t)seed,
                                             (uint32_t)(seed >> 32)).z) < P.train_prob) {
            const uint32_t slot = atomicAdd(&P.nrc_counters[1], 1u);
            if (slot < P.max_train) {
                aux = (slot + 1u) << 8;
                P.train_id[slot] = id;
                P.train_nv[slot] = 0;
            }
        }
        P.aux[id] = aux;
    }
}

// Radiance-cache hook: records the vertices of training paths (features, radiance so far,
// throughput) and ends other paths at their second diffuse-ish vertex with a cache query.
struct NrcHook {
    const WfParams* P;
    uint32_t id;
    uint32_t aux;
    __device__ __forceinline__ bool operator()(float3 x, float3 wo, float3 n, const DMat& M, const PathState& ps,
                                               uint32_t k) {
        const float r = effective_roughness(M);
        const uint32_t slot1 = aux >> 8;
        // the cache learns outgoing radiance divided by the vertex's albedo (+ 0.01), so it
        // need not reproduce colour steps between materials: the records carry beta times that
        // factor, which both the cache's output (k_nrc_apply) and the targets use
        const float3 fb = NRC_FACTOR_ALBEDO ? ps.beta * (nrc_albedo(M) + splat3(0.01f)) : ps.beta;
        if (slot1 && k < P->rec_per_path) {
            float4* rec = reinterpret_cast<float4*>(P->train_rec + ((size_t)(slot1 - 1) * P->rec_per_path + k) * 16);
            rec[0] = make_float4(x.x, x.y, x.z, wo.x);
            rec[1] = make_float4(wo.y, wo.z, n.x, n.y);
            rec[2] = make_float4(n.z, r, ps.L.x, ps.L.y);
            rec[3] = make_float4(ps.L.z, fb.x, fb.y, fb.z);
            P->train_nv[slot1 - 1] = k + 1;
        }
        if (r >= 0.25f) {
            const uint32_t cnt = min((aux & 0xffu) + 1u, 255u);
            aux = (aux & ~0xffu) | cnt;
            // rendering paths end into the cache at their second diffuse-ish vertex; training
            // paths go NRC_TRAIN_END - 2 such vertices further and end into the cache there
            // too (self-training: their suffix targets then include the cache's estimate of
            // the rest of the path, and the terminal vertex itself is not a training record)
            const bool train_end = slot1 && cnt == NRC_TRAIN_END;
            if (train_end && k < P->rec_per_path) P->train_nv[slot1 - 1] = k;
            if ((cnt == 2u && !slot1) || train_end) {
                // warp-aggregated append: the lanes that reach this point take consecutive slots
                const uint32_t active = __activemask();
                const uint32_t lane = threadIdx.x & 31u;
                const int leader = __ffs(active) - 1;
                uint32_t q0 = 0;
                if ((int)lane == leader) q0 = atomicAdd(&P->nrc_counters[0], (uint32_t)__popc(active));
                q0 = __shfl_sync(active, q0, leader);
                const uint32_t q = q0 + __popc(active & ((1u << lane) - 1u));
                float4* rec = reinterpret_cast<float4*>(P->nrc_q + (size_t)q * 16);
                rec[0] = make_float4(x.x, x.y, x.z, wo.x);
                rec[1] = make_float4(wo.y, wo.z, n.x, n.y);
                rec[2] = make_float4(n.z, r, fb.x, fb.y);
                rec[3] = make_float4(fb.z, __uint_as_float(id), 0.0f, 0.0f);
                return true;
            }
        }
        return false;
    }
};

// radiance of the paths the cache ended: L += beta * max(cache, 0)
__global__ void k_nrc_apply(WfParams P) {
    const uint32_t nq = P.nrc_counters[0];
    if (blockIdx.x == 0 && threadIdx.x == 0 && nq) atomicAdd(&P.stats[ST_NRC], (unsigned long long)nq);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const float* rec = P.nrc_q + (size_t)q * 16;
        const uint32_t id = __float_as_uint(rec[13]);
        const float* y = P.nrc_out + 4ull * q;
        float4 L = P.radiance[id];
        L.x += rec[10] * fmaxf(y[0], 0.0f);
        L.y += rec[11] * fmaxf(y[1], 0.0f);
        L.z += rec[12] * fmaxf(y[2], 0.0f);
        P.radiance[id] = L;
    }
}

// training samples from the path suffixes: target_j = (L_end - L_j) / beta_j per channel
__global__ void k_nrc_targets(WfParams P) {
    const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= min(P.nrc_counters[1], P.max_train)) return;
    const uint32_t id = P.train_id[slot];
    const float4 Le = P.radiance[id];
    const uint32_t nv = min(P.train_nv[slot], P.rec_per_path);
    for (uint32_t j = 0; j < nv; ++j) {
        const float* rec = P.train_rec + ((size_t)slot * P.rec_per_path + j) * 16;
        const float L[3] = {Le.x - rec[10], Le.y - rec[11], Le.z - rec[12]};
        const float b[3] = {rec[13], rec[14], rec[15]};
        float t[3];
        bool ok = isfinite(Le.x) && isfinite(Le.y) && isfinite(Le.z);
        for (int c = 0; c < 3; ++c) t[c] = b[c] > 1e-4f ? fmaxf(L[c], 0.0f) / b[c] : 0.0f;
        if (!ok) continue;
        const uint32_t o = atomicAdd(&P.nrc_counters[2], 1u);
        if (o >= P.sample_cap) return;
        float* out = P.train_samples + (size_t)o * 16;
        for (int c = 0; c < 10; ++c) out[c] = rec[c];
        out[10] = t[0]; out[11] = t[1]; out[12] = t[2];
        out[13] = 0.0f; out[14] = 0.0f; out[15] = 0.0f;
    }
}

__global__ void k_wf_setup(uint32_t* counters, int out_q, uint32_t n_keys) {
    const uint32_t t = threadIdx.x;
    if (t == 0) {
        counters[out_q] = 0;
        counters[C_SH] = 0;
        counters[C_HEAD_TRACE] = 0;
        counters[C_HEAD_SHADOW] = 0;
    }
    for (uint32_t k = t; k < n_keys; k += blockDim.x) counters[C_BUCKETS + k] = 0;
}

__device__ __forceinline__ uint32_t hit_key(const DScene& S, const HitRec& h, uint32_t n_mats) {
    if (h.tri == PT_NO_HIT) return n_mats;
    const uint32_t code = __float_as_uint(__ldg(S.tris + 3u * h.tri + 1).w);
    return (code & PT_LIGHT_BIT) ? n_mats + 1 : code;
}

// Persistent closest-hit over the input queue.  A warp takes 32 queue slots with one atomic,
// each lane carries its ray through the per-ray step loop (one BVH node per step), and the
// warp takes the next 32 once all of its rays are done (lane refill was measured slower).
template <bool COUNT, bool MULTI = false>
__global__ void __launch_bounds__(128) k_wf_trace(WfParams P, int in_q) {
    __shared__ uint32_t hist[MAX_SORT_KEYS];
    if (P.counters[C_TAIL]) return;
    const bool sort = P.n_keys > 0;
    if (sort)
        for (uint32_t k = threadIdx.x; k < P.n_keys; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    const uint32_t count = P.counters[in_q];
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&P.stats[ST_EXT], (unsigned long long)count);
    const uint32_t lane = lane_id();
    TravCount tc = {0, 0, 0};
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&P.counters[C_HEAD_TRACE], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= count) break;
        const uint32_t slot = base + lane;
        if (slot < count) {
            const float4 ro = P.ray_o[in_q][slot], rd = P.ray_d[in_q][slot];
            HitRec h;
            uint32_t key = 0;
            if (MULTI) {
                // merged batch waves: the ray carries its job in the w word of its origin
                const DJob& J = P.jobs[__float_as_uint(ro.w)];
                const DScene S = J.S;
                trace_closest_t<COUNT>(S, xyz(ro), xyz(rd), __int_as_float(0x7f800000), h, tc);
                if (sort) key = J.key_base + hit_key(S, h, J.n_mats);
            } else {
                trace_closest_t<COUNT>(P.S, xyz(ro), xyz(rd), __int_as_float(0x7f800000), h, tc);
                if (sort) key = hit_key(P.S, h, P.n_keys - 2);
            }
            P.hit[slot] = make_float4(h.t, h.u, h.v, __uint_as_float(h.tri));
            if (sort) {
                P.keys[slot] = key;
                atomicAdd(&hist[key], 1u);
            }
        }
    }
    if (COUNT) {
        const unsigned long long nn = warp_sum_u64(tc.nodes), nt = warp_sum_u64(tc.tris),
                                 nb = warp_sum_u64(tc.boxes);
        if (lane == 0) {
            atomicAdd(&P.stats[ST_BOXES], nb);
            atomicAdd(&P.stats[ST_NODES], nn);
            atomicAdd(&P.stats[ST_TRIS], nt);
        }
    }
    if (sort) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < P.n_keys; k += blockDim.x)
            if (hist[k]) atomicAdd(&P.counters[C_BUCKETS + k], hist[k]);
    }
}

// exclusive scan of the bucket counts into bucket cursors (one block)
__global__ void k_wf_sort_scan(uint32_t* counters, uint32_t n_keys) {
    if (counters[C_TAIL]) return;
    __shared__ uint32_t part[MAX_SORT_KEYS];
    const uint32_t t = threadIdx.x;
    const uint32_t v = t < n_keys ? counters[C_BUCKETS + t] : 0u;
    part[t] = v;
    __syncthreads();
    for (uint32_t off = 1; off < blockDim.x; off <<= 1) {
        const uint32_t a = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += a;
        __syncthreads();
    }
    if (t < n_keys) counters[C_BUCKETS + t] = part[t] - v;
}

// Counting-sort scatter: each block ranks a chunk of SORT_ITEMS x SORT_THREADS slots in shared
// memory (warp-aggregated shared atomics per key), reserves each key's run of the chunk with
// one global atomic, then writes the permutation.  (One global atomic per key and warp made
// the few material buckets a point of contention: 8.3M slots gave 0.8M atomics on 5 words.)
constexpr uint32_t SORT_THREADS = 256, SORT_ITEMS = 16;

__global__ void __launch_bounds__(SORT_THREADS) k_wf_sort_scatter(WfParams P, int in_q) {
    __shared__ uint32_t s_cnt[MAX_SORT_KEYS];
    if (P.counters[C_TAIL]) return;
    const uint32_t count = P.counters[in_q];
    const uint32_t n_keys = P.n_keys;
    const uint32_t lane = lane_id(), tid = threadIdx.x;
    const uint32_t lt = (1u << lane) - 1u;
    constexpr uint32_t CHUNK = SORT_THREADS * SORT_ITEMS;
    for (uint32_t c0 = blockIdx.x * CHUNK; c0 < count; c0 += gridDim.x * CHUNK) {
        for (uint32_t k = tid; k < n_keys; k += SORT_THREADS) s_cnt[k] = 0u;
        __syncthreads();
        uint32_t key[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
        for (uint32_t i = 0; i < SORT_ITEMS; ++i) {
            const uint32_t slot = c0 + i * SORT_THREADS + tid;
            key[i] = slot < count ? min(P.keys[slot], n_keys - 1u) : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, key[i]);
            const uint32_t leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (key[i] != 0xffffffffu && lane == leader) b = atomicAdd(&s_cnt[key[i]], __popc(peers));
            rank[i] = __shfl_sync(0xffffffffu, b, leader) + __popc(peers & lt);
        }
        __syncthreads();
        // the chunk's run of each key: counts -> global positions (in place)
        for (uint32_t k = tid; k < n_keys; k += SORT_THREADS) {
            const uint32_t c = s_cnt[k];
            s_cnt[k] = c ? atomicAdd(&P.counters[C_BUCKETS + k], c) : 0u;
        }
        __syncthreads();
#pragma unroll
        for (uint32_t i = 0; i < SORT_ITEMS; ++i)
            if (key[i] != 0xffffffffu) P.perm[s_cnt[key[i]] + rank[i]] = c0 + i * SORT_THREADS + tid;
        __syncthreads();
    }
}

// ReSTIR DI, pass 1 (bounce 0, after the closest hits, queue 0 whose slot is the path id):
// the primary surface of every path and its initial reservoir.  M candidates from the
// next-event light sampler (source pdf in area measure on a quad, solid angle for the
// environment) are resampled with the cheap target p0 = lum(L_e) G |cos| (restir_target0);
// the reservoir keeps candidate i with probability w_i / sum w (u * sum w < w_i, streaming)
// and W = sum w / (M p0).  Paths with no surface to light get triangle PT_NO_HIT.
__global__ void __launch_bounds__(128, 6) k_restir_init(WfParams P) {
    if (P.counters[C_TAIL]) return;
    const uint32_t count = P.counters[C_Q0];
    const uint32_t sbase = wf_sample_base(P);
    const uint64_t seed = wf_seed(P);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const DScene& S = P.S;
    const bool has_env = S.env_w > 0 && S.env_total > 0.0f;
    for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < count; slot += gridDim.x * blockDim.x) {
        const float4 ro = P.ray_o[0][slot], rd = P.ray_d[0][slot];
        const float4 hh = P.hit[slot];
        const uint32_t id = __float_as_uint(rd.w);
        const uint32_t tri = __float_as_uint(hh.w);
        float4 g1 = make_float4(0.0f, 0.0f, 0.0f, __uint_as_float(PT_NO_HIT));
        float4 r0 = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(LIGHT_NONE));
        float4 r1 = make_float4(0.0f, (float)P.restir_M, 0.0f, 0.0f);
        bool valid = tri != PT_NO_HIT && P.max_depth > 0 && (has_env || S.n_quads > 0);
        if (valid) valid = !(__float_as_uint(__ldg(S.tris + 3u * tri + 1).w) & PT_LIGHT_BIT);
        RSurf g;
        if (valid) {
            const float3 x = xyz(ro) + xyz(rd) * hh.x;
            rsurf_make(S, x, -xyz(rd), tri, g);
            valid = g.C.has_smooth;
        }
        if (valid) {
            const float3 wo_w = -xyz(rd);
            const bool transmits = (1.0f - g.C.m) * g.C.t > 0.0f;
            P.rs_g0[id] = make_float4(g.x.x, g.x.y, g.x.z, hh.x);
            P.rs_gn[id] = make_float4(g.n.x, g.n.y, g.n.z, transmits ? 1.0f : 0.0f);
            g1 = make_float4(wo_w.x, wo_w.y, wo_w.z, __uint_as_float(tri));
            const uint32_t lp = P.pb + id % P.npix;
            const uint32_t p = (P.y0 + lp / P.cw) * P.cam.width + (P.x0 + lp % P.cw);
            const uint32_t s = sbase + id / P.npix;
            int sel;
            float3 y_sel;
            float W, ph_sel;
            restir_ris(S, g.x, g.n, transmits, p, s, RESTIR_CANDIDATES, P.restir_M, k0, k1, sel, y_sel, W, ph_sel);
            r0 = make_float4(y_sel.x, y_sel.y, y_sel.z, __int_as_float(sel));
            r1 = make_float4(W, (float)P.restir_M, ph_sel, 0.0f);
        }
        P.rs_g1[id] = g1;
        P.rs_i[2u * id] = r0;
        P.rs_i[2u * id + 1] = r1;
    }
}

// ReSTIR DI, pass 2: one spatial pass.  Up to K neighbours of the same sample (offsets
// uniform in [-R, R]^2 from the raw Philox words by multiply-shift, so every build picks the
// same pixels), skipped outside the window, on the pixel itself, without a surface, with
// normal cosine < 0.9 or depth differing by more than 10 %.  This pixel's and their initial
// reservoirs are resampled with the full target here (restir_target),
// w = target_here(y_j) W_j M_j; the result gets the unbiased weight
// W = sum w / (Z target_here(y)), Z = the sum of M over the combined reservoirs whose own
// initial target p0 is positive at y (those that could have drawn y).  The wave holds whole
// windows.
__global__ void __launch_bounds__(128, 6) k_restir_spatial(WfParams P, uint32_t n) {
    if (P.counters[C_TAIL]) return;
    const uint32_t sbase = wf_sample_base(P);
    const uint64_t seed = wf_seed(P);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t ch = P.npix / P.cw;
    const uint32_t side = 2u * P.restir_R + 1u;
    for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < n; id += gridDim.x * blockDim.x) {
        const float4 g1 = P.rs_g1[id];
        const uint32_t tri = __float_as_uint(g1.w);
        float4 f0 = P.rs_i[2u * id], f1 = P.rs_i[2u * id + 1];
        if (tri != PT_NO_HIT) {
            const float4 g0 = P.rs_g0[id];
            RSurf g;
            rsurf_make(P.S, xyz(g0), xyz(g1), tri, g);
            const uint32_t lp = id % P.npix, base = id - lp;
            const uint32_t rx = lp % P.cw, ry = lp / P.cw;
            const uint32_t p = (P.y0 + ry) * P.cam.width + (P.x0 + rx);
            const uint32_t s = sbase + id / P.npix;
            float3 c0, ld0;
            float wsum = restir_target(P.S, g.x, g.tt, g.bb, g.n, g.C, g.wo, __float_as_int(f0.w), xyz(f0), c0, ld0) *
                         f1.x * f1.y;
            const float Mq = f1.y;
            const bool transmits = P.rs_gn[id].w != 0.0f;
            int light = __float_as_int(f0.w);
            float3 y = xyz(f0);
            uint32_t used[64];
            uint32_t n_used = 0;
            for (uint32_t j = 0; j < P.restir_K; ++j) {
                const uint4 r = philox4x32_10(make_uint4(p, s, RESTIR_SPATIAL, j), k0, k1);
                const int dx = (int)(((uint64_t)r.x * side) >> 32) - (int)P.restir_R;
                const int dy = (int)(((uint64_t)r.y * side) >> 32) - (int)P.restir_R;
                const float u_sel = u24(r.z);
                const int nx = (int)rx + dx, ny = (int)ry + dy;
                if ((dx == 0 && dy == 0) || nx < 0 || ny < 0 || nx >= (int)P.cw || ny >= (int)ch) continue;
                const uint32_t nid = base + (uint32_t)ny * P.cw + (uint32_t)nx;
                if (__float_as_uint(P.rs_g1[nid].w) == PT_NO_HIT) continue;
                const float4 ng0 = P.rs_g0[nid], nn = P.rs_gn[nid];
                if (dot3(xyz(nn), g.n) < 0.9f || fabsf(ng0.w - g0.w) > 0.1f * g0.w) continue;
                used[n_used++] = nid;
                const float4 a0 = P.rs_i[2u * nid], a1 = P.rs_i[2u * nid + 1];
                float3 c, ld;
                const float ph = restir_target(P.S, g.x, g.tt, g.bb, g.n, g.C, g.wo, __float_as_int(a0.w), xyz(a0), c, ld);
                const float w = ph * a1.x * a1.y;
                if (!(w > 0.0f)) continue;
                wsum += w;
                if (u_sel * wsum < w) {
                    light = __float_as_int(a0.w);
                    y = xyz(a0);
                }
            }
            float3 c, ld;
            const float ph = restir_target(P.S, g.x, g.tt, g.bb, g.n, g.C, g.wo, light, y, c, ld);
            float Z = restir_target0(P.S, g.x, g.n, transmits, light, y) > 0.0f ? Mq : 0.0f;
            for (uint32_t u = 0; u < n_used; ++u) {
                const uint32_t nid = used[u];
                const float4 nn = P.rs_gn[nid];
                if (restir_target0(P.S, xyz(P.rs_g0[nid]), xyz(nn), nn.w != 0.0f, light, y) > 0.0f)
                    Z += P.rs_i[2u * nid + 1].y;
            }
            f0 = make_float4(y.x, y.y, y.z, __int_as_float(light));
            f1 = make_float4((ph > 0.0f && Z > 0.0f) ? wsum / (Z * ph) : 0.0f, Z, ph, 0.0f);
        }
        P.rs_f[2u * id] = f0;
        P.rs_f[2u * id + 1] = f1;
    }
}

template <bool NRC, bool RIS, bool FUZZ = true, bool MULTI = false>
__global__ void __launch_bounds__(128, 5) k_wf_shade(WfParams P, int in_q, int out_q, uint32_t k) {
    if (P.counters[C_TAIL]) return;
    const uint32_t count = P.counters[in_q];
    const uint32_t sbase = wf_sample_base(P);
    const uint64_t seed = wf_seed(P);
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    unsigned long long rr_cnt = 0;
    for (uint32_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; base < count; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        const bool valid = i < count;
        bool cont = false, shadow = false;
        float3 no = splat3(0.0f), nd = splat3(0.0f);
        ShadowRay sh;
        uint32_t id = 0;
        float tag = 0.0f;   // merged batch waves: the job, carried by the appended rays
        float4 b4 = make_float4(0, 0, 0, 0);
        if (valid) {
            const uint32_t slot = P.n_keys ? P.perm[i] : i;
            const float4 ro = P.ray_o[in_q][slot], rd = P.ray_d[in_q][slot];
            const float4 hh = P.hit[slot];
            id = __float_as_uint(rd.w);
            HitRec h;
            h.t = hh.x; h.u = hh.y; h.v = hh.z; h.tri = __float_as_uint(hh.w);
            b4 = P.beta[id];
            const float4 L4 = P.radiance[id];
            PathState ps;
            ps.beta = xyz(b4);
            ps.prev_pdf = b4.w;
            ps.L = xyz(L4);
            VertexRng rng;
            DScene Sm;
            uint32_t md = 0, fl = 0, job = 0;
            if constexpr (MULTI) {
                wfm_context(P, __float_as_uint(L4.w), id, Sm, rng, md, fl, job);
            } else {
                const uint32_t lp = P.pb + id % P.npix;
                rng.p = (P.y0 + lp / P.cw) * P.cam.width + (P.x0 + lp % P.cw);
                rng.s = sbase + id / P.npix;
                rng.k0 = (uint32_t)seed;
                rng.k1 = (uint32_t)(seed >> 32);
            }
            rng.k = k;
            ShadeOut so;
            int r;
            if constexpr (MULTI) {
                r = shade_vertex<false, FUZZ>(Sm, h, xyz(ro), xyz(rd), k, md, fl, rng, ps, so, nullptr, 0u);
            } else if (NRC) {
                NrcHook hook;
                hook.P = &P;
                hook.id = id;
                hook.aux = P.aux[id];
                r = shade_vertex_h(P.S, h, xyz(ro), xyz(rd), k, P.max_depth, P.flags, rng, ps, so, hook);
                P.aux[id] = hook.aux;
            } else {
                const float4* rres = (P.restir_on && k == 0) ? P.rs_f + 2u * id : nullptr;
                r = shade_vertex<RIS, FUZZ>(P.S, h, xyz(ro), xyz(rd), k, P.max_depth, P.flags, rng, ps, so, rres,
                                            P.restir_on ? P.restir_L : 0u);
            }
            P.radiance[id] = make_float4(ps.L.x, ps.L.y, ps.L.z, MULTI ? L4.w : 0.0f);
            if (so.rr_end) rr_cnt++;
            tag = MULTI ? __uint_as_float(job) : 0.0f;
            cont = r == SHADE_CONTINUE;
            shadow = so.has_shadow;
            if (cont) {
                no = so.next_o;
                nd = so.next_d;
                P.beta[id] = make_float4(ps.beta.x, ps.beta.y, ps.beta.z, ps.prev_pdf);
            }
            sh = so.sh;
        }
        // warp-aggregated appends to the next-ray queue and the shadow queue
        const uint32_t mc = __ballot_sync(0xffffffffu, cont);
        const uint32_t ms = __ballot_sync(0xffffffffu, shadow);
        uint32_t bc = 0, bs = 0;
        if (lane == 0) {
            if (mc) bc = atomicAdd(&P.counters[out_q], __popc(mc));
            if (ms) bs = atomicAdd(&P.counters[C_SH], __popc(ms));
        }
        bc = __shfl_sync(0xffffffffu, bc, 0);
        bs = __shfl_sync(0xffffffffu, bs, 0);
        if (cont) {
            const uint32_t pos = bc + __popc(mc & lt);
            P.ray_o[out_q][pos] = make_float4(no.x, no.y, no.z, tag);
            P.ray_d[out_q][pos] = make_float4(nd.x, nd.y, nd.z, __uint_as_float(id));
        }
        if (shadow) {
            const uint32_t pos = bs + __popc(ms & lt);
            P.sh_o[pos] = make_float4(sh.o.x, sh.o.y, sh.o.z, sh.tmax);
            P.sh_d[pos] = make_float4(sh.d.x, sh.d.y, sh.d.z, __uint_as_float(id));
            P.sh_c[pos] = make_float4(sh.contrib.x, sh.contrib.y, sh.contrib.z, tag);
        }
    }
    rr_cnt = warp_sum_u64(rr_cnt);
    if (lane == 0 && rr_cnt) atomicAdd(&P.stats[ST_RR], rr_cnt);
}

// Persistent shadow any-hit over the shadow queue, with the same lane refilling; an
// unoccluded shadow ray adds its contribution to its path's radiance.
template <bool COUNT, bool MULTI = false>
__global__ void __launch_bounds__(128) k_wf_shadow(WfParams P) {
    const uint32_t count = P.counters[C_SH];
    if (blockIdx.x == 0 && threadIdx.x == 0 && count) atomicAdd(&P.stats[ST_SHADOW], (unsigned long long)count);
    const uint32_t lane = lane_id();
    TravCount tc = {0, 0, 0};
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&P.counters[C_HEAD_SHADOW], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= count) break;
        const uint32_t slot = base + lane;
        if (slot < count) {
            const float4 so = P.sh_o[slot], sd = P.sh_d[slot];
            bool occ;
            if (MULTI) {
                // merged batch waves: the job rides in the w word of the contribution
                const DScene S = P.jobs[__float_as_uint(P.sh_c[slot].w)].S;
                occ = trace_any_t<COUNT>(S, xyz(so), xyz(sd), so.w, tc);
            } else {
                occ = trace_any_t<COUNT>(P.S, xyz(so), xyz(sd), so.w, tc);
            }
            if (!occ) {
                const uint32_t id = __float_as_uint(sd.w);
                const float4 c = P.sh_c[slot];
                float4 L = P.radiance[id];
                L.x += c.x; L.y += c.y; L.z += c.z;
                P.radiance[id] = L;
            }
        }
    }
    if (COUNT) {
        const unsigned long long nn = warp_sum_u64(tc.nodes), nt = warp_sum_u64(tc.tris),
                                 nb = warp_sum_u64(tc.boxes);
        if (lane == 0) {
            atomicAdd(&P.stats[ST_SH_BOXES], nb);
            atomicAdd(&P.stats[ST_SH_NODES], nn);
            atomicAdd(&P.stats[ST_SH_TRIS], nt);
        }
    }
}

// Cooperative variants of the two traversal passes (PT_TRAVERSAL_COOP): a group of COOP_W = 8
// lanes carries one ray (pt_device.cuh, coop_*), so a warp holds 4 rays and its lanes test a
// node's 8 child boxes, or a node's leaf triangles, side by side.  A warp claims 32 queue
// slots with one atomic and hands them out one by one as its groups finish their rays; the
// warp leaves once the queue is drained and its groups are done.  Hits, node and triangle
// counts equal the per-lane kernels' above.  Measured on the 1080p CAD frame: 20 of 32 lanes
// active per instruction (per-lane: 9), but every lane of a group decodes and sets up the
// node and takes part in the scans, so a ray costs 5x the thread instructions and the pass
// takes 2.7x as long; the per-lane kernels stay the default.
__device__ __forceinline__ void coop_hand_out(uint32_t* head, uint32_t count, uint32_t lane, uint32_t gbase,
                                              bool active, uint32_t& wb, uint32_t& we, bool& drained,
                                              uint32_t& taken) {
    // taken: the slot handed to this lane's group (~0u: none)
    taken = 0xffffffffu;
    uint32_t idle = __ballot_sync(0xffffffffu, !active) & 0x01010101u;
    while (idle != 0u && !drained) {
        if (wb >= we) {
            uint32_t b = 0;
            if (lane == 0) b = atomicAdd(head, 32u);
            b = __shfl_sync(0xffffffffu, b, 0);
            if (b >= count) { drained = true; break; }
            wb = b;
            we = min(b + 32u, count);
        }
        if (gbase == (uint32_t)(__ffs(idle) - 1)) taken = wb;
        ++wb;
        idle &= idle - 1u;
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(128) k_wf_trace_coop(WfParams P, int in_q) {
    __shared__ uint32_t hist[MAX_SORT_KEYS];
    __shared__ CoopShared gsh[128 / COOP_W];
    if (P.counters[C_TAIL]) return;
    const bool sort = P.n_keys > 0;
    if (sort)
        for (uint32_t k = threadIdx.x; k < P.n_keys; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    const uint32_t count = P.counters[in_q];
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&P.stats[ST_EXT], (unsigned long long)count);
    const uint32_t lane = lane_id(), gl = lane & (COOP_W - 1u), gbase = lane & ~(COOP_W - 1u);
    const uint32_t gm = 0xffu << gbase;
    CoopShared& sh = gsh[threadIdx.x / COOP_W];
    TravCount tc = {0, 0, 0};
    CoopClosest st;
    uint32_t slot = 0, wb = 0, we = 0;
    bool active = false, drained = false;
    for (;;) {
        uint32_t taken;
        coop_hand_out(&P.counters[C_HEAD_TRACE], count, lane, gbase, active, wb, we, drained, taken);
        if (taken != 0xffffffffu) {
            slot = taken;
            active = true;
            const float4 ro = P.ray_o[in_q][slot], rd = P.ray_d[in_q][slot];
            coop_closest_init(P.S, xyz(ro), xyz(rd), __int_as_float(0x7f800000), st);
        }
        if (__ballot_sync(0xffffffffu, active) == 0u) break;
        if (active && coop_closest_step<COUNT>(P.S, st, sh, gl, gm, gbase, tc)) {
            HitRec h;
            if (coop_closest_finish(st, gl, gm, gbase, h)) {
                P.hit[slot] = make_float4(h.t, h.u, h.v, __uint_as_float(h.tri));
                if (sort) {
                    const uint32_t key = hit_key(P.S, h, P.n_keys - 2);
                    P.keys[slot] = key;
                    atomicAdd(&hist[key], 1u);
                }
            }
            active = false;
        }
    }
    if (COUNT) {
        const unsigned long long nn = warp_sum_u64(tc.nodes), nt = warp_sum_u64(tc.tris),
                                 nb = warp_sum_u64(tc.boxes);
        if (lane == 0) {
            atomicAdd(&P.stats[ST_BOXES], nb);
            atomicAdd(&P.stats[ST_NODES], nn);
            atomicAdd(&P.stats[ST_TRIS], nt);
        }
    }
    if (sort) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < P.n_keys; k += blockDim.x)
            if (hist[k]) atomicAdd(&P.counters[C_BUCKETS + k], hist[k]);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(128) k_wf_shadow_coop(WfParams P) {
    __shared__ CoopShared gsh[128 / COOP_W];
    const uint32_t count = P.counters[C_SH];
    if (blockIdx.x == 0 && threadIdx.x == 0 && count) atomicAdd(&P.stats[ST_SHADOW], (unsigned long long)count);
    const uint32_t lane = lane_id(), gl = lane & (COOP_W - 1u), gbase = lane & ~(COOP_W - 1u);
    const uint32_t gm = 0xffu << gbase;
    CoopShared& sh = gsh[threadIdx.x / COOP_W];
    TravCount tc = {0, 0, 0};
    CoopAny st;
    uint32_t slot = 0, wb = 0, we = 0;
    bool active = false, drained = false;
    for (;;) {
        uint32_t taken;
        coop_hand_out(&P.counters[C_HEAD_SHADOW], count, lane, gbase, active, wb, we, drained, taken);
        if (taken != 0xffffffffu) {
            slot = taken;
            active = true;
            const float4 so = P.sh_o[slot], sd = P.sh_d[slot];
            coop_any_init(P.S, xyz(so), xyz(sd), so.w, st);
        }
        if (__ballot_sync(0xffffffffu, active) == 0u) break;
        if (active && coop_any_step<COUNT>(P.S, st, sh, gl, gm, gbase, tc)) {
            if (!st.hit && gl == 0) {
                const uint32_t id = __float_as_uint(P.sh_d[slot].w);
                const float4 c = P.sh_c[slot];
                float4 L = P.radiance[id];
                L.x += c.x; L.y += c.y; L.z += c.z;
                P.radiance[id] = L;
            }
            active = false;
        }
    }
    if (COUNT) {
        const unsigned long long nn = warp_sum_u64(tc.nodes), nt = warp_sum_u64(tc.tris),
                                 nb = warp_sum_u64(tc.boxes);
        if (lane == 0) {
            atomicAdd(&P.stats[ST_SH_BOXES], nb);
            atomicAdd(&P.stats[ST_SH_NODES], nn);
            atomicAdd(&P.stats[ST_SH_TRIS], nt);
        }
    }
}

// Tail of a wave: when few paths are left, a per-bounce kernel lasts about as long as its
// slowest ray (a chain of dependent node and triangle loads), and the wave pays that once per
// stage and bounce.  This kernel takes the remaining queue instead and carries each path to
// its end in one thread: closest hit, shade_vertex_h (the same per-vertex code and random
// numbers as k_wf_shade), then the shadow ray, whose contribution is added after the vertex's
// own terms exactly as k_wf_shadow adds it.  It appends nothing, so the later per-bounce
// launches of the wave find empty queues (and C_TAIL makes the rest of this bounce skip).
template <bool NRC, bool COUNT, bool RIS, bool FUZZ = true, bool MULTI = false>
__global__ void __launch_bounds__(128, 4) k_wf_tail(WfParams P, int in_q, uint32_t k0, uint32_t limit) {
    const uint32_t count = P.counters[in_q];
    if (count == 0 || count > limit) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) P.counters[C_TAIL] = 1u;
    const uint32_t sbase = wf_sample_base(P);
    const uint64_t seed = wf_seed(P);
    unsigned long long n_ext = 0, n_sh = 0, n_rr = 0;
    TravCount tc = {0, 0, 0}, sc = {0, 0, 0};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float4 ro = P.ray_o[in_q][i], rd = P.ray_d[in_q][i];
        const uint32_t id = __float_as_uint(rd.w);
        const float4 b4 = P.beta[id];
        const float4 L4 = P.radiance[id];
        PathState ps;
        ps.beta = xyz(b4);
        ps.prev_pdf = b4.w;
        ps.L = xyz(L4);
        VertexRng rng;
        DScene Sm;
        uint32_t md = 0, fl = 0, job = 0;
        if constexpr (MULTI) {
            wfm_context(P, __float_as_uint(L4.w), id, Sm, rng, md, fl, job);
        } else {
            const uint32_t lp = P.pb + id % P.npix;
            rng.p = (P.y0 + lp / P.cw) * P.cam.width + (P.x0 + lp % P.cw);
            rng.s = sbase + id / P.npix;
            rng.k0 = (uint32_t)seed;
            rng.k1 = (uint32_t)(seed >> 32);
        }
        const DScene& S = MULTI ? Sm : P.S;
        const uint32_t max_depth = MULTI ? md : P.max_depth, flags = MULTI ? fl : P.flags;
        NrcHook hook;
        if (NRC) {
            hook.P = &P;
            hook.id = id;
            hook.aux = P.aux[id];
        }
        float3 o = xyz(ro), d = xyz(rd);
        for (uint32_t k = k0;; ++k) {
            HitRec h;
            if (COUNT) trace_closest_t<true, true>(S, o, d, __int_as_float(0x7f800000), h, tc);
            else trace_closest(S, o, d, __int_as_float(0x7f800000), h);
            n_ext++;
            rng.k = k;
            ShadeOut so;
            int r;
            if (NRC) r = shade_vertex_h(S, h, o, d, k, max_depth, flags, rng, ps, so, hook);
            else r = shade_vertex<RIS, FUZZ>(S, h, o, d, k, max_depth, flags, rng, ps, so, nullptr,
                                             P.restir_on ? P.restir_L : 0u);
            if (so.rr_end) n_rr++;
            if (so.has_shadow) {
                n_sh++;
                const bool occ = COUNT ? trace_any_t<true>(S, so.sh.o, so.sh.d, so.sh.tmax, sc)
                                       : trace_any(S, so.sh.o, so.sh.d, so.sh.tmax);
                if (!occ) {
                    ps.L.x += so.sh.contrib.x;
                    ps.L.y += so.sh.contrib.y;
                    ps.L.z += so.sh.contrib.z;
                }
            }
            if (r != SHADE_CONTINUE) break;
            o = so.next_o;
            d = so.next_d;
        }
        P.radiance[id] = make_float4(ps.L.x, ps.L.y, ps.L.z, MULTI ? L4.w : 0.0f);
        if (NRC) P.aux[id] = hook.aux;
        (void)job;
    }
    n_ext = warp_sum_u64(n_ext);
    n_sh = warp_sum_u64(n_sh);
    n_rr = warp_sum_u64(n_rr);
    if (lane_id() == 0) {
        if (n_ext) { atomicAdd(&P.stats[ST_EXT], n_ext); atomicAdd(&P.stats[ST_TAIL_EXT], n_ext); }
        if (n_sh) { atomicAdd(&P.stats[ST_SHADOW], n_sh); atomicAdd(&P.stats[ST_TAIL_SH], n_sh); }
        if (n_rr) atomicAdd(&P.stats[ST_RR], n_rr);
    }
    if (COUNT) {
        const unsigned long long a = warp_sum_u64(tc.nodes), b = warp_sum_u64(tc.tris),
                                 c = warp_sum_u64(sc.nodes), e = warp_sum_u64(sc.tris),
                                 f = warp_sum_u64(tc.boxes), g = warp_sum_u64(sc.boxes);
        if (lane_id() == 0) {
            atomicAdd(&P.stats[ST_TAIL_BOXES], f);
            atomicAdd(&P.stats[ST_TAIL_SH_BOXES], g);
            atomicAdd(&P.stats[ST_TAIL_NODES], a);
            atomicAdd(&P.stats[ST_TAIL_TRIS], b);
            atomicAdd(&P.stats[ST_TAIL_SH_NODES], c);
            atomicAdd(&P.stats[ST_TAIL_SH_TRIS], e);
        }
    }
}

// ---- merged batch waves: raygen and accumulation over a wave's segments
__global__ void k_wfm_raygen(WfParams P, uint32_t n_paths) {
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id == 0) {
        P.counters[C_Q0] = n_paths;
        P.counters[C_TAIL] = 0;
    }
    if (id >= n_paths) return;
    const uint32_t si = wfm_seg_of(P, id);
    const WfmSeg g = P.segs[si];
    const DJob& J = P.jobs[g.job];
    const uint32_t local = id - g.path0;
    const uint32_t lp = g.pb + local % g.npix;
    const uint32_t s = J.s0 + g.i0 + local / g.npix;
    const uint32_t px = J.x0 + lp % J.cw, py = J.y0 + lp / J.cw;
    const uint32_t p = py * J.cam.width + px;
    float3 o, d;
    camera_ray_ps(J.cam, px, py, p, s, (uint32_t)J.seed, (uint32_t)(J.seed >> 32), o, d);
    P.ray_o[0][id] = make_float4(o.x, o.y, o.z, __uint_as_float(g.job));
    P.ray_d[0][id] = make_float4(d.x, d.y, d.z, __uint_as_float(id));
    P.beta[id] = make_float4(1.0f, 1.0f, 1.0f, -1.0f);
    P.radiance[id] = make_float4(0.0f, 0.0f, 0.0f, __uint_as_float(si));
    if (id == 0) atomicAdd(&P.stats[ST_PATHS], (unsigned long long)n_paths);
}

// each segment pixel of the wave adds its samples in sample order (Kahan), as k_wf_accum does
__global__ void k_wfm_accum(WfParams P, uint32_t n_pix) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pix) return;
    uint32_t lo = 0, hi = P.n_segs;
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (P.segs[mid].pix0 <= t) lo = mid;
        else hi = mid;
    }
    const WfmSeg g = P.segs[lo];
    const DJob& J = P.jobs[g.job];
    const uint32_t j = t - g.pix0;
    const uint32_t lp = g.pb + j;
    float* sp = J.sum + 3ull * lp;
    float* cp = J.comp + 3ull * lp;
    float s0 = sp[0], s1 = sp[1], s2 = sp[2], c0 = cp[0], c1 = cp[1], c2 = cp[2];
    unsigned long long nan_cnt = 0;
    for (uint32_t q = 0; q < g.ns; ++q) {
        float4 L = P.radiance[g.path0 + q * g.npix + j];
        if (!isfinite(L.x) || !isfinite(L.y) || !isfinite(L.z)) {
            nan_cnt++;
            L = make_float4(0, 0, 0, 0);
        }
        kahan_add(s0, c0, L.x);
        kahan_add(s1, c1, L.y);
        kahan_add(s2, c2, L.z);
    }
    sp[0] = s0; sp[1] = s1; sp[2] = s2;
    cp[0] = c0; cp[1] = c1; cp[2] = c2;
    if (nan_cnt) atomicAdd(&P.stats[ST_NAN], nan_cnt);
}

// Launches with the fuzz layer compiled in only for scenes that have a material with fuzz
// (the kernels without it are the same code as before the layer existed, with fewer spills).
template <bool NRC, bool COUNT, bool RIS>
static void launch_tail(bool fuzz, uint32_t grid, cudaStream_t st, const WfParams& P, int in_q, uint32_t k,
                        uint32_t limit) {
    if (fuzz) PT_LAUNCH((k_wf_tail<NRC, COUNT, RIS, true>), grid, 128, 0, st, P, in_q, k, limit);
    else PT_LAUNCH((k_wf_tail<NRC, COUNT, RIS, false>), grid, 128, 0, st, P, in_q, k, limit);
}
template <bool NRC, bool RIS>
static void launch_shade(bool fuzz, uint32_t grid, cudaStream_t st, const WfParams& P, int in_q, int out_q,
                         uint32_t k) {
    if (fuzz) PT_LAUNCH((k_wf_shade<NRC, RIS, true>), grid, 128, 0, st, P, in_q, out_q, k);
    else PT_LAUNCH((k_wf_shade<NRC, RIS, false>), grid, 128, 0, st, P, in_q, out_q, k);
}

__global__ void k_wf_accum(WfParams P) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nan_cnt = 0;
    if (j < P.npix) {
        const uint32_t lp = P.pb + j;
        float* sp = P.sum + 3ull * lp;
        float* cp = P.comp + 3ull * lp;
        float s0 = sp[0], s1 = sp[1], s2 = sp[2], c0 = cp[0], c1 = cp[1], c2 = cp[2];
        for (uint32_t q = 0; q < P.nsamp; ++q) {
            float4 L = P.radiance[j + q * P.npix];
            if (!isfinite(L.x) || !isfinite(L.y) || !isfinite(L.z)) {
                nan_cnt++;
                L = make_float4(0, 0, 0, 0);
            }
            if (P.sample_out) {
                float* o3 = P.sample_out + 3ull * ((uint64_t)lp * P.spp_call + (P.i0 + q));
                o3[0] = L.x; o3[1] = L.y; o3[2] = L.z;
            }
            kahan_add(s0, c0, L.x);
            kahan_add(s1, c1, L.y);
            kahan_add(s2, c2, L.z);
        }
        sp[0] = s0; sp[1] = s1; sp[2] = s2;
        cp[0] = c0; cp[1] = c1; cp[2] = c2;
    }
    nan_cnt = warp_sum_u64(nan_cnt);
    if (lane_id() == 0 && nan_cnt) atomicAdd(&P.stats[ST_NAN], nan_cnt);
}

pt_status pt_free_wave(WaveBuffers& w) {
    void* ps[] = {w.ray_o[0], w.ray_o[1], w.ray_d[0], w.ray_d[1], w.hit, w.beta, w.radiance,
                  w.sh_o, w.sh_d, w.sh_c, w.perm, w.keys, w.counters, w.aux, w.nrc_q, w.nrc_out,
                  w.nrc_counters, w.train_rec, w.train_nv, w.train_id, w.train_samples,
                  w.rs_g0, w.rs_g1, w.rs_gn, w.rs_i, w.rs_f};
    for (void* p : ps)
        if (p) cudaFree(p);
    w = WaveBuffers();
    return PT_OK;
}

static pt_status ensure_wave(WaveBuffers& w, uint32_t capacity) {
    if (w.capacity >= capacity) return PT_OK;
    pt_free_wave(w);
    const size_t c = capacity;
    float4** f4[] = {&w.ray_o[0], &w.ray_o[1], &w.ray_d[0], &w.ray_d[1], &w.hit, &w.beta, &w.radiance,
                     &w.sh_o, &w.sh_d, &w.sh_c};
    for (float4** p : f4) {
        cudaError_t e = cudaMalloc((void**)p, c * sizeof(float4));
        if (e != cudaSuccess) {
            pt_free_wave(w);
            pt_set_error(std::string("wavefront buffers: ") + cudaGetErrorString(e));
            return PT_ERR_OOM;
        }
    }
    if (cudaMalloc(&w.perm, c * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&w.keys, c * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&w.counters, (C_BUCKETS + MAX_SORT_KEYS) * sizeof(uint32_t)) != cudaSuccess) {
        pt_free_wave(w);
        pt_set_error("wavefront buffers: out of memory");
        return PT_ERR_OOM;
    }
    w.capacity = capacity;
    w.bytes = c * (10 * sizeof(float4) + 2 * sizeof(uint32_t));
    return PT_OK;
}

// radiance-cache buffers: queries (one per path at most), training records and samples
// (`samples` per frame, collected from samples / 2 training paths)
static pt_status ensure_nrc_buffers(WaveBuffers& w, uint32_t rec_per_path, uint32_t samples) {
    const uint32_t cap = w.capacity, slots = std::max(samples / 2, 1u);
    if (w.nrc_capacity >= cap && w.rec_per_path >= rec_per_path && w.sample_cap == samples) return PT_OK;
    void* ps[] = {w.aux, w.nrc_q, w.nrc_out, w.nrc_counters, w.train_rec, w.train_nv, w.train_id, w.train_samples};
    for (void* q : ps)
        if (q) cudaFree(q);
    PT_CUDA_TRY(cudaMalloc(&w.aux, (size_t)cap * sizeof(uint32_t)));
    PT_CUDA_TRY(cudaMalloc(&w.nrc_q, (size_t)cap * 16 * sizeof(float)));
    PT_CUDA_TRY(cudaMalloc(&w.nrc_out, (size_t)cap * 4 * sizeof(float)));
    PT_CUDA_TRY(cudaMalloc(&w.nrc_counters, 8 * sizeof(uint32_t)));
    PT_CUDA_TRY(cudaMalloc(&w.train_rec, (size_t)slots * rec_per_path * 16 * sizeof(float)));
    PT_CUDA_TRY(cudaMalloc(&w.train_nv, slots * sizeof(uint32_t)));
    PT_CUDA_TRY(cudaMalloc(&w.train_id, slots * sizeof(uint32_t)));
    PT_CUDA_TRY(cudaMalloc(&w.train_samples, (size_t)samples * 16 * sizeof(float)));
    w.nrc_capacity = cap;
    w.train_slots = slots;
    w.rec_per_path = rec_per_path;
    w.sample_cap = samples;
    return PT_OK;
}

// ReSTIR DI buffers for every path of a wave
static pt_status ensure_restir_buffers(WaveBuffers& w) {
    if (w.restir_capacity >= w.capacity) return PT_OK;
    void* ps[] = {w.rs_g0, w.rs_g1, w.rs_gn, w.rs_i, w.rs_f};
    for (void* q : ps)
        if (q) cudaFree(q);
    w.rs_g0 = w.rs_g1 = w.rs_gn = w.rs_i = w.rs_f = nullptr;
    w.restir_capacity = 0;
    const size_t c = w.capacity;
    PT_CUDA_TRY(cudaMalloc(&w.rs_g0, c * sizeof(float4)));
    PT_CUDA_TRY(cudaMalloc(&w.rs_g1, c * sizeof(float4)));
    PT_CUDA_TRY(cudaMalloc(&w.rs_gn, c * sizeof(float4)));
    PT_CUDA_TRY(cudaMalloc(&w.rs_i, 2 * c * sizeof(float4)));
    PT_CUDA_TRY(cudaMalloc(&w.rs_f, 2 * c * sizeof(float4)));
    w.restir_capacity = w.capacity;
    return PT_OK;
}

static int g_trace_blocks_per_sm = 0, g_shade_blocks_per_sm = 0, g_shadow_blocks_per_sm = 0, g_tail_blocks_per_sm = 0;
static int g_coop_trace_bps = 0, g_coop_shadow_bps = 0;

// resident blocks per SM of the per-bounce kernels, queried once
static void wf_occupancy() {
    if (g_trace_blocks_per_sm != 0) return;
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_trace<false>, 128, 0);
    g_trace_blocks_per_sm = std::max(b, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_shade<false, false>, 128, 0);
    g_shade_blocks_per_sm = std::max(b, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_shadow<false>, 128, 0);
    g_shadow_blocks_per_sm = std::max(b, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_trace_coop<false>, 128, 0);
    g_coop_trace_bps = std::max(b, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_shadow_coop<false>, 128, 0);
    g_coop_shadow_bps = std::max(b, 1);
}

// the closest-hit and shadow passes, per-lane or cooperative (the same hits and counts)
template <bool COUNT>
static void launch_trace(bool coop, int sms, cudaStream_t st, const WfParams& P, int in_q) {
    if (coop) PT_LAUNCH(k_wf_trace_coop<COUNT>, sms * g_coop_trace_bps, 128, 0, st, P, in_q);
    else PT_LAUNCH(k_wf_trace<COUNT>, sms * g_trace_blocks_per_sm, 128, 0, st, P, in_q);
}
template <bool COUNT>
static void launch_shadow(bool coop, int sms, cudaStream_t st, const WfParams& P) {
    if (coop) PT_LAUNCH(k_wf_shadow_coop<COUNT>, sms * g_coop_shadow_bps, 128, 0, st, P);
    else PT_LAUNCH(k_wf_shadow<COUNT>, sms * g_shadow_blocks_per_sm, 128, 0, st, P);
}

pt_status pt_wavefront_tail_limit(int* out) {
    if (g_tail_blocks_per_sm == 0) {
        int b = 0;
        PT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_tail<true, false, false>, 128, 0));
        g_tail_blocks_per_sm = std::max(b, 1);
    }
    *out = pt_num_sms() * g_tail_blocks_per_sm * 128;
    return PT_OK;
}

// Everything that shapes the launch sequence of a wavefront call (the per-call words, first
// sample and seed, live in device memory): equal keys mean the same captured graph replays.
struct WfGraphKey {
    WfParams P;             // with the per-wave fields cleared
    uint32_t spp, npix_total, pix_chunk, samp_per_wave, tail_limit, tail_grid, count, coop;
    int sms, trace_bps, shade_bps, shadow_bps;
    uint64_t nrc_serial;    // the radiance cache the launches read and train (0: none)
};

static pt_status render_wavefront(pt_scene* s, const pt_camera& cam, uint32_t spp, uint32_t max_depth, uint64_t seed,
                                  pt_accum* acc, const pt_render_opts& o, cudaStream_t user_st) {
    cudaStream_t st = user_st;   // the stream the wave loops below issue to (a capture stream while capturing)
    const uint32_t npix_total = acc->width * acc->height;
    uint32_t cap = o.wave_paths ? o.wave_paths : (1u << 21);
    cap = std::max(cap, 32u);
    // waves hold whole samples of a pixel range: pixel chunk <= cap, then samples per wave;
    // with ReSTIR the chunk is the whole window (the spatial pass reads any pixel of it)
    const bool restir = o.restir != nullptr;
    const bool coop = o.traversal == PT_TRAVERSAL_COOP;
    const uint32_t pix_chunk = restir ? npix_total : std::min(npix_total, cap);
    const uint32_t samp_per_wave = std::max(1u, std::min(spp, cap / pix_chunk));
    pt_status r = ensure_wave(s->wave, pix_chunk * samp_per_wave);
    if (r != PT_OK) return r;
    WaveBuffers& w = s->wave;
    if (restir) {
        r = ensure_restir_buffers(w);
        if (r != PT_OK) return r;
    }
    const bool sort = o.sort_by_material == 1 || (o.sort_by_material < 0 && s->n_mats + 2 <= MAX_SORT_KEYS && s->n_mats > 1);
    const uint32_t n_keys = (sort && s->n_mats + 2 <= MAX_SORT_KEYS) ? s->n_mats + 2 : 0;
    wf_occupancy();
    if (g_tail_blocks_per_sm == 0) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_tail<true, false, false>, 128, 0);
        g_tail_blocks_per_sm = std::max(b, 1);
    }
    const int sms = pt_num_sms();
    // tail: the paths one launch of k_wf_tail holds resident, unless the caller says otherwise
    const uint32_t tail_grid = (uint32_t)(sms * g_tail_blocks_per_sm);
    const uint32_t tail_limit = o.tail_paths < 0 ? 0u : o.tail_paths > 0 ? (uint32_t)o.tail_paths : tail_grid * 128u;
    WfParams P;
    std::memset(&P, 0, sizeof(P));
    P.S = s->view();
    P.cam = to_dcam(cam);
    P.x0 = o.crop_x0;
    P.y0 = o.crop_y0;
    P.cw = acc->width;
    P.spp_call = spp;
    P.max_depth = max_depth;
    P.flags = o.flags;
    P.n_keys = n_keys;
    P.tail_bounce = tail_limit ? o.tail_bounce : 0u;   // part of the graph key: it shapes the launches
    for (int q = 0; q < 2; ++q) { P.ray_o[q] = w.ray_o[q]; P.ray_d[q] = w.ray_d[q]; }
    P.hit = w.hit; P.beta = w.beta; P.radiance = w.radiance;
    P.sh_o = w.sh_o; P.sh_d = w.sh_d; P.sh_c = w.sh_c;
    P.perm = w.perm; P.keys = w.keys; P.counters = w.counters;
    P.sum = acc->sum; P.comp = acc->comp; P.sample_out = o.sample_out;
    P.stats = s->d_stats;
    if (restir) {
        P.flags |= FLAG_RESTIR;
        P.restir_on = 1;
        P.restir_M = o.restir->candidates;
        P.restir_K = o.restir->spatial_neighbors;
        P.restir_R = o.restir->spatial_radius;
        P.restir_L = o.restir->later_candidates;
        P.rs_g0 = w.rs_g0; P.rs_g1 = w.rs_g1; P.rs_gn = w.rs_gn; P.rs_i = w.rs_i; P.rs_f = w.rs_f;
    }
    if (o.nrc) {
        r = ensure_nrc_buffers(w, std::min(max_depth + 1, 16u), pt_nrc_frame_samples(o.nrc));
        if (r != PT_OK) return r;
        r = pt_nrc_render_prepare(o.nrc, pix_chunk * samp_per_wave, w.sample_cap);
        if (r != PT_OK) return r;
        P.nrc_on = 1;
        P.rec_per_path = w.rec_per_path;
        P.max_train = o.nrc_train ? w.train_slots : 0;
        P.sample_cap = w.sample_cap;
        P.aux = w.aux; P.nrc_q = w.nrc_q; P.nrc_out = w.nrc_out; P.nrc_counters = w.nrc_counters;
        P.train_rec = w.train_rec; P.train_nv = w.train_nv; P.train_id = w.train_id;
        P.train_samples = w.train_samples;
    }
    uint64_t launches = 0;
    const bool count = (o.flags & FLAG_COUNT) != 0;
    // optional per-kind timing: an event pair around every launch of a kind
    const bool timed = o.kernel_ms != nullptr;
    // the per-call words first, on the caller's stream (graph or not)
    PT_LAUNCH(k_wf_frame, 1, 32, 0, user_st, w.counters, (uint32_t)acc->spp_done, seed);
    ++launches;
    const bool graph = o.use_graph && !timed;
    WfGraphKey key;
    if (graph) {
        std::memset(&key, 0, sizeof(key));
        key.P = P;
        key.spp = spp; key.npix_total = npix_total; key.pix_chunk = pix_chunk; key.samp_per_wave = samp_per_wave;
        key.tail_limit = tail_limit; key.tail_grid = tail_grid; key.count = count ? 1u : 0u;
        key.coop = coop ? 1u : 0u;
        key.sms = sms; key.trace_bps = g_trace_blocks_per_sm; key.shade_bps = g_shade_blocks_per_sm;
        key.shadow_bps = g_shadow_blocks_per_sm;
        key.nrc_serial = pt_nrc_serial(o.nrc);
        if (s->wf_graph && s->wf_key.size() == sizeof(key) && std::memcmp(s->wf_key.data(), &key, sizeof(key)) == 0) {
            PT_CUDA_TRY(cudaGraphLaunch(s->wf_graph, user_st));
            pt_count_launch(s->wf_graph_launches);
            s->launches += launches + s->wf_graph_launches;
            s->graph_replays++;
            return PT_OK;
        }
        if (s->wf_graph) {
            cudaGraphExecDestroy(s->wf_graph);
            s->wf_graph = nullptr;
            s->wf_key.clear();
        }
        if (!s->cap_stream) PT_CUDA_TRY(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
        // capture on the library's own stream (the caller's may be the legacy default stream,
        // which cannot be captured); the graph then runs on the caller's stream
        PT_CUDA_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        st = s->cap_stream;
    }
    const uint64_t global_before = g_pt_launches.load();
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PT_K_KINDS];
    auto begin = [&](int kind) -> cudaEvent_t {
        if (!timed) return nullptr;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        ev[kind].push_back({a, b});
        return b;
    };
    auto end = [&](cudaEvent_t b) {
        if (b) cudaEventRecord(b, st);
    };
    auto issue = [&]() -> pt_status {
        for (uint32_t pb = 0; pb < npix_total; pb += pix_chunk) {
            const uint32_t npix = std::min(pix_chunk, npix_total - pb);
            for (uint32_t i0 = 0; i0 < spp; i0 += samp_per_wave) {
                const uint32_t ns = std::min(samp_per_wave, spp - i0);
                P.pb = pb;
                P.npix = npix;
                P.i0 = i0;
                P.nsamp = ns;
                // whole groups of 4 rows, 8-pixel tiles across; ReSTIR's first pass needs slot = path id
                P.tiled = (!restir && pb % P.cw == 0 && npix % (4u * P.cw) == 0 && P.cw % 8u == 0) ? 1u : 0u;
                const uint32_t n = npix * ns;
                if (P.nrc_on) {
                    P.train_prob = std::min(1.0f, (float)w.train_slots / (float)n);
                    PT_CUDA_TRY(cudaMemsetAsync(w.nrc_counters, 0, 8 * sizeof(uint32_t), st));
                }
                cudaEvent_t e = begin(PT_K_RAYGEN);
                PT_LAUNCH(k_wf_raygen, (n + 255) / 256, 256, 0, st, P);
                end(e);
                ++launches;
                for (uint32_t k = 0; k <= max_depth; ++k) {
                    const int in_q = (int)(k & 1u), out_q = (int)((k + 1) & 1u);
                    PT_LAUNCH(k_wf_setup, 1, 256, 0, st, w.counters, out_q, n_keys);
                    ++launches;
                    if (tail_limit && !(restir && k == 0)) {
                        // at the forced bounce the tail kernel takes the paths whatever their number
                        const bool force = P.tail_bounce != 0 && k == P.tail_bounce;
                        const uint32_t lim = force ? 0xFFFFFFFFu : tail_limit;
                        e = begin(PT_K_TAIL);
                        const bool fz = s->has_fuzz;
                        if (P.nrc_on) {
                            if (count) launch_tail<true, true, false>(fz, tail_grid, st, P, in_q, k, lim);
                            else launch_tail<true, false, false>(fz, tail_grid, st, P, in_q, k, lim);
                        } else if (restir) {
                            if (count) launch_tail<false, true, true>(fz, tail_grid, st, P, in_q, k, lim);
                            else launch_tail<false, false, true>(fz, tail_grid, st, P, in_q, k, lim);
                        } else {
                            if (count) launch_tail<false, true, false>(fz, tail_grid, st, P, in_q, k, lim);
                            else launch_tail<false, false, false>(fz, tail_grid, st, P, in_q, k, lim);
                        }
                        end(e);
                        ++launches;
                        if (force) break;   // no path is left for the later bounces
                    }
                    e = begin(PT_K_TRACE);
                    if (count) launch_trace<true>(coop, sms, st, P, in_q);
                    else launch_trace<false>(coop, sms, st, P, in_q);
                    end(e);
                    ++launches;
                    if (n_keys) {
                        e = begin(PT_K_SORT);
                        PT_LAUNCH(k_wf_sort_scan, 1, MAX_SORT_KEYS, 0, st, w.counters, n_keys);
                        PT_LAUNCH(k_wf_sort_scatter, sms * 2, SORT_THREADS, 0, st, P, in_q);
                        end(e);
                        launches += 2;
                    }
                    if (restir && k == 0) {
                        e = begin(PT_K_RESTIR);
                        PT_LAUNCH(k_restir_init, sms * 6, 128, 0, st, P);
                        PT_LAUNCH(k_restir_spatial, sms * 6, 128, 0, st, P, n);
                        end(e);
                        launches += 2;
                    }
                    e = begin(PT_K_SHADE);
                    const uint32_t shade_grid = sms * g_shade_blocks_per_sm;
                    if (P.nrc_on) launch_shade<true, false>(s->has_fuzz, shade_grid, st, P, in_q, out_q, k);
                    else if (restir) launch_shade<false, true>(s->has_fuzz, shade_grid, st, P, in_q, out_q, k);
                    else launch_shade<false, false>(s->has_fuzz, shade_grid, st, P, in_q, out_q, k);
                    end(e);
                    e = begin(PT_K_SHADOW);
                    if (count) launch_shadow<true>(coop, sms, st, P);
                    else launch_shadow<false>(coop, sms, st, P);
                    end(e);
                    launches += 2;
                }
                if (P.nrc_on) {
                    // cache inference for the paths that ended at their second diffuse-ish vertex,
                    // then training on this wave's training-path suffixes; the counts stay on the
                    // device, so nothing here waits for the GPU
                    pt_status rr = pt_nrc_render_infer_dev(o.nrc, w.nrc_q, w.nrc_counters, n, w.nrc_out, st);
                    if (rr != PT_OK) return rr;
                    PT_LAUNCH(k_nrc_apply, sms * 4, 256, 0, st, P);
                    ++launches;
                    if (P.max_train) {
                        PT_LAUNCH(k_nrc_targets, (P.max_train + 127) / 128, 128, 0, st, P);
                        ++launches;
                        rr = pt_nrc_render_train_dev(o.nrc, w.train_samples, w.nrc_counters + 2, P.sample_cap, st);
                        if (rr != PT_OK) return rr;
                    }
                }
                e = begin(PT_K_ACCUM);
                PT_LAUNCH(k_wf_accum, (npix + 255) / 256, 256, 0, st, P);
                end(e);
                ++launches;
            }
        }
        return PT_OK;
    };
    pt_status ir = issue();
    if (graph) {
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
        st = user_st;
        // captured launches were recorded, not run: they count when the graph runs
        const uint64_t captured = g_pt_launches.load() - global_before;
        g_pt_launches.fetch_sub(captured);
        if (ir != PT_OK) {
            if (g) cudaGraphDestroy(g);
            return ir;
        }
        if (ce != cudaSuccess) {
            pt_set_error(std::string("graph capture: ") + cudaGetErrorString(ce));
            return PT_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            pt_set_error(std::string("graph instantiate: ") + cudaGetErrorString(ie));
            return PT_ERR_CUDA;
        }
        s->wf_graph = ex;
        s->wf_key.assign(reinterpret_cast<const unsigned char*>(&key), reinterpret_cast<const unsigned char*>(&key) + sizeof(key));
        s->wf_graph_launches = captured;
        PT_CUDA_TRY(cudaGraphLaunch(ex, user_st));
        pt_count_launch(captured);
    } else if (ir != PT_OK) {
        return ir;
    }
    s->launches += launches;
    PT_CUDA_TRY(cudaGetLastError());
    if (timed) {
        PT_CUDA_TRY(cudaStreamSynchronize(st));
        for (int kind = 0; kind < PT_K_KINDS; ++kind) {
            for (auto& pr : ev[kind]) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, pr.first, pr.second);
                o.kernel_ms[kind] += ms;
                if (o.kernel_launches) o.kernel_launches[kind] += 1;
                cudaEventDestroy(pr.first);
                cudaEventDestroy(pr.second);
            }
        }
    }
    return PT_OK;
}

// ------------------------------------------------------------------ entry points
static DJob make_job(pt_scene* s, const pt_camera& cam, uint32_t x0, uint32_t y0, const pt_accum* acc, uint32_t spp,
                     uint32_t max_depth, uint64_t seed, uint32_t flags, float* sample_out) {
    DJob j;
    std::memset(&j, 0, sizeof(j));
    j.S = s->view();
    j.cam = to_dcam(cam);
    j.x0 = x0;
    j.y0 = y0;
    j.cw = acc->width;
    j.ch = acc->height;
    j.s0 = (uint32_t)acc->spp_done;
    j.spp = spp;
    j.max_depth = max_depth;
    j.flags = flags;
    j.seed = seed;
    j.sum = acc->sum;
    j.comp = acc->comp;
    j.sample_out = sample_out;
    j.stats = s->d_stats;
    j.n_mats = s->n_mats;
    return j;
}


extern "C" pt_status pt_render(pt_scene* s, const pt_camera* camera, uint32_t spp, uint32_t max_depth, uint64_t seed,
                               pt_accum* acc, const pt_render_opts* opts, void* cuda_stream) {
    PT_CHECK_ARG(s && camera && acc, "NULL argument");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    PT_CHECK_ARG(acc->sum && acc->comp, "accumulator buffers are NULL");
    PT_CHECK_ARG(camera->width > 0 && camera->height > 0, "empty frame");
    PT_CHECK_ARG(camera->vfov_deg > 0.0f && camera->vfov_deg < 180.0f, "vfov outside (0, 180)");
    PT_CHECK_ARG(lens_ok(*camera), "lens_radius must be finite and >= 0, with focus_distance > 0 when it is > 0");
    pt_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.sort_by_material = -1;
    if (opts) o = *opts;
    PT_CHECK_ARG(acc->width > 0 && acc->height > 0, "empty window");
    PT_CHECK_ARG((uint64_t)o.crop_x0 + acc->width <= camera->width &&
                     (uint64_t)o.crop_y0 + acc->height <= camera->height, "window outside the frame");
    PT_CHECK_ARG(acc->spp_done + spp < (1ull << 32), "sample index overflows 32 bits");
    PT_CHECK_ARG(o.mode <= PT_MODE_MEGAKERNEL, "unknown mode");
    PT_CHECK_ARG(o.traversal <= PT_TRAVERSAL_COOP, "unknown traversal");
    PT_CHECK_ARG(!o.nrc || o.mode != PT_MODE_MEGAKERNEL, "the radiance cache runs in wavefront mode");
    if (o.restir) {
        const pt_restir_opts& ro = *o.restir;
        PT_CHECK_ARG(ro.candidates >= 1 && ro.candidates <= 4096, "restir candidates must be 1..4096");
        PT_CHECK_ARG(ro.spatial_neighbors <= 64, "restir spatial_neighbors must be 0..64");
        PT_CHECK_ARG(ro.spatial_radius >= 1 && ro.spatial_radius <= 4096, "restir spatial_radius must be 1..4096");
        PT_CHECK_ARG(ro.later_candidates <= 4096, "restir later_candidates must be 0..4096");
        PT_CHECK_ARG(!(o.flags & PT_FLAG_NO_NEE), "ReSTIR DI replaces next-event estimation: not with PT_FLAG_NO_NEE");
        if (o.mode == PT_MODE_MEGAKERNEL || o.nrc) {
            pt_set_error("ReSTIR DI runs in wavefront mode without the radiance cache");
            return PT_ERR_UNSUPPORTED;
        }
    }
    if (spp == 0) return PT_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->last_stream = st;
    uint32_t mode = o.mode;
    if (mode == PT_MODE_AUTO) {
        if (s->tuned && s->tuned_w == acc->width && s->tuned_h == acc->height && !o.nrc) {
            // the schedule pt_autotune measured fastest for frames of this size
            mode = s->tuned_opts.mode;
            o.wave_paths = s->tuned_opts.wave_paths;
            o.sort_by_material = s->tuned_opts.sort_by_material;
            o.tail_paths = s->tuned_opts.tail_paths;
            o.block_size = s->tuned_opts.block_size;
            o.use_graph = s->tuned_opts.use_graph;
            o.traversal = s->tuned_opts.traversal;
            o.tail_bounce = s->tuned_opts.tail_bounce;
        } else {
            mode = (o.nrc || (uint64_t)acc->width * acc->height >= (1u << 16)) ? PT_MODE_WAVEFRONT : PT_MODE_MEGAKERNEL;
        }
        if (o.restir) mode = PT_MODE_WAVEFRONT;
    }
    pt_status r;
    if (mode == PT_MODE_WAVEFRONT) {
        r = render_wavefront(s, *camera, spp, max_depth, seed, acc, o, st);
    } else {
        const uint32_t tile = o.block_size ? std::max(32u, o.block_size & ~31u) : 64u;
        r = launch_megakernel_one(make_job(s, *camera, o.crop_x0, o.crop_y0, acc, spp, max_depth, seed, o.flags,
                                           o.sample_out), tile, 0, st, s->d_head, &s->launches);
    }
    if (r == PT_OK) acc->spp_done += spp;
    return r;
}

// Streams of the wavefront batch, per device: created on first use, kept for the process.
struct BatchStreams {
    cudaStream_t s[16] = {};
    cudaEvent_t fork = nullptr, join[16] = {};
};
static std::mutex g_bstream_mutex;
static BatchStreams g_bstreams[64];

static pt_status batch_streams(int dev, BatchStreams** out) {
    PT_CHECK_ARG(dev >= 0 && dev < 64, "device index");
    std::lock_guard<std::mutex> lock(g_bstream_mutex);
    BatchStreams& b = g_bstreams[dev];
    if (!b.fork) {
        PT_CUDA_TRY(cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming));
        for (int k = 0; k < 16; ++k) {
            PT_CUDA_TRY(cudaStreamCreateWithFlags(&b.s[k], cudaStreamNonBlocking));
            PT_CUDA_TRY(cudaEventCreateWithFlags(&b.join[k], cudaEventDisableTiming));
        }
    }
    *out = &b;
    return PT_OK;
}

// Wavefront batch: each job through pt_render (wavefront, graph replay) on one of K streams
// forked from the caller's stream; jobs go, largest first, to the least-loaded stream, except
// that all jobs of a scene share a stream (they share its wave buffers).
static pt_status batch_wavefront(const pt_job* jobs, uint32_t n_jobs, uint32_t K, cudaStream_t st) {
    int dev = 0;
    PT_CUDA_TRY(cudaGetDevice(&dev));
    BatchStreams* B = nullptr;
    pt_status r = batch_streams(dev, &B);
    if (r != PT_OK) return r;
    PT_CUDA_TRY(cudaEventRecord(B->fork, st));
    for (uint32_t k = 0; k < K; ++k) PT_CUDA_TRY(cudaStreamWaitEvent(B->s[k], B->fork, 0));
    std::vector<uint32_t> order(n_jobs);
    for (uint32_t i = 0; i < n_jobs; ++i) order[i] = i;
    auto work = [&](uint32_t i) {
        return (double)jobs[i].camera.width * jobs[i].camera.height * std::max(jobs[i].spp, 1u) * (jobs[i].max_depth + 1);
    };
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return work(a) > work(b); });
    std::vector<double> load(K, 0.0);
    std::vector<std::pair<const pt_scene*, uint32_t>> placed;
    pt_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.mode = PT_MODE_WAVEFRONT;
    o.sort_by_material = -1;
    o.use_graph = 1;
    for (uint32_t i : order) {
        const pt_job& j = jobs[i];
        uint32_t k = K;
        for (auto& pl : placed)
            if (pl.first == j.scene) k = pl.second;
        if (k == K) {
            k = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
            placed.push_back({j.scene, k});
        }
        load[k] += work(i);
        r = pt_render(j.scene, &j.camera, j.spp, j.max_depth, j.seed, j.accum, &o, B->s[k]);
        if (r != PT_OK) break;
    }
    for (uint32_t k = 0; k < K; ++k) {
        cudaEventRecord(B->join[k], B->s[k]);
        cudaStreamWaitEvent(st, B->join[k], 0);
    }
    for (uint32_t i = 0; i < n_jobs; ++i) jobs[i].scene->last_stream = st;
    return r;
}

// ---- merged batch: the paths of every job share the wavefront waves
// A wave is a list of segments (WfmSeg), filled in job order: each job's (pixel range x
// sample range) blocks are the ones a single-scene wavefront of that job would make, and a
// block that does not fit in the wave's remaining room is split along its pixels.  Every
// wave runs the single-scene launch sequence (raygen, per bounce: setup, tail, closest hit,
// shade, shadow rays; accumulation) once for all its jobs, the kernels looking each path's
// scene, camera, depth and seed up through its segment.  The launch sequence of a batch
// layout is captured once as a CUDA graph (with the job table copied in from pinned memory
// at its start, so seeds, first samples and cameras may change between calls) and replayed.
struct MergedBatch {
    int device = -1;
    std::vector<uint64_t> key;      // per job: scene, width, height, spp, max depth; wave size
    std::vector<WfmSeg> segs;
    std::vector<uint32_t> wave_seg0, wave_paths, wave_pix;   // per wave: first segment, paths, pixels
    WaveBuffers wave;
    DJob* h_jobs = nullptr;
    DJob* d_jobs = nullptr;
    WfmSeg* d_segs = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    cudaStream_t cap = nullptr;
    uint64_t launches = 0;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (done) cudaEventDestroy(done);
        if (cap) cudaStreamDestroy(cap);
        if (h_jobs) cudaFreeHost(h_jobs);
        if (d_jobs) cudaFree(d_jobs);
        if (d_segs) cudaFree(d_segs);
        pt_free_wave(wave);
        exec = nullptr; done = nullptr; cap = nullptr; h_jobs = nullptr; d_jobs = nullptr; d_segs = nullptr;
        key.clear();
        launches = 0;
    }
};
static MergedBatch g_merged;   // guarded by g_batch_mutex

static void merged_layout(const std::vector<DJob>& dj, uint32_t cap, MergedBatch& m) {
    m.segs.clear();
    m.wave_seg0.clear();
    m.wave_paths.clear();
    m.wave_pix.clear();
    uint32_t fill = 0, pix = 0;
    auto close = [&]() {
        if (fill == 0) return;
        m.wave_paths.push_back(fill);
        m.wave_pix.push_back(pix);
        fill = 0;
        pix = 0;
    };
    for (uint32_t j = 0; j < dj.size(); ++j) {
        const uint32_t npix = dj[j].cw * dj[j].ch, spp = dj[j].spp;
        if (npix == 0 || spp == 0) continue;
        const uint32_t chunk = std::min(npix, cap);
        const uint32_t spw = std::max(1u, std::min(spp, cap / chunk));
        for (uint32_t pb = 0; pb < npix; pb += chunk) {
            const uint32_t np = std::min(chunk, npix - pb);
            for (uint32_t i0 = 0; i0 < spp; i0 += spw) {
                const uint32_t ns = std::min(spw, spp - i0);
                for (uint32_t done = 0; done < np;) {
                    if (cap - fill < ns) {
                        close();
                        continue;
                    }
                    const uint32_t take = std::min(np - done, (cap - fill) / ns);
                    // a wave holds each pixel of a job once: one accumulation thread adds all of
                    // the pixel's samples of the wave, in order (a later sample block of the same
                    // pixels waits for the next wave)
                    bool overlap = false;
                    if (fill > 0)
                        for (size_t k = m.wave_seg0.back(); k < m.segs.size() && !overlap; ++k)
                            overlap = m.segs[k].job == j && m.segs[k].pb < pb + done + take &&
                                      pb + done < m.segs[k].pb + m.segs[k].npix;
                    if (overlap) {
                        close();
                        continue;
                    }
                    if (fill == 0) m.wave_seg0.push_back((uint32_t)m.segs.size());
                    m.segs.push_back(WfmSeg{j, pb + done, take, i0, ns, fill, pix, 0u});
                    fill += take * ns;
                    pix += take;
                    done += take;
                    if (fill == cap) close();
                }
            }
        }
    }
    close();
}

static pt_status merged_launches(MergedBatch& m, const WfParams& base, uint32_t max_depth, bool fuzz, cudaStream_t st,
                                 uint64_t* launches) {
    const int sms = pt_num_sms();
    const uint32_t tail_grid = (uint32_t)(sms * g_tail_blocks_per_sm);
    const uint32_t tail_limit = tail_grid * 128u;
    for (size_t w = 0; w < m.wave_paths.size(); ++w) {
        WfParams P = base;
        const uint32_t seg_end = w + 1 < m.wave_seg0.size() ? m.wave_seg0[w + 1] : (uint32_t)m.segs.size();
        P.segs = m.d_segs + m.wave_seg0[w];
        P.n_segs = seg_end - m.wave_seg0[w];
        const uint32_t n = m.wave_paths[w];
        PT_LAUNCH(k_wfm_raygen, (n + 255) / 256, 256, 0, st, P, n);
        ++*launches;
        for (uint32_t k = 0; k <= max_depth; ++k) {
            const int in_q = (int)(k & 1u), out_q = (int)((k + 1) & 1u);
            PT_LAUNCH(k_wf_setup, 1, 256, 0, st, m.wave.counters, out_q, P.n_keys);
            if (fuzz) PT_LAUNCH((k_wf_tail<false, false, false, true, true>), tail_grid, 128, 0, st, P, in_q, k, tail_limit);
            else PT_LAUNCH((k_wf_tail<false, false, false, false, true>), tail_grid, 128, 0, st, P, in_q, k, tail_limit);
            PT_LAUNCH((k_wf_trace<false, true>), sms * g_trace_blocks_per_sm, 128, 0, st, P, in_q);
            if (P.n_keys) {
                PT_LAUNCH(k_wf_sort_scan, 1, MAX_SORT_KEYS, 0, st, m.wave.counters, P.n_keys);
                PT_LAUNCH(k_wf_sort_scatter, sms * 2, SORT_THREADS, 0, st, P, in_q);
                *launches += 2;
            }
            if (fuzz) PT_LAUNCH((k_wf_shade<false, false, true, true>), sms * g_shade_blocks_per_sm, 128, 0, st, P, in_q, out_q, k);
            else PT_LAUNCH((k_wf_shade<false, false, false, true>), sms * g_shade_blocks_per_sm, 128, 0, st, P, in_q, out_q, k);
            PT_LAUNCH((k_wf_shadow<false, true>), sms * g_shadow_blocks_per_sm, 128, 0, st, P);
            *launches += 5;
        }
        PT_LAUNCH(k_wfm_accum, (m.wave_pix[w] + 255) / 256, 256, 0, st, P, m.wave_pix[w]);
        ++*launches;
    }
    PT_CUDA_TRY(cudaGetLastError());
    return PT_OK;
}

static pt_status batch_merged(const pt_job* jobs, uint32_t n_jobs, const pt_batch_opts& bo, cudaStream_t st) {
    std::vector<DJob> dj;
    std::vector<uint64_t> key;
    bool fuzz = false;
    uint32_t max_depth = 0;
    const uint32_t cap = std::max(bo.wave_paths ? bo.wave_paths : (1u << 22), 1024u);
    uint32_t n_keys = 0;   // material sort keys: (job, material) pairs, plus miss and light per job
    for (uint32_t i = 0; i < n_jobs; ++i) {
        const pt_job& j = jobs[i];
        dj.push_back(make_job(j.scene, j.camera, 0, 0, j.accum, j.spp, j.max_depth, j.seed, 0, nullptr));
        dj.back().key_base = n_keys;
        n_keys += j.scene->n_mats + 2;
        fuzz = fuzz || j.scene->has_fuzz;
        max_depth = std::max(max_depth, j.max_depth);
        // the scene's serial, not its address: the graph holds the first scene's statistics
        // pointer, and a new scene may reuse a destroyed one's address
        key.insert(key.end(), {j.scene->serial, j.camera.width, j.camera.height, j.spp, j.max_depth});
    }
    key.push_back(cap);
    key.push_back(fuzz ? 1u : 0u);
    wf_occupancy();
    if (g_tail_blocks_per_sm == 0) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wf_tail<true, false, false>, 128, 0);
        g_tail_blocks_per_sm = std::max(b, 1);
    }
    int dev = 0;
    PT_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    MergedBatch& m = g_merged;
    const bool same = m.device == dev && m.key == key && m.d_jobs != nullptr;
    if (!same) {
        // a new layout: wait for what the old one may still run, then rebuild
        if (m.done) cudaEventSynchronize(m.done);
        m.release();
        m.device = dev;
        merged_layout(dj, cap, m);
        pt_status r = ensure_wave(m.wave, cap);
        if (r != PT_OK) { m.release(); return r; }
        if (cudaMallocHost((void**)&m.h_jobs, dj.size() * sizeof(DJob)) != cudaSuccess ||
            cudaMalloc((void**)&m.d_jobs, dj.size() * sizeof(DJob)) != cudaSuccess ||
            cudaMalloc((void**)&m.d_segs, std::max<size_t>(m.segs.size(), 1) * sizeof(WfmSeg)) != cudaSuccess) {
            m.release();
            pt_set_error("merged batch tables: out of memory");
            return PT_ERR_OOM;
        }
        PT_CUDA_TRY(cudaMemcpy(m.d_segs, m.segs.data(), m.segs.size() * sizeof(WfmSeg), cudaMemcpyHostToDevice));
        PT_CUDA_TRY(cudaEventCreateWithFlags(&m.done, cudaEventDisableTiming));
        m.key = key;
    } else {
        // the previous call may still read the pinned job table
        PT_CUDA_TRY(cudaEventSynchronize(m.done));
    }
    std::memcpy(m.h_jobs, dj.data(), dj.size() * sizeof(DJob));
    WfParams P;
    std::memset(&P, 0, sizeof(P));
    const WaveBuffers& w = m.wave;
    for (int q = 0; q < 2; ++q) { P.ray_o[q] = w.ray_o[q]; P.ray_d[q] = w.ray_d[q]; }
    P.hit = w.hit; P.beta = w.beta; P.radiance = w.radiance;
    P.sh_o = w.sh_o; P.sh_d = w.sh_d; P.sh_c = w.sh_c;
    P.perm = w.perm; P.keys = w.keys; P.counters = w.counters;
    P.stats = jobs[0].scene->d_stats;
    P.jobs = m.d_jobs;
    P.n_keys = n_keys <= MAX_SORT_KEYS ? n_keys : 0u;
    uint64_t launches = 0;
    if (bo.use_graph) {
        if (!m.exec) {
            if (!m.cap) PT_CUDA_TRY(cudaStreamCreateWithFlags(&m.cap, cudaStreamNonBlocking));
            PT_CUDA_TRY(cudaStreamBeginCapture(m.cap, cudaStreamCaptureModeThreadLocal));
            const uint64_t before = g_pt_launches.load();
            cudaMemcpyAsync(m.d_jobs, m.h_jobs, dj.size() * sizeof(DJob), cudaMemcpyHostToDevice, m.cap);
            uint64_t n_l = 0;
            const pt_status r = merged_launches(m, P, max_depth, fuzz, m.cap, &n_l);
            g_pt_launches.fetch_sub(g_pt_launches.load() - before);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(m.cap, &graph);
            if (r != PT_OK || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                m.release();
                if (r != PT_OK) return r;
                pt_set_error(std::string("merged batch capture: ") + cudaGetErrorString(ce));
                return PT_ERR_CUDA;
            }
            const cudaError_t ie = cudaGraphInstantiate(&m.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                m.release();
                pt_set_error(std::string("merged batch instantiate: ") + cudaGetErrorString(ie));
                return PT_ERR_CUDA;
            }
            m.launches = n_l;
        }
        PT_CUDA_TRY(cudaGraphLaunch(m.exec, st));
        pt_count_launch(m.launches);
        launches = m.launches;
    } else {
        PT_CUDA_TRY(cudaMemcpyAsync(m.d_jobs, m.h_jobs, dj.size() * sizeof(DJob), cudaMemcpyHostToDevice, st));
        pt_status r = merged_launches(m, P, max_depth, fuzz, st, &launches);
        if (r != PT_OK) return r;
    }
    PT_CUDA_TRY(cudaEventRecord(m.done, st));
    for (uint32_t i = 0; i < n_jobs; ++i) {
        jobs[i].scene->last_stream = st;
        jobs[i].accum->spp_done += jobs[i].spp;
    }
    jobs[0].scene->launches += launches;
    return PT_OK;
}

extern "C" pt_status pt_render_batch(const pt_job* jobs, uint32_t n_jobs, const pt_batch_opts* opts, void* cuda_stream) {
    PT_CHECK_ARG(jobs != nullptr || n_jobs == 0, "jobs is NULL");
    if (n_jobs == 0) return PT_OK;
    pt_batch_opts bo;
    std::memset(&bo, 0, sizeof(bo));
    if (opts) bo = *opts;
    const uint32_t tile = bo.tile_pixels ? bo.tile_pixels : 64;
    PT_CHECK_ARG(tile % 32 == 0, "tile_pixels must be a multiple of 32");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<DJob> dj;
    dj.reserve(n_jobs);
    for (uint32_t i = 0; i < n_jobs; ++i) {
        const pt_job& j = jobs[i];
        PT_CHECK_ARG(j.scene && j.accum && j.accum->sum && j.accum->comp, "job with NULL scene or accumulator");
        if (!j.scene->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
        PT_CHECK_ARG(lens_ok(j.camera), "job camera: bad lens_radius / focus_distance");
        PT_CHECK_ARG(j.accum->width == j.camera.width && j.accum->height == j.camera.height,
                     "batch accumulators cover the whole frame");
        PT_CHECK_ARG(j.accum->spp_done + j.spp < (1ull << 32), "sample index overflows 32 bits");
        dj.push_back(make_job(j.scene, j.camera, 0, 0, j.accum, j.spp, j.max_depth, j.seed, 0, nullptr));
        j.scene->last_stream = st;
    }
    PT_CHECK_ARG(bo.mode == PT_MODE_AUTO || bo.mode == PT_MODE_WAVEFRONT || bo.mode == PT_MODE_MEGAKERNEL, "unknown mode");
    if (bo.mode == PT_MODE_WAVEFRONT && bo.merged) return batch_merged(jobs, n_jobs, bo, st);
    if (bo.mode == PT_MODE_WAVEFRONT) {
        const uint32_t K = std::min(bo.streams ? bo.streams : 4u, 16u);
        return batch_wavefront(jobs, n_jobs, K, st);
    }
    uint64_t launches = 0;
    pt_status r;
    if (bo.use_graph) {
        r = launch_megakernel_graph(dj, tile, bo.blocks_per_sm, st, &launches);
    } else {
        // per-call device job table and queue head from the stream-ordered allocator:
        // allocated, used and released in stream order, so the call does not wait for the GPU
        DJob* d_jobs = nullptr;
        uint32_t* d_head = nullptr;
        PT_CUDA_TRY(cudaMallocAsync((void**)&d_jobs, dj.size() * sizeof(DJob), st));
        if (cudaMallocAsync((void**)&d_head, sizeof(uint32_t), st) != cudaSuccess) {
            cudaFreeAsync(d_jobs, st);
            pt_set_error("batch queue head: out of memory");
            return PT_ERR_OOM;
        }
        r = launch_megakernel(dj, tile, bo.blocks_per_sm, st, d_head, d_jobs, &launches);
        cudaFreeAsync(d_jobs, st);
        cudaFreeAsync(d_head, st);
    }
    if (r != PT_OK) return r;
    for (uint32_t i = 0; i < n_jobs; ++i) jobs[i].accum->spp_done += jobs[i].spp;
    jobs[0].scene->launches += launches;
    return PT_OK;
}

// ------------------------------------------------------------------ render without allocation
// Some callers cannot call cudaMalloc: code running where the allocator is off limits
// (a memory budget fixed up front, an embedding host that owns all device memory, a
// real-time loop that must not hit the allocator's locks or its possible synchronisation).
// pt_render_noalloc serves them: the same wavefront kernels as pt_render, but the work
// queues live in the fixed-size array below, which every GPU that loads this library keeps
// until the process exits.  The kernels themselves reset every counter that must start at
// zero (raygen sets the input queue size, the per-bounce setup kernel clears the output
// queue, the shadow queue, the fetch heads and the sort buckets) and initialise every path
// slot they read, so stale contents from an earlier call are never used.
constexpr uint32_t NOALLOC_MAX_PATHS = 16384;
constexpr size_t NOALLOC_F4 = 10;   // float4 arrays per path: 2 x ray o/d, hit, beta, radiance, 3 x shadow
constexpr size_t NOALLOC_BYTES =
    (size_t)NOALLOC_MAX_PATHS * (NOALLOC_F4 * sizeof(float4) + 2 * sizeof(uint32_t)) +
    (C_BUCKETS + MAX_SORT_KEYS) * sizeof(uint32_t);
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch in the current context.  In host code the array's name
// is only a host-side stand-in, so every call asks the runtime for the address that goes to
// the kernels.  The lookup allocates nothing once the library's device code is loaded in the
// context; looking it up on each call, rather than caching it per device ordinal, keeps the
// address right after cudaDeviceReset or under a context other than the primary one.
static pt_status noalloc_scratch(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        pt_set_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
        return PT_ERR_CUDA;
    }
    *out = p;
    return PT_OK;
}

extern "C" pt_status pt_render_noalloc(pt_scene* s, const pt_camera* camera, uint32_t spp, uint32_t max_depth,
                                       uint64_t seed, pt_accum* acc, const pt_render_opts* opts, void* cuda_stream) {
    PT_CHECK_ARG(s && camera && acc, "NULL argument");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    PT_CHECK_ARG(acc->sum && acc->comp, "accumulator buffers are NULL");
    PT_CHECK_ARG(camera->width > 0 && camera->height > 0, "empty frame");
    PT_CHECK_ARG(camera->vfov_deg > 0.0f && camera->vfov_deg < 180.0f, "vfov outside (0, 180)");
    PT_CHECK_ARG(lens_ok(*camera), "lens_radius must be finite and >= 0, with focus_distance > 0 when it is > 0");
    pt_render_opts o;
    std::memset(&o, 0, sizeof(o));
    o.sort_by_material = -1;
    if (opts) o = *opts;
    PT_CHECK_ARG(acc->width > 0 && acc->height > 0, "empty window");
    PT_CHECK_ARG((uint64_t)o.crop_x0 + acc->width <= camera->width &&
                     (uint64_t)o.crop_y0 + acc->height <= camera->height, "window outside the frame");
    PT_CHECK_ARG((uint64_t)acc->width * acc->height <= NOALLOC_MAX_PATHS,
                 "pt_render_noalloc renders windows of at most 16384 pixels; render larger images tile by tile");
    PT_CHECK_ARG(acc->spp_done + spp < (1ull << 32), "sample index overflows 32 bits");
    PT_CHECK_ARG(o.nrc == nullptr, "the radiance cache needs allocations: use pt_render");
    PT_CHECK_ARG(o.restir == nullptr, "ReSTIR DI needs allocations: use pt_render");
    PT_CHECK_ARG(o.kernel_ms == nullptr && o.kernel_launches == nullptr, "kernel timing is not available here");
    PT_CHECK_ARG((o.flags & ~(uint32_t)(FLAG_NO_NEE | FLAG_NO_RR)) == 0,
                 "only PT_FLAG_NO_NEE and PT_FLAG_NO_RR are available here (no PT_FLAG_COUNT)");
    if (spp == 0) return PT_OK;
    void* base = nullptr;
    pt_status r = noalloc_scratch(&base);
    if (r != PT_OK) return r;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->last_stream = st;
    // carve the fixed array into the wavefront buffers
    const size_t c = NOALLOC_MAX_PATHS;
    float4* f4 = reinterpret_cast<float4*>(base);
    WaveBuffers w;
    w.capacity = NOALLOC_MAX_PATHS;
    w.ray_o[0] = f4 + 0 * c; w.ray_o[1] = f4 + 1 * c;
    w.ray_d[0] = f4 + 2 * c; w.ray_d[1] = f4 + 3 * c;
    w.hit = f4 + 4 * c; w.beta = f4 + 5 * c; w.radiance = f4 + 6 * c;
    w.sh_o = f4 + 7 * c; w.sh_d = f4 + 8 * c; w.sh_c = f4 + 9 * c;
    uint32_t* u = reinterpret_cast<uint32_t*>(f4 + NOALLOC_F4 * c);
    w.perm = u; w.keys = u + c; w.counters = u + 2 * c;
    const uint32_t npix = acc->width * acc->height;
    const uint32_t samp_per_wave = std::max(1u, std::min(spp, NOALLOC_MAX_PATHS / npix));
    const bool sort = o.sort_by_material == 1 || (o.sort_by_material < 0 && s->n_mats + 2 <= MAX_SORT_KEYS && s->n_mats > 1);
    const uint32_t n_keys = (sort && s->n_mats + 2 <= MAX_SORT_KEYS) ? s->n_mats + 2 : 0;
    wf_occupancy();
    const int sms = pt_num_sms();
    WfParams P;
    std::memset(&P, 0, sizeof(P));
    P.S = s->view();
    P.cam = to_dcam(*camera);
    P.x0 = o.crop_x0;
    P.y0 = o.crop_y0;
    P.cw = acc->width;
    P.spp_call = spp;
    P.max_depth = max_depth;
    P.flags = o.flags & (FLAG_NO_NEE | FLAG_NO_RR);
    P.n_keys = n_keys;
    for (int q = 0; q < 2; ++q) { P.ray_o[q] = w.ray_o[q]; P.ray_d[q] = w.ray_d[q]; }
    P.hit = w.hit; P.beta = w.beta; P.radiance = w.radiance;
    P.sh_o = w.sh_o; P.sh_d = w.sh_d; P.sh_c = w.sh_c;
    P.perm = w.perm; P.keys = w.keys; P.counters = w.counters;
    P.sum = acc->sum; P.comp = acc->comp; P.sample_out = o.sample_out;
    P.stats = s->d_stats;
    P.pb = 0;
    P.npix = npix;
    PT_LAUNCH(k_wf_frame, 1, 32, 0, st, w.counters, (uint32_t)acc->spp_done, seed);
    uint64_t launches = 1;
    for (uint32_t i0 = 0; i0 < spp; i0 += samp_per_wave) {
        const uint32_t ns = std::min(samp_per_wave, spp - i0);
        P.i0 = i0;
        P.nsamp = ns;
        const uint32_t n = npix * ns;
        PT_LAUNCH(k_wf_raygen, (n + 255) / 256, 256, 0, st, P);
        ++launches;
        for (uint32_t k = 0; k <= max_depth; ++k) {
            const int in_q = (int)(k & 1u), out_q = (int)((k + 1) & 1u);
            PT_LAUNCH(k_wf_setup, 1, 256, 0, st, w.counters, out_q, n_keys);
            launch_trace<false>(false, sms, st, P, in_q);
            launches += 2;
            if (n_keys) {
                PT_LAUNCH(k_wf_sort_scan, 1, MAX_SORT_KEYS, 0, st, w.counters, n_keys);
                PT_LAUNCH(k_wf_sort_scatter, sms * 2, SORT_THREADS, 0, st, P, in_q);
                launches += 2;
            }
            launch_shade<false, false>(s->has_fuzz, sms * g_shade_blocks_per_sm, st, P, in_q, out_q, k);
            launch_shadow<false>(false, sms, st, P);
            launches += 2;
        }
        PT_LAUNCH(k_wf_accum, (npix + 255) / 256, 256, 0, st, P);
        ++launches;
    }
    s->launches += launches;
    PT_CUDA_TRY(cudaGetLastError());
    acc->spp_done += spp;
    return PT_OK;
}
