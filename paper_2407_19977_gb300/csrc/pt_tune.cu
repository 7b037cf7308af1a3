// pt_tune.cu -- autotuner of the execution schedule (beyond the paper, which runs one fixed
// WebGPU pipeline).  Every candidate renders the same samples with the same random numbers
// into scratch accumulators; the schedule changes only how the work is laid out on the GPU,
// never the image (a BVH of another leaf size finds the same closest hits, ties included).
// Candidates are timed with CUDA events on the caller's stream.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pt_internal.h"

namespace {

struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    float* alloc(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, n * sizeof(float)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<float*>(p);
    }
};

// ms per frame of `frames` frames after one warm-up frame (the warm-up also captures graphs)
template <class F>
static pt_status time_frames(F&& frame, uint32_t frames, cudaStream_t st, float* ms) {
    pt_status r = frame();
    if (r != PT_OK) return r;
    cudaEvent_t a, b;
    PT_CUDA_TRY(cudaEventCreate(&a));
    PT_CUDA_TRY(cudaEventCreate(&b));
    cudaEventRecord(a, st);
    for (uint32_t f = 0; f < frames && r == PT_OK; ++f) r = frame();
    cudaEventRecord(b, st);
    const cudaError_t e = cudaEventSynchronize(b);
    float t = 0.0f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r != PT_OK) return r;
    if (e != cudaSuccess) {
        pt_set_error(std::string("autotune: ") + cudaGetErrorString(e));
        return PT_ERR_CUDA;
    }
    *ms = t / (float)std::max(frames, 1u);
    return PT_OK;
}

}  // namespace

extern "C" pt_status pt_autotune(pt_scene* s, const pt_camera* camera, uint32_t spp, uint32_t max_depth,
                                 uint32_t frames, uint32_t tune_flags, pt_render_opts* best, float* best_ms,
                                 void* cuda_stream) {
    PT_CHECK_ARG(s && camera && best, "NULL argument");
    if (!s->built) { pt_set_error("pt_bvh_build has not run"); return PT_ERR_NOT_BUILT; }
    PT_CHECK_ARG(camera->width > 0 && camera->height > 0, "empty frame");
    PT_CHECK_ARG(lens_ok(*camera), "lens_radius must be finite and >= 0, with focus_distance > 0 when it is > 0");
    PT_CHECK_ARG((tune_flags & ~PT_TUNE_BVH) == 0, "unknown tune flags");
    if (spp == 0) spp = 1;
    if (frames == 0) frames = 2;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint32_t W = camera->width, H = camera->height;
    Scratch sc;
    float* sum = sc.alloc((size_t)W * H * 3);
    float* comp = sc.alloc((size_t)W * H * 3);
    if (!sum || !comp) {
        pt_set_error("autotune: scratch accumulator out of memory");
        return PT_ERR_OOM;
    }
    auto run = [&](const pt_render_opts& o, float* ms) {
        pt_accum acc{sum, comp, 0, W, H};
        return time_frames([&]() { return pt_render(s, camera, spp, max_depth, 1234567u, &acc, &o, st); }, frames, st,
                           ms);
    };
    pt_render_opts base;
    std::memset(&base, 0, sizeof(base));
    base.mode = PT_MODE_WAVEFRONT;
    base.sort_by_material = -1;
    base.use_graph = 1;
    // BVH builder and leaf size first, then the width on that tree (one default schedule), then
    // the schedule on the chosen tree
    if (tune_flags & PT_TUNE_BVH) {
        pt_bvh_opts best_bo{s->leaf_size, s->builder, s->collapse, s->tri_cost, s->box_cost, s->max_width};
        float best_t = 3.4e38f;
        auto try_tree = [&](const pt_bvh_opts& bo) {
            pt_status r = pt_bvh_build(s, &bo, cuda_stream);
            if (r != PT_OK) return r;
            float t = 0.0f;
            r = run(base, &t);
            if (r != PT_OK) return r;
            if (t < best_t) { best_t = t; best_bo = bo; }
            return PT_OK;
        };
        for (uint32_t builder : {(uint32_t)PT_BVH_PLOC, (uint32_t)PT_BVH_LBVH})
            for (uint32_t leaf = 1; leaf <= 4; ++leaf) {
                const pt_status r = try_tree(pt_bvh_opts{leaf, builder, s->collapse, s->tri_cost, s->box_cost, 8u});
                if (r != PT_OK) return r;
            }
        const pt_bvh_opts tree8 = best_bo;
        for (uint32_t width : {4u, 6u}) {
            pt_bvh_opts bo = tree8;
            bo.max_width = width;
            const pt_status r = try_tree(bo);
            if (r != PT_OK) return r;
        }
        // the last tree tried is 6 wide: rebuild the winner (same collapse rule and costs)
        if (best_bo.max_width != 6u) {
            const pt_status r = pt_bvh_build(s, &best_bo, cuda_stream);
            if (r != PT_OK) return r;
        }
    }
    std::vector<pt_render_opts> cand;
    const uint32_t npix = W * H;
    for (int sort = 0; sort <= 1; ++sort)
        for (int tail : {-1, 0, 1, 2})   // off, automatic, a quarter of it, four times it
            for (uint32_t wave : {1u << 20, 1u << 21, 1u << 22, 1u << 23}) {
                if (wave > (1u << 20) && (uint64_t)npix * spp <= wave / 2) continue;   // the smaller wave holds it all
                pt_render_opts o = base;
                o.sort_by_material = sort;
                o.tail_paths = tail;   // resolved below
                o.wave_paths = wave;
                cand.push_back(o);
            }
    for (uint32_t tile : {32u, 64u, 128u}) {
        pt_render_opts o = base;
        o.mode = PT_MODE_MEGAKERNEL;
        o.block_size = tile;
        o.use_graph = 0;
        cand.push_back(o);
    }
    // the automatic tail limit, to scale it
    int tb = 0;
    pt_status r = pt_wavefront_tail_limit(&tb);
    if (r != PT_OK) return r;
    pt_render_opts win = base;
    float win_t = 3.4e38f;
    for (pt_render_opts o : cand) {
        if (o.mode == PT_MODE_WAVEFRONT) {
            if (o.tail_paths == 1) o.tail_paths = std::max(tb / 4, 1);
            else if (o.tail_paths == 2) o.tail_paths = tb * 4;
        }
        float t = 0.0f;
        r = run(o, &t);
        if (r != PT_OK) return r;
        if (t < win_t) { win_t = t; win = o; }
    }
    // the traversal passes of the winning wavefront schedule: one ray per lane (the default)
    // or one ray per group of 8 lanes
    if (win.mode == PT_MODE_WAVEFRONT) {
        pt_render_opts o = win;
        o.traversal = PT_TRAVERSAL_COOP;
        float t = 0.0f;
        r = run(o, &t);
        if (r != PT_OK) return r;
        if (t < win_t) { win_t = t; win = o; }
    }
    // a wavefront winner with a tail limit: the tail kernel forced to take every remaining path
    // at bounce 3..6, which drops the later bounces' launches (they would find nothing to do)
    if (win.mode == PT_MODE_WAVEFRONT && win.tail_paths >= 0) {
        const pt_render_opts base_win = win;
        for (uint32_t kb = 3; kb <= std::min(6u, max_depth); ++kb) {
            pt_render_opts o = base_win;
            o.tail_bounce = kb;
            float t = 0.0f;
            r = run(o, &t);
            if (r != PT_OK) return r;
            if (t < win_t) { win_t = t; win = o; }
        }
    }
    *best = win;
    if (best_ms) *best_ms = win_t;
    s->tuned = true;
    s->tuned_w = W;
    s->tuned_h = H;
    s->tuned_opts = win;
    return PT_OK;
}

extern "C" pt_status pt_autotune_batch(const pt_job* jobs, uint32_t n_jobs, uint32_t frames, uint32_t tune_flags,
                                       pt_batch_opts* best, float* best_ms, void* cuda_stream) {
    PT_CHECK_ARG((jobs || n_jobs == 0) && best, "NULL argument");
    PT_CHECK_ARG((tune_flags & ~PT_TUNE_BVH) == 0, "unknown tune flags");
    std::memset(best, 0, sizeof(*best));
    if (n_jobs == 0) return PT_OK;
    if (frames == 0) frames = 2;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the same jobs on scratch accumulators starting at each job's sample index
    Scratch sc;
    std::vector<pt_accum> accs(n_jobs);
    std::vector<pt_job> tj(jobs, jobs + n_jobs);
    for (uint32_t i = 0; i < n_jobs; ++i) {
        PT_CHECK_ARG(jobs[i].accum != nullptr, "job without accumulator");
        const size_t n = (size_t)jobs[i].accum->width * jobs[i].accum->height * 3;
        float* a = sc.alloc(n);
        float* b = sc.alloc(n);
        if (!a || !b) {
            pt_set_error("autotune: scratch accumulators out of memory");
            return PT_ERR_OOM;
        }
        accs[i] = *jobs[i].accum;
        accs[i].sum = a;
        accs[i].comp = b;
        tj[i].accum = &accs[i];
    }
    pt_batch_opts win;
    std::memset(&win, 0, sizeof(win));
    float win_t = 3.4e38f;
    std::vector<pt_batch_opts> cand;
    for (uint32_t tile : {32u, 64u, 128u, 256u})
        for (uint32_t bps : {0u, 2u, 4u}) {
            pt_batch_opts o;
            std::memset(&o, 0, sizeof(o));
            o.mode = PT_MODE_MEGAKERNEL;
            o.tile_pixels = tile;
            o.blocks_per_sm = bps;
            o.use_graph = 1;
            cand.push_back(o);
        }
    for (uint32_t k : {1u, 2u, 4u, 8u}) {
        pt_batch_opts o;
        std::memset(&o, 0, sizeof(o));
        o.mode = PT_MODE_WAVEFRONT;
        o.streams = k;
        cand.push_back(o);
    }
    // one merged wavefront for all jobs (a captured graph), at three wave sizes
    for (uint32_t wp : {1u << 22, 1u << 23, 1u << 24}) {
        pt_batch_opts o;
        std::memset(&o, 0, sizeof(o));
        o.mode = PT_MODE_WAVEFRONT;
        o.merged = 1;
        o.wave_paths = wp;
        o.use_graph = 1;
        cand.push_back(o);
    }
    auto time_batch = [&](const pt_batch_opts& o, float* t) {
        for (auto& a : accs) a.spp_done = 0;
        return time_frames([&]() { return pt_render_batch(tj.data(), n_jobs, &o, cuda_stream); }, frames, st, t);
    };
    // BVH width first: every scene of the batch rebuilt at 4, 6 and 8 children per node (each
    // keeps its own builder, leaf size and collapse rule), timed with one merged wavefront
    if (tune_flags & PT_TUNE_BVH) {
        std::vector<pt_scene*> scenes;
        for (uint32_t i = 0; i < n_jobs; ++i) {
            PT_CHECK_ARG(jobs[i].scene != nullptr && jobs[i].scene->built, "job scene is NULL or not built");
            if (std::find(scenes.begin(), scenes.end(), jobs[i].scene) == scenes.end()) scenes.push_back(jobs[i].scene);
        }
        auto rebuild = [&](uint32_t width) {
            for (pt_scene* sc : scenes) {
                pt_bvh_opts bo{sc->leaf_size, sc->builder, sc->collapse, sc->tri_cost, sc->box_cost, width};
                const pt_status r = pt_bvh_build(sc, &bo, cuda_stream);
                if (r != PT_OK) return r;
            }
            return PT_OK;
        };
        pt_batch_opts probe;
        std::memset(&probe, 0, sizeof(probe));
        probe.mode = PT_MODE_WAVEFRONT;
        probe.merged = 1;
        probe.wave_paths = 1u << 23;
        probe.use_graph = 1;
        uint32_t best_w = 8;
        float best_t = 3.4e38f;
        for (uint32_t width : {8u, 6u, 4u}) {
            pt_status r = rebuild(width);
            if (r != PT_OK) return r;
            float t = 0.0f;
            r = time_batch(probe, &t);
            if (r != PT_OK) return r;
            if (t < best_t) { best_t = t; best_w = width; }
        }
        if (best_w != 4u) {
            const pt_status r = rebuild(best_w);
            if (r != PT_OK) return r;
        }
    }
    for (const pt_batch_opts& o : cand) {
        float t = 0.0f;
        const pt_status r = time_batch(o, &t);
        if (r != PT_OK) return r;
        if (t < win_t) { win_t = t; win = o; }
    }
    *best = win;
    if (best_ms) *best_ms = win_t;
    return PT_OK;
}
