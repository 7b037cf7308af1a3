// pt_nrc.cu -- neural radiance cache entry points (placeholder until the cache kernels land).
#include "pt_internal.h"

extern "C" pt_status pt_nrc_create(const pt_nrc_opts*, void*, pt_nrc** out) {
    if (out) *out = nullptr;
    pt_set_error("radiance cache not available in this build");
    return PT_ERR_UNSUPPORTED;
}
extern "C" pt_status pt_nrc_train(pt_nrc*, const float*, uint32_t, void*) { return PT_ERR_UNSUPPORTED; }
extern "C" pt_status pt_nrc_infer(pt_nrc*, const float*, uint32_t, float*, void*) { return PT_ERR_UNSUPPORTED; }
extern "C" pt_status pt_nrc_params(pt_nrc*, int, float**, uint64_t*) { return PT_ERR_UNSUPPORTED; }
extern "C" pt_status pt_nrc_last_loss(pt_nrc*, float*) { return PT_ERR_UNSUPPORTED; }
extern "C" void pt_nrc_destroy(pt_nrc*) {}
