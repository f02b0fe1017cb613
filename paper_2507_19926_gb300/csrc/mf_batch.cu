// Batched persistent launch -- placeholder until the kernel lands.
#include "mf_registry.h"

extern "C" {
int mf_batch_plan_create(const mf_image_desc *, int, mf_batch_plan **out) {
    if (out) *out = nullptr;
    mf::set_error("batched launch not built");
    return MF_ERR_UNSUPPORTED;
}
int mf_batch_run(mf_batch_plan *, mf_stream_t) { return MF_ERR_UNSUPPORTED; }
int mf_batch_plan_destroy(mf_batch_plan *) { return MF_OK; }
}
