// sr_pending.cu -- entry points whose kernels are not in this build yet.
#include "sr_runtime.cuh"

extern "C" sr_status sr_sort_keys_learned(void *, size_t, sr_key_type, const sr_learned_opts *, sr_stream) {
    return SR_ERR_UNSUPPORTED;
}
extern "C" sr_status sr_model_loss_grad(const float *, const float *, size_t, const float *, float *,
                                        float *, sr_stream) {
    return SR_ERR_UNSUPPORTED;
}
extern "C" sr_status sr_model_train(const float *, const float *, size_t, float *, uint32_t, float,
                                    float *, sr_stream) {
    return SR_ERR_UNSUPPORTED;
}
extern "C" sr_status sr_model_buckets(const void *, size_t, sr_key_type, const float *, uint64_t,
                                      uint64_t, uint32_t, uint32_t *, sr_stream) {
    return SR_ERR_UNSUPPORTED;
}

namespace sr {
sr_status learned_stats(const void *, sr_stats *) { return SR_OK; }
}  // namespace sr
