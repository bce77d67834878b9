// sr_segmented.cu -- the C entry points of the segmented sort, its
// statistics and the description of its launch configurations.  The sort
// itself is in sr_segmented.cuh; its instantiations per key type are in
// sr_seg_{i32,u32,f32,k8}.cu.
#include "sr_segmented.cuh"

namespace sr {

sr_status segmented_stats(const void *aux, sr_stats *out) {
    const SegCtrl *c = (const SegCtrl *)aux;
    out->big_segments = c->n_big;
    out->passes_skipped = 0;
    return SR_OK;
}

template <typename CFG> static sr_segmented_config describe() {
    sr_segmented_config d;
    std::memset(&d, 0, sizeof(d));
    d.strategy = CFG::BUCKETS;
    d.sort_threads = CFG::SNT;
    d.pack_items = CFG::BUCKETS ? 0 : CFG::IPT_P;
    d.tile_items = CFG::IPT;
    d.fan_in = CFG::F;
    d.merge_threads = CFG::MNT;
    d.tile_keys = (int64_t)CFG::SNT * CFG::IPT;
    d.cta_keys = (int64_t)CFG::F * CFG::SNT * CFG::IPT;
    d.small_keys = CFG::BUCKETS ? small_cap(CFG::LADDER, NSMALL - 1) : (int64_t)CFG::SNT * CFG::IPT_P / 2;
    d.ladder = CFG::BUCKETS ? CFG::LADDER : -1;
    return d;
}

int segmented_num_configs(int key_bytes) { return key_bytes == 4 ? SEG_NCFG_K4 : SEG_NCFG_K8; }

static sr_status describe_cfg(int key_bytes, int cfg, sr_segmented_config *out) {
    if (key_bytes == 4) {
        switch (cfg) {
        case 0: *out = describe<SegK4_0>(); return SR_OK;
        case 1: *out = describe<SegK4_1>(); return SR_OK;
        case 2: *out = describe<SegK4_2>(); return SR_OK;
        case 3: *out = describe<SegK4_3>(); return SR_OK;
        case 4: *out = describe<SegK4_4>(); return SR_OK;
        case 5: *out = describe<SegK4_5>(); return SR_OK;
        case 6: *out = describe<SegK4_6>(); return SR_OK;
        case 7: *out = describe<SegK4_7>(); return SR_OK;
        default: return SR_ERR_INVALID_ARG;
        }
    }
    switch (cfg) {
    case 0: *out = describe<SegK8_0>(); return SR_OK;
    case 1: *out = describe<SegK8_1>(); return SR_OK;
    case 2: *out = describe<SegK8_2>(); return SR_OK;
    case 3: *out = describe<SegK8_3>(); return SR_OK;
    case 4: *out = describe<SegK8_4>(); return SR_OK;
    default: return SR_ERR_INVALID_ARG;
    }
}

static sr_status segmented_dispatch(void *d_keys, size_t n_keys, const int64_t *d_off, size_t nseg,
                                    sr_key_type kt, int cfg, cudaStream_t s) {
    switch (kt) {
    case SR_KEY_I32:
        return segmented_run_cfg<SR_KEY_I32>((const uint32_t *)d_keys, (uint32_t *)d_keys, n_keys, d_off, nseg, s,
                                             true, cfg);
    case SR_KEY_U32:
        return segmented_run_cfg<SR_KEY_U32>((const uint32_t *)d_keys, (uint32_t *)d_keys, n_keys, d_off, nseg, s,
                                             true, cfg);
    case SR_KEY_F32:
        return segmented_run_cfg<SR_KEY_F32>((const uint32_t *)d_keys, (uint32_t *)d_keys, n_keys, d_off, nseg, s,
                                             true, cfg);
    case SR_KEY_U64:
        return segmented_run_cfg<SR_KEY_U64>((const unsigned long long *)d_keys, (unsigned long long *)d_keys,
                                             n_keys, d_off, nseg, s, true, cfg);
    case SR_KEY_I64:
        return segmented_run_cfg<SR_KEY_I64>((const unsigned long long *)d_keys, (unsigned long long *)d_keys,
                                             n_keys, d_off, nseg, s, true, cfg);
    default: return SR_ERR_INVALID_ARG;
    }
}

}  // namespace sr

using namespace sr;

extern "C" int sr_segmented_num_configs(sr_key_type kt) {
    if (!valid_key_type(kt)) return 0;
    return segmented_num_configs(key_bytes_of(kt));
}

extern "C" sr_status sr_segmented_config_info(sr_key_type kt, int config, sr_segmented_config *out) {
    if (!valid_key_type(kt) || !out) return SR_ERR_INVALID_ARG;
    if (config == SR_SEG_CONFIG_DEFAULT) config = segmented_default_cfg(key_bytes_of(kt), false);
    return describe_cfg(key_bytes_of(kt), config, out);
}

extern "C" sr_status sr_sort_segmented_cfg(void *d_keys, size_t n_keys, const int64_t *d_offsets,
                                           size_t num_segments, sr_key_type kt, int config, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (num_segments > 0 && !d_offsets) return SR_ERR_INVALID_ARG;
    if (n_keys > 0 && !d_keys) return SR_ERR_INVALID_ARG;
    if (n_keys > 0 && ((uintptr_t)d_keys % key_bytes_of(kt)) != 0) return SR_ERR_INVALID_ARG;
    if (((uintptr_t)d_offsets % 8) != 0) return SR_ERR_INVALID_ARG;
    if (config == SR_SEG_CONFIG_DEFAULT) config = segmented_default_cfg(key_bytes_of(kt), false);
    if (config < 0 || config >= segmented_num_configs(key_bytes_of(kt))) return SR_ERR_INVALID_ARG;
    if (num_segments >= (size_t)0x7fffffff || n_keys >= (1ull << 40)) return SR_ERR_UNSUPPORTED;
    return segmented_dispatch(d_keys, n_keys, d_offsets, num_segments, kt, config, (cudaStream_t)stream);
}

extern "C" sr_status sr_sort_segmented_ex(void *d_keys, size_t n_keys, const int64_t *d_offsets,
                                          size_t num_segments, sr_key_type kt, sr_stream stream) {
    return sr_sort_segmented_cfg(d_keys, n_keys, d_offsets, num_segments, kt, SR_SEG_CONFIG_DEFAULT, stream);
}

extern "C" sr_status sr_sort_segmented(void *d_keys, const int64_t *d_offsets, size_t num_segments,
                                       sr_key_type kt, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (num_segments == 0) return SR_OK;
    if (!d_offsets || ((uintptr_t)d_offsets % 8) != 0) return SR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t total = 0;
    if (cudaMemcpyAsync(&total, d_offsets + num_segments, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return SR_ERR_CUDA;
    }
    if (total < 0) return SR_ERR_BAD_SEGMENTS;
    return sr_sort_segmented_ex(d_keys, (size_t)total, d_offsets, num_segments, kt, stream);
}
