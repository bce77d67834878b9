// sr_seg_k8.cu -- the segmented sort's configurations for 8-byte keys
// (uint64, int64).
#include "sr_segmented.cuh"

namespace sr {

template <int KT>
static sr_status run_k8(const unsigned long long *in, unsigned long long *out, size_t n, const int64_t *off,
                        size_t nseg, cudaStream_t s, bool record, int cfg) {
    switch (cfg) {
    case 0: return segmented_run_t<KT, SegK8_0>(in, out, n, off, nseg, s, record);
    case 1: return segmented_run_t<KT, SegK8_1>(in, out, n, off, nseg, s, record);
    case 2: return segmented_run_t<KT, SegK8_2>(in, out, n, off, nseg, s, record);
    case 3: return segmented_run_t<KT, SegK8_3>(in, out, n, off, nseg, s, record);
    case 4: return segmented_run_t<KT, SegK8_4>(in, out, n, off, nseg, s, record);
    default: return SR_ERR_INVALID_ARG;
    }
}
static_assert(SEG_NCFG_K8 == 5, "every configuration needs a case");

template <>
sr_status segmented_run_cfg<SR_KEY_U64>(const unsigned long long *in, unsigned long long *out, size_t n,
                                        const int64_t *off, size_t nseg, cudaStream_t s, bool record, int cfg) {
    return run_k8<SR_KEY_U64>(in, out, n, off, nseg, s, record, cfg);
}
template <>
sr_status segmented_run_cfg<SR_KEY_I64>(const unsigned long long *in, unsigned long long *out, size_t n,
                                        const int64_t *off, size_t nseg, cudaStream_t s, bool record, int cfg) {
    return run_k8<SR_KEY_I64>(in, out, n, off, nseg, s, record, cfg);
}

}  // namespace sr
