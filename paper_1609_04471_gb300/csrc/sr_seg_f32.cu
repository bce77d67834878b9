// sr_seg_f32.cu -- the segmented sort's configurations for float32 keys
// (one translation unit per key type, so they compile in parallel).
#include "sr_segmented.cuh"

namespace sr {

template <int KT>
static sr_status run_k4(const uint32_t *in, uint32_t *out, size_t n, const int64_t *off, size_t nseg,
                        cudaStream_t s, bool record, int cfg) {
    switch (cfg) {
    case 0: return segmented_run_t<KT, SegK4_0>(in, out, n, off, nseg, s, record);
    case 1: return segmented_run_t<KT, SegK4_1>(in, out, n, off, nseg, s, record);
    case 2: return segmented_run_t<KT, SegK4_2>(in, out, n, off, nseg, s, record);
    case 3: return segmented_run_t<KT, SegK4_3>(in, out, n, off, nseg, s, record);
    case 4: return segmented_run_t<KT, SegK4_4>(in, out, n, off, nseg, s, record);
    case 5: return segmented_run_t<KT, SegK4_5>(in, out, n, off, nseg, s, record);
    case 6: return segmented_run_t<KT, SegK4_6>(in, out, n, off, nseg, s, record);
    case 7: return segmented_run_t<KT, SegK4_7>(in, out, n, off, nseg, s, record);
    default: return SR_ERR_INVALID_ARG;
    }
}
static_assert(SEG_NCFG_K4 == 8, "every configuration needs a case");

template <>
sr_status segmented_run_cfg<SR_KEY_F32>(const uint32_t *in, uint32_t *out, size_t n, const int64_t *off, size_t nseg,
                                      cudaStream_t s, bool record, int cfg) {
    return run_k4<SR_KEY_F32>(in, out, n, off, nseg, s, record, cfg);
}

}  // namespace sr
