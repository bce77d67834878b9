// sr_sort.cu -- the plain comparison sort: sr_sort_keys, sr_sort_pairs,
// sr_sort_keys_host and sr_detect_runs.
//
// One call is a fixed launch sequence on the caller's stream, with every
// data-dependent decision taken on the device (so a call can be captured in a
// CUDA graph):
//
//   k_detect     run-detection scan (Section 2's Run(A); Section 3 process 1):
//                counts descents and non-descents of neighbour pairs.
//   k_reverse    if every pair strictly descends, reverse the whole array in
//                one read + write (Section 3 technique (a); Section 4's remark
//                that sorted and reversely sorted lists take O(n)).
//   k_block_sort sort each tile of SORT_NT*IPT keys in shared memory; a tile
//                that is already ascending is left alone, a strictly
//                descending one is reversed (techniques (a), (b); Section 4 (f)).
//   per merge pass p (run width w = tile << p), policy e1 of Section 3:
//     k_partition  merge-path split of every output tile of NT*IPT keys, and a
//                  count of run pairs whose runs overlap (A.last > B.first);
//                  a pass where no pair overlaps is skipped -- nothing moves
//                  (technique (f) applied to whole passes).
//     k_merge      each CTA stages its A and B ranges in shared memory and
//                  merges them, IPT outputs per thread, stably.
//   k_copy_back  if skipped passes left the result in scratch, copy it home.
//
// If every pair is in order (the input is sorted) nothing after the scan moves
// any data.
#include <algorithm>
#include <cstring>

#include "sr_device.cuh"
#include "sr_kernels.cuh"
#include "sr_runtime.cuh"

namespace sr {

// --------------------------------------------------------------- host

static int grid_for(long long work, int per_block, int cap) {
    long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename F>
static sr_status allow_smem(F *kernel, size_t bytes) {
    if (bytes > 48 * 1024) {
        if (cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return launch_status();
    }
    return SR_OK;
}

template <int KT, bool VALS>
static sr_status sort_impl(void *d_keys, uint32_t *d_vals, size_t n, cudaStream_t s, int call) {
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    typedef Shape<sizeof(T), VALS> S;
    constexpr int NT = S::NT, IPT = S::IPT, SNT = S::SORT_NT;
    constexpr int NV = NT * IPT;    // keys per merge CTA
    constexpr int TS = SNT * IPT;   // keys per block-sort tile
    static_assert(TS % NV == 0, "sort tile must be a whole number of merge tiles");

    CallRecord &rec = call_record();
    rec = CallRecord();
    rec.host.call = call;
    rec.host.n = n;
    rec.host.key_type = KT;
    rec.host.tile = TS;
    rec.host.merge_tile = NV;
    rec.stream = s;
    rec.key_bytes = (int)sizeof(T);
    rec.val_bytes = VALS ? 4 : 0;
    if (n < 2) return SR_OK;

    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    const long long N = (long long)n;
    const long long tiles = (N + TS - 1) / TS;
    const int P = ceil_log2((unsigned long long)tiles);
    if (P > MAX_PASSES) return SR_ERR_UNSUPPORTED;
    const long long mtiles = (N + NV - 1) / NV;
    const size_t kbytes = align_up(n * sizeof(T), 256);
    const size_t vbytes = VALS ? align_up(n * 4, 256) : 0;
    const size_t sbytes = align_up((size_t)(mtiles + 1) * 8, 256);
    const size_t cbytes = align_up(sizeof(Ctrl), 256);
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, (P > 0 ? kbytes + vbytes + sbytes : 0) + cbytes, s));
    unsigned char *sp = (unsigned char *)scratch;
    Ctrl *ctrl = (Ctrl *)sp;
    T *sk = (T *)(sp + cbytes);
    uint32_t *sv = (uint32_t *)(sp + cbytes + kbytes);
    long long *splits = (long long *)(sp + cbytes + kbytes + vbytes);
    T *uk = (T *)d_keys;
    uint32_t *uv = d_vals;
    const int cur0 = P & 1;          // the block sort writes where the last pass must not
    rec.cur0 = cur0;
    rec.host.passes_planned = P;

    sr_status st = SR_OK;
    do {
        if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) { st = launch_status(); break; }
        const size_t det_smem = (size_t)(TS + 1) * sizeof(U);
        if ((st = allow_smem(k_detect<KT, SNT, IPT>, det_smem)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT, det_smem, s,
                  uk, N, ctrl);
        SR_LAUNCH(SR_KERNEL_REVERSE, (k_reverse<KT, VALS>), grid_for(N / 2, 256, 152 * 16), 256, 0, s,
                  uk, uv, N, ctrl);
        const size_t bs_smem = (size_t)TS * (sizeof(U) + (VALS ? 4 : 0));
        if ((st = allow_smem(k_block_sort<KT, SNT, IPT, VALS>, bs_smem)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_BLOCK_SORT, (k_block_sort<KT, SNT, IPT, VALS>), (unsigned)tiles, SNT,
                  bs_smem, s, uk, uv, cur0 ? sk : uk, cur0 ? sv : uv, N, ctrl);
        const size_t m_smem = (size_t)(NV + 16) * (sizeof(U) + (VALS ? 4 : 0));
        const bool vec = ((uintptr_t)uk % 16) == 0 && (!VALS || ((uintptr_t)uv % 16) == 0);
        if ((st = allow_smem(k_merge<KT, NT, IPT, VALS, true>, m_smem)) != SR_OK) break;
        if ((st = allow_smem(k_merge<KT, NT, IPT, VALS, false>, m_smem)) != SR_OK) break;
        for (int p = 0; p < P; ++p) {
            const long long w = (long long)TS << p;
            const long long nb = mtiles + 1;
            SR_LAUNCH(SR_KERNEL_PARTITION, (k_partition<KT>), (unsigned)((nb + 7) / 8), 256, 0, s,
                      uk, sk, N, w, NV, nb, splits, ctrl, cur0, p);
            if (vec) {
                SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS, true>), (unsigned)mtiles, NT, m_smem,
                          s, uk, uv, sk, sv, N, w, splits, ctrl, cur0, p);
            } else {
                SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS, false>), (unsigned)mtiles, NT, m_smem,
                          s, uk, uv, sk, sv, N, w, splits, ctrl, cur0, p);
            }
        }
        if (st != SR_OK) break;
        if (P > 0) {
            SR_LAUNCH(SR_KERNEL_COPY, (k_copy_back<KT, VALS>), grid_for(N, 256, 152 * 16), 256, 0, s,
                      uk, uv, sk, sv, N, ctrl, cur0, P);
        }
        if (cudaMemcpyAsync(ds->last_ctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess) {
            st = launch_status();
            break;
        }
        rec.has_ctrl = true;
    } while (0);
    scratch_free(scratch, s);
    return st;
}

template <bool VALS>
static sr_status dispatch_sort(void *d_keys, uint32_t *d_vals, size_t n, sr_key_type kt,
                               cudaStream_t s, int call) {
    switch (kt) {
    case SR_KEY_I32: return sort_impl<SR_KEY_I32, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_U32: return sort_impl<SR_KEY_U32, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_F32: return sort_impl<SR_KEY_F32, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_U64: return sort_impl<SR_KEY_U64, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_I64: return sort_impl<SR_KEY_I64, VALS>(d_keys, d_vals, n, s, call);
    default: return SR_ERR_INVALID_ARG;
    }
}

template <int KT>
static sr_status detect_impl(const void *d_keys, size_t n, sr_run_info *out, cudaStream_t s) {
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef Shape<sizeof(T), false> S;
    constexpr int SNT = S::SORT_NT, IPT = S::IPT, TS = SNT * IPT;
    std::memset(out, 0, sizeof(*out));
    out->n = n;
    out->tile = TS;
    if (n == 0) return SR_OK;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    const long long N = (long long)n;
    const long long tiles = (N + TS - 1) / TS;
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, sizeof(Ctrl), s));
    Ctrl *ctrl = (Ctrl *)scratch;
    Ctrl h;
    sr_status st = SR_OK;
    do {
        if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) { st = launch_status(); break; }
        const size_t smem = (size_t)(TS + 1) * sizeof(typename K::U);
        if ((st = allow_smem(k_detect<KT, SNT, IPT>, smem)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT, smem, s,
                  (const T *)d_keys, N, ctrl);
        if (cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = launch_status();
            if (st == SR_OK) st = SR_ERR_CUDA;
            break;
        }
        out->runs = h.descents + 1;
        out->sorted = h.descents == 0;
        out->strictly_descending = (h.nondescents == 0 && n > 1) || n == 1;
        out->tiles = (uint64_t)tiles;
        out->tiles_ascending = h.tiles_ascending;
        out->tiles_descending = h.tiles_descending;
    } while (0);
    scratch_free(scratch, s);
    return st;
}

}  // namespace sr

using namespace sr;

extern "C" sr_status sr_sort_keys(void *d_keys, size_t n, sr_key_type kt, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && !d_keys) return SR_ERR_INVALID_ARG;
    if (n > 1 && ((uintptr_t)d_keys % key_bytes_of(kt)) != 0) return SR_ERR_INVALID_ARG;
    return dispatch_sort<false>(d_keys, nullptr, n, kt, (cudaStream_t)stream, 1);
}

extern "C" sr_status sr_sort_pairs(void *d_keys, uint32_t *d_vals, size_t n, sr_key_type kt,
                                   sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && (!d_keys || !d_vals)) return SR_ERR_INVALID_ARG;
    if (n > 1 && (((uintptr_t)d_keys % key_bytes_of(kt)) != 0 || ((uintptr_t)d_vals % 4) != 0))
        return SR_ERR_INVALID_ARG;
    return dispatch_sort<true>(d_keys, d_vals, n, kt, (cudaStream_t)stream, 2);
}

extern "C" sr_status sr_sort_keys_host(void *h_keys, size_t n, sr_key_type kt, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && !h_keys) return SR_ERR_INVALID_ARG;
    if (n < 2) return SR_OK;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = n * key_bytes_of(kt);
    void *d = nullptr;
    SR_TRY(scratch_alloc(ds, &d, bytes, s));
    sr_status st = SR_OK;
    if (cudaMemcpyAsync(d, h_keys, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) st = launch_status();
    if (st == SR_OK) st = dispatch_sort<false>(d, nullptr, n, kt, s, 1);
    if (st == SR_OK && cudaMemcpyAsync(h_keys, d, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = launch_status();
    scratch_free(d, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == SR_OK) st = launch_status();
    return st;
}

extern "C" sr_status sr_detect_runs(const void *d_keys, size_t n, sr_key_type kt, sr_run_info *out,
                                    sr_stream stream) {
    if (!valid_key_type(kt) || !out) return SR_ERR_INVALID_ARG;
    if (n > 0 && !d_keys) return SR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    switch (kt) {
    case SR_KEY_I32: return detect_impl<SR_KEY_I32>(d_keys, n, out, s);
    case SR_KEY_U32: return detect_impl<SR_KEY_U32>(d_keys, n, out, s);
    case SR_KEY_F32: return detect_impl<SR_KEY_F32>(d_keys, n, out, s);
    case SR_KEY_U64: return detect_impl<SR_KEY_U64>(d_keys, n, out, s);
    case SR_KEY_I64: return detect_impl<SR_KEY_I64>(d_keys, n, out, s);
    default: return SR_ERR_INVALID_ARG;
    }
}
