// sr_sort.cu -- the plain comparison sort: sr_sort_keys, sr_sort_pairs,
// sr_sort_keys_host and sr_detect_runs.
//
// One call is the fixed launch sequence of sr_plain.cuh on the caller's stream,
// with every data-dependent decision taken on the device (so a call can be
// captured in a CUDA graph).  Scratch comes from the library's stream-ordered
// pool and goes back to it at the end of the call.
#include <algorithm>
#include <cstring>

#include "sr_device.cuh"
#include "sr_kernels.cuh"
#include "sr_plain.cuh"
#include "sr_runtime.cuh"

namespace sr {

// --------------------------------------------------------------- host

template <int KT, bool VALS>
static sr_status sort_impl(void *d_keys, uint32_t *d_vals, size_t n, cudaStream_t s, int call) {
    typedef PlainSort<KT, VALS> PS;
    typedef typename PS::T T;
    const PS plan(n, !VALS && SR_REM_KEYS);
    CallRecord &rec = call_record();
    rec = CallRecord();
    rec.host.call = call;
    rec.host.n = n;
    rec.host.key_type = KT;
    rec.host.tile = PS::TS;
    rec.host.merge_tile = PS::NV;
    rec.stream = s;
    rec.key_bytes = (int)sizeof(T);
    rec.val_bytes = VALS ? 4 : 0;
    if (n < 2) return SR_OK;
    if (plan.passes > MAX_PASSES) return SR_ERR_UNSUPPORTED;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, plan.bytes, s));
    rec.cur0 = plan.passes & 1;
    rec.host.passes_planned = plan.passes;
    sr_status st = plan.launch((T *)d_keys, d_vals, (unsigned char *)scratch, s);
    if (st == SR_OK) {
        if (cudaMemcpyAsync(ds->last_ctrl, scratch, sizeof(Ctrl), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            st = launch_status();
        else
            rec.has_ctrl = true;
    }
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
        SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT, 0, s,
                  (const T *)d_keys, N, ctrl, (const int *)nullptr, (typename K::U *)nullptr, 1);
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

// Copy in, sort, copy out, all on stream s (the device copy is pool scratch,
// freed in stream order).
static sr_status host_sort_enqueue(void *h_keys, size_t n, sr_key_type kt, cudaStream_t s) {
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    const size_t bytes = n * key_bytes_of(kt);
    void *d = nullptr;
    SR_TRY(scratch_alloc(ds, &d, bytes, s));
    sr_status st = SR_OK;
    if (cudaMemcpyAsync(d, h_keys, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) st = launch_status();
    if (st == SR_OK) st = dispatch_sort<false>(d, nullptr, n, kt, s, 1);
    if (st == SR_OK && cudaMemcpyAsync(h_keys, d, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = launch_status();
    scratch_free(d, s);
    return st;
}

extern "C" sr_status sr_sort_keys_host(void *h_keys, size_t n, sr_key_type kt, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && !h_keys) return SR_ERR_INVALID_ARG;
    if (n < 2) return SR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    sr_status st = host_sort_enqueue(h_keys, n, kt, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == SR_OK) st = launch_status();
    return st;
}

extern "C" sr_status sr_sort_keys_host_async(void *h_keys, size_t n, sr_key_type kt, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && !h_keys) return SR_ERR_INVALID_ARG;
    if (n < 2) return SR_OK;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, h_keys) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return SR_ERR_INVALID_ARG;                 // must be page-locked host memory
    }
    return host_sort_enqueue(h_keys, n, kt, (cudaStream_t)stream);
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
