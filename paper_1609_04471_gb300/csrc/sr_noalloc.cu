// sr_noalloc.cu -- sr_sort_keys_noalloc: the key sort for callers that must
// not allocate device memory.
//
// Who needs it.  sr_sort_keys takes its scratch (a second key buffer, the
// merge-path split table and a small control block) from a stream-ordered
// pool at every call.  Some callers cannot let a library allocate while they
// run: a service that reserves all of its device memory at start-up so that it
// can never fail with out-of-memory in the middle of a request; a host
// framework that owns the device memory and forbids allocations behind its
// back; code on a latency-critical path, where an allocation can stall or
// synchronise.  This entry point gives them the same sort with no allocation
// of any kind: its scratch is one file-scope device array of fixed size, which
// the CUDA runtime creates when it loads this library's device code and which
// every GPU that loads the library keeps until the process exits.
//
// Limits and sharing.
//   * n may be at most SR_NOALLOC_MAX_KEYS (2^20) keys of any key type; larger
//     n returns SR_ERR_INVALID_ARG before anything runs.
//   * All calls on a device share the one array, and it keeps the previous
//     call's contents; each call clears the control block it needs zeroed.
//     Calls whose device work overlaps -- on different streams, or from
//     different host threads without ordering -- race on the array and give
//     wrong results: order them on one stream, or synchronise between them.
//   * The first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make
//     that first call before any stream capture.
//   * sr_get_stats does not describe these calls.
#include <cstring>
#include <mutex>

#include "sr_device.cuh"
#include "sr_kernels.cuh"
#include "sr_plain.cuh"
#include "sr_runtime.cuh"

namespace sr {
namespace {

// Scratch for the largest n of any key type under either merge fan-in:
// PlainSort's own layout function (control block, tile extremes for the pass
// planner, split tables, merge-tile samples, key buffer) evaluated at compile
// time, so a layout that outgrows the array fails the build.
template <int KT> constexpr size_t plain_bytes(bool fan4) {
    return PlainSort<KT, false>::layout(SR_NOALLOC_MAX_KEYS, false, fan4).bytes;
}
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kScratchBytes =
    cmax(cmax(cmax(plain_bytes<SR_KEY_I32>(true), plain_bytes<SR_KEY_I32>(false)),
              cmax(plain_bytes<SR_KEY_U32>(true), plain_bytes<SR_KEY_U32>(false))),
         cmax(cmax(cmax(plain_bytes<SR_KEY_F32>(true), plain_bytes<SR_KEY_F32>(false)),
                   cmax(plain_bytes<SR_KEY_U64>(true), plain_bytes<SR_KEY_U64>(false))),
              cmax(plain_bytes<SR_KEY_I64>(true), plain_bytes<SR_KEY_I64>(false))));
static_assert(plain_bytes<SR_KEY_I32>(true) <= kScratchBytes && plain_bytes<SR_KEY_U64>(true) <= kScratchBytes &&
                  plain_bytes<SR_KEY_I64>(false) <= kScratchBytes,
              "every key type's layout at SR_NOALLOC_MAX_KEYS fits the fixed scratch");
static_assert(kScratchBytes <= (size_t)16 << 20, "the fixed scratch stays modest");

// The scratch itself.  In host code this name is only a host-side stand-in
// for the device symbol; host code must use the address from
// cudaGetSymbolAddress (scratch_base below), never the name.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_base[kMaxDevices];

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
sr_status scratch_base(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SR_ERR_CUDA;
        }
        g_base[dev] = p;
    }
    *out = (unsigned char *)g_base[dev];
    return SR_OK;
}

// The launch sequence of sr_sort_keys (keys only) over the fixed scratch.
template <int KT>
sr_status noalloc_impl(void *d_keys, size_t n, cudaStream_t s, unsigned char *base) {
    typedef PlainSort<KT, false> PS;
    const PS plan(n);
    if (plan.bytes > kScratchBytes) return SR_ERR_INTERNAL;      // excluded at compile time
    return plan.launch((typename PS::T *)d_keys, nullptr, base, s);
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" sr_status sr_sort_keys_noalloc(void *d_keys, size_t n, sr_key_type kt, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > SR_NOALLOC_MAX_KEYS) return SR_ERR_INVALID_ARG;
    if (n > 1 && !d_keys) return SR_ERR_INVALID_ARG;
    if (n > 1 && ((uintptr_t)d_keys % key_bytes_of(kt)) != 0) return SR_ERR_INVALID_ARG;
    if (n < 2) return SR_OK;
    unsigned char *base = nullptr;
    SR_TRY(scratch_base(&base));
    cudaStream_t s = (cudaStream_t)stream;
    switch (kt) {
    case SR_KEY_I32: return noalloc_impl<SR_KEY_I32>(d_keys, n, s, base);
    case SR_KEY_U32: return noalloc_impl<SR_KEY_U32>(d_keys, n, s, base);
    case SR_KEY_F32: return noalloc_impl<SR_KEY_F32>(d_keys, n, s, base);
    case SR_KEY_U64: return noalloc_impl<SR_KEY_U64>(d_keys, n, s, base);
    case SR_KEY_I64: return noalloc_impl<SR_KEY_I64>(d_keys, n, s, base);
    default: return SR_ERR_INVALID_ARG;
    }
}
