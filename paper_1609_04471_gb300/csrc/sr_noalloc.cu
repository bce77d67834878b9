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
#include "sr_runtime.cuh"

namespace sr {
namespace {

// Layout of the scratch array: [control block | split table | key buffer].
constexpr size_t kCtrlBytes = 256;
constexpr size_t kMinMergeTile = Shape<8, false>::NT * Shape<8, false>::IPT;   // 2816 keys
constexpr size_t kSplitBytes =
    ((SR_NOALLOC_MAX_KEYS + kMinMergeTile - 1) / kMinMergeTile + 1) * 8 + 255 & ~size_t(255);
constexpr size_t kKeyBytes = (size_t)SR_NOALLOC_MAX_KEYS * 8;
constexpr size_t kScratchBytes = kCtrlBytes + kSplitBytes + kKeyBytes;
static_assert(sizeof(Ctrl) <= kCtrlBytes, "control block does not fit");

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
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    typedef Shape<sizeof(T), false> S;
    constexpr int NT = S::NT, IPT = S::IPT, SNT = S::SORT_NT;
    constexpr int NV = NT * IPT;
    constexpr int TS = SNT * IPT;
    // every kernel below fits the default 48 KB of dynamic shared memory
    static_assert((TS + 1) * sizeof(U) <= 48 * 1024, "detect tile too large");
    static_assert(TS * sizeof(U) <= 48 * 1024, "block-sort tile too large");
    static_assert((NV + 16) * sizeof(U) <= 48 * 1024, "merge tile too large");
    if (n < 2) return SR_OK;
    const long long N = (long long)n;
    const long long tiles = (N + TS - 1) / TS;
    const int P = ceil_log2((unsigned long long)tiles);
    const long long mtiles = (N + NV - 1) / NV;
    if ((size_t)(mtiles + 1) * 8 > kSplitBytes || n * sizeof(T) > kKeyBytes) return SR_ERR_INVALID_ARG;
    Ctrl *ctrl = (Ctrl *)base;
    long long *splits = (long long *)(base + kCtrlBytes);
    T *sk = (T *)(base + kCtrlBytes + kSplitBytes);
    T *uk = (T *)d_keys;
    const int cur0 = P & 1;
    const bool vec = ((uintptr_t)uk % 16) == 0;      // the scratch array is 256-byte aligned
    sr_status st = SR_OK;
    do {
        // the array keeps the previous call's contents: zero the counters
        if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) { st = launch_status(); break; }
        SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT,
                  (size_t)(TS + 1) * sizeof(U), s, uk, N, ctrl);
        SR_LAUNCH(SR_KERNEL_REVERSE, (k_reverse<KT, false>), (unsigned)((N / 2 + 255) / 256 > 0 ? (N / 2 + 255) / 256 : 1),
                  256, 0, s, uk, (uint32_t *)nullptr, N, ctrl);
        SR_LAUNCH(SR_KERNEL_BLOCK_SORT, (k_block_sort<KT, SNT, IPT, false>), (unsigned)tiles, SNT,
                  (size_t)TS * sizeof(U), s, uk, (const uint32_t *)nullptr, cur0 ? sk : uk,
                  (uint32_t *)nullptr, N, ctrl);
        for (int p = 0; p < P; ++p) {
            const long long w = (long long)TS << p;
            const long long nb = mtiles + 1;
            SR_LAUNCH(SR_KERNEL_PARTITION, (k_partition<KT>), (unsigned)((nb + 7) / 8), 256, 0, s,
                      uk, sk, N, w, NV, nb, splits, ctrl, cur0, p);
            if (vec) {
                SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, false, true>), (unsigned)mtiles, NT,
                          (size_t)(NV + 16) * sizeof(U), s, uk, (uint32_t *)nullptr, sk, (uint32_t *)nullptr,
                          N, w, splits, ctrl, cur0, p);
            } else {
                SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, false, false>), (unsigned)mtiles, NT,
                          (size_t)(NV + 16) * sizeof(U), s, uk, (uint32_t *)nullptr, sk, (uint32_t *)nullptr,
                          N, w, splits, ctrl, cur0, p);
            }
        }
        if (st != SR_OK) break;
        if (P > 0) {
            SR_LAUNCH(SR_KERNEL_COPY, (k_copy_back<KT, false>), (unsigned)((N + 255) / 256), 256, 0, s,
                      uk, (uint32_t *)nullptr, sk, (const uint32_t *)nullptr, N, ctrl, cur0, P);
        }
    } while (0);
    return st;
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
