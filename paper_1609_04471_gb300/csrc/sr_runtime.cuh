// sr_runtime.cuh -- host-side runtime shared by the sort entry points:
// per-device state (a stream-ordered scratch pool, the device status word,
// the last call's control block), thread-local call statistics and error
// mapping.  Nothing here is on the device's hot path.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sortrace.h"
#include "sr_device.cuh"

namespace sr {

struct DeviceState {
    int device = -1;
    cudaMemPool_t pool = nullptr;   // scratch: stream-ordered, kept cached
    int *status = nullptr;          // device status word (sr_status codes)
    Ctrl *last_ctrl = nullptr;      // copy of the last call's control block
    void *last_aux = nullptr;       // copy of the last segmented / learned call's control block
};
constexpr size_t kAuxBytes = 2048;

// Per-device state of the current device, created on first use (the first
// call on a device must not be inside a stream capture).
sr_status device_state(DeviceState **out);

// Scratch of `bytes` from the device pool, ordered on `s`.  Honours the
// SR_INJECT_OOM environment variable (any non-empty value but "0") by failing
// with SR_ERR_OOM, so the error path can be tested without exhausting memory.
sr_status scratch_alloc(DeviceState *ds, void **p, size_t bytes, cudaStream_t s);
void scratch_free(void *p, cudaStream_t s);

// Maps the last CUDA error to a status (and clears it).
sr_status launch_status();

// Thread-local record of the last call, completed by sr_get_stats.
struct CallRecord {
    sr_stats host;                  // fields known on the host
    cudaStream_t stream = nullptr;
    bool has_ctrl = false;          // last_ctrl holds this call's control block
    int key_bytes = 4;
    int val_bytes = 0;
    int cur0 = 0;
    int aux_kind = 0;               // 3: last_aux holds a segmented call's block, 4: a learned call's
};

// The segmented sort from `in` to `out` (in == out: in place) under launch
// configuration `cfg` (an index into the configurations of the key width;
// sr_seg_k4.cu / sr_seg_k8.cu); `record` makes it this thread's last call for
// sr_get_stats.  SR_ERR_INVALID_ARG for an unknown cfg.
template <int KT>
sr_status segmented_run_cfg(const typename Key<KT>::T *in, typename Key<KT>::T *out, size_t n_keys,
                            const int64_t *d_off, size_t nseg, cudaStream_t s, bool record, int cfg);
// Configurations of the segmented sort per key width, and the two defaults:
// small segments in packs (general batches) and one CTA per small segment
// (segments of moderate, similar sizes such as learned buckets).
int segmented_num_configs(int key_bytes);
inline int segmented_default_cfg(int key_bytes, bool buckets) {
    // buckets: 4-byte keys take the ladder sized for learned buckets (~2,048 keys)
    return buckets ? (key_bytes == 4 ? 7 : 2) : 0;
}

// Fill the stats fields of a segmented / learned call from its control block.
sr_status segmented_stats(const void *aux, sr_stats *out);
sr_status learned_stats(const void *aux, sr_stats *out);
CallRecord &call_record();

// Whether per-launch profiling is on for this thread (sr_profile_begin), and
// an adjustment of the launch count (graph replays count their kernels).
bool profiling_on();
void count_launches(long long k);
unsigned long long host_launch_count();     // the launches counted on the host
unsigned long long thread_launch_count();   // ... by this host thread
// Kernels that graph replays ran beyond those counted on the host (read on
// the device after it finishes its queued work; 0 if no graph ran).
unsigned long long graph_kernel_count();

// Graph conditional nodes (sr_sort.cu), for launch sequences that branch on
// the device inside a stream capture: a handle in the graph that s is
// capturing into; and a conditional node of `type` with `size` bodies
// (returned in bodies) after s's current capture dependencies, which then
// becomes the capture's only dependency.
sr_status new_handle(cudaStream_t s, cudaGraphConditionalHandle *h);
sr_status add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                          unsigned size, cudaGraph_t *bodies);

// Captures `fn(cb)` into the graph `body` on stream cb (which must not be
// capturing); *kernels = the kernels it launched.
template <typename F>
sr_status capture_into(cudaGraph_t body, cudaStream_t cb, F fn, unsigned int *kernels) {
    const unsigned long long l0 = thread_launch_count();
    if (cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return launch_status();
    sr_status st = fn(cb);
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(cb, &out) != cudaSuccess && st == SR_OK) st = launch_status();
    *kernels = (unsigned int)(thread_launch_count() - l0);
    return st;
}

// Kernel instrumentation: every launch site calls launch_begin / launch_end
// around its <<<>>> (see SR_LAUNCH).
void launch_begin(int kind, cudaStream_t s);
sr_status launch_end(int kind, cudaStream_t s);

size_t align_up(size_t x, size_t a);
// Streaming multiprocessors of the current device (looked up once per device;
// 152 if the query fails).
int device_sm_count();
int ceil_log2(unsigned long long x);
size_t key_bytes_of(sr_key_type kt);
bool valid_key_type(int kt);

}  // namespace sr

#define SR_TRY(expr)                               \
    do {                                           \
        sr_status _st = (expr);                    \
        if (_st != SR_OK) return _st;              \
    } while (0)

namespace sr {
// Whether launches use programmatic dependent launch (on unless the
// environment variable SR_PDL is "0").
bool pdl_enabled();

// Launches kernel on stream s.  With programmatic dependent launch the
// kernel's CTAs may be scheduled while the previous kernel on the stream is
// still finishing; every kernel of the library therefore begins with
// griddep_wait() (see sr_device.cuh) before it touches memory the previous
// kernel wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}
}  // namespace sr

// Launches `kernel` with (grid, block, smem, stream, args...), counts it,
// times it when profiling is on, and breaks out of the enclosing loop with the
// status in `st` if the launch failed.
#define SR_LAUNCH(kind, kernel, grid, block, smem, stream, ...)                              \
    {                                                                                         \
        ::sr::launch_begin((kind), (stream));                                                 \
        ::sr::launch_kernel(kernel, dim3(grid), dim3(block), (smem), (stream), __VA_ARGS__);  \
        st = ::sr::launch_end((kind), (stream));                                              \
        if (st != SR_OK) break;                                                               \
    }

#define SR_LAUNCHED()                              \
    do {                                           \
        sr_status _st = ::sr::launch_status();     \
        if (_st != SR_OK) return _st;              \
    } while (0)
