// sr_sort.cu -- the plain comparison sort: sr_sort_keys, sr_sort_pairs,
// sr_sort_keys_host and sr_detect_runs.
//
// One call is the fixed launch sequence of sr_plain.cuh on the caller's stream,
// with every data-dependent decision taken on the device (so a call can be
// captured in a CUDA graph).  Scratch comes from the library's stream-ordered
// pool and goes back to it at the end of the call.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <cstring>

#include "sr_device.cuh"
#include "sr_kernels.cuh"
#include "sr_plain.cuh"
#include "sr_runtime.cuh"

namespace sr {

// ------------------------------------------------- repeated calls as graphs
//
// A call repeated with the same arguments (key type, payloads, n, buffers)
// replays a CUDA graph of its launch sequence: the scan and the whole-input
// paths, a one-thread kernel that reads the call's mode, and a conditional
// node whose body -- the block sort, planner, merge passes and copy-back --
// runs only when the mode is MODE_SORT.  Inputs that a whole-input path
// finishes (sorted, strictly descending, few distinct or few displaced keys)
// then skip the ~2 launches per merge pass whose kernels would return at once.
// The graph owns its scratch.  Not used inside a stream capture, while
// profiling, or with SORTRACE_GRAPHS=0; the first call with new arguments
// takes the ordinary launches.

__global__ void k_sort_cond(cudaGraphConditionalHandle h, const Ctrl *__restrict__ c, long long n) {
    griddep_wait();
    cudaGraphSetConditional(h, call_mode(c, n) == MODE_SORT ? 1u : 0u);
}

namespace {
struct GraphEntry {
    int dev = -1, kt = -1;
    bool vals = false;
    size_t n = 0;
    const void *keys = nullptr, *pay = nullptr;
    unsigned hits = 0;
    bool failed = false;             // the graph could not be built: ordinary launches
    unsigned long long used = 0;     // recency tick
    void *scratch = nullptr;         // owned by the graph
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;           // kernel nodes of the graph (the launch count per replay)
    cudaStream_t last = nullptr;     // stream of the last replay
};
constexpr int kGraphSlots = 16;
constexpr size_t kGraphMinKeys = 1u << 16;
std::mutex g_gmu;
GraphEntry g_graph[kGraphSlots];
unsigned long long g_tick = 0;
cudaStream_t g_cap_stream[2][64];    // per device: the two capture streams

bool graphs_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("SORTRACE_GRAPHS");
        return !(e && e[0] == '0');
    }();
    return on;
}
}  // namespace

// Builds the conditional graph of `plan` over `scratch` (capture on private
// streams; nothing runs).
template <typename PS>
static sr_status build_graph(const PS &plan, typename PS::T *uk, uint32_t *uv, unsigned char *scratch, int dev,
                             cudaGraphExec_t *exec, long long *kernels) {
    cudaStream_t *cs = &g_cap_stream[0][dev], *cb = &g_cap_stream[1][dev];
    if (!*cs && cudaStreamCreateWithFlags(cs, cudaStreamNonBlocking) != cudaSuccess) return launch_status();
    if (!*cb && cudaStreamCreateWithFlags(cb, cudaStreamNonBlocking) != cudaSuccess) return launch_status();
    const unsigned long long l0 = sr_launch_count();
    cudaGraph_t g = nullptr;
    sr_status st = SR_OK;
    if (cudaStreamBeginCapture(*cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) return launch_status();
    do {
        cudaStreamCaptureStatus cst;
        if (cudaStreamGetCaptureInfo(*cs, &cst, nullptr, &g) != cudaSuccess) { st = launch_status(); break; }
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) { st = launch_status(); break; }
        if ((st = plan.launch_prefix(uk, uv, scratch, *cs)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_PARTITION, k_sort_cond, 1, 32, 0, *cs, h, (const Ctrl *)(scratch + plan.off_ctrl),
                  (long long)plan.n);
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edata = nullptr;
        size_t ndeps = 0;
        if (cudaStreamGetCaptureInfo(*cs, &cst, nullptr, &g, &deps, &edata, &ndeps) != cudaSuccess) {
            st = launch_status();
            break;
        }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        if (cudaGraphAddNode(&cnode, g, deps, edata, ndeps, &cp) != cudaSuccess) { st = launch_status(); break; }
        if (cudaStreamBeginCaptureToGraph(*cb, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            st = launch_status();
            break;
        }
        st = plan.launch_sort(uk, uv, scratch, *cb);
        cudaGraph_t body = nullptr;
        if (cudaStreamEndCapture(*cb, &body) != cudaSuccess && st == SR_OK) st = launch_status();
        if (st != SR_OK) break;
        if (cudaStreamUpdateCaptureDependencies(*cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) !=
            cudaSuccess) {
            st = launch_status();
            break;
        }
    } while (0);
    cudaGraph_t done = nullptr;
    if (cudaStreamEndCapture(*cs, &done) != cudaSuccess && st == SR_OK) st = launch_status();
    if (st == SR_OK && cudaGraphInstantiate(exec, done, 0) != cudaSuccess) st = launch_status();
    if (done) cudaGraphDestroy(done);
    cudaGetLastError();
    *kernels = (long long)(sr_launch_count() - l0);
    count_launches(-*kernels);                   // captured, not launched
    return st;
}

// Replays (or builds, on the second identical call) the graph of this call.
// Returns SR_OK with *done = true when the call went through a graph.
template <int KT, bool VALS>
static sr_status graph_call(const PlainSort<KT, VALS> &plan, int kt, void *d_keys, uint32_t *d_vals, cudaStream_t s,
                            DeviceState *ds, bool *done) {
    typedef PlainSort<KT, VALS> PS;
    *done = false;
    if (!graphs_enabled() || plan.n < (long long)kGraphMinKeys || profiling_on()) return SR_OK;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess || cst != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return SR_OK;
    }
    std::lock_guard<std::mutex> lock(g_gmu);
    GraphEntry *e = nullptr, *victim = &g_graph[0];
    for (auto &x : g_graph) {
        if (x.hits && x.dev == ds->device && x.kt == kt && x.vals == VALS && x.n == (size_t)plan.n &&
            x.keys == d_keys && x.pay == d_vals) {
            e = &x;
            break;
        }
        if (!x.hits || x.used < victim->used) victim = &x;
    }
    ++g_tick;
    if (!e) {                                    // first sight: remember, launch ordinarily
        if (victim->exec) {
            if (victim->last) cudaStreamSynchronize(victim->last);
            cudaGraphExecDestroy(victim->exec);
        }
        if (victim->scratch) scratch_free(victim->scratch, victim->last ? victim->last : s);
        *victim = GraphEntry();
        victim->dev = ds->device; victim->kt = kt; victim->vals = VALS; victim->n = (size_t)plan.n;
        victim->keys = d_keys; victim->pay = d_vals; victim->hits = 1; victim->used = g_tick;
        return SR_OK;
    }
    e->used = g_tick;
    if (e->failed) return SR_OK;
    if (!e->exec) {
        void *scratch = nullptr;
        SR_TRY(scratch_alloc(ds, &scratch, plan.bytes, s));
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;
        const sr_status st = build_graph(plan, (typename PS::T *)d_keys, d_vals, (unsigned char *)scratch,
                                         ds->device, &exec, &kernels);
        if (st != SR_OK) {                       // fall back to the ordinary launches for good
            if (exec) cudaGraphExecDestroy(exec);
            scratch_free(scratch, s);
            e->failed = true;
            return SR_OK;
        }
        e->exec = exec;
        e->scratch = scratch;
        e->kernels = kernels;
    }
    if (cudaGraphLaunch(e->exec, s) != cudaSuccess) return launch_status();
    e->last = s;
    count_launches(e->kernels);
    if (cudaMemcpyAsync(ds->last_ctrl, (unsigned char *)e->scratch + plan.off_ctrl, sizeof(Ctrl),
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return launch_status();
    *done = true;
    return SR_OK;
}

// --------------------------------------------------------------- host

template <int KT, bool VALS>
static sr_status sort_impl(void *d_keys, uint32_t *d_vals, size_t n, cudaStream_t s, int call, bool graphs) {
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
    rec.cur0 = plan.passes & 1;
    rec.host.passes_planned = plan.passes;
    if (graphs) {                                // caller's buffers: a repeated call replays its graph
        bool done = false;
        SR_TRY(graph_call(plan, KT, d_keys, d_vals, s, ds, &done));
        if (done) {
            rec.has_ctrl = true;
            return SR_OK;
        }
    }
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, plan.bytes, s));
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
                               cudaStream_t s, int call, bool graphs) {
    switch (kt) {
    case SR_KEY_I32: return sort_impl<SR_KEY_I32, VALS>(d_keys, d_vals, n, s, call, graphs);
    case SR_KEY_U32: return sort_impl<SR_KEY_U32, VALS>(d_keys, d_vals, n, s, call, graphs);
    case SR_KEY_F32: return sort_impl<SR_KEY_F32, VALS>(d_keys, d_vals, n, s, call, graphs);
    case SR_KEY_U64: return sort_impl<SR_KEY_U64, VALS>(d_keys, d_vals, n, s, call, graphs);
    case SR_KEY_I64: return sort_impl<SR_KEY_I64, VALS>(d_keys, d_vals, n, s, call, graphs);
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
    return dispatch_sort<false>(d_keys, nullptr, n, kt, (cudaStream_t)stream, 1, true);
}

extern "C" sr_status sr_sort_pairs(void *d_keys, uint32_t *d_vals, size_t n, sr_key_type kt,
                                   sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && (!d_keys || !d_vals)) return SR_ERR_INVALID_ARG;
    if (n > 1 && (((uintptr_t)d_keys % key_bytes_of(kt)) != 0 || ((uintptr_t)d_vals % 4) != 0))
        return SR_ERR_INVALID_ARG;
    return dispatch_sort<true>(d_keys, d_vals, n, kt, (cudaStream_t)stream, 2, true);
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
    if (st == SR_OK) st = dispatch_sort<false>(d, nullptr, n, kt, s, 1, false);
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
