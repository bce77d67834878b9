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
// replays a CUDA graph of its launch sequence.  After the scan, a one-thread
// kernel reads the call's state and picks one branch of a switch node:
//   0 sorted input: nothing more;
//   1 strictly descending: the reversal;
//   2 a few-distinct-keys candidate: count and write (then the few-displaced-
//     keys path and the sort section behind an IF node, for a candidate the
//     count rejects);
//   3 few displaced keys: that path, then the sort section behind an IF node
//     (for a bucket overflow);
//   4 the sort section.
// Inputs a whole-input path finishes so skip every launch of the other
// paths and the ~2 launches per merge pass.  The graph owns its scratch.  Not
// used inside a stream capture, while profiling, or with SORTRACE_GRAPHS=0;
// the first call with new arguments takes the ordinary launches.  The
// deciding kernels add the kernels of the branch they pick to a device
// counter that sr_launch_count reads.

__device__ unsigned long long g_branch_kernels;

struct BranchKernels {
    unsigned int reverse, few_rem, rem, sort;
};

__global__ void k_route(cudaGraphConditionalHandle h, const Ctrl *__restrict__ c, long long n, long long rtiles,
                        long long dmax, int rem, BranchKernels k) {
    griddep_wait();
    if (threadIdx.x != 0) return;                 // one setter of the condition
    unsigned int v, cnt;
    if (c->descents == 0) { v = 0; cnt = 0; }
    else if (c->nondescents == 0 && n > 1) { v = 1; cnt = k.reverse; }
    else if (c->few_cand) { v = 2; cnt = k.few_rem; }
    else if (rem && 2 * c->descents >= (unsigned long long)rtiles && c->descents <= (unsigned long long)dmax) {
        v = 3;
        cnt = k.rem;
    } else { v = 4; cnt = k.sort; }
    cudaGraphSetConditional(h, v);
    if (cnt) atomicAdd(&g_branch_kernels, (unsigned long long)cnt);
}

__global__ void k_sort_cond(cudaGraphConditionalHandle h, const Ctrl *__restrict__ c, long long n,
                            unsigned int sort_kernels) {
    griddep_wait();
    if (threadIdx.x != 0) return;                 // one setter of the condition
    const bool go = call_mode(c, n) == MODE_SORT;
    cudaGraphSetConditional(h, go ? 1u : 0u);
    if (go) atomicAdd(&g_branch_kernels, (unsigned long long)sort_kernels);
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
    long long kernels = 0;           // kernels every replay runs (the rest is counted on the device)
    cudaEvent_t done = nullptr;      // recorded after every replay
};
constexpr int kGraphSlots = 16;
constexpr size_t kGraphMinKeys = 1u << 16;
constexpr int kMaxDev = 64;
std::mutex g_gmu;
GraphEntry g_graph[kGraphSlots];
unsigned long long g_tick = 0;
cudaStream_t g_cap_stream[3][kMaxDev];   // per device: capture streams (top, branch, nested)
bool g_graph_used[kMaxDev];

bool graphs_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("SORTRACE_GRAPHS");
        return !(e && e[0] == '0');
    }();
    return on;
}
}  // namespace

// Adds a conditional node of `type` with `size` bodies after the current
// capture dependencies of s, and makes it the capture's only dependency.
sr_status add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                          unsigned size, cudaGraph_t *bodies) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &edata, &ndeps) != cudaSuccess) return launch_status();
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = size;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, edata, ndeps, &cp) != cudaSuccess) return launch_status();
    for (unsigned i = 0; i < size; ++i) bodies[i] = cp.conditional.phGraph_out[i];
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
        return launch_status();
    return SR_OK;
}

// A handle for a conditional node in the graph that s is capturing into.
sr_status new_handle(cudaStream_t s, cudaGraphConditionalHandle *h) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &g) != cudaSuccess) return launch_status();
    if (cudaGraphConditionalHandleCreate(h, g, 0, 0) != cudaSuccess) return launch_status();
    return SR_OK;
}

// The kernels fn would launch (captured into a scratch graph and dropped).
template <typename F>
static sr_status count_kernels(cudaStream_t cb, F fn, unsigned int *kernels) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return launch_status();
    const sr_status st = capture_into(g, cb, fn, kernels);
    cudaGraphDestroy(g);
    return st;
}

// Builds the routed graph of `plan` over `scratch` (capture on private
// streams; nothing runs).  *kernels: the kernels every replay runs (the scan
// and the router; the rest is counted on the device).
template <typename PS>
static sr_status build_graph(const PS &plan, typename PS::T *uk, uint32_t *uv, unsigned char *scratch, int dev,
                             cudaGraphExec_t *exec, long long *kernels) {
    cudaStream_t cs[3];
    for (int i = 0; i < 3; ++i) {
        if (!g_cap_stream[i][dev] &&
            cudaStreamCreateWithFlags(&g_cap_stream[i][dev], cudaStreamNonBlocking) != cudaSuccess)
            return launch_status();
        cs[i] = g_cap_stream[i][dev];
    }
    const Ctrl *ctrl = (const Ctrl *)(scratch + plan.off_ctrl);
    const long long n = plan.n;
    const unsigned long long l_start = thread_launch_count();
    auto part = [&](int parts) { return [&, parts](cudaStream_t x) {
        return plan.launch_prefix(uk, uv, scratch, x, nullptr, parts); }; };
    auto sort = [&](cudaStream_t x) { return plan.launch_sort(uk, uv, scratch, x); };
    // kernels per part, for the device-side count
    unsigned int k_scan = 0, k_rev = 0, k_few = 0, k_rem = 0, k_sort = 0;
    sr_status st = count_kernels(cs[1], part(PS::PART_SCAN), &k_scan);
    if (st == SR_OK) st = count_kernels(cs[1], part(PS::PART_REVERSE), &k_rev);
    if (st == SR_OK) st = count_kernels(cs[1], part(PS::PART_FEW), &k_few);
    if (st == SR_OK) st = count_kernels(cs[1], part(PS::PART_REM), &k_rem);
    if (st == SR_OK) st = count_kernels(cs[1], sort, &k_sort);
    // a branch body: `parts` of the prefix, then the sort section behind an
    // IF node that a one-thread kernel sets from the call's mode
    auto guarded = [&](int parts) { return [&, parts](cudaStream_t x) -> sr_status {
        sr_status s2 = plan.launch_prefix(uk, uv, scratch, x, nullptr, parts);
        cudaGraphConditionalHandle hi;
        if (s2 == SR_OK) s2 = new_handle(x, &hi);
        if (s2 != SR_OK) return s2;
        do {
            sr_status &st = s2;     // SR_LAUNCH reports into `st`
            SR_LAUNCH(SR_KERNEL_PARTITION, k_sort_cond, 1, 32, 0, x, hi, ctrl, n, k_sort);
        } while (0);
        cudaGraph_t ifb[1];
        if (s2 == SR_OK) s2 = add_conditional(x, hi, cudaGraphCondTypeIf, 1, ifb);
        unsigned int k = 0;
        if (s2 == SR_OK) s2 = capture_into(ifb[0], cs[2], sort, &k);
        return s2;
    }; };
    if (st != SR_OK) return st;
    if (cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeRelaxed) != cudaSuccess) return launch_status();
    do {
        if ((st = plan.launch_prefix(uk, uv, scratch, cs[0], nullptr, PS::PART_SCAN)) != SR_OK) break;
        cudaGraphConditionalHandle hs;
        if ((st = new_handle(cs[0], &hs)) != SR_OK) break;
        const BranchKernels bk = {k_rev, k_few + k_rem + 1, k_rem + 1, k_sort};
        SR_LAUNCH(SR_KERNEL_PARTITION, k_route, 1, 32, 0, cs[0], hs, ctrl, n, plan.rtiles, plan.rem_dmax,
                  plan.rem ? 1 : 0, bk);
        cudaGraph_t br[5];
        if ((st = add_conditional(cs[0], hs, cudaGraphCondTypeSwitch, 5, br)) != SR_OK) break;
        cudaGraphNode_t empty;
        if (cudaGraphAddEmptyNode(&empty, br[0], nullptr, 0) != cudaSuccess) { st = launch_status(); break; }
        unsigned int k = 0;
        if ((st = capture_into(br[1], cs[1], part(PS::PART_REVERSE), &k)) != SR_OK) break;
        if ((st = capture_into(br[2], cs[1], guarded(PS::PART_FEW | PS::PART_REM), &k)) != SR_OK) break;
        if (plan.rem) {
            if ((st = capture_into(br[3], cs[1], guarded(PS::PART_REM), &k)) != SR_OK) break;
        } else if (cudaGraphAddEmptyNode(&empty, br[3], nullptr, 0) != cudaSuccess) {
            st = launch_status();
            break;
        }
        if ((st = capture_into(br[4], cs[1], sort, &k)) != SR_OK) break;
    } while (0);
    cudaGraph_t done = nullptr;
    if (cudaStreamEndCapture(cs[0], &done) != cudaSuccess && st == SR_OK) st = launch_status();
    if (st == SR_OK && cudaGraphInstantiate(exec, done, 0) != cudaSuccess) st = launch_status();
    if (done) cudaGraphDestroy(done);
    cudaGetLastError();
    count_launches(-(long long)(thread_launch_count() - l_start));  // captured, not launched
    *kernels = (long long)k_scan + 1;                                // the scan kernels and the router
    return st;
}

// Drops every cached graph of the current device and returns its scratch.
static sr_status graph_cache_clear() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return launch_status();
    std::lock_guard<std::mutex> lock(g_gmu);
    sr_status st = SR_OK;
    for (auto &x : g_graph) {
        if (!x.hits || x.dev != dev) continue;
        if (x.done && cudaEventSynchronize(x.done) != cudaSuccess) st = launch_status();
        if (x.exec) cudaGraphExecDestroy(x.exec);
        scratch_free(x.scratch, nullptr);           // idle now: its last replay has finished
        if (x.done) cudaEventDestroy(x.done);
        x = GraphEntry();
    }
    return st;
}

unsigned long long graph_kernel_count() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 0;
    }
    {
        std::lock_guard<std::mutex> lock(g_gmu);
        if (!g_graph_used[dev]) return 0;
    }
    unsigned long long v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&v, g_branch_kernels, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
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
    GraphEntry *e = nullptr, *victim = nullptr;
    for (auto &x : g_graph) {
        if (x.hits && x.dev == ds->device && x.kt == kt && x.vals == VALS && x.n == (size_t)plan.n &&
            x.keys == d_keys && x.pay == d_vals) {
            e = &x;
            break;
        }
        // the slot to reuse: an empty one, else the least recent of this device
        if (!x.hits) {
            if (!victim || victim->hits) victim = &x;
        } else if (x.dev == ds->device && (!victim || (victim->hits && x.used < victim->used))) {
            victim = &x;
        }
    }
    ++g_tick;
    if (!e && !victim) return SR_OK;             // every slot holds another device's graph
    if (!e) {                                    // first sight: remember, launch ordinarily
        if (victim->done) cudaEventSynchronize(victim->done);     // its last replay has finished
        if (victim->exec) cudaGraphExecDestroy(victim->exec);
        if (victim->scratch) scratch_free(victim->scratch, s);
        if (victim->done) cudaEventDestroy(victim->done);
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
    if (!e->done && cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming) != cudaSuccess)
        return launch_status();
    if (cudaGraphLaunch(e->exec, s) != cudaSuccess || cudaEventRecord(e->done, s) != cudaSuccess)
        return launch_status();
    g_graph_used[ds->device] = true;
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
    PS plan(n, !VALS && SR_REM_KEYS);
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
    plan.status = ds->status;
    rec.cur0 = plan.steps & 1;
    rec.host.passes_planned = plan.steps;
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
                  (const T *)d_keys, N, ctrl, (const int *)nullptr, (typename K::U *)nullptr, 1,
                  (typename K::U *)nullptr, (typename K::U *)nullptr);
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

// Per-device streams for sr_sort_keys_host_many: one for the copies in, and
// two lanes of (sort, copy out) that take the arrays in turn, so a short sort
// and its copy out need not wait behind a long one.
static cudaStream_t g_pipe[5][64];

extern "C" sr_status sr_sort_keys_host_many(void *const *h_keys, const size_t *n, int count, sr_key_type kt,
                                            sr_stream stream) {
    if (!valid_key_type(kt) || count < 0 || (count > 0 && (!h_keys || !n))) return SR_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 2) continue;
        cudaPointerAttributes pa;
        if (!h_keys[i] || cudaPointerGetAttributes(&pa, h_keys[i]) != cudaSuccess ||
            pa.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return SR_ERR_INVALID_ARG;             // every array page-locked
        }
    }
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    const int dev = ds->device;
    if (dev < 0 || dev >= 64) return SR_ERR_UNSUPPORTED;
    for (int k = 0; k < 5; ++k)
        if (!g_pipe[k][dev] && cudaStreamCreateWithFlags(&g_pipe[k][dev], cudaStreamNonBlocking) != cudaSuccess)
            return launch_status();
    cudaStream_t cin = g_pipe[0][dev];
    cudaStream_t comp[2] = {g_pipe[1][dev], g_pipe[2][dev]}, cout[2] = {g_pipe[3][dev], g_pipe[4][dev]};
    const cudaStream_t s = (cudaStream_t)stream;
    auto link = [&](cudaStream_t from, cudaStream_t to) -> sr_status {   // `to` waits for `from`'s work so far
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return launch_status();
        const bool ok = cudaEventRecord(e, from) == cudaSuccess && cudaStreamWaitEvent(to, e, 0) == cudaSuccess;
        cudaEventDestroy(e);
        return ok ? SR_OK : launch_status();
    };
    // the pipeline starts after the caller's earlier work on `stream`
    SR_TRY(link(s, cin));
    for (int k = 0; k < 2; ++k) {
        SR_TRY(link(s, comp[k]));
        SR_TRY(link(s, cout[k]));
    }
    const size_t kb = key_bytes_of(kt);
    sr_status st = SR_OK;
    int lane = 0;
    for (int i = 0; i < count && st == SR_OK; ++i) {
        if (n[i] < 2) continue;
        const size_t bytes = n[i] * kb;
        cudaStream_t cs = comp[lane], co = cout[lane];
        lane ^= 1;
        void *d = nullptr;
        if ((st = scratch_alloc(ds, &d, bytes, cin)) != SR_OK) break;
        if (cudaMemcpyAsync(d, h_keys[i], bytes, cudaMemcpyHostToDevice, cin) != cudaSuccess) {
            st = launch_status();
            break;
        }
        if ((st = link(cin, cs)) != SR_OK) break;              // array i is on the device
        if ((st = dispatch_sort<false>(d, nullptr, n[i], kt, cs, 1, false)) != SR_OK) break;
        if ((st = link(cs, co)) != SR_OK) break;               // array i is sorted
        if (cudaMemcpyAsync(h_keys[i], d, bytes, cudaMemcpyDeviceToHost, co) != cudaSuccess) {
            st = launch_status();
            break;
        }
        scratch_free(d, co);
    }
    // the caller's later work on `stream` waits for all of it (also after an
    // error: the arrays queued before it are still in flight)
    sr_status st2 = link(cin, s);
    for (int k = 0; k < 2; ++k) {
        if (st2 == SR_OK) st2 = link(comp[k], s);
        if (st2 == SR_OK) st2 = link(cout[k], s);
    }
    return st != SR_OK ? st : st2;
}

extern "C" sr_status sr_release_cached(void) { return graph_cache_clear(); }

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
