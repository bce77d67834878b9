// sr_runtime.cu -- per-device state, scratch pool, status word and statistics.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "sr_runtime.cuh"

namespace sr {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceState g_dev[kMaxDevices];
thread_local CallRecord g_rec;
std::atomic<unsigned long long> g_launches{0};

struct Timed {
    int kind;
    cudaEvent_t a, b;
};
thread_local bool g_prof_on = false;
thread_local unsigned long long g_thread_launches = 0;   // this thread's launches (captures count with it)
thread_local std::vector<Timed> g_prof;
thread_local cudaEvent_t g_prof_pending = nullptr;
}  // namespace

void launch_begin(int kind, cudaStream_t s) {
    (void)kind;
    if (!g_prof_on) return;
    cudaEvent_t a = nullptr;
    if (cudaEventCreate(&a) == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
        g_prof_pending = a;
    } else {
        if (a) cudaEventDestroy(a);
        g_prof_pending = nullptr;
        cudaGetLastError();
    }
}

sr_status launch_end(int kind, cudaStream_t s) {
    sr_status st = launch_status();
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++g_thread_launches;
    if (g_prof_on && g_prof_pending) {
        cudaEvent_t b = nullptr;
        if (cudaEventCreate(&b) == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess) {
            g_prof.push_back(Timed{kind, g_prof_pending, b});
        } else {
            cudaEventDestroy(g_prof_pending);
            if (b) cudaEventDestroy(b);
            cudaGetLastError();
        }
        g_prof_pending = nullptr;
    }
    return st;
}

bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("SR_PDL");
        return !(e && std::strcmp(e, "0") == 0);
    }();
    return on;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int device_sm_count() {
    static int cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        cached[dev] = v;
    }
    return cached[dev];
}

int ceil_log2(unsigned long long x) {
    int r = 0;
    while ((1ull << r) < x) ++r;
    return r;
}

size_t key_bytes_of(sr_key_type kt) { return (kt == SR_KEY_U64 || kt == SR_KEY_I64) ? 8 : 4; }

bool valid_key_type(int kt) { return kt >= SR_KEY_I32 && kt <= SR_KEY_I64; }

CallRecord &call_record() { return g_rec; }

sr_status launch_status() {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return SR_OK;
    if (e == cudaErrorMemoryAllocation) return SR_ERR_OOM;
    return SR_ERR_CUDA;
}

sr_status device_state(DeviceState **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &ds = g_dev[dev];
    if (ds.device < 0) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&ds.pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return SR_ERR_CUDA;
        }
        // keep freed scratch cached in the pool between calls
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(ds.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (cudaMalloc(&ds.status, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&ds.last_ctrl, sizeof(Ctrl)) != cudaSuccess ||
            cudaMalloc(&ds.last_aux, kAuxBytes) != cudaSuccess ||
            cudaMemset(ds.last_aux, 0, kAuxBytes) != cudaSuccess ||
            cudaMemset(ds.status, 0, sizeof(int)) != cudaSuccess ||
            cudaMemset(ds.last_ctrl, 0, sizeof(Ctrl)) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            return SR_ERR_CUDA;
        }
        ds.device = dev;
    }
    *out = &ds;
    return SR_OK;
}

sr_status scratch_alloc(DeviceState *ds, void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    const char *inj = std::getenv("SR_INJECT_OOM");
    if (inj && inj[0] && std::strcmp(inj, "0") != 0) return SR_ERR_OOM;
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ds->pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
    }
    return SR_OK;
}

void scratch_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

}  // namespace sr

using namespace sr;

extern "C" const char *sr_status_string(sr_status s) {
    switch (s) {
    case SR_OK: return "SR_OK";
    case SR_ERR_INVALID_ARG: return "SR_ERR_INVALID_ARG";
    case SR_ERR_UNSUPPORTED: return "SR_ERR_UNSUPPORTED";
    case SR_ERR_OOM: return "SR_ERR_OOM";
    case SR_ERR_CUDA: return "SR_ERR_CUDA";
    case SR_ERR_TIMEOUT: return "SR_ERR_TIMEOUT";
    case SR_ERR_INTERNAL: return "SR_ERR_INTERNAL";
    case SR_ERR_BAD_SEGMENTS: return "SR_ERR_BAD_SEGMENTS";
    default: return "SR_ERR_UNKNOWN";
    }
}

namespace sr {
bool profiling_on() { return g_prof_on; }
void count_launches(long long k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }
unsigned long long host_launch_count() { return g_launches.load(); }
unsigned long long thread_launch_count() { return g_thread_launches; }
}  // namespace sr

extern "C" uint64_t sr_launch_count(void) { return g_launches.load() + sr::graph_kernel_count(); }

extern "C" sr_status sr_profile_begin(void) {
    for (auto &t : g_prof) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    g_prof.clear();
    g_prof_on = true;
    return SR_OK;
}

extern "C" sr_status sr_profile_end(sr_kernel_time *out, int count) {
    g_prof_on = false;
    if (out && count > 0) {
        for (int k = 0; k < count; ++k) { out[k].launches = 0; out[k].ms = 0.0; }
    }
    sr_status st = SR_OK;
    for (auto &t : g_prof) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) {
            cudaGetLastError();
            st = SR_ERR_CUDA;
        } else if (out && t.kind >= 0 && t.kind < count) {
            out[t.kind].launches += 1;
            out[t.kind].ms += ms;
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    g_prof.clear();
    return st;
}

extern "C" sr_status sr_stream_status(sr_stream stream) {
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return SR_ERR_CUDA; }
    int word = 0;
    if (cudaMemcpy(&word, ds->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(ds->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SR_ERR_CUDA;
    }
    return (sr_status)word;
}

extern "C" sr_status sr_get_stats(sr_stats *out) {
    if (!out) return SR_ERR_INVALID_ARG;
    CallRecord &r = call_record();
    *out = r.host;
    out->abi_version = SR_ABI_VERSION;
    if (r.aux_kind) {
        DeviceState *ds = nullptr;
        SR_TRY(device_state(&ds));
        if (cudaStreamSynchronize(r.stream) != cudaSuccess) { cudaGetLastError(); return SR_ERR_CUDA; }
        unsigned char aux[kAuxBytes];
        if (cudaMemcpy(aux, ds->last_aux, kAuxBytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return SR_ERR_CUDA;
        }
        if (r.aux_kind == 3) return segmented_stats(aux, out);
        if (r.aux_kind == 4) return learned_stats(aux, out);
    }
    if (!r.has_ctrl) return SR_OK;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    if (cudaStreamSynchronize(r.stream) != cudaSuccess) { cudaGetLastError(); return SR_ERR_CUDA; }
    Ctrl c;
    if (cudaMemcpy(&c, ds->last_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return SR_ERR_CUDA;
    }
    const unsigned long long n = out->n;
    const unsigned long long elem = (unsigned long long)(r.key_bytes + r.val_bytes);
    out->runs = n ? c.descents + 1 : 0;
    out->input_class = c.descents == 0 ? 1
                       : (c.nondescents == 0 && n > 1 ? 2 : (c.few_active ? 3 : (c.rem_gate ? 4 : 0)));
    unsigned long long bytes = n * (unsigned long long)r.key_bytes;     // the scan reads the keys
    int skipped = 0, merged = 0;
    if (out->input_class == 0) {
        bytes += 2 * n * elem;                                          // block sort
        const bool repaired = c.repair && !c.repair_fail;
        merged = out->passes_planned > 0 && !repaired ? c.nsteps : 0;   // steps the natural runs needed
        skipped = out->passes_planned - merged;
        bytes += (unsigned long long)merged * 2 * n * elem;
        if (repaired) bytes += 2 * c.repair_keys * elem;                  // the boundary windows, in place
        const int cur = r.cur0 | (c.tile_perm ? 1 : 0);                  // where the block sort wrote
        if (((cur + merged) & 1) != 0) bytes += 2 * n * elem;            // copy back
    } else if (out->input_class == 2) {
        bytes += 2 * n * elem;                                          // one reversal
    } else if (out->input_class == 3) {
        bytes += 2 * n * elem;                                          // counted, then written as runs
    } else if (out->input_class == 4) {
        out->displaced = c.rem_dcount;
        bytes += 2 * n * elem;                                          // split: in-order keys and buckets
        bytes += 2 * c.rem_dcount * elem;                               // bucket sorts
        bytes += 2 * n * elem;                                          // per-tile merges into place
    }
    out->passes_skipped = skipped;
    out->bytes_moved = bytes;
    return SR_OK;
}
