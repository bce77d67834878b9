// sr_learned.cu -- sr_sort_keys_learned and the router network's kernels
// (sr_model_loss_grad, sr_model_train, sr_model_buckets).
//
// The paper has no learned component; this is the split-then-sort-the-parts
// shape of its quicksort (Section 4) with the split points read off a small
// monotone network that predicts each key's CDF.  Launch sequence, all on the
// caller's stream, nothing read back to the host:
//
//   k_sample      every stride-th key's order image -> sample
//   (plain sort)  the sample, sorted as unsigned order images
//   k_train       one CTA: training points = quantiles of the sorted sample,
//                 quantile start, full-batch Adam steps (forward + backward),
//                 then the routing tables
//   k_hist        bucket of every key -> histogram
//   k_bucket_scan bucket offsets, largest bucket
//   k_scatter     every key to its bucket (scratch)
//   (segmented)   every bucket sorted, scratch -> caller's buffer
//   k_bucket_check every bucket's last key <= the next bucket's first key;
//                 else the fallback flag is set
//   (plain sort)  gated by that flag: runs only if the check failed
//
// The network (H = 32 hidden units; theta = [x0, delta[H], beta[H]]):
//   d_j = softplus(delta_j), x_j = x0 + sum_{i<j} d_i, h_j = ramp((x - x_j)/d_j),
//   w = softmax(beta), y = sum_j w_j h_j.
// Because the ramps tile the key axis, for x in segment k (x_k <= x < x_{k+1})
// every ramp before k is 1 and every ramp after k is 0, so
//   y = P_k + w_k * ramp((x - x_k)/d_k),  P_k = sum_{j<k} w_j.
// The kernels evaluate this form.  With P computed as a sequential float sum
// (P_{k+1} = fl(P_k + w_k)) it is non-decreasing in the key in float
// arithmetic: within a segment every step is monotone, and across a knot the
// left side is at most fl(P_k + w_k * 1) = P_{k+1}, the right side at least
// P_{k+1}.  So equal keys share a bucket and buckets come in key order; the
// check catches any router for which that fails (the SR_MODEL_FORCE_BAD hook).
#include <algorithm>
#include <cstring>

#include "sr_device.cuh"
#include "sr_plain.cuh"
#include "sr_runtime.cuh"

namespace sr {

constexpr int H = SR_MODEL_HIDDEN;
constexpr int NPARAM = SR_MODEL_PARAMS;
static_assert(NPARAM == 2 * H + 1, "parameter layout");

struct Router {
    float knot[H + 1];           // x_0 .. x_H
    float invd[H];               // 1 / d_j
    float P[H + 1];              // P_0 = 0, P_{j+1} = fl(P_j + w_j)
    float w[H];
    unsigned long long lo;       // order image mapped to x = 0
    float inv_span;              // 1 / (hi - lo)
    int model;
    int nbuckets;
    int pad;
};

struct LearnCtrl {
    Router r;
    float theta[NPARAM];
    float grad[NPARAM];
    float loss;
    float loss0;                 // loss of the starting parameters
    int fallback;                // 1 when the bucket check failed
    int steps_done;
    unsigned long long max_bucket;
    unsigned long long bucket_sq;  // sum of squared bucket sizes
    unsigned long long nkeys;
    int nbuckets;
    int pad2;
};
static_assert(sizeof(LearnCtrl) <= kAuxBytes, "learned control block too large for the stats buffer");

// ------------------------------------------------------------ device math

__device__ __forceinline__ float softplus_f(float v) { return v > 20.f ? v : log1pf(expf(v)); }
__device__ __forceinline__ float sigmoid_f(float v) { return 1.f / (1.f + expf(-v)); }

// x = (u - lo) / (hi - lo) for an order image u, monotone in u.
// Explicitly rounded operations throughout routing, so every kernel that routes
// a key computes the same bucket whatever the compiler fuses.
__device__ __forceinline__ float norm_x(unsigned long long u, unsigned long long lo, float inv_span) {
    const float d = u >= lo ? __ull2float_rn(u - lo) : -__ull2float_rn(lo - u);
    return __fmul_rn(d, inv_span);
}

// Segment k of x: the number of interior knots x_1..x_{H-1} that are <= x.
__device__ __forceinline__ int segment_of(const float *knot, float x) {
    int lo = 0, hi = H - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (knot[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int route_bucket(const Router &r, float x) {
    float y;
    if (r.model == SR_MODEL_EQUAL_WIDTH) {
        y = x;
    } else {
        const int k = segment_of(r.knot, x);
        const float u = fminf(fmaxf(__fmul_rn(__fsub_rn(x, r.knot[k]), r.invd[k]), 0.f), 1.f);
        y = __fmaf_rn(r.w[k], u, r.P[k]);
    }
    const float yb = __fmul_rn(y, (float)r.nbuckets);
    int b = yb > 0.f ? (int)fminf(yb, (float)(r.nbuckets - 1)) : 0;
    if (b > r.nbuckets - 1) b = r.nbuckets - 1;
    if (r.model == SR_MODEL_FORCE_BAD) b = r.nbuckets - 1 - b;      // test hook: not monotone
    return b;
}

// The parameters' derived tables (one warp; lane j owns hidden unit j).
struct Derived {
    float d[H], sig[H], invd[H], w[H];
    float knot[H + 1], P[H + 1];
};

__device__ void derive(const float *theta, Derived &dv, int lane) {
    const float delta = theta[1 + lane], beta = theta[1 + H + lane];
    const float d = softplus_f(delta);
    dv.d[lane] = d;
    dv.sig[lane] = sigmoid_f(delta);
    dv.invd[lane] = 1.f / d;
    float mx = beta;
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float e = expf(beta - mx);
    float sum = e;
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    dv.w[lane] = e / sum;
    __syncwarp();
    if (lane == 0) {
        // sequential float sums: the knots must not decrease and P must satisfy
        // P_{j+1} = fl(P_j + w_j) exactly (the monotonicity argument above)
        float x = theta[0], p = 0.f;
        for (int j = 0; j < H; ++j) {
            dv.knot[j] = x;
            dv.P[j] = p;
            x = __fadd_rn(x, dv.d[j]);
            p = __fadd_rn(p, dv.w[j]);
        }
        dv.knot[H] = x;
        dv.P[H] = p;
    }
    __syncwarp();
}

__device__ void derived_to_router(const Derived &dv, Router &r, int lane) {
    r.invd[lane] = dv.invd[lane];
    r.w[lane] = dv.w[lane];
    r.knot[lane] = dv.knot[lane];
    r.P[lane] = dv.P[lane];
    if (lane == 0) { r.knot[H] = dv.knot[H]; r.P[H] = dv.P[H]; }
}

// ------------------------------------------------------------- training

enum { TRAIN_PIPELINE = 0, TRAIN_GRAD = 1, TRAIN_STEPS = 2 };
constexpr int TRAIN_NT = 1024;

// One CTA.  TRAIN_PIPELINE: builds the training points from the sorted
// sample (order images), starts from the quantile knots and trains `steps`
// Adam steps, then writes the routing tables.  TRAIN_GRAD: loss and gradient
// of lc->theta over the given points.  TRAIN_STEPS: `steps` Adam steps from
// lc->theta over the given points.
template <typename U>
__global__ void __launch_bounds__(TRAIN_NT)
k_train(const U *__restrict__ sample, long long m, float *__restrict__ px, float *__restrict__ pt, long long np,
        int mode, int steps, float lr, int cap, int model, int nbuckets, LearnCtrl *__restrict__ lc) {
    griddep_wait();
    __shared__ float th[NPARAM], am[NPARAM], av[NPARAM], gr[NPARAM];
    __shared__ Derived dv;
    __shared__ float acc_w[H], acc_s[H], acc_kn[H], acc_d[H];
    __shared__ float s_loss;
    __shared__ long long s_np;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;

    if (mode == TRAIN_PIPELINE) {
        const unsigned long long lo = (unsigned long long)sample[0];
        const unsigned long long hi = (unsigned long long)sample[m - 1];
        const float inv_span = hi > lo ? (float)(1.0 / (double)(hi - lo)) : 0.f;
        const long long S = min((long long)cap, m);
        for (long long i = t; i < S; i += TRAIN_NT) {
            const long long idx = S > 1 ? (i * (m - 1)) / (S - 1) : 0;
            px[i] = norm_x((unsigned long long)sample[idx], lo, inv_span);
            pt[i] = (float)(((double)idx + 0.5) / (double)m);
        }
        if (t == 0) {
            lc->r.lo = lo;
            lc->r.inv_span = inv_span;
            lc->r.model = model;
            lc->r.nbuckets = nbuckets;
            s_np = S;
        }
        __syncthreads();
        __threadfence_block();
        if (t == 0) {
            // quantile start: knots at the points' 0, 1/H, ..., 1 quantiles
            float prev = px[0];
            th[0] = prev;
            for (int j = 0; j < H; ++j) {
                const long long q = ((long long)(j + 1) * (S - 1) + H / 2) / H;
                const float kx = px[q];
                const float gap = fmaxf(kx - prev, 1e-7f);
                th[1 + j] = gap > 20.f ? gap : logf(expm1f(gap));
                th[1 + H + j] = 0.f;
                prev += gap;                                  // the model's knot x_{j+1}
            }
        }
    } else {
        if (t < NPARAM) th[t] = lc->theta[t];
        if (t == 0) s_np = np;
    }
    if (t < NPARAM) { am[t] = 0.f; av[t] = 0.f; }
    if (t < H) { acc_w[t] = 0.f; acc_s[t] = 0.f; acc_kn[t] = 0.f; acc_d[t] = 0.f; }
    if (t == 0) s_loss = 0.f;
    __syncthreads();
    const long long S = s_np;
    const long long ppt = (S + TRAIN_NT - 1) / TRAIN_NT;
    const long long p0 = min(S, (long long)t * ppt), p1 = min(S, p0 + ppt);
    const int total_steps = mode == TRAIN_GRAD ? 1 : steps + 1;   // the last pass only measures the loss

    for (int it = 0; it < total_steps; ++it) {
        if (wid == 0) derive(th, dv, lane);
        __syncthreads();
        // forward and backward over this thread's (sorted) points
        float loss = 0.f, gw = 0.f, gs = 0.f, gkn = 0.f, gd = 0.f;
        int kc = -1;
        const float gscale = 2.f / (float)S;
        for (long long i = p0; i < p1; ++i) {
            const float x = px[i];
            const int k = segment_of(dv.knot, x);
            if (k != kc) {
                if (kc >= 0) {
                    atomicAdd(&acc_w[kc], gw); atomicAdd(&acc_s[kc], gs);
                    atomicAdd(&acc_kn[kc], gkn); atomicAdd(&acc_d[kc], gd);
                }
                gw = gs = gkn = gd = 0.f;
                kc = k;
            }
            const float u = (x - dv.knot[k]) * dv.invd[k];
            const float h = fminf(fmaxf(u, 0.f), 1.f);
            const float y = fmaf(dv.w[k], h, dv.P[k]);
            const float r = y - pt[i];
            loss += r * r;
            const float g = gscale * r;
            gs += g;                                  // every unit before k is saturated at 1
            gw += g * h;
            if (u > 0.f && u < 1.f) {
                const float gu = g * dv.w[k];
                gkn -= gu * dv.invd[k];               // d u / d x_k = -1/d_k
                gd -= gu * u * dv.invd[k];            // d u / d d_k = -u/d_k
            }
        }
        if (kc >= 0) {
            atomicAdd(&acc_w[kc], gw); atomicAdd(&acc_s[kc], gs);
            atomicAdd(&acc_kn[kc], gkn); atomicAdd(&acc_d[kc], gd);
        }
        for (int o = 16; o; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
        if (lane == 0) atomicAdd(&s_loss, loss);
        __syncthreads();
        if (wid == 0) {
            const float Lmean = s_loss / (float)S;
            // dL/dw_j = acc_w[j] + sum_{k > j} acc_s[k]
            float suf = acc_s[lane];
            for (int o = 1; o < 32; o <<= 1) {                 // inclusive suffix sum
                const float v = __shfl_down_sync(0xffffffffu, suf, o);
                if (lane + o < 32) suf += v;
            }
            const float dw = acc_w[lane] + (suf - acc_s[lane]);
            float swd = dv.w[lane] * dw;
            for (int o = 16; o; o >>= 1) swd += __shfl_xor_sync(0xffffffffu, swd, o);
            const float dbeta = dv.w[lane] * (dw - swd);
            // knot x_j = x0 + sum_{i<j} d_i:  dL/dd_j = acc_d[j] + sum_{i > j} acc_kn[i]
            float kn = acc_kn[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const float v = __shfl_down_sync(0xffffffffu, kn, o);
                if (lane + o < 32) kn += v;
            }
            const float dd = acc_d[lane] + (kn - acc_kn[lane]);
            const float ddelta = dd * dv.sig[lane];
            float dx0 = acc_kn[lane];
            for (int o = 16; o; o >>= 1) dx0 += __shfl_xor_sync(0xffffffffu, dx0, o);
            gr[1 + lane] = ddelta;
            gr[1 + H + lane] = dbeta;
            if (lane == 0) gr[0] = dx0;
            __syncwarp();
            if (it == 0 && lane == 0) lc->loss0 = Lmean;
            const bool last = it == total_steps - 1;
            if (last) {
                if (lane == 0) lc->loss = Lmean;
                for (int q = lane; q < NPARAM; q += 32) lc->grad[q] = gr[q];
            } else {
                // Adam (Kingma and Ba, 2015), bias-corrected
                const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
                const float c1 = 1.f - powf(b1, (float)(it + 1)), c2 = 1.f - powf(b2, (float)(it + 1));
                for (int q = lane; q < NPARAM; q += 32) {
                    am[q] = b1 * am[q] + (1.f - b1) * gr[q];
                    av[q] = b2 * av[q] + (1.f - b2) * gr[q] * gr[q];
                    th[q] -= lr * (am[q] / c1) / (sqrtf(av[q] / c2) + eps);
                }
            }
            acc_w[lane] = 0.f; acc_s[lane] = 0.f; acc_kn[lane] = 0.f; acc_d[lane] = 0.f;
            if (lane == 0) s_loss = 0.f;
        }
        __syncthreads();
    }
    if (wid == 0) {
        derive(th, dv, lane);
        derived_to_router(dv, lc->r, lane);
        for (int q = lane; q < NPARAM; q += 32) lc->theta[q] = th[q];
        if (lane == 0) lc->steps_done = total_steps - 1;
    }
}

// Routing tables from lc->theta (one warp), for sr_model_buckets.
__global__ void k_router(LearnCtrl *__restrict__ lc) {
    griddep_wait();
    __shared__ Derived dv;
    derive(lc->theta, dv, threadIdx.x & 31);
    derived_to_router(dv, lc->r, threadIdx.x & 31);
}

// ------------------------------------------------------------- routing

template <int KT>
__global__ void k_sample(const typename Key<KT>::T *__restrict__ keys, long long m, long long stride,
                         typename Key<KT>::U *__restrict__ sample) {
    griddep_wait();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) sample[i] = Key<KT>::ord(keys[i * stride]);
}

template <int KT>
__global__ void k_hist(const typename Key<KT>::T *__restrict__ keys, long long n, const LearnCtrl *__restrict__ lc,
                       unsigned int *__restrict__ hist) {
    griddep_wait();
    __shared__ Router r;
    if (threadIdx.x < sizeof(Router) / 4) ((uint32_t *)&r)[threadIdx.x] = ((const uint32_t *)&lc->r)[threadIdx.x];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = norm_x((unsigned long long)Key<KT>::ord(keys[i]), r.lo, r.inv_span);
        atomicAdd(&hist[route_bucket(r, x)], 1u);
    }
}

// Every key to the next free slot of its bucket.  A slot beyond the bucket's
// end (impossible while routing is deterministic) is not written; it raises
// the fallback flag and SR_ERR_INTERNAL in the status word instead.
template <int KT>
__global__ void k_scatter(const typename Key<KT>::T *__restrict__ keys, long long n,
                          LearnCtrl *__restrict__ lc, unsigned long long *__restrict__ cursor,
                          const long long *__restrict__ off, typename Key<KT>::T *__restrict__ out,
                          int *__restrict__ status_word) {
    griddep_wait();
    __shared__ Router r;
    if (threadIdx.x < sizeof(Router) / 4) ((uint32_t *)&r)[threadIdx.x] = ((const uint32_t *)&lc->r)[threadIdx.x];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const typename Key<KT>::T key = keys[i];
        const float x = norm_x((unsigned long long)Key<KT>::ord(key), r.lo, r.inv_span);
        const int b = route_bucket(r, x);
        const unsigned long long pos = atomicAdd(&cursor[b], 1ull);
        if (pos < (unsigned long long)off[b + 1]) {
            out[pos] = key;
        } else {
            atomicExch(&lc->fallback, 1);
            atomicExch(status_word, (int)SR_ERR_INTERNAL);
        }
    }
}

// Exclusive scan of the histogram into offsets (one CTA); off[nb] = n.
__global__ void __launch_bounds__(1024)
k_bucket_scan(const unsigned int *__restrict__ hist, int nb, long long n, long long *__restrict__ off,
              unsigned long long *__restrict__ cursor, LearnCtrl *__restrict__ lc) {
    griddep_wait();
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned int s_max;
    __shared__ unsigned long long s_sq;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int per = (nb + 1023) / 1024;
    const int b0 = min(nb, t * per), b1 = min(nb, b0 + per);
    unsigned long long sum = 0, sq = 0;
    unsigned int mx = 0;
    for (int b = b0; b < b1; ++b) {
        const unsigned long long h = hist[b];
        sum += h;
        sq += h * h;
        mx = max(mx, hist[b]);
    }
    if (t == 0) { s_max = 0; s_sq = 0; }
    unsigned long long x = sum;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = s_warp[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        s_warp[lane] = w;
    }
    atomicMax(&s_max, mx);
    atomicAdd(&s_sq, sq);
    __syncthreads();
    unsigned long long run = (wid ? s_warp[wid - 1] : 0ull) + x - sum;
    for (int b = b0; b < b1; ++b) {
        off[b] = (long long)run;
        cursor[b] = run;
        run += hist[b];
    }
    if (t == 0) {
        off[nb] = n;
        lc->max_bucket = s_max;
        lc->bucket_sq = s_sq;
        lc->nkeys = (unsigned long long)n;
        lc->nbuckets = nb;
    }
}

// Every bucket's last key <= the next bucket's first key (buckets sorted).
template <int KT>
__global__ void k_bucket_check(const typename Key<KT>::T *__restrict__ keys, const long long *__restrict__ off,
                               int nb, long long n, LearnCtrl *__restrict__ lc) {
    griddep_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < 1 || b >= nb) return;
    const long long p = off[b];
    if (p > 0 && p < n && Key<KT>::ord(keys[p - 1]) > Key<KT>::ord(keys[p])) atomicExch(&lc->fallback, 1);
}

// ------------------------------------------------------------- host

static int sm_count_l() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <int KB> struct UKey;
template <> struct UKey<4> { enum { KT = SR_KEY_U32 }; };
template <> struct UKey<8> { enum { KT = SR_KEY_U64 }; };

template <int KT>
static sr_status learned_impl(void *d_keys, size_t n, const sr_learned_opts *o, cudaStream_t s) {
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    constexpr int KTU = UKey<sizeof(U)>::KT;
    const uint32_t nb = o && o->num_buckets ? o->num_buckets : (1u << 16);
    const uint32_t stride = o && o->sample_stride ? o->sample_stride : 100u;
    const uint32_t cap = o && o->train_points ? o->train_points : 8192u;
    uint32_t steps = o && o->train_steps ? o->train_steps : 64u;
    const float lr = o && o->learning_rate > 0.f ? o->learning_rate : 3e-3f;
    const uint32_t model = o ? o->model : 0u;
    if (nb < 16 || nb > (1u << 20) || (nb & (nb - 1)) || model > SR_MODEL_FORCE_BAD || cap < 2 || cap > (1u << 20))
        return SR_ERR_INVALID_ARG;
    if (model == SR_MODEL_UNTRAINED || model == SR_MODEL_EQUAL_WIDTH) steps = 0;

    CallRecord &rec = call_record();
    rec = CallRecord();
    rec.host.call = 4;
    rec.host.n = n;
    rec.host.key_type = KT;
    rec.stream = s;
    if (n < 2) return SR_OK;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));

    const long long N = (long long)n;
    const long long m = (N + stride - 1) / stride;
    const PlainSort<KTU, false> sample_sort((size_t)m);
    const PlainSort<KT, false> fallback_sort(n);
    // scratch: control | sample | sample-sort scratch | points | histogram |
    //          offsets | cursors | bucketed keys | fallback scratch
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off += align_up(bytes, 256); return at; };
    const size_t o_ctrl = take(sizeof(LearnCtrl));
    const size_t o_sample = take((size_t)m * sizeof(U));
    const size_t o_ss = take(sample_sort.bytes);
    const size_t o_px = take((size_t)cap * 4);
    const size_t o_pt = take((size_t)cap * 4);
    const size_t o_hist = take((size_t)nb * 4);
    const size_t o_off = take((size_t)(nb + 1) * 8);
    const size_t o_cur = take((size_t)nb * 8);
    const size_t o_keys = take(n * sizeof(T));
    const size_t o_fb = take(fallback_sort.bytes);
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, off, s));
    unsigned char *sp = (unsigned char *)scratch;
    LearnCtrl *lc = (LearnCtrl *)(sp + o_ctrl);
    U *sample = (U *)(sp + o_sample);
    float *px = (float *)(sp + o_px), *pt = (float *)(sp + o_pt);
    unsigned int *hist = (unsigned int *)(sp + o_hist);
    long long *boff = (long long *)(sp + o_off);
    unsigned long long *cursor = (unsigned long long *)(sp + o_cur);
    T *bucketed = (T *)(sp + o_keys);
    T *uk = (T *)d_keys;

    sr_status st = SR_OK;
    do {
        if (cudaMemsetAsync(lc, 0, sizeof(LearnCtrl), s) != cudaSuccess ||
            cudaMemsetAsync(hist, 0, (size_t)nb * 4, s) != cudaSuccess) {
            st = launch_status();
            break;
        }
        SR_LAUNCH(SR_KERNEL_MODEL, k_sample<KT>, (unsigned)((m + 255) / 256), 256, 0, s, uk, m, (long long)stride,
                  sample);
        if ((st = sample_sort.launch((typename PlainSort<KTU, false>::T *)sample, nullptr, sp + o_ss, s)) != SR_OK)
            break;
        SR_LAUNCH(SR_KERNEL_MODEL, k_train<U>, 1, TRAIN_NT, 0, s, sample, m, px, pt, (long long)0,
                  (int)TRAIN_PIPELINE, (int)steps, lr, (int)cap, (int)model, (int)nb, lc);
        const int grid = sm_count_l() * 8;
        SR_LAUNCH(SR_KERNEL_MODEL, k_hist<KT>, grid, 256, 0, s, uk, N, lc, hist);
        SR_LAUNCH(SR_KERNEL_MODEL, k_bucket_scan, 1, 1024, 0, s, hist, (int)nb, N, boff, cursor, lc);
        SR_LAUNCH(SR_KERNEL_MODEL, k_scatter<KT>, grid, 256, 0, s, uk, N, lc, cursor, boff, bucketed, ds->status);
        if ((st = segmented_run<KT>(bucketed, uk, n, (const int64_t *)boff, nb, s, false)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_MODEL, k_bucket_check<KT>, (unsigned)((nb + 255) / 256), 256, 0, s, uk, boff, (int)nb,
                  N, lc);
        if ((st = fallback_sort.launch(uk, nullptr, sp + o_fb, s, &lc->fallback)) != SR_OK) break;
        if (cudaMemcpyAsync(ds->last_aux, lc, sizeof(LearnCtrl), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            st = launch_status();
            break;
        }
        rec.aux_kind = 4;
    } while (0);
    scratch_free(scratch, s);
    return st;
}

sr_status learned_stats(const void *aux, sr_stats *out) {
    const LearnCtrl *c = (const LearnCtrl *)aux;
    out->fallback = c->fallback;
    out->max_bucket = c->max_bucket;
    out->model_loss = c->loss;
    out->bucket_imbalance =
        c->nkeys ? (float)((double)c->nbuckets * (double)c->bucket_sq / ((double)c->nkeys * (double)c->nkeys)) : 0.f;
    return SR_OK;
}

// Synchronous helper for the model entry points: runs k_train in `mode` over
// the given points from theta; returns the control block.
static sr_status model_run(const float *d_x, const float *d_t, size_t m, const float *h_theta, int mode,
                           uint32_t steps, float lr, LearnCtrl *h_out, cudaStream_t s) {
    if (!d_x || !d_t || !h_theta || m == 0) return SR_ERR_INVALID_ARG;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, sizeof(LearnCtrl), s));
    LearnCtrl *lc = (LearnCtrl *)scratch;
    sr_status st = SR_OK;
    do {
        if (cudaMemsetAsync(lc, 0, sizeof(LearnCtrl), s) != cudaSuccess ||
            cudaMemcpyAsync(lc->theta, h_theta, NPARAM * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = launch_status();
            break;
        }
        SR_LAUNCH(SR_KERNEL_MODEL, k_train<uint32_t>, 1, TRAIN_NT, 0, s, (const uint32_t *)nullptr, (long long)0,
                  const_cast<float *>(d_x), const_cast<float *>(d_t), (long long)m, mode, (int)steps, lr, 0,
                  (int)SR_MODEL_TRAINED, 1, lc);
        if (cudaMemcpyAsync(h_out, lc, sizeof(LearnCtrl), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            st = launch_status();
            break;
        }
    } while (0);
    scratch_free(scratch, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == SR_OK) st = launch_status();
    return st;
}

template <int KT>
__global__ void k_buckets_out(const typename Key<KT>::T *__restrict__ keys, long long n,
                              const LearnCtrl *__restrict__ lc, uint32_t *__restrict__ out) {
    griddep_wait();
    __shared__ Router r;
    if (threadIdx.x < sizeof(Router) / 4) ((uint32_t *)&r)[threadIdx.x] = ((const uint32_t *)&lc->r)[threadIdx.x];
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)route_bucket(r, norm_x((unsigned long long)Key<KT>::ord(keys[i]), r.lo, r.inv_span));
}

template <int KT>
static sr_status buckets_impl(const void *d_keys, size_t n, const float *h_theta, uint64_t lo, uint64_t hi,
                              uint32_t nb, uint32_t *d_out, cudaStream_t s) {
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, sizeof(LearnCtrl), s));
    LearnCtrl *lc = (LearnCtrl *)scratch;
    Router hr;
    std::memset(&hr, 0, sizeof(hr));
    hr.lo = lo;
    hr.inv_span = hi > lo ? (float)(1.0 / (double)(hi - lo)) : 0.f;
    hr.model = SR_MODEL_TRAINED;
    hr.nbuckets = (int)nb;
    sr_status st = SR_OK;
    do {
        if (cudaMemcpyAsync(&lc->r, &hr, sizeof(Router), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(lc->theta, h_theta, NPARAM * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = launch_status();
            break;
        }
        SR_LAUNCH(SR_KERNEL_MODEL, k_router, 1, 32, 0, s, lc);
        SR_LAUNCH(SR_KERNEL_MODEL, k_buckets_out<KT>, (unsigned)((n + 255) / 256), 256, 0, s,
                  (const typename Key<KT>::T *)d_keys, (long long)n, lc, d_out);
    } while (0);
    scratch_free(scratch, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == SR_OK) st = launch_status();
    return st;
}

}  // namespace sr

using namespace sr;

extern "C" sr_status sr_sort_keys_learned(void *d_keys, size_t n, sr_key_type kt, const sr_learned_opts *opts,
                                          sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && !d_keys) return SR_ERR_INVALID_ARG;
    if (n > 1 && ((uintptr_t)d_keys % key_bytes_of(kt)) != 0) return SR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    switch (kt) {
    case SR_KEY_I32: return learned_impl<SR_KEY_I32>(d_keys, n, opts, s);
    case SR_KEY_U32: return learned_impl<SR_KEY_U32>(d_keys, n, opts, s);
    case SR_KEY_F32: return learned_impl<SR_KEY_F32>(d_keys, n, opts, s);
    case SR_KEY_U64: return learned_impl<SR_KEY_U64>(d_keys, n, opts, s);
    case SR_KEY_I64: return learned_impl<SR_KEY_I64>(d_keys, n, opts, s);
    default: return SR_ERR_INVALID_ARG;
    }
}

extern "C" sr_status sr_model_loss_grad(const float *d_x, const float *d_t, size_t m, const float *h_theta,
                                        float *h_loss, float *h_grad, sr_stream stream) {
    if (!h_loss || !h_grad) return SR_ERR_INVALID_ARG;
    LearnCtrl out;
    SR_TRY(model_run(d_x, d_t, m, h_theta, TRAIN_GRAD, 0, 0.f, &out, (cudaStream_t)stream));
    *h_loss = out.loss;
    std::memcpy(h_grad, out.grad, sizeof(out.grad));
    return SR_OK;
}

extern "C" sr_status sr_model_train(const float *d_x, const float *d_t, size_t m, float *h_theta, uint32_t steps,
                                    float learning_rate, float *h_loss, sr_stream stream) {
    if (!h_loss || !(learning_rate > 0.f)) return SR_ERR_INVALID_ARG;
    LearnCtrl out;
    SR_TRY(model_run(d_x, d_t, m, h_theta, TRAIN_STEPS, steps, learning_rate, &out, (cudaStream_t)stream));
    std::memcpy(h_theta, out.theta, sizeof(out.theta));
    *h_loss = out.loss;
    return SR_OK;
}

extern "C" sr_status sr_model_buckets(const void *d_keys, size_t n, sr_key_type kt, const float *h_theta,
                                      uint64_t lo, uint64_t hi, uint32_t num_buckets, uint32_t *d_out,
                                      sr_stream stream) {
    if (!valid_key_type(kt) || !h_theta || num_buckets < 1) return SR_ERR_INVALID_ARG;
    if (n == 0) return SR_OK;
    if (!d_keys || !d_out) return SR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    switch (kt) {
    case SR_KEY_I32: return buckets_impl<SR_KEY_I32>(d_keys, n, h_theta, lo, hi, num_buckets, d_out, s);
    case SR_KEY_U32: return buckets_impl<SR_KEY_U32>(d_keys, n, h_theta, lo, hi, num_buckets, d_out, s);
    case SR_KEY_F32: return buckets_impl<SR_KEY_F32>(d_keys, n, h_theta, lo, hi, num_buckets, d_out, s);
    case SR_KEY_U64: return buckets_impl<SR_KEY_U64>(d_keys, n, h_theta, lo, hi, num_buckets, d_out, s);
    case SR_KEY_I64: return buckets_impl<SR_KEY_I64>(d_keys, n, h_theta, lo, hi, num_buckets, d_out, s);
    default: return SR_ERR_INVALID_ARG;
    }
}
