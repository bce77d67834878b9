// sr_learned.cu -- sr_sort_keys_learned and the router network's kernels
// (sr_model_loss_grad, sr_model_train, sr_model_buckets).
//
// The paper has no learned component; this is the split-then-sort-the-parts
// shape of its quicksort (Section 4) with the split points read off a small
// monotone network that predicts each key's CDF.  Launch sequence, on the
// caller's stream:
//
//   k_sample      every stride-th key's order image -> sample
//   (plain sort)  the sample, sorted as unsigned order images
//   k_train       one CTA: training points = quantiles of the sorted sample,
//                 quantile start, full-batch Adam steps (forward + backward),
//                 then the routing tables
//   two-level split of the bucket id (coarse digit, then fine digit): per
//                 level k_split_tiles, k_split_hist (shared-memory counts per
//                 tile), k_scan_* (positions), k_split_scatter
//   (segmented)   every bucket sorted, one CTA per bucket, scratch -> the
//                 caller's buffer
//   k_bucket_check every bucket's last key <= the next bucket's first key;
//                 else the fallback flag is set
//   (plain sort)  only if the check failed (the flag is read back: this call
//                 waits for its stream once; inside a stream capture the
//                 plain sort is the body of an IF node that a one-thread
//                 kernel sets from the flag, so nothing is read back)
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
#include <mutex>

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

// Routing state a CTA keeps in shared memory: per segment k the float4
// (x_k, 1/d_k, w_k, P_k), and the interior knots for the search.
struct RouteSmem {
    float4 seg[H];
    float knot[H + 1];
    unsigned long long lo;
    float inv_span;
    int model, nbuckets;
};

__device__ __forceinline__ void load_route(const Router &r, RouteSmem &rs) {
    const int t = threadIdx.x;
    if (t < H) rs.seg[t] = make_float4(r.knot[t], r.invd[t], r.w[t], r.P[t]);
    if (t <= H) rs.knot[t] = r.knot[t];
    if (t == 0) { rs.lo = r.lo; rs.inv_span = r.inv_span; rs.model = r.model; rs.nbuckets = r.nbuckets; }
}

// The same bucket as route_bucket (same operations in the same order), with
// the segment found by an unrolled branch-free search and one 128-bit load.
__device__ __forceinline__ int route_fast(const RouteSmem &rs, float x) {
    float y;
    if (rs.model == SR_MODEL_EQUAL_WIDTH) {
        y = x;
    } else {
        int k = 0;                                   // largest k in [0, H-1] with x_k <= x
#pragma unroll
        for (int step = H / 2; step >= 1; step >>= 1) k += (rs.knot[k + step] <= x) ? step : 0;
        const float4 g = rs.seg[k];
        const float u = fminf(fmaxf(__fmul_rn(__fsub_rn(x, g.x), g.y), 0.f), 1.f);
        y = __fmaf_rn(g.z, u, g.w);
    }
    const float yb = __fmul_rn(y, (float)rs.nbuckets);
    int b = yb > 0.f ? (int)fminf(yb, (float)(rs.nbuckets - 1)) : 0;
    if (b > rs.nbuckets - 1) b = rs.nbuckets - 1;
    if (rs.model == SR_MODEL_FORCE_BAD) b = rs.nbuckets - 1 - b;
    return b;
}

template <int KT>
__device__ __forceinline__ float norm_key(typename Key<KT>::T key, const RouteSmem &rs) {
    if (sizeof(typename Key<KT>::U) == 4) {
        const uint32_t u = (uint32_t)Key<KT>::ord(key), lo = (uint32_t)rs.lo;
        const float d = u >= lo ? __uint2float_rn(u - lo) : -__uint2float_rn(lo - u);
        return __fmul_rn(d, rs.inv_span);
    }
    return norm_x((unsigned long long)Key<KT>::ord(key), rs.lo, rs.inv_span);
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

// `exact`: the knots and P as sequential float sums (what routing needs);
// otherwise warp scans (the training steps, where only the gradient matters).
__device__ void derive(const float *theta, Derived &dv, int lane, bool exact = true) {
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
    if (!exact) {
        float xs = d, ps = dv.w[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const float a = __shfl_up_sync(0xffffffffu, xs, o), b = __shfl_up_sync(0xffffffffu, ps, o);
            if (lane >= o) { xs += a; ps += b; }
        }
        dv.knot[lane] = theta[0] + xs - d;
        dv.P[lane] = ps - dv.w[lane];
        if (lane == 31) { dv.knot[H] = theta[0] + xs; dv.P[H] = ps; }
        __syncwarp();
        return;
    }
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
    __shared__ float s_lossw[TRAIN_NT / 32];
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
    __syncthreads();
    const long long S = s_np;
    const long long ppt = (S + TRAIN_NT - 1) / TRAIN_NT;
    const long long p0 = min(S, (long long)t * ppt), p1 = min(S, p0 + ppt);
    const int total_steps = mode == TRAIN_GRAD ? 1 : steps + 1;   // the last pass only measures the loss

    float b1t = 1.f, b2t = 1.f;                    // running powers of Adam's betas
    // up to PREG points per thread stay in registers across the steps
    constexpr int PREG = 8;
    const bool in_regs = ppt <= PREG;
    float rx[PREG], rt[PREG];
#pragma unroll
    for (int q = 0; q < PREG; ++q) {
        const long long i = p0 + q;
        rx[q] = (in_regs && i < p1) ? px[i] : 0.f;
        rt[q] = (in_regs && i < p1) ? pt[i] : 0.f;
    }
    if (wid == 0) derive(th, dv, lane, false);
    __syncthreads();
    for (int it = 0; it < total_steps; ++it) {
        // forward and backward over this thread's points; per segment k of the
        // run of points the thread is in, the partial sums (gw, gs, gkn, gd)
        float loss = 0.f, gw = 0.f, gs = 0.f, gkn = 0.f, gd = 0.f;
        int kc = -1;
        const float gscale = 2.f / (float)S;
        auto point = [&](float x, float tgt) {
            // points arrive in ascending order: walk on from the last segment
            int k = kc;
            if (k < 0 || x < dv.knot[k]) k = segment_of(dv.knot, x);
            while (k < H - 1 && dv.knot[k + 1] <= x) ++k;
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
            const float r = y - tgt;
            loss += r * r;
            const float g = gscale * r;
            gs += g;                                  // every unit before k is saturated at 1
            gw += g * h;
            if (u > 0.f && u < 1.f) {
                const float gu = g * dv.w[k];
                gkn -= gu * dv.invd[k];               // d u / d x_k = -1/d_k
                gd -= gu * u * dv.invd[k];            // d u / d d_k = -u/d_k
            }
        };
        if (in_regs) {
#pragma unroll
            for (int q = 0; q < PREG; ++q)
                if (p0 + q < p1) point(rx[q], rt[q]);
        } else {
            for (long long i = p0; i < p1; ++i) point(px[i], pt[i]);
        }
        // the open run of every lane: lanes of one warp hold non-decreasing
        // segments when the points are sorted, so equal segments are adjacent
        // lanes; a segmented suffix sum leaves each run's total at its first
        // lane, which adds it once (otherwise every lane adds its own)
        const int kprev = __shfl_up_sync(0xffffffffu, kc, 1);
        const bool ordered = __all_sync(0xffffffffu, lane == 0 || kc < 0 || (kprev >= 0 && kprev <= kc));
        if (ordered) {
            for (int o = 1; o < 32; o <<= 1) {
                const int k2 = __shfl_down_sync(0xffffffffu, kc, o);
                const float w2 = __shfl_down_sync(0xffffffffu, gw, o);
                const float s2v = __shfl_down_sync(0xffffffffu, gs, o);
                const float kn2 = __shfl_down_sync(0xffffffffu, gkn, o);
                const float d2 = __shfl_down_sync(0xffffffffu, gd, o);
                if (lane + o < 32 && k2 == kc) { gw += w2; gs += s2v; gkn += kn2; gd += d2; }
            }
        }
        if (kc >= 0 && (!ordered || lane == 0 || kprev != kc)) {
            atomicAdd(&acc_w[kc], gw); atomicAdd(&acc_s[kc], gs);
            atomicAdd(&acc_kn[kc], gkn); atomicAdd(&acc_d[kc], gd);
        }
        for (int o = 16; o; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
        if (lane == 0) s_lossw[wid] = loss;
        __syncthreads();
        if (wid == 0) {
            float lsum = s_lossw[lane];
            for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            const float Lmean = lsum / (float)S;
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
                b1t *= b1;
                b2t *= b2;
                const float c1 = 1.f - b1t, c2 = 1.f - b2t;
                for (int q = lane; q < NPARAM; q += 32) {
                    am[q] = b1 * am[q] + (1.f - b1) * gr[q];
                    av[q] = b2 * av[q] + (1.f - b2) * gr[q] * gr[q];
                    th[q] -= lr * (am[q] / c1) / (sqrtf(av[q] / c2) + eps);
                }
                __syncwarp();
                derive(th, dv, lane, false);       // the next step's tables
            }
            acc_w[lane] = 0.f; acc_s[lane] = 0.f; acc_kn[lane] = 0.f; acc_d[lane] = 0.f;
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

// ----------------------------------------------------- two-level split
//
// A key's bucket b (0 .. B-1) is split into two digits, b >> s2 and
// b & (D2 - 1).  Each level moves every key once: tiles of SPLIT_T keys of
// the level's input segments count their keys per digit in shared memory, one
// exclusive scan over (segment, digit, tile) turns the counts into output
// positions, and the tiles move their keys to those positions, taking slots
// from shared-memory counters.  Level 1 has one segment (the whole input) and
// produces D1 coarse buckets; level 2 splits every coarse bucket into D2 fine
// ones, which are the buckets.  No key needs a global atomic.
constexpr int SPLIT_T = 8192;
constexpr int SPLIT_NT = 512;
constexpr int SCAN_PER_CTA = 8192;

// Tile table of a level (one CTA; at most 1024 segments): tile_base[s] = first
// tile of segment s, tile_base[S] = number of tiles; tile_seg / tile_local
// give every tile's segment and its index inside the segment.
__global__ void __launch_bounds__(1024)
k_split_tiles(const long long *__restrict__ seg_off, int S, int *__restrict__ tile_base, int *__restrict__ tile_seg,
              int *__restrict__ tile_local) {
    griddep_wait();
    __shared__ int s_warp[32];
    __shared__ int s_cnt[1024];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int cnt = t < S ? (int)((seg_off[t + 1] - seg_off[t] + SPLIT_T - 1) / SPLIT_T) : 0;
    int x = cnt;
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = s_warp[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int before = (wid ? s_warp[wid - 1] : 0) + x - cnt;
    s_cnt[t] = t < S ? before : s_warp[31];
    if (t < S) tile_base[t] = before;
    if (t == S - 1) tile_base[S] = before + cnt;
    __syncthreads();
    // every tile finds its segment: the last s with s_cnt[s] <= tile (bases are
    // non-decreasing; empty segments share their base with the next one)
    const int total = s_warp[31];
    for (int tile = t; tile < total; tile += blockDim.x) {
        int lo = 0, hi = S - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_cnt[mid] <= tile) lo = mid;
            else hi = mid - 1;
        }
        tile_seg[tile] = lo;
        tile_local[tile] = tile - s_cnt[lo];
    }
}

__device__ __forceinline__ int digit_of(int b, int level, int s2, int mask2) {
    return level == 1 ? (b >> s2) : (b & mask2);
}

// Loads/stores of VW consecutive bucket ids as one vector (VW * sizeof(BT) is
// 4, 8 or 16 bytes; the address must be aligned to it).
template <typename BT, int VW>
__device__ __forceinline__ void load_ids(const BT *p, int (&b)[VW]) {
    if constexpr (VW * sizeof(BT) == 16) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < VW; ++e) b[e] = sizeof(BT) == 4 ? (int)w[e] : (int)((w[e / 2] >> (16 * (e & 1))) & 0xffffu);
    } else if constexpr (VW * sizeof(BT) == 8) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        const uint32_t w[2] = {q.x, q.y};
#pragma unroll
        for (int e = 0; e < VW; ++e) b[e] = sizeof(BT) == 4 ? (int)w[e] : (int)((w[e / 2] >> (16 * (e & 1))) & 0xffffu);
    } else {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(p);
#pragma unroll
        for (int e = 0; e < VW; ++e) b[e] = sizeof(BT) == 4 ? (int)w : (int)((w >> (16 * (e & 1))) & 0xffffu);
    }
}
template <typename BT, int VW>
__device__ __forceinline__ void store_ids(BT *p, const int (&b)[VW]) {
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < VW; ++e) {
        if (sizeof(BT) == 4) w[e] = (uint32_t)b[e];
        else w[e / 2] |= ((uint32_t)b[e] & 0xffffu) << (16 * (e & 1));
    }
    if constexpr (VW * sizeof(BT) == 16) *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    else if constexpr (VW * sizeof(BT) == 8) *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    else *reinterpret_cast<uint32_t *>(p) = w[0];
}

// Level 1 counts: routes every key once, writes its bucket id (BT) beside it
// and counts the coarse digit per tile.  Level 2 counts: reads the ids only.
// Each thread takes 16-byte vectors of keys (and the ids beside them) where
// the tile is aligned, single keys otherwise.
template <int KT, typename BT, int LEVEL>
__global__ void __launch_bounds__(SPLIT_NT)
k_split_hist(const typename Key<KT>::T *__restrict__ in, const BT *__restrict__ bid_in, BT *__restrict__ bid_out,
             const long long *__restrict__ seg_off, int S, const int *__restrict__ tile_base,
             const int *__restrict__ tile_seg, const int *__restrict__ tile_local, int D, int s2,
             const LearnCtrl *__restrict__ lc, unsigned int *__restrict__ counts) {
    griddep_wait();
    typedef typename Key<KT>::T T;
    constexpr int VW = 16 / sizeof(T);             // keys per 16-byte vector
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NW = SPLIT_NT / 32;
    unsigned int *hall = reinterpret_cast<unsigned int *>(smem);     // [NW][D]: one histogram per warp
    __shared__ RouteSmem rs;
    const int tile = blockIdx.x;
    if (tile >= tile_base[S]) return;
    const int t = threadIdx.x;
    if (LEVEL == 1) load_route(lc->r, rs);
    for (int d = t; d < NW * D; d += SPLIT_NT) hall[d] = 0u;
    unsigned int *hist = hall + (t >> 5) * D;
    __syncthreads();
    const int s = tile_seg[tile], tl = tile_local[tile];
    const int nt = tile_base[s + 1] - tile_base[s];
    const long long start = seg_off[s] + (long long)tl * SPLIT_T;
    const int cnt = (int)(min(start + SPLIT_T, seg_off[s + 1]) - start);
    const int mask2 = (1 << s2) - 1;
    if constexpr (LEVEL == 1) {
        const T *tin = in + start;
        BT *tout = bid_out + start;
        const bool vec = (((uintptr_t)tin) & 15) == 0 && (((uintptr_t)tout) & (VW * sizeof(BT) - 1)) == 0;
        const int nvec = vec ? cnt / VW : 0;
        for (int v = t; v < nvec; v += SPLIT_NT) {
            T k[VW];
            if constexpr (VW == 4) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(tin) + v);
                k[0] = (T)q.x; k[1] = (T)q.y; k[2] = (T)q.z; k[3] = (T)q.w;
            } else {
                const ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2 *>(tin) + v);
                k[0] = (T)q.x; k[1] = (T)q.y;
            }
            int b[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                b[e] = route_fast(rs, norm_key<KT>(k[e], rs));
                atomicAdd(&hist[b[e] >> s2], 1u);
            }
            store_ids<BT, VW>(tout + (long long)v * VW, b);
        }
        for (int i = nvec * VW + t; i < cnt; i += SPLIT_NT) {
            const int b = route_fast(rs, norm_key<KT>(__ldg(tin + i), rs));
            tout[i] = (BT)b;
            atomicAdd(&hist[b >> s2], 1u);
        }
    } else {
        const BT *tin = bid_in + start;
        constexpr int BW = 16 / sizeof(BT);        // ids per 16-byte vector
        const bool vec = (((uintptr_t)tin) & 15) == 0;
        const int nvec = vec ? cnt / BW : 0;
        for (int v = t; v < nvec; v += SPLIT_NT) {
            int b[BW];
            load_ids<BT, BW>(tin + (long long)v * BW, b);
#pragma unroll
            for (int e = 0; e < BW; ++e) atomicAdd(&hist[b[e] & mask2], 1u);
        }
        for (int i = nvec * BW + t; i < cnt; i += SPLIT_NT) atomicAdd(&hist[(int)tin[i] & mask2], 1u);
    }
    __syncthreads();
    const long long base_e = (long long)D * tile_base[s];
    for (int d = t; d < D; d += SPLIT_NT) {
        unsigned int c = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) c += hall[w * D + d];
        counts[base_e + (long long)d * nt + tl] = c;
    }
}

// Moves one tile's keys (and, at level 1, their bucket ids) to the level's
// output: first into shared memory grouped by digit (the tile's own counts,
// scanned, give each digit's stretch; a shared counter hands out slots), then
// out with every digit's stretch written contiguously by one warp.
template <int KT, typename BT, int LEVEL>
__global__ void __launch_bounds__(SPLIT_NT)
k_split_scatter(const typename Key<KT>::T *__restrict__ in, const BT *__restrict__ bid_in,
                typename Key<KT>::T *__restrict__ out, BT *__restrict__ bid_out, const long long *__restrict__ seg_off,
                int S, const int *__restrict__ tile_base, const int *__restrict__ tile_seg,
                const int *__restrict__ tile_local, int D, int s2, LearnCtrl *__restrict__ lc,
                const unsigned int *__restrict__ counts, const unsigned long long *__restrict__ pos,
                int *__restrict__ status_word) {
    griddep_wait();
    typedef typename Key<KT>::T T;
    constexpr int VW = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smem[];
    T *stage_k = reinterpret_cast<T *>(smem);                                       // [SPLIT_T]
    unsigned long long *gbase = reinterpret_cast<unsigned long long *>(stage_k + SPLIT_T);   // [D]
    unsigned int *tstart = reinterpret_cast<unsigned int *>(gbase + D);             // [D + 1]
    unsigned int *taken = tstart + D + 1;                                           // [D]
    BT *stage_b = reinterpret_cast<BT *>(taken + D);                                // [SPLIT_T] (level 1)
    __shared__ unsigned int s_warp[32];
    const int tile = blockIdx.x;
    if (tile >= tile_base[S]) return;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int s = tile_seg[tile], tl = tile_local[tile];
    const int nt = tile_base[s + 1] - tile_base[s];
    const long long base_e = (long long)D * tile_base[s];
    // exclusive scan of this tile's counts over the digits (D <= 1024, two per thread)
    const int d0 = 2 * t, d1 = 2 * t + 1;
    const unsigned int c0 = d0 < D ? counts[base_e + (long long)d0 * nt + tl] : 0u;
    const unsigned int c1 = d1 < D ? counts[base_e + (long long)d1 * nt + tl] : 0u;
    unsigned int x = c0 + c1;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned int w = lane < SPLIT_NT / 32 ? s_warp[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const unsigned int before = (wid ? s_warp[wid - 1] : 0u) + x - (c0 + c1);
    if (d0 < D) { tstart[d0] = before; taken[d0] = before; gbase[d0] = pos[base_e + (long long)d0 * nt + tl]; }
    if (d1 < D) { tstart[d1] = before + c0; taken[d1] = before + c0; gbase[d1] = pos[base_e + (long long)d1 * nt + tl]; }
    if (t == 0) tstart[D] = s_warp[SPLIT_NT / 32 - 1];
    __syncthreads();
    const long long start = seg_off[s] + (long long)tl * SPLIT_T;
    const int cnt = (int)(min(start + SPLIT_T, seg_off[s + 1]) - start);
    const int mask2 = (1 << s2) - 1;
    const T *tin = in + start;
    const BT *bin = bid_in + start;
    bool bad = false;
    auto stage = [&](T k, int b) {
        const int d = LEVEL == 1 ? (b >> s2) : (b & mask2);
        const unsigned int q = atomicAdd(&taken[d], 1u);         // taken[d] starts at the digit's stretch
        if (q < (unsigned int)cnt) {
            stage_k[q] = k;
            if (LEVEL == 1) stage_b[q] = (BT)b;
        } else {
            bad = true;                                          // impossible: the counts came from the same ids
        }
    };
    const bool vec = (((uintptr_t)tin) & 15) == 0 && (((uintptr_t)bin) & (VW * sizeof(BT) - 1)) == 0;
    const int nvec = vec ? cnt / VW : 0;
    for (int v = t; v < nvec; v += SPLIT_NT) {
        T k[VW];
        if constexpr (VW == 4) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(tin) + v);
            k[0] = (T)q.x; k[1] = (T)q.y; k[2] = (T)q.z; k[3] = (T)q.w;
        } else {
            const ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2 *>(tin) + v);
            k[0] = (T)q.x; k[1] = (T)q.y;
        }
        int b[VW];
        load_ids<BT, VW>(bin + (long long)v * VW, b);
#pragma unroll
        for (int e = 0; e < VW; ++e) stage(k[e], b[e]);
    }
    for (int i = nvec * VW + t; i < cnt; i += SPLIT_NT) stage(__ldg(tin + i), (int)bin[i]);
    if (bad) {
        atomicExch(&lc->fallback, 1);
        atomicExch(status_word, (int)SR_ERR_INTERNAL);
    }
    __syncthreads();
    // one warp per digit stretch: contiguous shared reads, contiguous global writes
    for (int d = wid; d < D; d += SPLIT_NT / 32) {
        const unsigned int q0 = tstart[d], q1 = tstart[d + 1];
        T *o = out + gbase[d];
        for (unsigned int q = q0 + lane; q < q1; q += 32) {
            o[q - q0] = stage_k[q];
            if (LEVEL == 1) bid_out[gbase[d] + (q - q0)] = stage_b[q];
        }
    }
}

// Exclusive scan of counts[0 .. E) into pos[0 .. E] (pos[E] = total), in three
// kernels: per-CTA sums, a scan of the sums, per-CTA rescans.
__global__ void __launch_bounds__(1024)
k_scan_sums(const unsigned int *__restrict__ counts, const int *__restrict__ tile_base, int S, int D,
            unsigned long long *__restrict__ sums) {
    griddep_wait();
    __shared__ unsigned long long s_w[32];
    const long long E = (long long)D * tile_base[S];
    const long long e0 = (long long)blockIdx.x * SCAN_PER_CTA;
    if (e0 >= E) return;
    unsigned long long v = 0;
    for (long long e = e0 + threadIdx.x; e < min(E, e0 + SCAN_PER_CTA); e += blockDim.x) v += counts[e];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = s_w[threadIdx.x];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024)
k_scan_top(unsigned long long *__restrict__ sums, const int *__restrict__ tile_base, int S, int D) {
    griddep_wait();
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    const long long E = (long long)D * tile_base[S];
    const long long nb = (E + SCAN_PER_CTA - 1) / SCAN_PER_CTA;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) s_carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < nb; b0 += 1024) {
        const long long i = b0 + t;
        const unsigned long long v = i < nb ? sums[i] : 0ull;
        unsigned long long x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long w = s_w[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const unsigned long long excl = s_carry + (wid ? s_w[wid - 1] : 0ull) + x - v;
        if (i < nb) sums[i] = excl;
        __syncthreads();
        if (t == 0) s_carry += s_w[31];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024)
k_scan_apply(const unsigned int *__restrict__ counts, const int *__restrict__ tile_base, int S, int D,
             const unsigned long long *__restrict__ sums, unsigned long long *__restrict__ pos) {
    griddep_wait();
    __shared__ unsigned long long s_w[32];
    constexpr int PER = SCAN_PER_CTA / 1024;
    const long long E = (long long)D * tile_base[S];
    const long long e0 = (long long)blockIdx.x * SCAN_PER_CTA;
    if (e0 >= E) return;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    unsigned long long v[PER], run = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const long long e = e0 + (long long)t * PER + j;
        v[j] = e < E ? counts[e] : 0u;
        run += v[j];
    }
    unsigned long long x = run;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = s_w[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    unsigned long long p = sums[blockIdx.x] + (wid ? s_w[wid - 1] : 0ull) + x - run;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const long long e = e0 + (long long)t * PER + j;
        if (e < E) pos[e] = p;
        p += v[j];
    }
    if (e0 + SCAN_PER_CTA >= E && t == 1023) pos[E] = p;     // the block holding the last entry
}

__global__ void k_whole_range(long long *__restrict__ seg_off, long long n) {
    griddep_wait();
    if (threadIdx.x == 0) { seg_off[0] = 0; seg_off[1] = n; }
}

// Level 1 -> coarse bucket offsets: coff[c] = position of (digit c, tile 0).
__global__ void k_coarse_off(const unsigned long long *__restrict__ pos, const int *__restrict__ tile_base,
                             int D1, long long n, long long *__restrict__ coff) {
    griddep_wait();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > D1) return;
    const int nt = tile_base[1];
    coff[c] = (c < D1 && nt > 0) ? (long long)pos[(long long)c * nt] : n;
}

// Level 2 -> bucket offsets: boff[c*D2 + f] = position of (coarse c, digit f, tile 0).
__global__ void k_bucket_off(const unsigned long long *__restrict__ pos, const int *__restrict__ tile_base,
                             const long long *__restrict__ coff, int D1, int D2, long long n,
                             long long *__restrict__ boff) {
    griddep_wait();
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long B = (long long)D1 * D2;
    if (b > B) return;
    if (b == B) { boff[B] = n; return; }
    const int c = (int)(b / D2), f = (int)(b % D2);
    const int nt = tile_base[c + 1] - tile_base[c];
    boff[b] = nt > 0 ? (long long)pos[(long long)D2 * tile_base[c] + (long long)f * nt] : coff[c];
}

// Every bucket's last key <= the next bucket's first key (buckets sorted).
// Also records the largest bucket and the sum of squared bucket sizes.
template <int KT>
__global__ void k_bucket_check(const typename Key<KT>::T *__restrict__ keys, const long long *__restrict__ off,
                               int nb, long long n, LearnCtrl *__restrict__ lc) {
    griddep_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;                       // nb is a multiple of 16; whole warps return together
    const unsigned long long len = (unsigned long long)(off[b + 1] - off[b]);
    unsigned long long mx = len, sq = len * len;
    for (int o = 16; o; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(__activemask(), mx, o));
        sq += __shfl_xor_sync(__activemask(), sq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&lc->max_bucket, mx);
        atomicAdd(&lc->bucket_sq, sq);
    }
    if (b == 0) { lc->nkeys = (unsigned long long)n; lc->nbuckets = nb; }
    const long long p = off[b];
    if (b > 0 && p > 0 && p < n && Key<KT>::ord(keys[p - 1]) > Key<KT>::ord(keys[p])) atomicExch(&lc->fallback, 1);
}

// One thread: the condition of the IF node that holds the plain sort inside a
// stream capture, from the bucket check's outcome.
__global__ void k_fallback_cond(cudaGraphConditionalHandle h, const LearnCtrl *__restrict__ lc) {
    griddep_wait();
    if (threadIdx.x != 0) return;              // one setter of the condition
    cudaGraphSetConditional(h, lc->fallback ? 1u : 0u);
}

// ------------------------------------------------------------- host


// A stream per device that captures the fallback IF node's body (it never
// runs work of its own).
static sr_status fallback_capture_stream(int dev, cudaStream_t *out) {
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static cudaStream_t streams[kMaxDev];
    if (dev < 0 || dev >= kMaxDev) return SR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        return launch_status();
    *out = streams[dev];
    return SR_OK;
}

template <int KB> struct UKey;
template <> struct UKey<4> { enum { KT = SR_KEY_U32 }; };
template <> struct UKey<8> { enum { KT = SR_KEY_U64 }; };

template <int KT, typename BT>
static sr_status learned_impl(void *d_keys, size_t n, const sr_learned_opts *o, cudaStream_t s) {
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    constexpr int KTU = UKey<sizeof(U)>::KT;
    const uint32_t nb = o && o->num_buckets ? o->num_buckets : (1u << 16);
    const uint32_t stride = o && o->sample_stride ? o->sample_stride : 100u;
    const uint32_t cap = o && o->train_points ? o->train_points : 2048u;
    uint32_t steps = o && o->train_steps ? o->train_steps : 16u;
    const float lr = o && o->learning_rate > 0.f ? o->learning_rate : 1e-3f;
    const uint32_t model = o ? o->model : 0u;
    const int seg_cfg = o && o->bucket_config ? (int)o->bucket_config - 1 : segmented_default_cfg((int)sizeof(T), true);
    if (nb < 16 || nb > (1u << 20) || (nb & (nb - 1)) || model > SR_MODEL_FORCE_BAD || cap < 2 || cap > (1u << 20) ||
        seg_cfg >= segmented_num_configs((int)sizeof(T)))
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
    cudaStream_t cb = nullptr;                     // made on the first call, before any capture that needs it
    SR_TRY(fallback_capture_stream(ds->device, &cb));

    const long long N = (long long)n;
    const long long m = (N + stride - 1) / stride;
    const PlainSort<KTU, false> sample_sort((size_t)m);
    const PlainSort<KT, false> fallback_sort(n);
    int lb = 0;
    while ((1u << lb) < nb) ++lb;
    const int D2 = 1 << (lb / 2), D1 = (int)(nb >> (lb / 2)), s2 = lb / 2;
    const long long tiles1 = (N + SPLIT_T - 1) / SPLIT_T;
    const long long tiles_max = tiles1 + D1;
    const long long E_max = (long long)std::max(D1, D2) * tiles_max;
    const long long sums_max = (E_max + SCAN_PER_CTA - 1) / SCAN_PER_CTA + 1;
    // scratch: control | sample | sample-sort scratch | points | split tables |
    //          counts | positions | CTA sums | coarse and bucket offsets |
    //          two key buffers | fallback scratch
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off += align_up(bytes, 256); return at; };
    const size_t o_ctrl = take(sizeof(LearnCtrl));
    const size_t o_sample = take((size_t)m * sizeof(U));
    const size_t o_ss = take(sample_sort.bytes);
    const size_t o_px = take((size_t)cap * 4);
    const size_t o_pt = take((size_t)cap * 4);
    const size_t o_range = take(2 * 8);
    const size_t o_tb = take((size_t)(D1 + 2) * 4);
    const size_t o_tseg = take((size_t)tiles_max * 4);
    const size_t o_tloc = take((size_t)tiles_max * 4);
    const size_t o_cnt = take((size_t)E_max * 4);
    const size_t o_pos = take((size_t)(E_max + 1) * 8);
    const size_t o_sums = take((size_t)sums_max * 8);
    const size_t o_coff = take((size_t)(D1 + 1) * 8);
    const size_t o_boff = take((size_t)(nb + 1) * 8);
    const size_t o_ka = take(n * sizeof(T));
    const size_t o_kb = take(n * sizeof(T));
    const size_t o_ba = take(n * sizeof(BT));
    const size_t o_bb = take(n * sizeof(BT));
    const size_t o_fb = take(fallback_sort.bytes);
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, off, s));
    unsigned char *sp = (unsigned char *)scratch;
    LearnCtrl *lc = (LearnCtrl *)(sp + o_ctrl);
    U *sample = (U *)(sp + o_sample);
    float *px = (float *)(sp + o_px), *pt = (float *)(sp + o_pt);
    long long *range = (long long *)(sp + o_range);
    int *tb = (int *)(sp + o_tb), *tseg = (int *)(sp + o_tseg), *tloc = (int *)(sp + o_tloc);
    unsigned int *cnt = (unsigned int *)(sp + o_cnt);
    unsigned long long *pos = (unsigned long long *)(sp + o_pos), *sums = (unsigned long long *)(sp + o_sums);
    long long *coff = (long long *)(sp + o_coff), *boff = (long long *)(sp + o_boff);
    T *ka = (T *)(sp + o_ka), *kb = (T *)(sp + o_kb);
    BT *ba = (BT *)(sp + o_ba), *bb = (BT *)(sp + o_bb);
    T *uk = (T *)d_keys;

    sr_status st = SR_OK;
    do {
        if (cudaMemsetAsync(lc, 0, sizeof(LearnCtrl), s) != cudaSuccess) { st = launch_status(); break; }
        SR_LAUNCH(SR_KERNEL_MODEL, k_sample<KT>, (unsigned)((m + 255) / 256), 256, 0, s, uk, m, (long long)stride,
                  sample);
        if ((st = sample_sort.launch((typename PlainSort<KTU, false>::T *)sample, nullptr, sp + o_ss, s)) != SR_OK)
            break;
        SR_LAUNCH(SR_KERNEL_MODEL, k_train<U>, 1, TRAIN_NT, 0, s, sample, m, px, pt, (long long)0,
                  (int)TRAIN_PIPELINE, (int)steps, lr, (int)cap, (int)model, (int)nb, lc);
        // level 1: the whole input -> D1 coarse buckets (ka)
        SR_LAUNCH(SR_KERNEL_MODEL, k_whole_range, 1, 32, 0, s, range, N);
        for (int level = 1; level <= 2; ++level) {
            const int S = level == 1 ? 1 : D1;
            const int D = level == 1 ? D1 : D2;
            const long long *segs = level == 1 ? range : coff;
            const T *in = level == 1 ? uk : ka;
            T *out = level == 1 ? ka : kb;
            const unsigned grid = (unsigned)(level == 1 ? tiles1 : tiles_max);
            const unsigned sgrid = (unsigned)(((long long)D * grid + SCAN_PER_CTA - 1) / SCAN_PER_CTA);
            // level 1 writes the bucket ids (ba) beside the keys; they move with the keys (bb)
            const BT *bin = level == 1 ? ba : bb;
            SR_LAUNCH(SR_KERNEL_MODEL, k_split_tiles, 1, 1024, 0, s, segs, S, tb, tseg, tloc);
            const size_t h_smem = (size_t)(SPLIT_NT / 32) * D * 4;
            auto hist_kernel = level == 1 ? k_split_hist<KT, BT, 1> : k_split_hist<KT, BT, 2>;
            if (h_smem > 48 * 1024 &&
                cudaFuncSetAttribute((const void *)hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)h_smem) != cudaSuccess) {
                st = launch_status();
                break;
            }
            SR_LAUNCH(SR_KERNEL_MODEL, hist_kernel, grid, SPLIT_NT, h_smem, s, in, bin, ba, segs, S, tb, tseg, tloc, D,
                      s2, lc, cnt);
            SR_LAUNCH(SR_KERNEL_MODEL, k_scan_sums, sgrid, 1024, 0, s, cnt, tb, S, D, sums);
            SR_LAUNCH(SR_KERNEL_MODEL, k_scan_top, 1, 1024, 0, s, sums, tb, S, D);
            SR_LAUNCH(SR_KERNEL_MODEL, k_scan_apply, sgrid, 1024, 0, s, cnt, tb, S, D, sums, pos);
            const size_t sc_smem = (size_t)SPLIT_T * (sizeof(T) + (level == 1 ? sizeof(BT) : 0)) + (size_t)D * 16 + 4;
            auto scatter_kernel = level == 1 ? k_split_scatter<KT, BT, 1> : k_split_scatter<KT, BT, 2>;
            if (sc_smem > 48 * 1024 &&
                cudaFuncSetAttribute((const void *)scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sc_smem) != cudaSuccess) {
                st = launch_status();
                break;
            }
            SR_LAUNCH(SR_KERNEL_MODEL, scatter_kernel, grid, SPLIT_NT, sc_smem, s, in, bin, out,
                      level == 1 ? bb : (BT *)nullptr, segs, S, tb, tseg, tloc, D, s2, lc, cnt, pos, ds->status);
            if (level == 1) {
                SR_LAUNCH(SR_KERNEL_MODEL, k_coarse_off, (unsigned)((D1 + 1 + 255) / 256), 256, 0, s, pos, tb, D1, N,
                          coff);
            } else {
                SR_LAUNCH(SR_KERNEL_MODEL, k_bucket_off, (unsigned)((nb + 1 + 255) / 256), 256, 0, s, pos, tb, coff,
                          D1, D2, N, boff);
            }
        }
        if (st != SR_OK) break;
        // every bucket sorted, kb -> the caller's buffer
        if ((st = segmented_run_cfg<KT>(kb, uk, n, (const int64_t *)boff, nb, s, false, seg_cfg)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_MODEL, k_bucket_check<KT>, (unsigned)((nb + 255) / 256), 256, 0, s, uk, boff, (int)nb,
                  N, lc);
        if (cudaMemcpyAsync(ds->last_aux, lc, sizeof(LearnCtrl), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            st = launch_status();
            break;
        }
        rec.aux_kind = 4;
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) { st = launch_status(); break; }
        if (cst == cudaStreamCaptureStatusActive) {
            // inside the caller's capture: the plain sort goes into the body of
            // an IF node whose condition the check's outcome sets on the device
            // (no host read); its kernels run only when a replay falls back
            cudaGraphConditionalHandle h;
            if ((st = new_handle(s, &h)) != SR_OK) break;
            SR_LAUNCH(SR_KERNEL_MODEL, k_fallback_cond, 1, 32, 0, s, h, (const LearnCtrl *)lc);
            cudaGraph_t body[1];
            if ((st = add_conditional(s, h, cudaGraphCondTypeIf, 1, body)) != SR_OK) break;
            unsigned int k = 0;
            st = capture_into(body[0], cb, [&](cudaStream_t x) { return fallback_sort.launch(uk, nullptr, sp + o_fb, x); },
                              &k);
            count_launches(-(long long)k);         // captured into the body, run only on a fallback
            break;
        }
        // the check's outcome decides whether the plain sort runs: read it back
        // (launching the plain sort gated on the device would still cost every
        // one of its kernels a full grid of empty CTAs)
        int fallback = 0;
        if (cudaMemcpyAsync(&fallback, &lc->fallback, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = launch_status();
            if (st == SR_OK) st = SR_ERR_CUDA;
            break;
        }
        if (fallback && (st = fallback_sort.launch(uk, nullptr, sp + o_fb, s)) != SR_OK) break;
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
    const bool wide = opts && opts->num_buckets > (1u << 16);     // bucket ids need 32 bits
    switch (kt) {
    case SR_KEY_I32: return wide ? learned_impl<SR_KEY_I32, uint32_t>(d_keys, n, opts, s)
                                 : learned_impl<SR_KEY_I32, uint16_t>(d_keys, n, opts, s);
    case SR_KEY_U32: return wide ? learned_impl<SR_KEY_U32, uint32_t>(d_keys, n, opts, s)
                                 : learned_impl<SR_KEY_U32, uint16_t>(d_keys, n, opts, s);
    case SR_KEY_F32: return wide ? learned_impl<SR_KEY_F32, uint32_t>(d_keys, n, opts, s)
                                 : learned_impl<SR_KEY_F32, uint16_t>(d_keys, n, opts, s);
    case SR_KEY_U64: return wide ? learned_impl<SR_KEY_U64, uint32_t>(d_keys, n, opts, s)
                                 : learned_impl<SR_KEY_U64, uint16_t>(d_keys, n, opts, s);
    case SR_KEY_I64: return wide ? learned_impl<SR_KEY_I64, uint32_t>(d_keys, n, opts, s)
                                 : learned_impl<SR_KEY_I64, uint16_t>(d_keys, n, opts, s);
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
