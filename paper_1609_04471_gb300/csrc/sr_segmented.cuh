// sr_segmented.cuh -- the segmented sort (many arrays, each sorted on its
// own, in one batched launch sequence), templated on its launch
// configuration; instantiated per key width in sr_seg_k4.cu / sr_seg_k8.cu,
// entry points in sr_segmented.cu.
//
// The paper sorts one array per call (Section 1); a batch is those calls side
// by side.  Segments are sorted in place by size class:
//
//   small   len <= C      Consecutive small segments that start in the same
//                         chunk of C keys form a "pack" of at most 2C keys.  One
//                         CTA sorts a pack as composite keys (index of the
//                         segment inside the pack, key): each segment comes out
//                         sorted in its own place.  At most one non-small
//                         segment starts in a chunk (it is longer than C), so a
//                         pack is always contiguous.
//   medium  C < len <= F*T  One CTA sorts the segment: F block-sort tiles of T
//                         keys merged in shared memory (F is the merge fan-in
//                         of the configuration).
//   big     len > F*T     Its F*T-key tiles are sorted that way, then merge passes
//                         (policy e1 of Section 3) run over every big segment
//                         at once; a segment that needs p passes keeps its
//                         data in the buffer that makes its last pass land home.
//
// Launches: k_seg_classify (one thread per segment: checks the offsets, marks
// the first segment of every chunk, lists medium and big segments),
// k_seg_bigscan (tile bases of big segments), k_seg_sort (one persistent
// kernel whose CTAs pull packs, medium segments and big-segment tiles from a
// work queue), k_seg_merge x passes (each exits at once when no big segment
// needs that pass), k_seg_finish (device status word).  No launch depends on a
// value read back to the host, so sr_sort_segmented_ex can be captured in a
// CUDA graph.
#pragma once
#include <algorithm>
#include <cstring>

#include "sr_device.cuh"
#include "sr_kernels.cuh"
#include "sr_runtime.cuh"

namespace sr {

// ---------------------------------------------------------- composite keys

// (segment index inside the pack, key image): ordering by the pair sorts every
// segment of a pack independently.
template <int KB> struct Comp;
template <> struct Comp<4> {
    typedef unsigned long long C;
    static __device__ __forceinline__ C make(unsigned int seg, uint32_t u) {
        return ((unsigned long long)seg << 32) | u;
    }
    template <typename U> static __device__ __forceinline__ U key(C c) { return (U)(uint32_t)c; }
};

struct Comp96 {
    unsigned long long key;
    unsigned int seg;
    unsigned int pad;
    __device__ __forceinline__ Comp96() {}
    __device__ __forceinline__ explicit Comp96(int) : key(0), seg(0), pad(0) {}
    __device__ __forceinline__ bool operator<(const Comp96 &o) const {
        return seg < o.seg || (seg == o.seg && key < o.key);
    }
    __device__ __forceinline__ bool operator>(const Comp96 &o) const { return o < *this; }
};
template <> __device__ __forceinline__ Comp96 umax_of<Comp96>() {
    Comp96 c(0);
    c.key = ~0ull;
    c.seg = ~0u;
    return c;
}
template <> struct Comp<8> {
    typedef Comp96 C;
    static __device__ __forceinline__ C make(unsigned int seg, unsigned long long u) {
        C c(0);
        c.key = u;
        c.seg = seg;
        return c;
    }
    template <typename U> static __device__ __forceinline__ U key(const C &c) { return (U)c.key; }
};

// ------------------------------------------------------------ configurations

// A launch configuration of the segmented sort (the autotuner picks one per
// workload):
//   BUCKETS  0: small segments (<= C = SNT*IPT_P/2) share a CTA as composite
//            keys ("packs"); 1: one CTA of the smallest of five fixed shapes
//            (from ladder LADDER, below) per small segment (<= 3840 keys).
//   SNT      threads of the persistent sort CTA.
//   IPT_P    composite keys per thread of a pack.
//   IPT      keys per thread of a block-sort tile (T = SNT * IPT).
//   F        merge fan-in: block-sort tiles one CTA merges in shared memory,
//            so one CTA sorts up to F*T keys and long segments start their
//            global merge passes from runs of F*T keys.
// Global merge passes over long segments use tiles of 256 * IPT keys.
template <int BUCKETS_, int SNT_, int IPT_P_, int IPT_, int F_, int LADDER_ = 0> struct SegCfg {
    enum { BUCKETS = BUCKETS_, SNT = SNT_, IPT_P = IPT_P_, IPT = IPT_, F = F_, MNT = 256, MIPT = IPT_,
           LADDER = LADDER_ };
};
// Bucket mode (segments of similar, moderate sizes): a small segment gets one
// CTA of the smallest shape that holds it, instead of sharing a pack.  Two
// ladders of shapes (threads x keys per thread, IPT odd):
//   ladder 0: 128x9, 128x15, 256x9, 256x11, 256x15
//   ladder 1:  64x9, 128x9, 128x15, 256x11, 256x15
//   ladder 2: 128x13, 128x17, 128x19, 128x23, 256x15 (segments of 1,200-3,000 keys:
//             one merge level fewer than 256-thread shapes)
enum { NSMALL = 5 };
__host__ __device__ constexpr int small_nt(int ladder, int c) {
    return ladder == 0 ? (c < 2 ? 128 : 256) : ladder == 1 ? (c == 0 ? 64 : c < 3 ? 128 : 256) : (c < 4 ? 128 : 256);
}
__host__ __device__ constexpr int small_ipt(int ladder, int c) {
    return ladder == 0 ? (c == 0 || c == 2 ? 9 : c == 1 || c == 4 ? 15 : 11)
         : ladder == 1 ? (c < 2 ? 9 : c == 2 ? 15 : c == 3 ? 11 : 15)
                       : (c == 0 ? 13 : c == 1 ? 17 : c == 2 ? 19 : c == 3 ? 23 : 15);
}
__host__ __device__ constexpr int small_cap(int ladder, int c) { return small_nt(ladder, c) * small_ipt(ladder, c); }
static_assert(small_cap(0, 0) == 1152 && small_cap(0, 1) == 1920 && small_cap(0, 2) == 2304 &&
                  small_cap(0, 3) == 2816 && small_cap(0, 4) == 3840 && small_cap(1, 0) == 576 &&
                  small_cap(1, 1) == 1152 && small_cap(1, 2) == 1920 && small_cap(1, 3) == 2816 &&
                  small_cap(1, 4) == 3840 && small_cap(2, 0) == 1664 && small_cap(2, 1) == 2176 &&
                  small_cap(2, 2) == 2432 && small_cap(2, 3) == 2944 && small_cap(2, 4) == 3840,
              "small-shape ladders");

struct SegCtrl {
    int status;                  // SR_ERR_BAD_SEGMENTS when the offsets fail the check
    unsigned int n_medium;
    unsigned int n_big;
    unsigned int n_big_tiles;    // block-sort tiles of all big segments
    unsigned int n_big_mtiles;   // merge tiles of all big segments
    int max_passes;              // most merge passes any big segment needs
    unsigned int work_next;      // work queue of k_seg_sort
    unsigned int pad1;
    unsigned long long big_keys;
    unsigned int n_small[NSMALL];  // bucket mode: segments per small shape
    unsigned int pad2;
};

__device__ __forceinline__ int dev_ceil_log2(long long x) {
    int r = 0;
    while ((1ll << r) < x) ++r;
    return r;
}

// ----------------------------------------------------------- kernels

// Packs mode: marks the first segment of every chunk and lists medium and big
// segments.  Bucket mode: lists every segment under the smallest small shape
// that holds it (lists[cls * nseg + i]), or as medium or big; no packs.
// Appends s to a list through one atomic per warp and list: the lanes that
// append to `counter` (all lanes of the warp call this with `take` set or not)
// get consecutive slots from the lowest lane's single atomicAdd.
__device__ __forceinline__ void warp_append(bool take, unsigned int *counter, unsigned int *list, unsigned int s) {
    const unsigned int lanes = __ballot_sync(0xffffffffu, take);
    if (!take) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(lanes) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned int)__popc(lanes));
    base = __shfl_sync(lanes, base, leader);
    list[base + __popc(lanes & ((1u << lane) - 1u))] = s;
}

static __global__ void k_seg_classify(const int64_t *__restrict__ off, long long nseg, long long nkeys, int chunk,
                               int tile, long long nchunks, int *__restrict__ chunk_first,
                               unsigned int *__restrict__ medium, unsigned int *__restrict__ big,
                               int bucket_mode, int ladder, unsigned int *__restrict__ lists,
                               SegCtrl *__restrict__ c) {
    griddep_wait();
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s < nseg;                    // every lane stays to the end (warp-wide appends)
    long long a = 0, b = 0, prev = 0;
    if (live) {
        a = off[s];
        b = off[s + 1];
        prev = s > 0 ? off[s - 1] : 0;
    }
    const bool bad = live && (b < a || a < 0 || b > nkeys || prev > a);
    if (bad) atomicExch(&c->status, (int)SR_ERR_BAD_SEGMENTS);
    const bool ok = live && !bad;
    const long long len = b - a;
    if (bucket_mode) {
        // (a single key still moves when in != out)
        int cls = NSMALL;
        if (ok && len >= 1)
            for (int q = NSMALL - 1; q >= 0; --q)
                if (len <= small_cap(ladder, q)) cls = q;
#pragma unroll
        for (int q = 0; q < NSMALL; ++q)
            warp_append(cls == q, &c->n_small[q], lists + (long long)q * nseg, (unsigned int)s);
        const bool med = ok && cls == NSMALL && len > chunk && len <= tile;
        const bool bg = ok && cls == NSMALL && len > tile;
        warp_append(med, &c->n_medium, medium, (unsigned int)s);
        warp_append(bg, &c->n_big, big, (unsigned int)s);
        if (bg) atomicAdd(&c->big_keys, (unsigned long long)len);
        return;
    }
    if (!ok) return;
    {
        // chunks (chunk of the previous start, chunk of this start] begin with s
        const long long cs = a / chunk;
        const long long cp = s > 0 ? prev / chunk : -1;
        for (long long q = cp + 1; q <= cs && q <= nchunks; ++q) chunk_first[q] = (int)s;
        if (s == nseg - 1)
            for (long long q = cs + 1; q <= nchunks; ++q) chunk_first[q] = (int)nseg;
    }
    if (len > chunk) {
        if (len <= tile) {
            medium[atomicAdd(&c->n_medium, 1u)] = (unsigned int)s;
        } else {
            big[atomicAdd(&c->n_big, 1u)] = (unsigned int)s;
            atomicAdd(&c->big_keys, (unsigned long long)len);
        }
    }
}

// Tile bases of the big segments, in list order (one CTA).
static __global__ void __launch_bounds__(1024)
k_seg_bigscan(const int64_t *__restrict__ off, const unsigned int *__restrict__ big, int tile, int mtile,
              unsigned int *__restrict__ tile_base, unsigned int *__restrict__ mtile_base,
              SegCtrl *__restrict__ c) {
    griddep_wait();
    __shared__ unsigned int s_carry[2];
    __shared__ unsigned int s_warp[2][32];
    __shared__ int s_maxp;
    if (c->status) return;
    const unsigned int nb = c->n_big;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) { s_carry[0] = 0; s_carry[1] = 0; s_maxp = 0; }
    __syncthreads();
    int maxp = 0;
    for (unsigned int base = 0; base < nb; base += blockDim.x) {
        const unsigned int i = base + t;
        unsigned int nt = 0, nm = 0;
        if (i < nb) {
            const long long len = off[big[i] + 1] - off[big[i]];
            nt = (unsigned int)((len + tile - 1) / tile);
            nm = (unsigned int)((len + mtile - 1) / mtile);
            maxp = max(maxp, dev_ceil_log2(nt));
        }
        // block-wide exclusive scan of (nt, nm)
        unsigned int xt = nt, xm = nm;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned int yt = __shfl_up_sync(0xffffffffu, xt, d);
            const unsigned int ym = __shfl_up_sync(0xffffffffu, xm, d);
            if (lane >= d) { xt += yt; xm += ym; }
        }
        if (lane == 31) { s_warp[0][wid] = xt; s_warp[1][wid] = xm; }
        __syncthreads();
        if (wid == 0) {
            unsigned int wt = lane < (int)(blockDim.x >> 5) ? s_warp[0][lane] : 0u;
            unsigned int wm = lane < (int)(blockDim.x >> 5) ? s_warp[1][lane] : 0u;
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned int yt = __shfl_up_sync(0xffffffffu, wt, d);
                const unsigned int ym = __shfl_up_sync(0xffffffffu, wm, d);
                if (lane >= d) { wt += yt; wm += ym; }
            }
            s_warp[0][lane] = wt;
            s_warp[1][lane] = wm;
        }
        __syncthreads();
        const unsigned int before_t = (wid ? s_warp[0][wid - 1] : 0u) + xt - nt + s_carry[0];
        const unsigned int before_m = (wid ? s_warp[1][wid - 1] : 0u) + xm - nm + s_carry[1];
        if (i < nb) { tile_base[i] = before_t; mtile_base[i] = before_m; }
        __syncthreads();
        if (t == 0) {
            s_carry[0] += s_warp[0][(blockDim.x >> 5) - 1];
            s_carry[1] += s_warp[1][(blockDim.x >> 5) - 1];
        }
        __syncthreads();
    }
    atomicMax(&s_maxp, maxp);
    __syncthreads();
    if (t == 0) {
        c->n_big_tiles = s_carry[0];
        c->n_big_mtiles = s_carry[1];
        c->max_passes = s_maxp;
        tile_base[nb] = s_carry[0];
        mtile_base[nb] = s_carry[1];
    }
}

// index i with base[i] <= j < base[i + 1] (base non-decreasing, base[0] = 0)
__device__ __forceinline__ unsigned int find_base(const unsigned int *__restrict__ base, unsigned int n,
                                                  unsigned int j) {
    unsigned int lo = 0, hi = n;                  // answer in [lo, hi)
    while (hi - lo > 1) {
        const unsigned int mid = (lo + hi) >> 1;
        if (base[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Sorts keys[g0 .. g0+cnt) in place with the plain block sort (cnt <= SNT*IPT),
// writing the result to dst (which may be keys).
template <int KT, int SNT, int IPT>
__device__ __forceinline__ void sort_range(const typename Key<KT>::T *src, typename Key<KT>::T *dst, long long g0,
                                           int cnt, typename Key<KT>::U *s) {
    typedef Key<KT> K;
    typedef typename K::U U;
    const int t = threadIdx.x;
    uint32_t dummy_v[IPT];
    U k[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int idx = i * SNT + t;
        s[idx] = idx < cnt ? K::ord(src[g0 + idx]) : umax_of<U>();
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) { k[i] = s[t * IPT + i]; dummy_v[i] = 0u; }
    __syncthreads();
    block_sort<U, SNT, IPT, false>(k, dummy_v, s, nullptr);
#pragma unroll
    for (int i = 0; i < IPT; ++i) s[t * IPT + i] = k[i];
    __syncthreads();
    for (int idx = t; idx < cnt; idx += SNT) dst[g0 + idx] = K::unord(s[idx]);
    __syncthreads();
}

// Sorts keys[g0 .. g0+cnt) (cnt <= F*SNT*IPT) into dst: each of the F tiles
// of SNT*IPT keys is block-sorted, then log2(F) rounds of pairwise merges in
// shared memory (s: 2*F*SNT*IPT images, two buffers) join the sorted tiles.
template <int KT, int SNT, int IPT, int F>
__device__ __forceinline__ void sort_range_f(const typename Key<KT>::T *src, typename Key<KT>::T *dst,
                                             long long g0, int cnt, typename Key<KT>::U *s) {
    if constexpr (F == 1) {
        sort_range<KT, SNT, IPT>(src, dst, g0, cnt, s);
    } else {
        typedef Key<KT> K;
        typedef typename K::U U;
        constexpr int TT = SNT * IPT, FT = F * TT;
        U *x = s, *y = s + FT;
        const int t = threadIdx.x;
        for (int idx = t; idx < FT; idx += SNT) x[idx] = idx < cnt ? K::ord(src[g0 + idx]) : umax_of<U>();
        __syncthreads();
        const int nt = (cnt + TT - 1) / TT;        // tiles holding keys; the rest are padding
        uint32_t dv[IPT];
        U k[IPT];
        for (int f = 0; f < nt; ++f) {
#pragma unroll
            for (int i = 0; i < IPT; ++i) { k[i] = x[f * TT + t * IPT + i]; dv[i] = 0u; }
            block_sort<U, SNT, IPT, false>(k, dv, y, nullptr);   // y: the block sort's own scratch
#pragma unroll
            for (int i = 0; i < IPT; ++i) x[f * TT + t * IPT + i] = k[i];
            __syncthreads();
        }
        U *from = x, *to = y;
        for (int len = TT; len < nt * TT; len <<= 1) {
            // merge runs [2j*len, (2j+1)*len) and [(2j+1)*len, (2j+2)*len)
            const int limit = ((nt * TT + 2 * len - 1) / (2 * len)) * (2 * len);
            for (int r = 0; r < F; ++r) {
                const int g = (r * SNT + t) * IPT;     // first output of this thread
                if (g < limit) {
                    const int base = (g / (2 * len)) * (2 * len), d = g - base;
                    const int sp = merge_path(from + base, len, from + base + len, len, d);
                    int ix[IPT];
                    serial_merge<U, IPT>(from, base + sp, base + len, base + len + d - sp, base + 2 * len, k, ix);
#pragma unroll
                    for (int i = 0; i < IPT; ++i) to[g + i] = k[i];
                }
            }
            __syncthreads();
            U *tmp = from; from = to; to = tmp;
        }
        for (int idx = t; idx < cnt; idx += SNT) dst[g0 + idx] = K::unord(from[idx]);
        __syncthreads();
    }
}

// Reads every segment from `in` and writes it sorted to `out` (in == out sorts
// in place).  Tiles of big segments that need an odd number of merge passes go
// to `alt`, the merge passes' other buffer (alt may be in when in != out).
template <int KT, typename CFG>
__global__ void __launch_bounds__(CFG::SNT)
k_seg_sort(const typename Key<KT>::T *in, typename Key<KT>::T *out, typename Key<KT>::T *alt,
           const int64_t *__restrict__ off,
           long long nchunks, const int *__restrict__ chunk_first, const unsigned int *__restrict__ medium,
           const unsigned int *__restrict__ big, const unsigned int *__restrict__ tile_base,
           SegCtrl *__restrict__ c) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    typedef Comp<sizeof(T)> CP;
    typedef typename CP::C C;
    constexpr int SNT = CFG::SNT, IPT_P = CFG::IPT_P, IPT = CFG::IPT, F = CFG::F;
    constexpr int PT = SNT * IPT_P;          // pack tile
    constexpr int CH = PT / 2;               // chunk
    constexpr int FT = F * SNT * IPT;        // keys one CTA sorts
    extern __shared__ __align__(16) unsigned char smem[];
    C *sc = reinterpret_cast<C *>(smem);                       // pack composites [PT]
    int *sf = reinterpret_cast<int *>(sc + PT);                // pack segment flags [PT]
    U *su = reinterpret_cast<U *>(smem);                       // plain tile [TT] (aliases sc)
    __shared__ unsigned int s_item;
    __shared__ int s_warp[SNT / 32];
    if (c->status) return;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned int n_medium = c->n_medium;
    const unsigned int n_big = c->n_big;
    const unsigned long long total = (unsigned long long)nchunks + n_medium + c->n_big_tiles;
    for (;;) {
        if (t == 0) s_item = atomicAdd(&c->work_next, 1u);
        __syncthreads();
        const unsigned long long item = s_item;
        __syncthreads();
        if (item >= total) break;
        if (!CFG::BUCKETS && item < (unsigned long long)nchunks) {
            // ---- a pack: the small segments that start in chunk `item`
            int sb = chunk_first[item], se = chunk_first[item + 1];
            if (se > sb && off[se] - off[se - 1] > CH) --se;   // the one non-small segment
            if (se - sb < 1) continue;
            const long long g0 = off[sb];
            const int cnt = (int)(off[se] - g0);
            if (cnt < 1) continue;                 // a single key still moves when in != out
            for (int i = t; i < PT; i += SNT) sf[i] = 0;
            __syncthreads();
            for (int q = sb + 1 + t; q < se; q += SNT) {
                const int pos = (int)(off[q] - g0);
                if (pos < cnt) atomicAdd(&sf[pos], 1);
            }
            __syncthreads();
            // inclusive scan of the flags over the thread-blocked layout:
            // segment index inside the pack of every position
            int run[IPT_P];
            int acc = 0;
#pragma unroll
            for (int i = 0; i < IPT_P; ++i) { acc += sf[t * IPT_P + i]; run[i] = acc; }
            int x = acc;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += y;
            }
            if (lane == 31) s_warp[wid] = x;
            __syncthreads();
            if (wid == 0) {
                int w = lane < SNT / 32 ? s_warp[lane] : 0;
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, w, d);
                    if (lane >= d) w += y;
                }
                if (lane < SNT / 32) s_warp[lane] = w;
            }
            __syncthreads();
            const int before = (wid ? s_warp[wid - 1] : 0) + x - acc;
            C kc[IPT_P];
            uint32_t dv[IPT_P];
#pragma unroll
            for (int i = 0; i < IPT_P; ++i) {
                const int pos = t * IPT_P + i;
                kc[i] = pos < cnt ? CP::make((unsigned int)(before + run[i]), K::ord(in[g0 + pos]))
                                  : umax_of<C>();
                dv[i] = 0u;
            }
            __syncthreads();
            block_sort<C, SNT, IPT_P, false>(kc, dv, sc, nullptr);
#pragma unroll
            for (int i = 0; i < IPT_P; ++i) sc[t * IPT_P + i] = kc[i];
            __syncthreads();
            for (int i = t; i < cnt; i += SNT) out[g0 + i] = K::unord(CP::template key<U>(sc[i]));
            __syncthreads();
        } else if (item < (unsigned long long)nchunks + n_medium) {
            // ---- a medium segment: one CTA sort
            const unsigned int sgi = medium[item - nchunks];
            const long long g0 = off[sgi];
            sort_range_f<KT, SNT, IPT, F>(in, out, g0, (int)(off[sgi + 1] - g0), su);
        } else {
            // ---- one block-sort tile of a big segment
            const unsigned int j = (unsigned int)(item - nchunks - n_medium);
            const unsigned int bi = find_base(tile_base, n_big, j);
            const unsigned int sgi = big[bi];
            const long long s0 = off[sgi], len = off[sgi + 1] - s0;
            const long long g0 = s0 + (long long)(j - tile_base[bi]) * FT;
            const int cnt = (int)min((long long)FT, s0 + len - g0);
            const int passes = dev_ceil_log2((len + FT - 1) / FT);
            sort_range_f<KT, SNT, IPT, F>(in, (passes & 1) ? alt : out, g0, cnt, su);
        }
    }
}

// Bucket mode: one CTA of NT threads per listed segment (at most NT*IPT keys).
template <int KT, int NT, int IPT>
__global__ void __launch_bounds__(NT)
k_seg_small(const typename Key<KT>::T *in, typename Key<KT>::T *out, const int64_t *__restrict__ off,
            const unsigned int *__restrict__ list, int cls, SegCtrl *__restrict__ c) {
    griddep_wait();
    typedef typename Key<KT>::U U;
    extern __shared__ __align__(16) unsigned char smem[];
    U *su = reinterpret_cast<U *>(smem);
    if (c->status) return;
    const unsigned int count = c->n_small[cls];
    for (unsigned int i = blockIdx.x; i < count; i += gridDim.x) {
        const unsigned int sgi = list[i];
        const long long g0 = off[sgi];
        sort_range<KT, NT, IPT>(in, out, g0, (int)(off[sgi + 1] - g0), su);
    }
}

// Merge pass p over the merge tiles of every big segment that needs it.
template <int KT, int NT, int IPT, bool VEC>
__global__ void __launch_bounds__(NT)
k_seg_merge(typename Key<KT>::T *out, typename Key<KT>::T *alt, long long nkeys,
            const int64_t *__restrict__ off, const unsigned int *__restrict__ big,
            const unsigned int *__restrict__ mtile_base, int tile, int p, SegCtrl *__restrict__ c) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    constexpr int NV = NT * IPT;
    constexpr int SV = NV + 16;
    if (c->status || p >= c->max_passes) return;
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    __shared__ long long s_split[2];
    const int t = threadIdx.x;
    const unsigned int n_big = c->n_big, n_mt = c->n_big_mtiles;
    for (unsigned int j = blockIdx.x; j < n_mt; j += gridDim.x) {
        const unsigned int bi = find_base(mtile_base, n_big, j);
        const unsigned int sgi = big[bi];
        const long long s0 = off[sgi], len = off[sgi + 1] - s0;
        const int passes = dev_ceil_log2((len + tile - 1) / tile);
        if (p >= passes) continue;
        const long long w = (long long)tile << p;
        const long long lo0 = (long long)(j - mtile_base[bi]) * NV;    // tile start inside the segment
        const long long lo1 = min(lo0 + NV, len);
        const long long pb = (lo0 / (2 * w)) * (2 * w);
        const long long a_beg = s0 + pb, a_end = s0 + min(pb + w, len);
        const long long b_beg = a_end, b_end = s0 + min(pb + 2 * w, len);
        const int cur = (passes - p) & 1;                             // 1: the data is in alt
        const T *src = cur ? alt : out;
        T *dst = cur ? out : alt;
        if (t < 64) {
            const int which = t >> 5;
            const long long out = which ? lo1 : lo0;
            long long sp;
            if (which && s0 + lo1 == b_end) sp = a_end - a_beg;
            else sp = warp_split<K>(src, a_beg, a_end - a_beg, b_beg, b_end - b_beg, out - pb, t & 31);
            if ((t & 31) == 0) s_split[which] = a_beg + sp;
        }
        __syncthreads();
        const long long a0 = s_split[0], a1 = s_split[1];
        const long long b0 = b_beg + (lo0 - pb) - (a0 - a_beg);
        merge_tile<KT, NT, IPT, false, VEC>(src, dst, nullptr, nullptr, nkeys, s0 + lo0, (int)(lo1 - lo0), a0, a1,
                                            b0, s, nullptr);
        __syncthreads();
    }
    (void)SV;
}

static __global__ void k_seg_finish(const SegCtrl *__restrict__ c, int *__restrict__ status_word) {
    griddep_wait();
    if (threadIdx.x == 0 && c->status) atomicExch(status_word, c->status);
}

// ------------------------------------------------------------- host

template <typename FN>
static sr_status allow_smem(FN *kernel, size_t bytes) {
    if (bytes > 48 * 1024 && cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)bytes) != cudaSuccess)
        return launch_status();
    return SR_OK;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <int KT, typename CFG>
sr_status segmented_run_t(const typename Key<KT>::T *in, typename Key<KT>::T *out, size_t n_keys,
                          const int64_t *d_off, size_t nseg, cudaStream_t s, bool record) {
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    typedef typename Comp<sizeof(T)>::C C;
    constexpr bool bucket_mode = CFG::BUCKETS != 0;
    constexpr int SNT = CFG::SNT, PT = SNT * CFG::IPT_P, CH = PT / 2;
    constexpr int TT = CFG::F * SNT * CFG::IPT;    // keys one CTA sorts: the run length before merge passes
    constexpr int MNT = CFG::MNT, MIPT = CFG::MIPT, NV = MNT * MIPT;
    static_assert(TT % NV == 0, "merge tiles must divide the sorted run");
    static_assert((TT / NV & (TT / NV - 1)) == 0, "merge tiles per run must be a power of two");

    CallRecord dummy;
    CallRecord &rec = record ? call_record() : dummy;
    rec = CallRecord();
    rec.host.call = 3;
    rec.host.n = n_keys;
    rec.host.key_type = KT;
    rec.host.tile = TT;
    rec.host.merge_tile = NV;
    rec.stream = s;
    if (nseg == 0) return SR_OK;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    const long long nchunks = (long long)(n_keys / CH) + 1;
    const int passes_upper = ceil_log2((unsigned long long)((n_keys + TT - 1) / TT + 1));
    rec.host.passes_planned = passes_upper;
    const size_t cb = align_up(sizeof(SegCtrl), 256);
    const size_t fb = align_up((size_t)(nchunks + 2) * 4, 256);
    const size_t lb = align_up((nseg + 1) * 4, 256);
    constexpr int SMAX = small_cap(CFG::LADDER, NSMALL - 1);
    const bool in_place = (const void *)in == (const void *)out;
    const size_t kb = in_place ? align_up(n_keys * sizeof(T), 256) : 0;
    void *scratch = nullptr;
    const size_t lsb = bucket_mode ? align_up((size_t)NSMALL * nseg * 4, 256) : 0;
    SR_TRY(scratch_alloc(ds, &scratch, cb + fb + 4 * lb + lsb + kb, s));
    unsigned char *sp = (unsigned char *)scratch;
    SegCtrl *ctrl = (SegCtrl *)sp;
    int *chunk_first = (int *)(sp + cb);
    unsigned int *medium = (unsigned int *)(sp + cb + fb);
    unsigned int *big = (unsigned int *)(sp + cb + fb + lb);
    unsigned int *tile_base = (unsigned int *)(sp + cb + fb + 2 * lb);
    unsigned int *mtile_base = (unsigned int *)(sp + cb + fb + 3 * lb);
    unsigned int *lists = (unsigned int *)(sp + cb + fb + 4 * lb);
    T *alt = in_place ? (T *)(sp + cb + fb + 4 * lb + lsb) : const_cast<T *>(in);
    const bool vec = ((uintptr_t)out % 16) == 0 && ((uintptr_t)alt % 16) == 0;
    sr_status st = SR_OK;
    do {
        if (cudaMemsetAsync(ctrl, 0, sizeof(SegCtrl), s) != cudaSuccess) { st = launch_status(); break; }
        const int chunk = bucket_mode ? SMAX : CH;
        SR_LAUNCH(SR_KERNEL_SEGMENTED, k_seg_classify, (unsigned)((nseg + 255) / 256), 256, 0, s, d_off,
                  (long long)nseg, (long long)n_keys, chunk, TT, nchunks, chunk_first, medium, big,
                  bucket_mode ? 1 : 0, (int)CFG::LADDER, lists, ctrl);
        SR_LAUNCH(SR_KERNEL_SEGMENTED, k_seg_bigscan, 1, 1024, 0, s, d_off, big, TT, NV, tile_base, mtile_base,
                  ctrl);
        const size_t sort_smem = std::max(bucket_mode ? (size_t)0 : (size_t)PT * (sizeof(C) + 4),
                                          (size_t)TT * sizeof(U) * (CFG::F > 1 ? 2 : 1));
        if ((st = allow_smem(k_seg_sort<KT, CFG>, sort_smem)) != SR_OK) break;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_sort<KT, CFG>, SNT, sort_smem);
        const int sort_grid = sm_count() * std::max(per_sm, 1);
        if constexpr (bucket_mode) {
#define SR_SMALL(cls)                                                                                     \
    SR_LAUNCH(SR_KERNEL_SEGMENTED,                                                                        \
              (k_seg_small<KT, small_nt(CFG::LADDER, cls), small_ipt(CFG::LADDER, cls)>),                \
              sm_count() * (2048 / small_nt(CFG::LADDER, cls)), small_nt(CFG::LADDER, cls),               \
              (size_t)small_cap(CFG::LADDER, cls) * sizeof(U), s, in, out, d_off,                        \
              lists + (size_t)(cls) * nseg, cls, ctrl)
            SR_SMALL(0);
            SR_SMALL(1);
            SR_SMALL(2);
            SR_SMALL(3);
            SR_SMALL(4);
#undef SR_SMALL
        }
        SR_LAUNCH(SR_KERNEL_SEGMENTED, (k_seg_sort<KT, CFG>), sort_grid, SNT, sort_smem, s, in, out, alt, d_off,
                  bucket_mode ? 0ll : nchunks, chunk_first, medium, big, tile_base, ctrl);
        const size_t m_smem = merge_tile_smem<U, MNT, MIPT, false>();
        if ((st = allow_smem(k_seg_merge<KT, MNT, MIPT, true>, m_smem)) != SR_OK) break;
        if ((st = allow_smem(k_seg_merge<KT, MNT, MIPT, false>, m_smem)) != SR_OK) break;
        const int merge_grid = sm_count() * 8;
        for (int p = 0; p < passes_upper; ++p) {
            if (vec) {
                SR_LAUNCH(SR_KERNEL_MERGE, (k_seg_merge<KT, MNT, MIPT, true>), merge_grid, MNT, m_smem, s, out,
                          alt, (long long)n_keys, d_off, big, mtile_base, TT, p, ctrl);
            } else {
                SR_LAUNCH(SR_KERNEL_MERGE, (k_seg_merge<KT, MNT, MIPT, false>), merge_grid, MNT, m_smem, s, out,
                          alt, (long long)n_keys, d_off, big, mtile_base, TT, p, ctrl);
            }
        }
        if (st != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_SEGMENTED, k_seg_finish, 1, 32, 0, s, ctrl, ds->status);
        if (record) {
            if (cudaMemcpyAsync(ds->last_aux, ctrl, sizeof(SegCtrl), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                st = launch_status();
                break;
            }
            rec.aux_kind = 3;
        }
    } while (0);
    scratch_free(scratch, s);
    return st;
}


// The configurations of each key width, in the order of the C ABI's config
// index (sr_segmented_config_info describes them).
typedef SegCfg<0, 512, 11, 15, 1> SegK4_0;      // packs 512x11, tiles 512x15, fan-in 1
typedef SegCfg<0, 256, 11, 15, 2> SegK4_1;      // packs 256x11, tiles 256x15, fan-in 2
typedef SegCfg<1, 512, 1, 15, 1, 0> SegK4_2;    // buckets (ladder 0), tiles 512x15, fan-in 1
typedef SegCfg<1, 256, 1, 15, 4, 0> SegK4_3;    // buckets (ladder 0), tiles 256x15, fan-in 4
typedef SegCfg<1, 512, 1, 15, 1, 1> SegK4_4;    // buckets (ladder 1), tiles 512x15, fan-in 1
typedef SegCfg<1, 256, 1, 15, 2, 1> SegK4_5;    // buckets (ladder 1), tiles 256x15, fan-in 2
typedef SegCfg<1, 512, 1, 15, 2, 1> SegK4_6;    // buckets (ladder 1), tiles 512x15, fan-in 2
typedef SegCfg<1, 512, 1, 15, 1, 2> SegK4_7;    // buckets (ladder 2), tiles 512x15, fan-in 1
enum { SEG_NCFG_K4 = 8 };
typedef SegCfg<0, 512, 7, 11, 1> SegK8_0;
typedef SegCfg<0, 256, 7, 11, 2> SegK8_1;
typedef SegCfg<1, 512, 1, 11, 1, 0> SegK8_2;
typedef SegCfg<1, 256, 1, 11, 4, 0> SegK8_3;
typedef SegCfg<1, 512, 1, 11, 1, 1> SegK8_4;
enum { SEG_NCFG_K8 = 5 };

}  // namespace sr
