// sr_rem.cuh -- the few-displaced-keys path of the plain key sort.
//
// A k-exchange list (Section 2) is a sorted list after k exchanges of key
// pairs: at most 2k keys are away from their final place, and the paper ties
// the class to the Rem measure (the fewest keys whose removal leaves a sorted
// sequence).  Run detection alone gains nothing on it -- each displaced key
// breaks the runs of its tile, so every tile and every merge pass has work --
// but when only a few keys are displaced, removing them leaves one sorted
// sequence, and the removed keys are few enough to sort on the side.  The path
// is chosen on the device after the run-detection scan, for keys only (the
// result is then unique: no payload order to keep), when the descents are at
// least one per two tiles (REM_TNT x IPT keys each) and at most n/32.
//
//   k_rem_bounds  one CTA: a value bound per tile -- the median of the 9
//                 keys around the tile's first position, which the
//                 run-detection scan records -- made nondecreasing by a
//                 running maximum (bound[0] is the smallest image).
//   k_rem_split   per tile: the keys inside the tile's value
//                 range [bound[b], bound[b+1]) are candidates; while two
//                 consecutive candidates are out of order, both stop being
//                 candidates (at most REM_ROUNDS rounds, else none are).  The
//                 candidates, in input order, are sorted and fit between the
//                 neighbouring tiles' candidates: they go to the tile's own
//                 slot of the scratch buffer.  Every other key goes to the
//                 bucket of the tile whose value range holds it (a fixed
//                 capacity of REM_CAP keys per bucket; overflow abandons the
//                 path and the ordinary sort runs on the untouched input).
//   k_rem_bsort   per bucket: sorts it in place (rank by counting in shared
//                 memory; the buckets are small); its last CTA computes the
//                 output offset of every tile's block (candidates plus bucket)
//                 and switches the call to MODE_REM.
//   k_rem_merge   per tile: merges the tile's candidates with its bucket into
//                 the tile's output block (one merge tile).
//
// Correctness does not depend on the bounds: any nondecreasing bounds
// partition the values into ordered ranges, the candidates kept are sorted by
// construction, and the buckets are sorted before the merge.  The bounds only
// decide how many keys land in buckets.
#pragma once

#include <type_traits>

#include "sr_device.cuh"
#include "sr_kernels.cuh"

namespace sr {

// REM_TNT: threads of a split CTA (a tile is REM_TNT x IPT keys); the merge of
// a tile's block (at most REM_TNT x IPT + REM_CAP keys) runs as one merge tile
// of REM_TNT x (IPT + REM_CAP / REM_TNT) keys.
enum { REM_ROUNDS = 8, REM_CAP = 512, REM_NT = 1024, REM_TNT = 256, REM_BSORT_NT = 256 };

// Inclusive maximum scan over the CTA (blockDim.x = REM_NT).
template <typename U>
__device__ __forceinline__ U rem_block_max_scan(U x, U *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const U y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o && y > x) x = y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        U w = lane < REM_NT / 32 ? s_warp[lane] : U(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const U y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o && y > w) w = y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    if (wid > 0 && s_warp[wid - 1] > x) x = s_warp[wid - 1];
    return x;
}

// Inclusive sum scan over the CTA of width NT.
template <int NT, typename V>
__device__ __forceinline__ V rem_block_sum_scan(V x, V *s_warp, V *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        V w = lane < NT / 32 ? s_warp[lane] : V(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const V y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    if (wid > 0) x += s_warp[wid - 1];
    *total = s_warp[NT / 32 - 1];
    return x;
}

// One CTA of REM_NT threads.  Leaves rem_active at 0 unless the call sorts
// and its descents are in [tiles / 2, dmax]; clears the bucket counts and
// turns the medians in bound[] into their running maximum.
template <int KT>
__global__ void __launch_bounds__(REM_NT)
k_rem_bounds(long long n, long long tiles, long long dmax, Ctrl *__restrict__ c, typename Key<KT>::U *__restrict__ bound,
             unsigned int *__restrict__ b_count) {
    griddep_wait();
    typedef typename Key<KT>::U U;
    __shared__ U s_warp[32];
    if (call_mode(c, n) != MODE_SORT) return;
    const unsigned long long d = c->descents;
    if (2 * d < (unsigned long long)tiles || d > (unsigned long long)dmax) return;
    const int t = threadIdx.x;
    const long long per = (tiles + REM_NT - 1) / REM_NT;
    const long long b0 = min((long long)t * per, tiles), b1 = min(b0 + per, tiles);
    U run = 0;
    for (long long b = b0; b < b1; ++b) {
        const U v = bound[b];                       // the scan's median (0 for b = 0)
        b_count[b] = 0u;
        if (v > run) run = v;
    }
    const U incl = rem_block_max_scan<U>(run, s_warp);
    const U up = __shfl_up_sync(0xffffffffu, incl, 1);          // thread t-1's inclusive maximum
    U carry = (t & 31) ? up : ((t >> 5) ? s_warp[(t >> 5) - 1] : U(0));
    for (long long b = b0; b < b1; ++b) {
        const U v = bound[b];
        if (v > carry) carry = v;
        bound[b] = carry;
    }
    if (t == 0) c->rem_active = 1;
}

// The bucket (tile) whose value range holds u: the last b with
// bound[b] <= u (bound[0] is the smallest image).
template <typename U>
__device__ __forceinline__ long long rem_dest(const U *__restrict__ bound, long long tiles, U u) {
    long long lo = 0, hi = tiles;          // bound[lo] <= u; the answer is in [lo, hi)
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (bound[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// CTAs loop over the tiles of NT*IPT keys.  Shared memory: NT*IPT
// images and NT*IPT drop flags.
#ifndef SR_REM_GRID
#define SR_REM_GRID 8           // CTAs per SM launched for the per-tile kernels (they loop over tiles)
#endif
#ifndef SR_REM_SPLIT_MINB
#define SR_REM_SPLIT_MINB 4     // 64 registers: four CTAs per SM
#endif
__device__ __forceinline__ unsigned int popc_mask(unsigned int m) { return __popc(m); }
__device__ __forceinline__ unsigned int popc_mask(unsigned long long m) { return __popcll(m); }

template <int KT, int NT, int IPT>
__global__ void __launch_bounds__(NT, SR_REM_SPLIT_MINB)
k_rem_split(const typename Key<KT>::T *__restrict__ keys, long long n, long long tiles, Ctrl *__restrict__ c,
            const typename Key<KT>::U *__restrict__ bound, typename Key<KT>::T *__restrict__ sslot,
            unsigned int *__restrict__ s_count, typename Key<KT>::T *__restrict__ dbuck,
            unsigned int *__restrict__ b_count) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int TS = NT * IPT;
    constexpr int NW = NT / 32;
    static_assert(IPT <= 64, "one bit per key of a thread");
    typedef typename std::conditional<(IPT > 32), unsigned long long, unsigned int>::type Mask;
    if (!c->rem_active) return;
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    unsigned char *dropf = reinterpret_cast<unsigned char *>(s + TS);
    __shared__ U w_val[NW];
    __shared__ int w_idx[NW];
    __shared__ unsigned int w_cnt[32];
    __shared__ int s_stop;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    __syncthreads();                               // the previous tile's shared buffers are free
    if (t == 0) s_stop = *(volatile const int *)&c->rem_over;   // another tile gave up the path
    __syncthreads();
    if (s_stop) return;
    const long long base = tile * TS;
    const int cnt = (int)min((long long)TS, n - base);
    const U lo = bound[tile];
    const bool top = tile == tiles - 1;
    const U hi = top ? U(0) : bound[tile + 1];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int idx = i * NT + t;
        if (idx < cnt) s[idx] = K::ord(keys[base + idx]);
        dropf[idx] = 0;
    }
    __syncthreads();
    U k[IPT];
    Mask keep = 0, valid = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int j = t * IPT + i;
        k[i] = j < cnt ? s[j] : U(0);
        if (j < cnt) {
            valid |= Mask(1) << i;
            if (k[i] >= lo && (top || k[i] < hi)) keep |= Mask(1) << i;
        }
    }
    // Are the candidates in order already (the usual case)?  Each must be at
    // least the largest candidate before it: a maximum scan, no positions.
    {
        U tmax = 0;
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if (((keep >> i) & Mask(1)) && k[i] > tmax) tmax = k[i];
        U incl = tmax;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const U y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o && y > incl) incl = y;
        }
        if (lane == 31) w_val[wid] = incl;
        __syncthreads();
        U run = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) run = 0;
        for (int w = 0; w < wid; ++w) run = w_val[w] > run ? w_val[w] : run;
        int bad = 0;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if ((keep >> i) & Mask(1)) {
                bad |= k[i] < run;
                run = k[i] > run ? k[i] : run;
            }
        }
        if (!__syncthreads_or(bad)) goto split_done;
    }
    for (int round = 0;; ++round) {
        // the last candidate of this thread's keys: (has, value, tile index)
        int has = 0, idx = -1;
        U val = 0;
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if ((keep >> i) & Mask(1)) { has = 1; val = k[i]; idx = t * IPT + i; }
        // inclusive scan over the CTA of "the latest candidate so far"
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int h2 = __shfl_up_sync(0xffffffffu, has, o);
            const U v2 = __shfl_up_sync(0xffffffffu, val, o);
            const int i2 = __shfl_up_sync(0xffffffffu, idx, o);
            if (lane >= o && !has && h2) { has = 1; val = v2; idx = i2; }
        }
        if (lane == 31) { w_val[wid] = val; w_idx[wid] = has ? idx : -1; }
        __syncthreads();
        // exclusive: from the previous lane, else from the previous warps
        int ph = __shfl_up_sync(0xffffffffu, has, 1);
        U pv = __shfl_up_sync(0xffffffffu, val, 1);
        int pi = __shfl_up_sync(0xffffffffu, idx, 1);
        if (lane == 0 || !ph) {
            ph = 0;
            for (int w = wid - 1; w >= 0; --w)
                if (w_idx[w] >= 0) { ph = 1; pv = w_val[w]; pi = w_idx[w]; break; }
        }
        // consecutive candidates out of order: both stop being candidates
        Mask drop = 0;
        int found = 0;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if ((keep >> i) & Mask(1)) {
                if (ph && pv > k[i]) {
                    found = 1;
                    drop |= Mask(1) << i;
                    const int pt = pi / IPT;
                    if (pt == t) drop |= Mask(1) << (pi - t * IPT);
                    else dropf[pi] = 1;
                }
                ph = 1; pv = k[i]; pi = t * IPT + i;
            }
        }
        keep &= ~drop;
        const int any = __syncthreads_or(found);
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if (dropf[t * IPT + i]) keep &= ~(Mask(1) << i);
        if (!any) break;
        if (round + 1 >= REM_ROUNDS) { keep = 0; break; }
        __syncthreads();                            // w_val / w_idx are rewritten next round
    }
split_done:
    // candidates to the front of s in input order, the other keys after them;
    // both counts in one scan ((candidates << 16) | others: a tile has fewer
    // than 2^16 keys)
    {
        const unsigned int ns = popc_mask(keep), nd = popc_mask(valid) - ns;
        unsigned int tot;
        const unsigned int mine = (ns << 16) | nd;
        const unsigned int ex = rem_block_sum_scan<NT, unsigned int>(mine, w_cnt, &tot) - mine;
        const unsigned int s_tot = tot >> 16, d_tot = tot & 0xffffu;
        unsigned int ps = ex >> 16, pd = s_tot + (ex & 0xffffu);
        __syncthreads();                            // every key is in registers: s is free
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if ((keep >> i) & Mask(1)) s[ps++] = k[i];
            else if ((valid >> i) & Mask(1)) s[pd++] = k[i];
        }
        if (t == 0) s_count[tile] = s_tot;
        __syncthreads();
        for (int j = t; j < (int)s_tot; j += NT) sslot[base + j] = K::unord(s[j]);
        // the others, one per thread: the bucket of their value range
        for (int j = t; j < (int)d_tot; j += NT) {
            const U u = s[s_tot + j];
            const long long b = rem_dest<U>(bound, tiles, u);
            const unsigned int q = atomicAdd(&b_count[b], 1u);
            if (q < (unsigned int)REM_CAP) dbuck[b * REM_CAP + q] = K::unord(u);
            else atomicExch(&c->rem_over, 1);
        }
    }
    }
}

// Block offsets (one CTA of REM_BSORT_NT threads), and the switch to
// MODE_REM (rem_gate = 1).
__device__ __forceinline__ void rem_scan(long long tiles, Ctrl *__restrict__ c,
                                         const unsigned int *__restrict__ s_count,
                                         const unsigned int *__restrict__ b_count, long long *__restrict__ blk_off,
                                         unsigned long long *s_warp) {
    constexpr int NT = REM_BSORT_NT;
    const int t = threadIdx.x;
    const long long per = (tiles + NT - 1) / NT;
    const long long b0 = min((long long)t * per, tiles), b1 = min(b0 + per, tiles);
    unsigned long long sum = 0, dsum = 0;
    for (long long b = b0; b < b1; ++b) {
        sum += (unsigned long long)s_count[b] + b_count[b];
        dsum += b_count[b];
    }
    if (dsum) atomicAdd(&c->rem_dcount, dsum);
    unsigned long long total;
    const unsigned long long incl = rem_block_sum_scan<NT, unsigned long long>(sum, s_warp, &total);
    unsigned long long off = incl - sum;
    for (long long b = b0; b < b1; ++b) {
        blk_off[b] = (long long)off;
        off += (unsigned long long)s_count[b] + b_count[b];
    }
    if (t == 0) {
        blk_off[tiles] = (long long)total;
        c->rem_gate = 1;
    }
}

// CTAs of REM_BSORT_NT threads loop over the buckets: each is sorted in
// place (rank by counting; equal keys by bucket position).  The last CTA
// computes the block offsets instead.  gridDim.x >= 2.
template <int KT>
__global__ void __launch_bounds__(REM_BSORT_NT)
k_rem_bsort(typename Key<KT>::T *__restrict__ buck, long long tiles, Ctrl *__restrict__ c,
            const unsigned int *__restrict__ s_count, const unsigned int *__restrict__ b_count,
            long long *__restrict__ blk_off) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int NT = REM_BSORT_NT, Q = (REM_CAP + NT - 1) / NT;
    __shared__ U s[REM_CAP];
    __shared__ unsigned long long s_warp[32];
    if (!c->rem_active || c->rem_over) return;     // not taken, or a bucket overflowed
    const int t = threadIdx.x;
    if (blockIdx.x == gridDim.x - 1) {              // the last CTA: the block offsets
        rem_scan(tiles, c, s_count, b_count, blk_off, s_warp);
        return;
    }
    for (long long b = blockIdx.x; b < tiles; b += gridDim.x - 1) {
    const int m = (int)b_count[b];                  // <= REM_CAP: no bucket overflowed
    typename K::T *bk = buck + b * REM_CAP;
    __syncthreads();                                // the previous bucket's reads of s are done
    for (int i = t; i < m; i += NT) s[i] = K::ord(bk[i]);
    __syncthreads();
    U r[Q];
    int rk[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int i = t + q * NT;
        rk[q] = 0;
        r[q] = i < m ? s[i] : U(0);
    }
    if (m <= NT) {                                  // one key per thread (the usual case)
        for (int j = 0; j < m; ++j) {
            const U x = s[j];
            rk[0] += (x < r[0]) || (x == r[0] && j < t);
        }
    } else {
        for (int j = 0; j < m; ++j) {
            const U x = s[j];
#pragma unroll
            for (int q = 0; q < Q; ++q) rk[q] += (x < r[q]) || (x == r[q] && j < t + q * NT);
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (t + q * NT < m) bk[rk[q]] = K::unord(r[q]);
    }
}

// CTAs loop over the tiles: each tile's candidates merged with its sorted
// bucket into the tile's output block, as one merge tile of NT x MIPT keys.
// src indexes the scratch buffer that holds the candidate slots (tile b at
// b*ts) followed, at index dofs, by the buckets (bucket b at dofs +
// b*REM_CAP); n_src bounds it.
#ifndef SR_REM_MERGE_MINB
#define SR_REM_MERGE_MINB 4     // 64 registers: four CTAs per SM
#endif
#if SR_REM_MERGE_MINB
#define SR_REM_MERGE_BOUNDS __launch_bounds__(NT, SR_REM_MERGE_MINB)
#else
#define SR_REM_MERGE_BOUNDS __launch_bounds__(NT)
#endif
template <int KT, int NT, int MIPT, bool VEC>
__global__ void SR_REM_MERGE_BOUNDS
k_rem_merge(typename Key<KT>::T *__restrict__ out, const typename Key<KT>::T *__restrict__ src, long long n_src,
            long long dofs, int ts, long long tiles, const Ctrl *__restrict__ c,
            const unsigned int *__restrict__ s_count, const unsigned int *__restrict__ b_count,
            const long long *__restrict__ blk_off, int *status) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    if (!c->rem_gate) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long bar;             // the bulk-copy staging's barrier, set up per tile
    U *s = reinterpret_cast<U *>(smem);
    for (long long b = blockIdx.x; b < tiles; b += gridDim.x) {
        const long long na = s_count[b], nb = b_count[b];
        const long long a_beg = b * ts, b_beg = dofs + b * REM_CAP;
        __syncthreads();                            // the previous tile's shared buffers are free
        if (na + nb > 0)                            // na <= ts and nb <= REM_CAP: one merge tile holds it
            merge_tile<KT, NT, MIPT, false, VEC>(src, out, nullptr, nullptr, n_src, blk_off[b], (int)(na + nb), a_beg,
                                                 a_beg + na, b_beg, s, nullptr, nullptr, 0, VEC ? &bar : nullptr,
                                                 status);
    }
}

}  // namespace sr
