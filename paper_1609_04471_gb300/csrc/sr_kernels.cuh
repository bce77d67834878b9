// sr_kernels.cuh -- the kernels of the plain sort (run detection, reversal,
// block sort, merge-path partition, merge pass, copy-back).  The launch
// sequence that drives them is described in sr_sort.cu.
#pragma once

#include <climits>

#include "sr_device.cuh"

#ifndef SR_SPLIT_SAMPLES
#define SR_SPLIT_SAMPLES 1  // merge splits searched over recorded tile samples first
#endif
#ifndef SR_MERGE_RAW_I32
// bulk-staged int32 merge tiles compare the raw keys as signed int32, with no
// pass over the staged tile to make order images (2^28: merge steps 5.78 ->
// 4.93 ms, 0.96 of the measured copy bandwidth)
#define SR_MERGE_RAW_I32 1
#endif
#ifndef SR_MERGE_1LD
#define SR_MERGE_1LD 1      // global merge tiles: one unguarded shared load per merge step (padded buffer)
#endif
#ifndef SR_REM_KEYS
#define SR_REM_KEYS 1       // the few-displaced-keys path (keys only)
#endif
#ifndef SR_FEW_KEYS
#define SR_FEW_KEYS 1       // the few-distinct-keys path (4-byte keys, keys only)
#endif

namespace sr {

enum { RUNS_NT = 1024 };          // threads of the one-CTA planners (k_tile_order, k_runs)
// Longest wait for a tile's bulk copies: tries of mbarrier.try_wait (each
// waits in hardware for a while); a tile that gives up reports
// SR_ERR_TIMEOUT in its status word.
enum { BULK_WAIT_TRIES = 1 << 22 };
// How a merge tile stages its windows into shared memory: one key at a time
// (arrays not 16-byte aligned), 4-key groups by 16-byte loads through
// registers, or the same groups by 1-D bulk copies.
enum { STAGE_SCALAR = 0, STAGE_VEC = 1, STAGE_BULK = 2 };

// ------------------------------------------------------------- kernels

// Run detection over tile blockIdx.x of NT*IPT keys: counts the descents
// a[i] > a[i+1] and non-descents of every pair whose left key lies in the tile
// (so the pair across two tiles is counted once), and whether the tile alone
// is ascending or strictly descending.  Keys arrive in 16-byte vectors when
// the array is 16-byte aligned; the right neighbour of a vector's last key is
// the next vector's first, read again through the read-only path.
// `gate` (optional): when it points at 0 the scan counts nothing, so the call
// sees a "sorted" input and every later kernel of the sequence returns at once.
// The median of the keys at positions p-4 .. p+4 (positions past n read the
// last key), as an order image.
template <int KT>
__device__ __forceinline__ typename Key<KT>::U median9_image(const typename Key<KT>::T *__restrict__ keys,
                                                             long long n, long long p) {
    typedef Key<KT> K;
    typedef typename K::U U;
    U x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = K::ord(keys[min(p - 4 + i, n - 1)]);
#pragma unroll
    for (int r = 0; r < 9; ++r) {
#pragma unroll
        for (int i = r & 1; i + 1 < 9; i += 2) {
            const U a = x[i], b = x[i + 1];
            x[i] = a < b ? a : b;
            x[i + 1] = a < b ? b : a;
        }
    }
    return x[4];
}

// `med` (optional): the scan also records, for every multiple b*mt of mt
// below n (mt divides NT*IPT), the median of the 9 keys around it in med[b]
// (med[0] = 0), for the few-displaced-keys path's value bounds.
// `tmin`, `tmax` (optional): the tile's smallest and largest key images.
template <int KT, int NT, int IPT>
__global__ void __launch_bounds__(NT) k_detect(const typename Key<KT>::T *__restrict__ keys,
                                               long long n, Ctrl *__restrict__ c,
                                               const int *__restrict__ gate,
                                               typename Key<KT>::U *__restrict__ med, int mt,
                                               typename Key<KT>::U *__restrict__ tmin,
                                               typename Key<KT>::U *__restrict__ tmax) {
    griddep_wait();
    if (gate && *gate == 0) return;
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    constexpr int TS = NT * IPT;
    constexpr int VW = 16 / sizeof(T);             // keys per 16-byte vector
    __shared__ unsigned int red[4];
    __shared__ U s_min, s_max;
    const int t = threadIdx.x;
    const long long base = (long long)blockIdx.x * TS;
    const int cnt = (int)(n - base < (long long)TS ? n - base : (long long)TS);   // keys of the tile
    const bool more = base + cnt < n;              // a key follows the tile
    const bool vec = (((uintptr_t)(keys + base)) & 15) == 0;
    if (t < 4) red[t] = 0;
    if (t == 0) { s_min = umax_of<U>(); s_max = U(0); }
    __syncthreads();
    unsigned int d = 0, nd = 0, din = 0, ndin = 0;
    U kmin = umax_of<U>(), kmax = U(0);
    const int ng = (cnt + VW - 1) / VW;
    // vectors whose VW pairs and next key all lie inside the tile: no bounds
    // tests; their non-descents are counted as pairs minus descents afterwards
    const int nfast = vec ? (cnt - 1) / VW : 0;    // vectors g with g*VW + VW < cnt
    unsigned int dfast = 0, pfast = 0;
    for (int g = t; g < nfast; g += NT) {
        const int j0 = g * VW;
        U x[VW + 1];
        if constexpr (VW == 4) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(keys + base + j0));
            x[0] = K::ord((T)q.x); x[1] = K::ord((T)q.y); x[2] = K::ord((T)q.z); x[3] = K::ord((T)q.w);
        } else {
            const ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2 *>(keys + base + j0));
            x[0] = K::ord((T)q.x); x[1] = K::ord((T)q.y);
        }
        x[VW] = K::ord(__ldg(keys + base + j0 + VW));
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            dfast += x[e] > x[e + 1];
            kmin = x[e] < kmin ? x[e] : kmin;
            kmax = x[e] > kmax ? x[e] : kmax;
        }
        pfast += VW;
    }
    d += dfast;
    nd += pfast - dfast;
    din |= dfast != 0;
    ndin |= pfast != dfast;
    for (int g = nfast + t; g < ng; g += NT) {
        const int j0 = g * VW;                     // tile index of the vector's first key
        U x[VW + 1];
        if (vec && j0 + VW <= cnt) {
            if constexpr (VW == 4) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(keys + base + j0));
                x[0] = K::ord((T)q.x); x[1] = K::ord((T)q.y); x[2] = K::ord((T)q.z); x[3] = K::ord((T)q.w);
            } else {
                const ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2 *>(keys + base + j0));
                x[0] = K::ord((T)q.x); x[1] = K::ord((T)q.y);
            }
        } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) x[e] = j0 + e < cnt ? K::ord(__ldg(keys + base + j0 + e)) : U(0);
        }
        const bool has_next = j0 + VW < cnt || (j0 + VW == cnt && more);
        x[VW] = has_next ? K::ord(__ldg(keys + base + j0 + VW)) : U(0);
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const int j = j0 + e;                  // pair (j, j+1)
            if (j < cnt) {
                kmin = x[e] < kmin ? x[e] : kmin;
                kmax = x[e] > kmax ? x[e] : kmax;
            }
            if (j + 1 < cnt || (j + 1 == cnt && more)) {
                const bool de = x[e] > x[e + 1];
                d += de;
                nd += !de;
                if (j + 1 < cnt) { din |= de; ndin |= !de; }
            }
        }
    }
    d = __reduce_add_sync(0xffffffffu, d);
    nd = __reduce_add_sync(0xffffffffu, nd);
    din = __reduce_or_sync(0xffffffffu, din);
    ndin = __reduce_or_sync(0xffffffffu, ndin);
    if (tmin) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const U a = __shfl_xor_sync(0xffffffffu, kmin, o), b = __shfl_xor_sync(0xffffffffu, kmax, o);
            kmin = a < kmin ? a : kmin;
            kmax = b > kmax ? b : kmax;
        }
    }
    if ((t & 31) == 0) {
        if (d) atomicAdd(&red[0], d);
        if (nd) atomicAdd(&red[1], nd);
        if (din) atomicOr(&red[2], din);
        if (ndin) atomicOr(&red[3], ndin);
        if (tmin) {
            atomicMin(&s_min, kmin);
            atomicMax(&s_max, kmax);
        }
    }
    __syncthreads();
    if (tmin && t == 0) {
        tmin[blockIdx.x] = s_min;
        tmax[blockIdx.x] = s_max;
    }
    if (t == 0) {
        if (red[0]) atomicAdd(&c->descents, (unsigned long long)red[0]);
        if (red[1]) atomicAdd(&c->nondescents, (unsigned long long)red[1]);
        if (!red[2]) atomicAdd(&c->tiles_ascending, 1ull);
        if (!red[3]) atomicAdd(&c->tiles_descending, 1ull);
    }
    // after the scan: the keys around this tile's multiples of mt are cached
    if (med && t < NT * IPT / mt) {
        const long long b = (long long)blockIdx.x * (NT * IPT / mt) + t;
        if (b * mt < n) med[b] = b == 0 ? U(0) : median9_image<KT>(keys, n, b * mt);
    }
}

// Technique (a) of Section 3 at the granularity of tiles: a chain of whole
// tiles in descending order (every key of tile t >= every key of tile t+1;
// strictly, when payloads must stay stable, since equal keys would change
// order) is a reversed run; the block sort writes its tiles in reversed order,
// so the chain leaves the block sort as one ascending run.  A chain is turned
// only when that lowers the count of natural runs (two tiles at the seam of
// two ascending runs also form a chain, and turning them would cut both runs).
// One CTA, from the scan's per-tile extremes: dest[t] = the tile position the
// block sort writes tile t to (dest[t] = t outside turned chains).  Sets
// c->tile_perm when some chain is turned; the block sort then writes to the
// scratch buffer whatever the step count (in place, a tile written elsewhere
// could overwrite one not yet read), and the run planner starts the steps there.
template <int KT>
__global__ void __launch_bounds__(RUNS_NT)
k_tile_order(const typename Key<KT>::U *__restrict__ tmin, const typename Key<KT>::U *__restrict__ tmax,
             long long n, long long ts, long long tiles, int strict, int *__restrict__ dest,
             Ctrl *__restrict__ c) {
    griddep_wait();
    if (call_mode(c, n) != MODE_SORT) return;
    __shared__ int s_carry;
    __shared__ int s_any;
    const int t = threadIdx.x;
    const long long full_tiles = n / ts;           // tiles of ts keys; a short last tile never moves
    // desc(q): tiles q-1 and q are full and in descending order (and not in
    // ascending order, which also holds when every key of both is equal)
    auto desc = [&](long long q) -> bool {
        if (q <= 0 || q >= full_tiles) return false;
        const bool down = strict ? tmax[q] < tmin[q - 1] : tmax[q] <= tmin[q - 1];
        return down && !(tmax[q - 1] <= tmin[q]);
    };
    if (t == 0) { s_carry = 0; s_any = 0; }
    __syncthreads();
    // forward: the first tile of each tile's chain, into dest
    for (long long t0 = 0; t0 < tiles; t0 += RUNS_NT) {
        const long long q = t0 + t;
        int start = (q < tiles && !desc(q)) ? (int)q : -1;
        // block-wide running maximum (chains start where desc is false)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, start, o);
            if ((t & 31) >= o) start = max(start, u);
        }
        __shared__ int s_w[RUNS_NT / 32];
        if ((t & 31) == 31) s_w[t >> 5] = start;
        __syncthreads();
        int before = s_carry;
        for (int w = 0; w < (t >> 5); ++w) before = max(before, s_w[w]);
        start = max(start, before);
        if (q < tiles) dest[q] = start;
        __syncthreads();
        if (t == RUNS_NT - 1) s_carry = start;
        __syncthreads();
    }
    // backward: the last tile of each chain; dest[q] = first + last - q
    if (t == 0) s_carry = (int)tiles - 1;
    __syncthreads();
    for (long long t1 = tiles; t1 > 0; t1 -= RUNS_NT) {
        const long long q = t1 - RUNS_NT + t;      // q < 0 for the first chunk's missing lanes
        int end = (q >= 0 && q < tiles && !desc(q + 1)) ? (int)q : INT_MAX;
        // block-wide running minimum from the right
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_down_sync(0xffffffffu, end, o);
            if ((t & 31) + o < 32) end = min(end, u);
        }
        __shared__ int s_w2[RUNS_NT / 32];
        if ((t & 31) == 0) s_w2[t >> 5] = end;
        __syncthreads();
        int after = s_carry;
        for (int w = (t >> 5) + 1; w < RUNS_NT / 32; ++w) after = min(after, s_w2[w]);
        end = min(end, after);
        if (q >= 0 && q < tiles) {
            const int first = dest[q];
            // reverse the chain only if that leaves fewer natural runs: its
            // L - 1 inner links become ascending, the links with the tiles on
            // either side may be lost or made
            auto asc = [&](long long x, long long y) -> int {   // tile x then tile y, in order
                return (x >= 0 && y < tiles && tmax[x] <= tmin[y]) ? 1 : 0;
            };
            const int gain = (end - first) + asc(first - 1, end) + asc(first, end + 1) - asc(first - 1, first) -
                             asc(end, end + 1);
            const bool flip = end > first && gain > 0;
            if (flip) s_any = 1;
            dest[q] = flip ? first + end - (int)q : (int)q;
        }
        __syncthreads();
        if (t == 0) s_carry = end;
        __syncthreads();
    }
    if (t == 0 && s_any) c->tile_perm = 1;
}

// Few distinct keys, step 1: FEW_SAMPLE keys spread over the whole array go
// into the call's set of distinct order images, in two phases.  Phase A
// (one CTA) takes the first FEW_SAMPLE_A keys of the sample; if
// they hold more than FEW_A_MAX distinct images the input has more than
// FEW_MAX (drawing FEW_SAMPLE_A keys from at most FEW_MAX values gives about
// 2,590 distinct ones when all are equally likely, fewer otherwise), the set
// is closed and phase B returns at once.  Phase B (k_few_sample2) takes the
// rest of the sample; its last CTA to finish (a ticket after a fence), if the
// call would sort and the set holds at most FEW_MAX images, sorts the set (a
// bitonic network in shared memory) into FewTables::sorted as the candidate.
// The counting pass checks every key against the set, so a sample that misses
// a key only costs that pass.  This is the multiway form of the fat (3-way)
// split of the paper's quicksorts (Section 4, techniques (d) and (g)): every
// distinct key is a pivot, keys equal to a pivot need no further comparisons,
// so the split alone sorts the input.  Phase A looks at its first
// FEW_SAMPLE_A0 keys first: more than FEW_A0_MAX distinct among them closes
// the set at once (1,024 draws from at most FEW_MAX values give about 906
// distinct ones, with a spread of about 12), so inputs with many distinct keys
// pay for one round of sample loads; sorted and strictly descending inputs
// skip the sample.
enum { FEW_SAMPLE = 65536, FEW_SAMPLE_A = 4096, FEW_A_MAX = 3072, FEW_A_ALONE = 256, FEW_NT2 = 1024 };
enum { FEW_SAMPLE_A0 = 1024, FEW_A0_MAX = 1000 };

// This CTA's `per` samples (sample indices from `first`) into a shared-memory
// set, then its images not yet in the call's set into it; the number it added
// goes to the call's count once.  Returns the CTA's added count (thread 0).
template <int KT, int NTH, int LOG2>
__device__ __forceinline__ void few_sample_cta(const typename Key<KT>::T *__restrict__ keys, long long n,
                                               long long first, Ctrl *__restrict__ c, FewTables *__restrict__ ft,
                                               unsigned long long *s_set, unsigned int *s_n, unsigned int *s_new,
                                               int *s_over) {
    const int t = threadIdx.x;
    for (int i = t; i < (1 << LOG2); i += NTH) s_set[i] = 0ull;
    if (t == 0) { *s_n = 0u; *s_over = 0; *s_new = 0u; }
    __syncthreads();
    const long long i = first + t;
    if (i < FEW_SAMPLE && n > 0)
        few_insert<LOG2>(s_set, s_n, s_over, (unsigned int)Key<KT>::ord(__ldg(keys + (i * n) / FEW_SAMPLE)),
                         NTH);
    __syncthreads();
    if (*s_over) {
        if (t == 0) atomicExch(&c->few_over, 1);
    } else {
        for (int q = t; q < (1 << LOG2); q += NTH)
            if (s_set[q] != 0ull && !((volatile int *)&c->few_over)[0])
                few_insert<FEW_SLOTS_LOG2>(ft->slot, s_new, &c->few_over, (unsigned int)(s_set[q] - 1ull),
                                           0xffffffffu);
    }
    __syncthreads();
    if (t == 0 && *s_new && atomicAdd(&c->few_n, *s_new) + *s_new > (unsigned int)FEW_MAX)
        atomicExch(&c->few_over, 1);
}

// Phase A: one CTA of FEW_NT2 threads puts the first FEW_SAMPLE_A samples
// into a set in shared memory (FEW_A_SLOTS slots, dynamic shared memory); more
// than FEW_A_MAX distinct images close the call's set at once; at most
// FEW_A_ALONE (each seen ~16 times or more on average) make the candidate
// here; else the images go into the call's set in global memory for phase B.
enum { FEW_A_SLOTS_LOG2 = 13, FEW_A_SLOTS = 1 << FEW_A_SLOTS_LOG2 };
template <int KT>
__global__ void __launch_bounds__(FEW_NT2) k_few_sample(const typename Key<KT>::T *__restrict__ keys, long long n,
                                                        Ctrl *__restrict__ c, FewTables *__restrict__ ft,
                                                        const int *__restrict__ gate) {
    griddep_wait();
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_tab = reinterpret_cast<unsigned long long *>(smem);
    __shared__ unsigned int s_n, s_new;
    __shared__ int s_over;
    if (gate && *gate == 0) return;
    const int mode = call_mode(c, n);
    if (mode == MODE_SORTED || mode == MODE_REVERSE) {           // the scan has settled the call
        if (threadIdx.x == 0) atomicExch(&c->few_over, 1);      // phase B returns at once too
        return;
    }
    const int t = threadIdx.x;
    for (int q = t; q < FEW_A_SLOTS; q += FEW_NT2) s_tab[q] = 0ull;
    if (t == 0) { s_n = 0u; s_new = 0u; s_over = 0; }
    __syncthreads();
    static_assert(FEW_SAMPLE_A0 <= FEW_NT2 && FEW_SAMPLE_A % FEW_NT2 == 0, "the first look is one round");
    if (n > 0) {
        if (t < FEW_SAMPLE_A0)
            few_insert<FEW_A_SLOTS_LOG2>(s_tab, &s_n, &s_over,
                                         (unsigned int)Key<KT>::ord(__ldg(keys + ((long long)t * n) / FEW_SAMPLE)),
                                         FEW_A_MAX);
        __syncthreads();
        if (s_n > FEW_A0_MAX) {
            if (t == 0) atomicExch(&c->few_over, 1);
            return;
        }
        for (int i = FEW_SAMPLE_A0 + t; i < FEW_SAMPLE_A; i += FEW_NT2)
            few_insert<FEW_A_SLOTS_LOG2>(s_tab, &s_n, &s_over,
                                         (unsigned int)Key<KT>::ord(__ldg(keys + ((long long)i * n) / FEW_SAMPLE)),
                                         FEW_A_MAX);
    }
    __syncthreads();
    if (s_over) {                                  // too many distinct keys: the path is off
        if (t == 0) atomicExch(&c->few_over, 1);
        return;
    }
    const unsigned int nd = s_n;
    if (nd <= FEW_A_ALONE) {
        // so few distinct keys that each showed up many times in this sample:
        // the set is taken as complete (the counting pass checks every key), it
        // is sorted here and phase B does nothing
        __shared__ unsigned int s_v[FEW_A_ALONE];
        __shared__ unsigned int s_k;
        if (t == 0) s_k = 0u;
        __syncthreads();
        for (int q = t; q < FEW_A_SLOTS; q += FEW_NT2)
            if (s_tab[q] != 0ull) s_v[atomicAdd(&s_k, 1u)] = (unsigned int)(s_tab[q] - 1ull);
        __syncthreads();
        if (t < (int)nd) {                         // rank of each image among at most FEW_A_ALONE
            unsigned int r = 0;
            for (unsigned int q = 0; q < nd; ++q) r += s_v[q] < s_v[t];
            ft->sorted[r] = s_v[t];
        }
        __syncthreads();
        if (t == 0 && call_mode(c, n) == MODE_SORT) {
            c->few_n = nd;
            __threadfence();
            c->few_cand = 1;
        }
        return;
    }
    for (int q = t; q < FEW_A_SLOTS; q += FEW_NT2)
        if (s_tab[q] != 0ull)
            few_insert<FEW_SLOTS_LOG2>(ft->slot, &s_new, &c->few_over, (unsigned int)(s_tab[q] - 1ull), 0xffffffffu);
    __syncthreads();
    if (t == 0) atomicAdd(&c->few_n, s_new);
}

template <int KT>
__global__ void __launch_bounds__(FEW_NT2) k_few_sample2(const typename Key<KT>::T *__restrict__ keys, long long n,
                                                         Ctrl *__restrict__ c, FewTables *__restrict__ ft,
                                                         const int *__restrict__ gate) {
    griddep_wait();
    __shared__ unsigned int s_v[FEW_MAX];
    __shared__ unsigned long long s_set[2 * FEW_NT2];
    __shared__ unsigned int s_n, s_new, s_k;
    __shared__ int s_over, s_last;
    if (gate && *gate == 0) return;
    if (((volatile int *)&c->few_over)[0] || c->few_cand) return;   // closed, or phase A settled it
    const int t = threadIdx.x;
    few_sample_cta<KT, FEW_NT2, 11>(keys, n, FEW_SAMPLE_A + (long long)blockIdx.x * FEW_NT2, c, ft, s_set, &s_n,
                                    &s_new, &s_over);
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(&c->few_ticket2, 1u) == gridDim.x - 1;
        s_k = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (call_mode(c, n) != MODE_SORT) return;
    const int over = ((volatile int *)&c->few_over)[0];
    const unsigned int nd = ((volatile unsigned int *)&c->few_n)[0];
    if (over || nd == 0u || nd > (unsigned int)FEW_MAX) return;
    for (int q = t; q < FEW_SLOTS; q += FEW_NT2) {
        const unsigned long long v = ((volatile unsigned long long *)ft->slot)[q];
        if (v != 0ull) {
            const unsigned int r = atomicAdd(&s_k, 1u);
            if (r < (unsigned int)FEW_MAX) s_v[r] = (unsigned int)(v - 1ull);
        }
    }
    __syncthreads();
    const unsigned int k = s_k;
    if (k != nd) return;                           // cannot happen; the ordinary sort then runs
    unsigned int P = 1;
    while (P < k) P <<= 1;
    for (unsigned int q = k + t; q < P; q += FEW_NT2) s_v[q] = 0xffffffffu;
    __syncthreads();
    // bitonic sort of s_v[0, P) ascending
    for (unsigned int size = 2; size <= P; size <<= 1) {
        for (unsigned int stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned int q = t; q < P / 2; q += FEW_NT2) {
                const unsigned int lo = 2 * stride * (q / stride) + (q % stride), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned int a = s_v[lo], b = s_v[hi];
                if ((a > b) == up) { s_v[lo] = b; s_v[hi] = a; }
            }
            __syncthreads();
        }
    }
    for (unsigned int q = t; q < k; q += FEW_NT2) ft->sorted[q] = s_v[q];
    __syncthreads();
    if (t == 0) {
        __threadfence();
        c->few_cand = 1;
    }
}

// Few distinct keys, step 2: counts the keys equal to each candidate image.
// Each CTA builds, in shared memory, a hash table from every image of the
// sorted set to its rank (FEW_A_SLOTS slots of image << 32 | rank + 1, at most
// half full), looks each key up in it (about 1.5 probes) and adds one to its
// own histogram, which goes to row blockIdx.x of `hist` with plain stores; a
// key outside the set raises few_miss and the ordinary sort runs instead.  At
// most FEW_COUNT_CTAS CTAs; dynamic shared memory: few_count_smem().
// With at most FEW_WARP_HIST distinct keys every warp counts into its own
// shared histogram row (the rows are summed at the end), so the warps of a CTA
// do not contend for the same few counters.
enum { FEW_COUNT_CTAS = 160, FEW_COUNT_NT = 1024, FEW_WARP_HIST = 64 };
constexpr size_t few_count_smem() {
    return (size_t)FEW_A_SLOTS * 8 + (size_t)FEW_MAX * 4 + (size_t)(FEW_COUNT_NT / 32) * FEW_WARP_HIST * 4;
}
template <int KT>
__global__ void __launch_bounds__(FEW_COUNT_NT) k_few_count(const typename Key<KT>::T *__restrict__ keys, long long n,
                                                            Ctrl *__restrict__ c, const FewTables *__restrict__ ft,
                                                            unsigned int *__restrict__ hist) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::T T;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_tab = reinterpret_cast<unsigned long long *>(smem);
    unsigned int *s_h = reinterpret_cast<unsigned int *>(s_tab + FEW_A_SLOTS);
    unsigned int *s_wh = s_h + FEW_MAX;            // per-warp rows when k <= FEW_WARP_HIST
    if (!c->few_cand) return;
    const int t = threadIdx.x;
    const int k = (int)c->few_n;
    const bool rows = k <= FEW_WARP_HIST;
    unsigned int *h_mine = rows ? s_wh + (t >> 5) * FEW_WARP_HIST : s_h;
    for (int q = t; q < FEW_A_SLOTS; q += FEW_COUNT_NT) s_tab[q] = 0ull;
    for (int q = t; q < k; q += FEW_COUNT_NT) s_h[q] = 0u;
    for (int q = t; q < (FEW_COUNT_NT / 32) * FEW_WARP_HIST; q += FEW_COUNT_NT) s_wh[q] = 0u;
    __syncthreads();
    constexpr unsigned int MASK = FEW_A_SLOTS - 1;
    for (int q = t; q < k; q += FEW_COUNT_NT) {    // the images are distinct: one slot each
        const unsigned int u = ft->sorted[q];
        const unsigned long long v = ((unsigned long long)u << 32) | (unsigned long long)(q + 1);
        for (unsigned int h = (u * 2654435761u) >> (32 - FEW_A_SLOTS_LOG2), probe = 0; probe < FEW_A_SLOTS;
             ++probe, h = (h + 1) & MASK)
            if (atomicCAS(&s_tab[h], 0ull, v) == 0ull) break;
    }
    __syncthreads();
    bool miss = false;
    auto count = [&](T key) {
        const unsigned int u = (unsigned int)K::ord(key);
        unsigned int h = (u * 2654435761u) >> (32 - FEW_A_SLOTS_LOG2);
        for (int probe = 0; probe < FEW_A_SLOTS; ++probe, h = (h + 1) & MASK) {   // ends at an empty slot
            const unsigned long long e2 = s_tab[h];
            if (e2 == 0ull) { miss = true; return; }
            if ((unsigned int)(e2 >> 32) == u) {
                atomicAdd(&h_mine[(unsigned int)e2 - 1u], 1u);
                return;
            }
        }
        miss = true;
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + t;
    long long tail = 0;
    if ((((uintptr_t)keys) & 15) == 0) {
        const long long nv = n / 4;
        const uint4 *q4 = reinterpret_cast<const uint4 *>(keys);
        for (long long v = gtid; v < nv; v += stride) {
            const uint4 q = __ldg(q4 + v);
            count((T)q.x); count((T)q.y); count((T)q.z); count((T)q.w);
        }
        tail = 4 * nv;
    }
    for (long long i = tail + gtid; i < n; i += stride) count(__ldg(keys + i));
    if (miss && !((volatile int *)&c->few_miss)[0]) atomicExch(&c->few_miss, 1);
    __syncthreads();
    if (rows) {
        for (int q = t; q < k; q += FEW_COUNT_NT) {
            unsigned int sum = 0;
            for (int w = 0; w < FEW_COUNT_NT / 32; ++w) sum += s_wh[w * FEW_WARP_HIST + q];
            s_h[q] = sum;
        }
        __syncthreads();
    }
    for (int q = t; q < k; q += FEW_COUNT_NT) hist[(long long)blockIdx.x * FEW_MAX + q] = s_h[q];
}

// Few distinct keys, step 2b: the count of every distinct image, summed over
// the rows of the count pass's histograms (one thread per image).
static __global__ void __launch_bounds__(256) k_few_reduce(const unsigned int *__restrict__ hist, int rows,
                                                    const Ctrl *__restrict__ c, FewTables *__restrict__ ft) {
    griddep_wait();
    if (!c->few_cand || c->few_miss) return;
    const int k = (int)c->few_n;
    const int warps = gridDim.x * (blockDim.x / 32);
    if (k > warps) {                               // many keys: one thread per key, its rows in sequence
        const int j = blockIdx.x * blockDim.x + threadIdx.x;
        if (j >= k) return;
        unsigned long long s = 0;
        for (int r = 0; r < rows; ++r) s += hist[(long long)r * FEW_MAX + j];
        ft->count[j] = s;
        return;
    }
    // few keys: one warp per key, its lanes sum the CTAs' rows, then a warp sum
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= k) return;
    unsigned long long s = 0;
    for (int r = lane; r < rows; r += 32) s += hist[(long long)r * FEW_MAX + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ft->count[j] = s;
}

// Few distinct keys, step 3: when every key was in the set, writes the sorted
// output, each distinct key repeated its count times (16-byte stores when the
// array is aligned), and switches the call to MODE_FEW: every later kernel of
// the ordinary sequence then returns at once.
template <int KT>
__global__ void __launch_bounds__(256) k_few_write(typename Key<KT>::T *__restrict__ keys, long long n,
                                                   Ctrl *__restrict__ c, const FewTables *__restrict__ ft) {
    griddep_wait();
    typedef Key<KT> K;
    constexpr int PER = FEW_MAX / 256;             // counts per thread in the scan
    __shared__ unsigned long long s_start[FEW_MAX + 1];
    __shared__ unsigned long long s_part[256];
    if (!c->few_cand || c->few_miss) return;
    const int t = threadIdx.x;
    if (blockIdx.x == 0 && t == 0) c->few_active = 1;
    const int k = (int)c->few_n;
    // s_start[q] = keys before distinct key q (an exclusive scan of the
    // counts): coalesced loads into shared memory, then PER contiguous per thread
    for (int q = t; q < FEW_MAX; q += 256) s_start[q] = q < k ? ft->count[q] : 0ull;
    __syncthreads();
    unsigned long long run = 0;
#pragma unroll
    for (int e = 0; e < PER; ++e) run += s_start[t * PER + e];
    s_part[t] = run;
    __syncthreads();
    if (t < 32) {
        unsigned long long acc = 0;
        for (int w = 0; w < 8; ++w) {              // 8 partial sums per lane, then a warp scan
            const unsigned long long x = s_part[t * 8 + w];
            s_part[t * 8 + w] = acc;
            acc += x;
        }
        unsigned long long incl = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (t >= o) incl += u;
        }
        const unsigned long long excl = incl - acc;
        for (int w = 0; w < 8; ++w) s_part[t * 8 + w] += excl;
    }
    __syncthreads();
    unsigned long long cnt[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) cnt[e] = s_start[t * PER + e];
    __syncthreads();
    run = s_part[t];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        s_start[t * PER + e] = run;
        run += cnt[e];
    }
    if (t == 255) s_start[FEW_MAX] = run;
    __syncthreads();
    // the last q < k with s_start[q] <= i
    auto which = [&](long long i) {
        int lo = 0, hi = k - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((long long)s_start[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    auto key_of = [&](int j) { return K::unord((typename K::U)__ldg(ft->sorted + j)); };
    if ((((uintptr_t)keys) & 15) == 0) {
        // each warp writes chunks of FEW_W_CHUNK consecutive 16-byte groups,
        // lane l the groups l, l + 32, ...: one search per lane per chunk, then
        // a key index that only moves forward
        const long long nv = n / 4;
        uint4 *q4 = reinterpret_cast<uint4 *>(keys);
        const int lane = t & 31;
        const long long warps = (long long)gridDim.x * (blockDim.x / 32);
        const long long wid = (long long)blockIdx.x * (blockDim.x / 32) + (t >> 5);
        constexpr int FEW_W_CHUNK = 32 * 8;
        for (long long c0 = wid * FEW_W_CHUNK; c0 < nv; c0 += warps * FEW_W_CHUNK) {
            const long long end = min(c0 + FEW_W_CHUNK, nv);
            long long v = c0 + lane;
            if (v >= end) continue;
            int j = which(4 * v);
            uint32_t kj = (uint32_t)key_of(j);      // the key of run j, and where run j ends
            long long ej = j + 1 < k ? (long long)s_start[j + 1] : LLONG_MAX;
            for (; v < end; v += 32) {
                const long long i = 4 * v;
                if (i + 4 <= ej) {                 // the whole vector lies in run j
                    q4[v] = make_uint4(kj, kj, kj, kj);
                    continue;
                }
                uint32_t e4[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    while (j + 1 < k && (long long)s_start[j + 1] <= i + m) ++j;
                    e4[m] = (uint32_t)key_of(j);
                }
                kj = e4[3];
                ej = j + 1 < k ? (long long)s_start[j + 1] : LLONG_MAX;
                q4[v] = make_uint4(e4[0], e4[1], e4[2], e4[3]);
            }
        }
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long i = 4 * nv + (long long)blockIdx.x * blockDim.x + t; i < n; i += stride)
            keys[i] = key_of(which(i));
    } else {
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long i = (long long)blockIdx.x * blockDim.x + t; i < n; i += stride) keys[i] = key_of(which(i));
    }
}

// Reverses p[0 .. n): 16-byte vectors from both ends when the array is
// aligned and a whole number of vectors, single elements otherwise.
template <typename E>
__device__ __forceinline__ void reverse_array(E *__restrict__ p, long long n, long long gtid, long long stride) {
    constexpr int VW = 16 / sizeof(E);
    if ((((uintptr_t)p) & 15) == 0 && n % VW == 0) {
        uint4 *q = reinterpret_cast<uint4 *>(p);
        const long long nv = n / VW;
        for (long long i = gtid; i < (nv + 1) / 2; i += stride) {
            const long long j = nv - 1 - i;
            const uint4 x = q[i], y = q[j];
            // reversed element order inside a vector (i == j: the middle vector, reversed in place)
            q[i] = VW == 4 ? make_uint4(y.w, y.z, y.y, y.x) : make_uint4(y.z, y.w, y.x, y.y);
            q[j] = VW == 4 ? make_uint4(x.w, x.z, x.y, x.x) : make_uint4(x.z, x.w, x.x, x.y);
        }
    } else {
        for (long long i = gtid; i < n / 2; i += stride) {
            const long long j = n - 1 - i;
            const E a = p[i], b = p[j];
            p[i] = b;
            p[j] = a;
        }
    }
}

template <int KT, bool VALS>
__global__ void k_reverse(typename Key<KT>::T *__restrict__ k, uint32_t *__restrict__ v,
                          long long n, const Ctrl *__restrict__ c) {
    griddep_wait();
    if (call_mode(c, n) != MODE_REVERSE) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    reverse_array(k, n, gtid, stride);
    if (VALS) reverse_array(v, n, gtid, stride);
}

// Sorts tile blockIdx.x of NT*IPT keys; records the tile's smallest and
// largest key images in tile_lo / tile_hi (if given) for the pass planner.
template <int KT, int NT, int IPT, bool VALS>
__global__ void __launch_bounds__(NT, Shape<sizeof(typename Key<KT>::T), VALS>::SORT_MINB)
k_block_sort(const typename Key<KT>::T *in_k, const uint32_t *in_v, typename Key<KT>::T *out_k0,
             uint32_t *out_v0, typename Key<KT>::T *alt_k, uint32_t *alt_v, long long n, const Ctrl *__restrict__ c,
             typename Key<KT>::U *__restrict__ tile_lo, typename Key<KT>::U *__restrict__ tile_hi,
             typename Key<KT>::U *__restrict__ samp0, long long smt, int mv, const int *__restrict__ dest) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int NV = NT * IPT;
    if (c && call_mode(c, n) != MODE_SORT) return;
    // the output buffer: out_k0 / out_v0, or the scratch pair alt_k / alt_v when
    // the tile planner turned chains and out_k0 is the input itself; tile
    // samples go with the buffer written (samp0 + smt for the scratch one)
    const bool to_alt = c && c->tile_perm && (const void *)out_k0 == (const void *)in_k;
    typename Key<KT>::T *out_k = to_alt ? alt_k : out_k0;
    uint32_t *out_v = to_alt ? alt_v : out_v0;
    U *samp = samp0 ? samp0 + ((const void *)out_k == (const void *)in_k ? 0 : smt) : nullptr;
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + NV);
    const int t = threadIdx.x;
    const long long base = (long long)blockIdx.x * NV;
    const int cnt = (int)(n - base < (long long)NV ? n - base : (long long)NV);
    // the tile's place in the output: reversed chains of descending tiles
    // (k_tile_order) land in reversed order; every moved tile is full.  Read
    // where the tile is written, so it is not held through the sort.
    auto out_tile = [&]() -> long long {
        return (dest && c && c->tile_perm) ? (long long)dest[blockIdx.x] : (long long)blockIdx.x;
    };
    // whole tiles of 16-byte aligned arrays move in 16-byte vectors
    typedef typename K::T T;
    constexpr int VW = 16 / sizeof(T);
    const bool vec = cnt == NV && (((uintptr_t)(in_k + base)) & 15) == 0 &&
                     (!VALS || (((uintptr_t)(in_v + base)) & 15) == 0);
    if (vec) {
        for (int g = t; g < NV / VW; g += NT) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(in_k + base) + g);
            if (sizeof(T) == 4) {
                *reinterpret_cast<uint4 *>(s + 4 * g) =
                    make_uint4((uint32_t)K::ord((T)q.x), (uint32_t)K::ord((T)q.y), (uint32_t)K::ord((T)q.z),
                               (uint32_t)K::ord((T)q.w));
            } else {
                *reinterpret_cast<ulonglong2 *>(s + 2 * g) =
                    make_ulonglong2((unsigned long long)K::ord((T)(((unsigned long long)q.y << 32) | q.x)),
                                    (unsigned long long)K::ord((T)(((unsigned long long)q.w << 32) | q.z)));
            }
        }
        if (VALS)
            for (int g = t; g < NV / 4; g += NT)
                *reinterpret_cast<uint4 *>(sv + 4 * g) = __ldg(reinterpret_cast<const uint4 *>(in_v + base) + g);
    } else {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int idx = i * NT + t;
            s[idx] = idx < cnt ? K::ord(in_k[base + idx]) : umax_of<U>();
            if (VALS) sv[idx] = idx < cnt ? in_v[base + idx] : 0u;
        }
    }
    __syncthreads();
    // presortedness of the tile
    int desc = 0, nondesc = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int j = t * IPT + i;
        if (j + 1 < cnt) {
            desc |= s[j] > s[j + 1];
            nondesc |= !(s[j] > s[j + 1]);
        }
    }
    const int any_desc = __syncthreads_or(desc);
    const int any_nondesc = __syncthreads_or(nondesc);
    // first and last key of every merge tile of mv keys in this tile, for the
    // first merge pass's split search; `rev` reads the tile back to front
    auto samples = [&](bool rev, long long otile) {
        if (!samp) return;
        const int per = NV / mv;
        for (int q = t; q < per && q * mv < cnt; q += NT) {
            const int f = q * mv, l = min(f + mv, cnt) - 1;
            samp[2 * (otile * per + q)] = rev ? s[cnt - 1 - f] : s[f];
            samp[2 * (otile * per + q) + 1] = rev ? s[cnt - 1 - l] : s[l];
        }
    };
    if (!any_desc) {                       // already ascending
        const long long otile = out_tile(), obase = otile * NV;
        if (t == 0 && tile_lo) { tile_lo[otile] = s[0]; tile_hi[otile] = s[cnt - 1]; }
        samples(false, otile);
        if (out_k != in_k || obase != base) {
            for (int idx = t; idx < cnt; idx += NT) {
                out_k[obase + idx] = K::unord(s[idx]);
                if (VALS) out_v[obase + idx] = sv[idx];
            }
        }
        return;
    }
    if (!any_nondesc) {                    // strictly descending: reverse
        const long long otile = out_tile(), obase = otile * NV;
        if (t == 0 && tile_lo) { tile_lo[otile] = s[cnt - 1]; tile_hi[otile] = s[0]; }
        samples(true, otile);
        for (int idx = t; idx < cnt; idx += NT) {
            out_k[obase + idx] = K::unord(s[cnt - 1 - idx]);
            if (VALS) out_v[obase + idx] = sv[cnt - 1 - idx];
        }
        return;
    }
    U k[IPT];
    uint32_t v[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        k[i] = s[t * IPT + i];
        v[i] = VALS ? sv[t * IPT + i] : 0u;
    }
    __syncthreads();
    if constexpr (!VALS && sizeof(U) == 4 && SR_BSORT_PP == 1) {
        s = block_sort_pp<U, NT, IPT>(k, s, s + block_sort_pp_keys<NT, IPT>());
    } else if constexpr (SR_BSORT_PP == 2) {
        uint32_t *va = reinterpret_cast<uint32_t *>(s + block_sort_pp_keys<NT, IPT>());
        s = block_sort_rs<U, NT, IPT, VALS>(k, v, s, va);
        sv = va;
    } else {
        block_sort<U, NT, IPT, VALS>(k, v, s, sv);
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            s[t * IPT + i] = k[i];
            if (VALS) sv[t * IPT + i] = v[i];
        }
        __syncthreads();
    }
    const long long otile = out_tile(), obase = otile * NV;
    if (t == 0 && tile_lo) { tile_lo[otile] = s[0]; tile_hi[otile] = s[cnt - 1]; }
    samples(false, otile);
    if (vec && (((uintptr_t)(out_k + obase)) & 15) == 0 && (!VALS || (((uintptr_t)(out_v + obase)) & 15) == 0)) {
        for (int g = t; g < NV / VW; g += NT) {
            uint4 q;
            if (sizeof(T) == 4) {
                const uint4 r = *reinterpret_cast<const uint4 *>(s + 4 * g);
                q = make_uint4((uint32_t)K::unord((U)r.x), (uint32_t)K::unord((U)r.y), (uint32_t)K::unord((U)r.z),
                               (uint32_t)K::unord((U)r.w));
            } else {
                const ulonglong2 r = *reinterpret_cast<const ulonglong2 *>(s + 2 * g);
                const unsigned long long e0 = (unsigned long long)K::unord((U)r.x);
                const unsigned long long e1 = (unsigned long long)K::unord((U)r.y);
                q = make_uint4((uint32_t)e0, (uint32_t)(e0 >> 32), (uint32_t)e1, (uint32_t)(e1 >> 32));
            }
            reinterpret_cast<uint4 *>(out_k + obase)[g] = q;
        }
        if (VALS)
            for (int g = t; g < NV / 4; g += NT)
                reinterpret_cast<uint4 *>(out_v + obase)[g] = *reinterpret_cast<const uint4 *>(sv + 4 * g);
        return;
    }
    for (int idx = t; idx < cnt; idx += NT) {
        out_k[obase + idx] = K::unord(s[idx]);
        if (VALS) out_v[obase + idx] = sv[idx];
    }
}

// Run planner (after the block sort), the natural runs of Section 3 at the
// granularity of whole tiles: tile t starts a new run unless the previous
// tile's largest key is <= its smallest (then the two sorted tiles are one
// sorted run already).  Merge step s of fan-in f merges groups of f
// consecutive runs of the step before, i.e. groups of f^(s+1) natural runs
// (policy e1 over the input's own runs), so an input made of m presorted
// stretches needs ceil(log_f(m)) steps whatever its length; an input with no
// presorted stretch longer than a tile has one run per tile.
//
// One CTA: rs0[q] = the first tile of natural run q (q < nruns), rs0[nruns] =
// tiles; nsteps = ceil(log_f(nruns)); src_buf[s] = the buffer holding the data
// before step s (the block sort's output buffer: cur0, or 1 when it turned chains of tiles).  Steps s >= nsteps of
// the launched sequence return at once.
template <int KT>
__global__ void __launch_bounds__(RUNS_NT)
k_runs(const typename Key<KT>::U *__restrict__ lo, const typename Key<KT>::U *__restrict__ hi, long long n,
       long long tiles, int fan, int cur0, int *__restrict__ rs0, Ctrl *__restrict__ c) {
    griddep_wait();
    if (call_mode(c, n) != MODE_SORT) return;
    __shared__ int s_warp[RUNS_NT / 32];
    __shared__ int s_total;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int base = 0;
    int far = 0;                                   // some tile's keys exceed the tile's two places on
    for (long long t0 = 0; t0 < tiles; t0 += RUNS_NT) {
        const long long q = t0 + t;
        const bool first = q < tiles && (q == 0 || hi[q - 1] > lo[q]);
        if (q + 2 < tiles && hi[q] > lo[q + 2]) far = 1;
        const unsigned ball = __ballot_sync(0xffffffffu, first);
        if (lane == 0) s_warp[wid] = __popc(ball);
        __syncthreads();
        if (wid == 0) {
            const int v = s_warp[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            s_warp[lane] = incl - v;               // exclusive prefix of the warps' counts
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
        if (first) rs0[base + s_warp[wid] + __popc(ball & ((1u << lane) - 1u))] = (int)q;
        base += s_total;
        __syncthreads();
    }
    far = __syncthreads_or(far);
    if (t == 0) {
        rs0[base] = (int)tiles;
        int steps = 0;
        for (long long m = base; m > 1; m = (m + fan - 1) / fan) ++steps;
        c->nruns = base;
        c->nsteps = steps;
        c->repair = (!far && steps > 0 && tiles >= 3) ? 1 : 0;
        const int cur = cur0 | (c->tile_perm ? 1 : 0);   // turned chains: the block sort wrote to scratch
        for (int s = 0; s <= steps; ++s) c->src_buf[s] = (signed char)(cur ^ (s & 1));
    }
}

// Neighbour repair, step 1 (when only neighbouring tiles overlap: every
// tile's keys are <= those of the tile two places on).  For each boundary
// between tiles t and t + 1 of the block sort's output: the keys of tile t
// above tile t+1's smallest (a suffix of t) and the keys of tile t+1 below
// tile t's largest (a prefix of t+1) are the only ones out of order there;
// win[2t], win[2t+1] = their counts.  A window larger than a merge tile
// (cap keys) sets repair_fail and the merge steps run instead.  These
// windows never overlap: a key of tile t below tile t-1's largest is <= tile
// t+1's smallest.
template <int KT>
__global__ void __launch_bounds__(256)
k_repair_plan(const typename Key<KT>::T *__restrict__ uk, const typename Key<KT>::T *__restrict__ sk,
              const typename Key<KT>::U *__restrict__ lo, const typename Key<KT>::U *__restrict__ hi, long long n,
              long long ts, long long tiles, int cap, int *__restrict__ win, Ctrl *__restrict__ c) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    if (call_mode(c, n) != MODE_SORT || !c->repair) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t + 1 >= tiles) return;
    const typename K::T *src = c->src_buf[0] ? sk : uk;
    const long long x0 = t * ts, x1 = x0 + ts, y0 = x1, y1 = min(y0 + ts, n);
    const U ymin = lo[t + 1], xmax = hi[t];
    long long a = x0, b = x1;                      // first key of tile t above ymin
    while (a < b) {
        const long long m = (a + b) >> 1;
        if (K::ord(src[m]) <= ymin) a = m + 1;
        else b = m;
    }
    long long e = y0, f = y1;                      // first key of tile t+1 not below xmax
    while (e < f) {
        const long long m = (e + f) >> 1;
        if (K::ord(src[m]) < xmax) e = m + 1;
        else f = m;
    }
    const long long na = x1 - a, nb = e - y0;
    win[2 * t] = (int)min(na, (long long)cap + 1);
    win[2 * t + 1] = (int)min(nb, (long long)cap + 1);
    if (na + nb > cap) atomicExch(&c->repair_fail, 1);
    else if (na && nb) atomicAdd(&c->repair_keys, (unsigned long long)(na + nb));
}

// Where natural run q starts (n for q >= nruns; keys, not tiles).
__device__ __forceinline__ long long nrun_pos(const int *__restrict__ rs0, int nruns, long long q, long long ts,
                                              long long n, long long tiles) {
    if (q >= nruns) return n;
    return min((nruns == tiles ? q : (long long)rs0[q]) * ts, n);   // every tile a run: no table read
}

// The natural run that holds tile t (the last q with rs0[q] <= t).
__device__ __forceinline__ long long nrun_of(const int *__restrict__ rs0, int nruns, long long tiles, long long t) {
    if (nruns == tiles) return t;                  // every tile a run of its own
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rs0[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The merge-path split of output position out of the merge of the adjacent
// sorted runs A = src[a_beg, a_end) and B = src[a_end, b_end) (run starts and
// out - a_beg are multiples of nv): the index in src where the share of A of
// the outputs from `out` on starts.  A group of 2^lg lanes computes it
// together (all lanes of the group get it).  samp (optional): the first and
// last key of every merge tile of src, as recorded when src was written; with
// it the search first narrows the split to one tile's stretch and then reads
// keys only there.
template <int KT>
__device__ __forceinline__ long long merge_split(const typename Key<KT>::T *__restrict__ src, long long a_beg,
                                                 long long a_end, long long b_end, long long out, int nv,
                                                 int lane, int lg, const typename Key<KT>::U *__restrict__ samp) {
    typedef Key<KT> K;
    typedef typename K::U U;
    const long long b_beg = a_end;
    const long long na = a_end - a_beg, nb = b_end - b_beg, d = out - a_beg;
    long long lo = max(0ll, d - nb), hi = min(d, na);
    if (samp && out < b_end && hi > lo) {
        // Coarse: the merge-path test at the multiples m = j*nv uses only the
        // first key of A's tile j and the last key of B's tile d/nv - j - 1.
        const long long jlo = (lo + nv - 1) / nv, jhi = (hi - 1) / nv, dj = d / nv;
        const long long ta = a_beg / nv, tb = b_beg / nv;
        const long long jt = group_search(jlo, jhi + 1, lane, lg, [&](long long j) {
            const U x = samp[2 * (ta + j)];
            const U y = samp[2 * (tb + dj - j - 1) + 1];
            return !(y < x);
        });
        if (jt > jlo) lo = max(lo, (jt - 1) * nv + 1);
        if (jt <= jhi) hi = min(hi, jt * nv);
    }
    // fine: the keys themselves, inside the stretch the samples left
    const long long sp = group_search(lo, hi, lane, lg, [&](long long m) {
        const U x = K::ord(src[a_beg + m]);
        const U y = K::ord(src[b_beg + d - 1 - m]);
        return !(y < x);
    });
    return a_beg + sp;
}

// Split of every output tile boundary b of merge step `step`, whose pairs
// are consecutive runs of `span` natural runs each (the pairs a 2-way step
// merges, or the AB and CD pairs of a 4-way step's groups); a group of 2^lg
// lanes per boundary.  splits[4b .. 4b + 3] = {where the tile's share of A
// starts, A's start, A's end = B's start, B's end}.  The tile samples of the
// buffer the step reads are at samp + smt * (that buffer).
template <int KT>
__global__ void __launch_bounds__(256)
k_partition(const typename Key<KT>::T *__restrict__ uk, const typename Key<KT>::T *__restrict__ sk,
            long long n, long long ts, long long tiles, int nv, long long nbound, long long *__restrict__ splits,
            const int *__restrict__ rs0, long long span, const Ctrl *__restrict__ c, int step, int lg,
            const typename Key<KT>::U *__restrict__ samp, long long smt) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> lg;
    if (b >= nbound) return;                       // uniform across the group
    if (step >= steps_of(c)) return;               // also when the input needs no sorting
    const bool leader = (lane & ((1 << lg) - 1)) == 0;
    const long long out = b * (long long)nv;
    if (out >= n) {                                // the end of the array: never a tile's start
        if (leader)
            for (int i = 0; i < 4; ++i) splits[4 * b + i] = n;
        return;
    }
    const int cur = c->src_buf[step];
    const int nruns = c->nruns;
    const long long q = nrun_of(rs0, nruns, tiles, out / ts);
    const long long p0 = (q / (2 * span)) * (2 * span);
    const long long a_beg = nrun_pos(rs0, nruns, p0, ts, n, tiles);
    const long long a_end = nrun_pos(rs0, nruns, p0 + span, ts, n, tiles);
    const long long b_end = nrun_pos(rs0, nruns, p0 + 2 * span, ts, n, tiles);
    const long long sp = merge_split<KT>(cur ? sk : uk, a_beg, a_end, b_end, out, nv, lane, lg,
                                         samp ? samp + cur * smt : nullptr);
    if (leader) {
        splits[4 * b + 0] = sp;
        splits[4 * b + 1] = a_beg;
        splits[4 * b + 2] = a_end;
        splits[4 * b + 3] = b_end;
    }
}

// Lanes per boundary for k_partition: about SR_PARTITION_LANES searching
// lanes in all, between 1 and 32 per boundary.
#ifndef SR_PARTITION_LANES
#define SR_PARTITION_LANES 160000
#endif
inline int partition_lg(long long nbound) {
    int lg = 5;
    while (lg > 0 && (nbound << lg) > SR_PARTITION_LANES) --lg;
    return lg;
}
// Lanes per boundary for k_partition4, whose probes each run two binary
// searches inside one merge tile: between 1 and 8 lanes, about
// SR_PARTITION4_LANES in all.
#ifndef SR_PARTITION4_LANES
#define SR_PARTITION4_LANES 160000
#endif
inline int partition4_lg(long long nbound) {
    int lg = 3;
    while (lg > 0 && (nbound << lg) > SR_PARTITION4_LANES) --lg;
    return lg;
}

// The end of a merge tile: every thread holds its IPT merged keys (and
// values) in registers; they go through shared memory (s, sv) so the tile
// leaves in coalesced (VEC: 16-byte) stores to dst at out0.  The tile's first
// and last key go to samp[2 * tile], samp[2 * tile + 1] if samp is given.
template <int KT, int NT, int IPT, bool VALS, bool VEC>
__device__ __forceinline__ void write_tile(const typename Key<KT>::U (&k)[IPT], const uint32_t (&v)[IPT],
                                           typename Key<KT>::U *s, uint32_t *sv,
                                           typename Key<KT>::T *__restrict__ dst_k, uint32_t *__restrict__ dst_v,
                                           long long out0, int cnt, typename Key<KT>::U *samp, long long tile,
                                           bool raw = false) {
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    const int t = threadIdx.x;
    // raw: the keys are the caller's own bit patterns (int32 compared as
    // signed), not order images; they leave unchanged and the samples get
    // their images
    auto out = [raw](U x) -> T { return raw ? (T)x : K::unord(x); };
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        s[t * IPT + i] = k[i];
        if (VALS) sv[t * IPT + i] = v[i];
    }
    __syncthreads();
    if (samp && t == 0) {                          // the output tile's first and last key, for the next pass
        samp[2 * tile] = raw ? K::ord((T)s[0]) : s[0];
        samp[2 * tile + 1] = raw ? K::ord((T)s[cnt - 1]) : s[cnt - 1];
    }
    if (VEC) {
        // keys before the first 4-key group boundary of the output go one by one
        const int head = min(cnt, (int)((4 - (out0 & 3)) & 3));
        if (t < head) {
            dst_k[out0 + t] = out(s[t]);
            if (VALS) dst_v[out0 + t] = sv[t];
        }
        const int full = (cnt - head) >> 2;
        if (head == 0) {
            // the tile starts on a group boundary: 16-byte shared loads as well
            for (int g = t; g < full; g += NT) {
                const int j = 4 * g;
                if (sizeof(T) == 4) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(s + j);
                    *reinterpret_cast<uint4 *>(dst_k + out0 + j) =
                        make_uint4((uint32_t)out((U)q.x), (uint32_t)out((U)q.y),
                                   (uint32_t)out((U)q.z), (uint32_t)out((U)q.w));
                } else {
                    const ulonglong2 q0 = *reinterpret_cast<const ulonglong2 *>(s + j);
                    const ulonglong2 q1 = *reinterpret_cast<const ulonglong2 *>(s + j + 2);
                    const unsigned long long e0 = (unsigned long long)out((U)q0.x);
                    const unsigned long long e1 = (unsigned long long)out((U)q0.y);
                    const unsigned long long e2 = (unsigned long long)out((U)q1.x);
                    const unsigned long long e3 = (unsigned long long)out((U)q1.y);
                    *reinterpret_cast<uint4 *>(dst_k + out0 + j) =
                        make_uint4((uint32_t)e0, (uint32_t)(e0 >> 32), (uint32_t)e1, (uint32_t)(e1 >> 32));
                    *reinterpret_cast<uint4 *>(dst_k + out0 + j + 2) =
                        make_uint4((uint32_t)e2, (uint32_t)(e2 >> 32), (uint32_t)e3, (uint32_t)(e3 >> 32));
                }
                if (VALS) *reinterpret_cast<uint4 *>(dst_v + out0 + j) = *reinterpret_cast<const uint4 *>(sv + j);
            }
        } else for (int g = t; g < full; g += NT) {
            const int j = head + 4 * g;
            if (sizeof(T) == 4) {
                uint4 q;
                q.x = (uint32_t)out(s[j + 0]);
                q.y = (uint32_t)out(s[j + 1]);
                q.z = (uint32_t)out(s[j + 2]);
                q.w = (uint32_t)out(s[j + 3]);
                *reinterpret_cast<uint4 *>(dst_k + out0 + j) = q;
            } else {
                const unsigned long long e0 = (unsigned long long)out(s[j + 0]);
                const unsigned long long e1 = (unsigned long long)out(s[j + 1]);
                const unsigned long long e2 = (unsigned long long)out(s[j + 2]);
                const unsigned long long e3 = (unsigned long long)out(s[j + 3]);
                *reinterpret_cast<uint4 *>(dst_k + out0 + j) =
                    make_uint4((uint32_t)e0, (uint32_t)(e0 >> 32), (uint32_t)e1, (uint32_t)(e1 >> 32));
                *reinterpret_cast<uint4 *>(dst_k + out0 + j + 2) =
                    make_uint4((uint32_t)e2, (uint32_t)(e2 >> 32), (uint32_t)e3, (uint32_t)(e3 >> 32));
            }
            if (VALS)
                *reinterpret_cast<uint4 *>(dst_v + out0 + j) = make_uint4(sv[j], sv[j + 1], sv[j + 2], sv[j + 3]);
        }
        for (int i = head + 4 * full + t; i < cnt; i += NT) {
            dst_k[out0 + i] = out(s[i]);
            if (VALS) dst_v[out0 + i] = sv[i];
        }
    } else {
        for (int i = t; i < cnt; i += NT) {
            dst_k[out0 + i] = out(s[i]);
            if (VALS) dst_v[out0 + i] = sv[i];
        }
    }
}

// The merge of one tile's staged windows A = s[sa, sa + acnt) and B = s[sb,
// sb + bcnt): thread outputs diag .. diag + IPT into k (with their staged
// positions in ix).  `marks`: the key after each window is `mark`, so when
// neither window holds it the steps compare once (serial_merge_marked).  C is
// the type the keys compare in (the order images, or int32 for raw int32 keys).
template <typename C, int IPT>
__device__ __forceinline__ void tile_merge(const C *s, int sa, int acnt, int sb, int bcnt, int cnt, int diag,
                                           bool marks, C mark, C (&k)[IPT], int (&ix)[IPT]) {
    const int sp = merge_path(s + sa, acnt, s + sb, bcnt, diag);
    const bool marked = marks && (acnt == 0 || s[sa + acnt - 1] != mark) && (bcnt == 0 || s[sb + bcnt - 1] != mark);
    if (marked) {
        serial_merge_marked<C, IPT>(s, sa + sp, sb + diag - sp, k, ix);
    } else if (SR_MERGE_1LD) {
        serial_merge_slack<C, IPT>(s, sa + sp, sa + acnt, sb + diag - sp, sb + bcnt, k, ix);
    } else {
        serial_merge<C, IPT>(s, sa + sp, sa + acnt, sb + diag - sp, sb + bcnt, k, ix);
    }
}

// Staged keys (and values) of a merge tile of NV keys: the two windows in
// 4-key groups, a spare group between them for A's end mark, and B's mark.
template <int NV> constexpr int merge_tile_sv() { return NV + 20; }

// Dynamic shared memory that merge_tile needs: merge_tile_sv staged keys (and
// as many values), plus the key slack the one-load merge step reads into.
template <typename U, int NT, int IPT, bool VALS>
constexpr size_t merge_tile_smem() {
    return (size_t)merge_tile_sv<NT * IPT>() * (sizeof(U) + (VALS ? 4 : 0)) +
           (SR_MERGE_1LD ? (size_t)(IPT + 8) * sizeof(U) : 0);
}

// Merges one output tile: outputs [out0, out0 + cnt) of the stable merge of
// the sorted ranges A = src[a0 .. a1) and B = src[b0 .. b0 + cnt - (a1 - a0)),
// written to dst at out0.  All threads of the CTA call it; s / sv are shared
// buffers of merge_tile_sv keys / values, and with SR_MERGE_1LD the key buffer
// must stay readable IPT + 8 keys further (the memory after it: the value
// buffer, or padding) -- merge_tile_smem gives the dynamic shared memory for
// s followed by sv.  `n` bounds the global buffers (loads stay below it).
//
// VEC (every buffer 16-byte aligned): the ranges are staged as windows of
// 4-key groups starting on a group boundary, so every group moves with 128-bit
// loads and shared-memory stores, all issued before the first is used; the
// output tile (which must start on a group boundary) leaves with 128-bit
// stores between scalar head and tail keys.  Keys before a range's start
// inside its first group are staged and ignored.
//
// bar (optional, VEC only): stage the two windows' whole 16-byte stretches by
// 1-D bulk copies that one thread starts, completed on this mbarrier (the
// keys past the array's last 16-byte boundary by plain loads), then turn them
// into order images in place; a tile whose copies do not complete within the
// wait's limit reports SR_ERR_TIMEOUT in `status` and writes nothing.  B's
// groups start one group after A's, and the key after each window is set to
// umax: when neither window holds a umax key, the merge steps compare once
// (serial_merge_marked).
template <int KT, int NT, int IPT, bool VALS, bool VEC>
__device__ __forceinline__ void merge_tile(const typename Key<KT>::T *__restrict__ src_k,
                                           typename Key<KT>::T *__restrict__ dst_k,
                                           const uint32_t *__restrict__ src_v, uint32_t *__restrict__ dst_v,
                                           long long n, long long out0, int cnt, long long a0, long long a1,
                                           long long b0, typename Key<KT>::U *s, uint32_t *sv,
                                           typename Key<KT>::U *samp = nullptr, long long tile = 0,
                                           unsigned long long *bar = nullptr, int *status = nullptr) {
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    constexpr int NV = NT * IPT;
    constexpr int SV = NV + 16;
    const int t = threadIdx.x;
    const int acnt = (int)(a1 - a0);
    const int bcnt = cnt - acnt;
    // bulk-staged int32 keys may stay raw and compare as signed int32 (no image pass)
    constexpr bool RAW_OK = KT == SR_KEY_I32 && SR_MERGE_RAW_I32;
    const bool raw = RAW_OK && VEC && bar;
    const U mark = raw ? (U)INT_MAX : umax_of<U>();
    int sa, sb;                                    // staged positions of A[a0] and B[b0]
    if (VEC && bar) {
        const long long g0[2] = {a0 & ~3ll, b0 & ~3ll};
        const long long ge[2] = {(a1 + 3) & ~3ll, (b0 + bcnt + 3) & ~3ll};
        const int nag = acnt > 0 ? (int)((ge[0] - g0[0]) >> 2) : 0;
        const int nbg = bcnt > 0 ? (int)((ge[1] - g0[1]) >> 2) : 0;
        const int first[2] = {0, nag + 1};        // a spare group between the windows
        const int ng[2] = {nag, nbg};
        sa = (int)(a0 - g0[0]);
        sb = 4 * (nag + 1) + (int)(b0 - g0[1]);
        const long long n4 = n & ~3ll;
        if (t == 0) mbar_init(bar, 1);
        __syncthreads();
        if (t == 0) {
            unsigned bytes = 0;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const long long hi = min(g0[i] + 4ll * ng[i], n4);
                if (hi > g0[i]) bytes += (unsigned)((hi - g0[i]) * (sizeof(T) + (VALS ? 4 : 0)));
            }
            mbar_arrive_expect(bar, bytes);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const long long hi = min(g0[i] + 4ll * ng[i], n4);
                if (hi > g0[i]) {
                    bulk_copy_g2s(s + 4 * first[i], src_k + g0[i], (unsigned)((hi - g0[i]) * sizeof(T)), bar);
                    if (VALS) bulk_copy_g2s(sv + 4 * first[i], src_v + g0[i], (unsigned)((hi - g0[i]) * 4), bar);
                }
            }
        }
        const long long e[2] = {a1, b0 + bcnt};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            if (ng[i] > 0 && e[i] > n4) {
                const long long from = max(n4, g0[i]);
                if (t < e[i] - from) {
                    const long long g = from + t;
                    s[4 * first[i] + (g - g0[i])] = (U)src_k[g];
                    if (VALS) sv[4 * first[i] + (g - g0[i])] = src_v[g];
                }
            }
        }
        const bool done = mbar_wait_bounded(bar, 0, BULK_WAIT_TRIES);
        if (!__syncthreads_and(done)) {
            if (t == 0 && status) atomicExch(status, (int)SR_ERR_TIMEOUT);
            mbar_wait_bounded(bar, 0, BULK_WAIT_TRIES);   // copies still in flight must land first
            return;
        }
        if (KT != SR_KEY_U32 && KT != SR_KEY_U64 && !raw) {   // raw keys -> order images, in place
            for (int g = t; g < nag + 1 + nbg; g += NT) {
                if (sizeof(U) == 4) {
                    uint4 q = *reinterpret_cast<uint4 *>(s + 4 * g);
                    q.x = (uint32_t)K::ord((T)q.x); q.y = (uint32_t)K::ord((T)q.y);
                    q.z = (uint32_t)K::ord((T)q.z); q.w = (uint32_t)K::ord((T)q.w);
                    *reinterpret_cast<uint4 *>(s + 4 * g) = q;
                } else {
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) s[4 * g + e2] = K::ord((T)s[4 * g + e2]);
                }
            }
            __syncthreads();
        }
        if (t == 0) {                              // the windows' end marks
            s[sa + acnt] = mark;
            s[sb + bcnt] = mark;
        }
    } else if (VEC) {
        const long long a0g = a0 & ~3ll, b0g = b0 & ~3ll;
        const int nag = (int)((((a1 + 3) & ~3ll) - a0g) >> 2);
        const int nbg = (int)((((b0 + bcnt + 3) & ~3ll) - b0g) >> 2);
        sa = (int)(a0 - a0g);
        const int offb = 4 * nag;
        sb = offb + (int)(b0 - b0g);
        constexpr int KMAX = (SV / 4 + NT - 1) / NT;
        U r[KMAX][4];
        uint4 rv[VALS ? KMAX : 1];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int g = t + k * NT;
            if (g < nag + nbg) {
                const long long gb = g < nag ? a0g + 4ll * g : b0g + 4ll * (g - nag);
                if (gb + 4 <= n) {
                    if (sizeof(T) == 4) {
                        const uint4 q = *reinterpret_cast<const uint4 *>(src_k + gb);
                        r[k][0] = (U)q.x; r[k][1] = (U)q.y; r[k][2] = (U)q.z; r[k][3] = (U)q.w;
                    } else {
                        const uint4 q0 = *reinterpret_cast<const uint4 *>(src_k + gb);
                        const uint4 q1 = *reinterpret_cast<const uint4 *>(src_k + gb + 2);
                        r[k][0] = (U)(((unsigned long long)q0.y << 32) | q0.x);
                        r[k][1] = (U)(((unsigned long long)q0.w << 32) | q0.z);
                        r[k][2] = (U)(((unsigned long long)q1.y << 32) | q1.x);
                        r[k][3] = (U)(((unsigned long long)q1.w << 32) | q1.z);
                    }
                    if (VALS) rv[k] = *reinterpret_cast<const uint4 *>(src_v + gb);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) r[k][e] = (gb + e < n) ? (U)src_k[gb + e] : U(0);
                    if (VALS) {
                        rv[k].x = (gb + 0 < n) ? src_v[gb + 0] : 0u;
                        rv[k].y = (gb + 1 < n) ? src_v[gb + 1] : 0u;
                        rv[k].z = (gb + 2 < n) ? src_v[gb + 2] : 0u;
                        rv[k].w = (gb + 3 < n) ? src_v[gb + 3] : 0u;
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int g = t + k * NT;
            if (g < nag + nbg) {
                const int o = g < nag ? 4 * g : offb + 4 * (g - nag);
                // one 16-byte shared store per 4-key group (o is a multiple of 4)
                if (sizeof(U) == 4) {
                    *reinterpret_cast<uint4 *>(s + o) =
                        make_uint4((uint32_t)K::ord((T)r[k][0]), (uint32_t)K::ord((T)r[k][1]),
                                   (uint32_t)K::ord((T)r[k][2]), (uint32_t)K::ord((T)r[k][3]));
                } else {
                    *reinterpret_cast<ulonglong2 *>(s + o) =
                        make_ulonglong2((unsigned long long)K::ord((T)r[k][0]), (unsigned long long)K::ord((T)r[k][1]));
                    *reinterpret_cast<ulonglong2 *>(s + o + 2) =
                        make_ulonglong2((unsigned long long)K::ord((T)r[k][2]), (unsigned long long)K::ord((T)r[k][3]));
                }
                if (VALS) *reinterpret_cast<uint4 *>(sv + o) = rv[k];
            }
        }
    } else {
        sa = 0;
        sb = acnt;
        for (int i = t; i < cnt; i += NT) {
            const long long g = i < acnt ? a0 + i : b0 + (i - acnt);
            s[i] = K::ord(src_k[g]);
            if (VALS) sv[i] = src_v[g];
        }
    }
    __syncthreads();
    const int diag = min(t * IPT, cnt);
    U k[IPT];
    int ix[IPT];
    if constexpr (RAW_OK) {
        if (raw) {
            int ki[IPT];
            tile_merge<int, IPT>(reinterpret_cast<const int *>(s), sa, acnt, sb, bcnt, cnt, diag, true, INT_MAX, ki,
                                 ix);
#pragma unroll
            for (int i = 0; i < IPT; ++i) k[i] = (U)ki[i];
        } else {
            tile_merge<U, IPT>(s, sa, acnt, sb, bcnt, cnt, diag, VEC && bar, mark, k, ix);
        }
    } else {
        tile_merge<U, IPT>(s, sa, acnt, sb, bcnt, cnt, diag, VEC && bar, mark, k, ix);
    }
    uint32_t v[IPT];
    if (VALS) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) v[i] = (diag + i < cnt) ? sv[ix[i]] : 0u;
    }
    write_tile<KT, NT, IPT, VALS, VEC>(k, v, s, sv, dst_k, dst_v, out0, cnt, samp, tile, raw);
}

// One CTA per output tile of NT*IPT keys of a 2-way merge step.  The tile's
// pair of runs and its share of each come from the split table.
template <int KT, int NT, int IPT, bool VALS, int STAGE>
__global__ void __launch_bounds__(NT, Shape<sizeof(typename Key<KT>::T), VALS>::MERGE_MINB)
k_merge(typename Key<KT>::T *uk, uint32_t *uv, typename Key<KT>::T *sk, uint32_t *svb, long long n,
        const long long *__restrict__ splits, const Ctrl *__restrict__ c, int step,
        typename Key<KT>::U *__restrict__ samp, long long smt, int *status) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int NV = NT * IPT;
    constexpr int SV = merge_tile_sv<NV>();        // staged keys, with room for window slack
    const long long b = blockIdx.x;
    // the tile's split entries (the table has a boundary past the last tile)
    // and the call's state, loaded together before any of them is tested
    const long long a0 = splits[4 * b], a_beg = splits[4 * b + 1], a_end = splits[4 * b + 2];
    const long long b_end = splits[4 * b + 3], a_next = splits[4 * (b + 1)];
    const int nsteps = steps_of(c);
    const int cur = c->src_buf[step];
    if (step >= nsteps) return;                    // also when the input needs no sorting
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + SV);
    const long long out0 = b * NV;
    const long long out1 = min(out0 + NV, n);
    const long long a1 = (out1 == b_end) ? a_end : a_next;
    const long long b0 = a_end + (out0 - a_beg) - (a0 - a_beg);
    // the output's tile samples go with the buffer it lands in
    __shared__ unsigned long long bar;
    merge_tile<KT, NT, IPT, VALS, STAGE != STAGE_SCALAR>(cur ? sk : uk, cur ? uk : sk, cur ? svb : uv,
                                                         cur ? uv : svb, n, out0, (int)(out1 - out0), a0, a1, b0, s,
                                                         sv, samp ? samp + (1 - cur) * smt : nullptr, b,
                                                         STAGE == STAGE_BULK ? &bar : nullptr, status);
}

// Neighbour repair, step 2: one CTA per tile boundary merges its window (the
// suffix of tile t and the prefix of tile t+1 found by k_repair_plan) in place,
// stably; keys outside the windows stay where the block sort put them.  After
// it the whole array is sorted: left of a window every key is <= tile t+1's
// smallest, right of it every key is >= tile t's largest.
template <int KT, int NT, int IPT, bool VALS>
__global__ void __launch_bounds__(NT)
k_repair(typename Key<KT>::T *uk, uint32_t *uv, typename Key<KT>::T *sk, uint32_t *svb, long long n, long long ts,
         long long tiles, const int *__restrict__ win, const Ctrl *__restrict__ c) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int SV = NT * IPT + 16;
    if (call_mode(c, n) != MODE_SORT || !c->repair || c->repair_fail) return;
    const long long t = blockIdx.x;
    if (t + 1 >= tiles) return;
    const int na = win[2 * t], nb = win[2 * t + 1];
    if (na == 0 || nb == 0) return;                // the boundary is already in order
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + SV);
    const bool scratch = c->src_buf[0] != 0;
    typename K::T *buf = scratch ? sk : uk;
    uint32_t *vbuf = scratch ? svb : uv;
    const long long mid = (t + 1) * ts;
    merge_tile<KT, NT, IPT, VALS, false>(buf, buf, vbuf, vbuf, n, mid - na, na + nb, mid - na, mid, mid, s, sv);
}

// ------------------------------------------------------------ 4-way merge steps
//
// A 4-way step merges every group of four consecutive runs A, B, C, D of w
// keys (the group at the end of the array may hold fewer or shorter runs) into
// one run: merge(merge(A, B), merge(C, D)), with A before B before C before D
// on equal keys -- the stable merge of the four runs (policy e1 of Section 3
// taken two rounds at a time), reading and writing every key once where two
// 2-way passes would do it twice.  The splits come from two launches:
// k_partition over the pairs (A, B) and (C, D) gives the 2-way split of every
// merge tile of the merged pairs AB and CD (which are never written), and
// k_partition4 runs, for every output tile boundary, a merge-path search of AB
// against CD whose probes read keys of AB and CD through those 2-way splits,
// then records where each of A, B, C and D starts for the tile.

// A merged pair P = merge(X, Y) of adjacent runs X = [x_beg, x_end) and
// Y = [x_end, y_end), seen through the 2-way splits of its merge tiles:
// split1[4 (t0 + j)] is where P's tile j (outputs j*nv ..) starts in X.
struct PairView {
    long long x_beg, x_end, y_end, t0, len;
};

__device__ __forceinline__ PairView pair_view(long long x_beg, long long x_end, long long y_end, int nv) {
    PairView P;
    P.x_beg = x_beg;
    P.x_end = x_end;
    P.y_end = y_end;
    P.t0 = x_beg / nv;
    P.len = y_end - x_beg;
    return P;
}

// The stretches X[xs, xe) and Y[ys, ye) that tile j of P (j * nv < P.len)
// is merged from.
__device__ __forceinline__ void pair_tile(const long long *__restrict__ split1, const PairView &P, int nv,
                                          long long j, long long &xs, long long &xe, long long &ys,
                                          long long &ye) {
    xs = split1[4 * (P.t0 + j)];
    const long long o1 = min((j + 1) * (long long)nv, P.len);
    xe = o1 == P.len ? P.x_end : split1[4 * (P.t0 + j + 1)];
    ys = P.x_end + j * (long long)nv - (xs - P.x_beg);
    ye = P.x_end + o1 - (xe - P.x_beg);
}

// First and last key images of P's tile j (j * nv < P.len).
template <int KT>
__device__ __forceinline__ typename Key<KT>::U pair_first(const typename Key<KT>::T *__restrict__ src,
                                                          const long long *__restrict__ split1, const PairView &P,
                                                          int nv, long long j) {
    typedef Key<KT> K;
    long long xs, xe, ys, ye;
    pair_tile(split1, P, nv, j, xs, xe, ys, ye);
    if (xs < xe && (ys >= ye || !(K::ord(src[ys]) < K::ord(src[xs])))) return K::ord(src[xs]);
    return K::ord(src[ys]);
}
template <int KT>
__device__ __forceinline__ typename Key<KT>::U pair_last(const typename Key<KT>::T *__restrict__ src,
                                                         const long long *__restrict__ split1, const PairView &P,
                                                         int nv, long long j) {
    typedef Key<KT> K;
    typedef typename K::U U;
    long long xs, xe, ys, ye;
    pair_tile(split1, P, nv, j, xs, xe, ys, ye);
    U v = 0;
    if (xe > xs) v = K::ord(src[xe - 1]);
    if (ye > ys) {
        const U y = K::ord(src[ye - 1]);
        v = v < y ? y : v;
    }
    return v;
}

// S_P(x), how many X keys are among the first x outputs of P (0 <= x <=
// P.len), at x = j * nv: a tile boundary of P (from the split table), or P's
// end.
__device__ __forceinline__ long long pair_count_at_tile(const long long *__restrict__ split1, const PairView &P,
                                                        int nv, long long j) {
    if (j <= 0) return 0;
    if (j * nv >= P.len) return P.x_end - P.x_beg;
    return split1[4 * (P.t0 + j)] - P.x_beg;
}

// Two known values of S_P: S_P(xl) = sl and S_P(xh) = sh, xl <= xh.  Since
// S_P and x - S_P never decrease, S_P(x) for xl <= x <= xh lies in
// [max(sl, sh - (xh - x)), min(sh, sl + (x - xl))].
struct PairAnchors {
    long long xl, sl, xh, sh;
};

// The bounded merge-path search for S_P(x) inside the anchors' range: about
// log2 of the anchors' distance dependent rounds of two loads.
template <int KT>
__device__ __forceinline__ long long pair_count(const typename Key<KT>::T *__restrict__ src, const PairView &P,
                                               const PairAnchors &q, long long x) {
    typedef Key<KT> K;
    const long long nx = P.x_end - P.x_beg, ny = P.y_end - P.x_end;
    long long lo = max(max(q.sl, q.sh - (q.xh - x)), max(0ll, x - ny));
    long long hi = min(min(q.sh, q.sl + (x - q.xl)), min(x, nx));
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (!(K::ord(src[P.x_end + x - 1 - mid]) < K::ord(src[P.x_beg + mid]))) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The 4-way split of boundary d (a multiple of nv, outputs counted from A's
// start) between AB and CD: the number x of AB keys among the first d outputs
// of merge(AB, CD), found in [lo, hi] (already narrowed to one tile of AB by
// the coarse search) by a group of 2^lg lanes, with S_AB(x) in *sab and
// S_CD(d - x) in *scd.  Each round the lanes probe evenly spaced m: AB[m]
// against CD[d - 1 - m], keys of the never-written merged pairs found by the
// bounded searches of pair_count; the lanes next to the round's answer hand
// their counts on as the anchors of the next round, so every search is about
// as long as the stretch the round leaves (the searches of one boundary take
// about log2(nv) + log2(nv / (G+1)) + ... rounds instead of log2(nv) per
// probe).
template <int KT>
__device__ __forceinline__ long long ab_cd_split(const typename Key<KT>::T *__restrict__ src,
                                                 const long long *__restrict__ split1, const PairView &AB,
                                                 const PairView &CD, int nv, long long d, long long lo, long long hi,
                                                 int lane, int lg, long long *sab, long long *scd) {
    typedef Key<KT> K;
    typedef typename K::U U;
    const int G = 1 << lg;
    const int j = lane & (G - 1);
    const int base = lane & ~(G - 1);
    const unsigned mask = lg == 5 ? 0xffffffffu : (((1u << G) - 1u) << base);
    // anchors: the AB tile boundaries around [lo, hi] and the CD boundaries
    // they face (probe m reads AB up to x = m + 1 and CD up to x = d - m)
    const long long j0 = lo / nv;
    PairAnchors ab, cd;
    ab.xl = j0 * nv;
    ab.sl = pair_count_at_tile(split1, AB, nv, j0);
    ab.xh = min((j0 + 1) * nv, AB.len);
    ab.sh = pair_count_at_tile(split1, AB, nv, j0 + 1);
    cd.xl = max(d - (j0 + 1) * nv, 0ll);
    cd.sl = pair_count_at_tile(split1, CD, nv, d / nv - j0 - 1);
    cd.xh = min(d - j0 * nv, CD.len);
    cd.sh = pair_count_at_tile(split1, CD, nv, d / nv - j0);
    while (hi > lo) {
        const long long step = (hi - lo + G) / (G + 1);
        const long long m = lo + (long long)(j + 1) * step - 1;
        bool before = false;
        long long s1 = 0, s2 = 0;
        if (m < hi) {
            const long long x1 = m + 1, x2 = d - m;
            s1 = pair_count<KT>(src, AB, ab, x1);
            s2 = pair_count<KT>(src, CD, cd, x2);
            U a = 0, c = 0;                        // AB[m], CD[d - 1 - m]: the later of the last keys taken
            if (s1 > 0) a = K::ord(src[AB.x_beg + s1 - 1]);
            if (x1 - 1 - s1 >= 0) {
                const U y = K::ord(src[AB.x_end + x1 - 1 - s1]);
                a = a < y ? y : a;
            }
            if (s2 > 0) c = K::ord(src[CD.x_beg + s2 - 1]);
            if (x2 - 1 - s2 >= 0) {
                const U y = K::ord(src[CD.x_end + x2 - 1 - s2]);
                c = c < y ? y : c;
            }
            before = !(c < a);
        }
        const int cnt = __popc(__ballot_sync(mask, before));
        const long long s1l = __shfl_sync(mask, s1, base + (cnt > 0 ? cnt - 1 : 0));
        const long long s2l = __shfl_sync(mask, s2, base + (cnt > 0 ? cnt - 1 : 0));
        const long long s1h = __shfl_sync(mask, s1, base + (cnt < G ? cnt : G - 1));
        const long long s2h = __shfl_sync(mask, s2, base + (cnt < G ? cnt : G - 1));
        const long long mlo = lo + (long long)cnt * step - 1;          // lane cnt - 1's probe
        const long long mhi = lo + (long long)(cnt + 1) * step - 1;    // lane cnt's probe
        if (cnt > 0) {
            ab.xl = mlo + 1; ab.sl = s1l;
            cd.xh = d - mlo; cd.sh = s2l;
        }
        if (cnt < G && mhi < hi) {
            ab.xh = mhi + 1; ab.sh = s1h;
            cd.xl = d - mhi; cd.sl = s2h;
        }
        const long long nhi = cnt == G ? hi : mhi;
        lo = lo + (long long)cnt * step;
        hi = min(hi, nhi);
    }
    *sab = pair_count<KT>(src, AB, ab, lo);
    *scd = pair_count<KT>(src, CD, cd, d - lo);
    return lo;
}

// 4-way splits of every output tile boundary of step `step`, whose groups
// are four consecutive runs of `span` natural runs each; a group of 2^lg
// lanes per boundary.  split4[8b + i] is where tile b's share of run i (A, B,
// C, D) starts in the source buffer, split4[8b + 4 + i] where run i of the
// tile's group ends.
template <int KT>
__global__ void __launch_bounds__(256)
k_partition4(const typename Key<KT>::T *__restrict__ uk, const typename Key<KT>::T *__restrict__ sk,
             long long n, long long ts, long long tiles, int nv, long long nbound,
             const long long *__restrict__ split1, long long *__restrict__ split4, const int *__restrict__ rs0,
             long long span, const Ctrl *__restrict__ c, int step, int lg) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> lg;
    if (b >= nbound) return;                       // uniform across the group
    if (step >= steps_of(c)) return;
    const bool leader = (lane & ((1 << lg) - 1)) == 0;
    const long long out = b * (long long)nv;
    if (out >= n) {                                // the end of the array: never a tile's start
        if (leader)
            for (int i = 0; i < 8; ++i) split4[8 * b + i] = n;
        return;
    }
    const typename Key<KT>::T *src = c->src_buf[step] ? sk : uk;
    const int nruns = c->nruns;
    const long long q = nrun_of(rs0, nruns, tiles, out / ts);
    const long long g0 = (q / (4 * span)) * (4 * span);
    long long e[5];                                // A = [e0, e1), B = [e1, e2), C = [e2, e3), D = [e3, e4)
#pragma unroll
    for (int i = 0; i < 5; ++i) e[i] = nrun_pos(rs0, nruns, g0 + i * span, ts, n, tiles);
    const PairView AB = pair_view(e[0], e[1], e[2], nv), CD = pair_view(e[2], e[3], e[4], nv);
    const long long d = out - e[0];                // a multiple of nv
    long long lo = max(0ll, d - CD.len), hi = min(d, AB.len);
    if (hi > lo) {
        // coarse: at m = j * nv, AB[m] is the first key of AB's tile j and
        // CD[d - 1 - m] the last key of CD's (full) tile d / nv - j - 1
        const long long jlo = (lo + nv - 1) / nv, jhi = (hi - 1) / nv, dj = d / nv;
        if (jlo <= jhi) {
            const long long jt = group_search(jlo, jhi + 1, lane, lg, [&](long long j) {
                return !(pair_last<KT>(src, split1, CD, nv, dj - j - 1) < pair_first<KT>(src, split1, AB, nv, j));
            });
            if (jt > jlo) lo = max(lo, (jt - 1) * nv + 1);
            if (jt <= jhi) hi = min(hi, jt * nv);
        }
    }
    // fine: AB outputs among the first d outputs of merge(AB, CD), and the
    // counts of A and C among them
    long long a, cc;
    const long long x = ab_cd_split<KT>(src, split1, AB, CD, nv, d, lo, hi, lane, lg, &a, &cc);
    if (leader) {
        split4[8 * b + 0] = e[0] + a;
        split4[8 * b + 1] = e[1] + (x - a);
        split4[8 * b + 2] = e[2] + cc;
        split4[8 * b + 3] = e[3] + (d - x - cc);
#pragma unroll
        for (int i = 0; i < 4; ++i) split4[8 * b + 4 + i] = e[i + 1];
    }
}

// One of four values by a run-time index, without indexing a local array
// (which would live in local memory).
template <typename V>
__device__ __forceinline__ V pick4(int i, V a, V b, V c, V d) {
    return i == 0 ? a : i == 1 ? b : i == 2 ? c : d;
}


// Staged key capacity of a 4-way merge tile: NV keys plus, per window, up to
// 3 keys before its first and after its last 4-key group boundary.
template <int NV> struct Merge4Cap { enum { SV = NV + 32 }; };

// Dynamic shared memory of k_merge4: the staged keys (and values), plus the
// slack the one-load merge step reads into.
template <typename U, int NT, int IPT, bool VALS>
constexpr size_t merge4_smem() {
    return (size_t)Merge4Cap<NT * IPT>::SV * (sizeof(U) + (VALS ? 4 : 0)) + (size_t)(IPT + 8) * sizeof(U);
}

// One output tile of a 4-way step: outputs [out0, out0 + cnt) of the stable
// merge of A = src[beg0, beg0 + len0), B, C and D likewise (len0 + .. + len3 =
// cnt), written to dst at out0.  The four windows are staged in shared memory
// (STAGE_VEC: 4-key groups by 16-byte loads through registers; STAGE_BULK:
// the same groups by 1-D bulk copies that one thread starts, completed on an
// mbarrier, then turned into order images in place; STAGE_SCALAR: one key at a
// time, for arrays that are not 16-byte aligned).  Level 1 merges A with B and
// C with D into [AB | CD] in registers, each thread IPT outputs (the thread
// whose outputs cross the end of AB finishes with the start of CD); level 2
// merges AB with CD.
template <int KT, int NT, int IPT, bool VALS, int STAGE>
__device__ __forceinline__ void merge_tile4(const typename Key<KT>::T *__restrict__ src_k,
                                            typename Key<KT>::T *__restrict__ dst_k,
                                            const uint32_t *__restrict__ src_v, uint32_t *__restrict__ dst_v,
                                            long long n, long long out0, int cnt, const long long (&beg)[4],
                                            const int (&len)[4], typename Key<KT>::U *s, uint32_t *sv,
                                            unsigned long long *bar, int *status, typename Key<KT>::U *samp,
                                            long long tile) {
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    constexpr int NV = NT * IPT;
    constexpr int SV = Merge4Cap<NV>::SV;
    const int t = threadIdx.x;
    int pos[4];                                    // staged position of each window's first key
    if (STAGE == STAGE_SCALAR) {
        int q = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) { pos[i] = q; q += len[i]; }
        for (int j = t; j < cnt; j += NT) {
            const int i = j < pos[1] ? 0 : j < pos[2] ? 1 : j < pos[3] ? 2 : 3;
            const long long g = pick4(i, beg[0], beg[1], beg[2], beg[3]) + (j - pick4(i, pos[0], pos[1], pos[2], pos[3]));
            s[j] = K::ord(src_k[g]);
            if (VALS) sv[j] = src_v[g];
        }
    } else {
        // window i as whole 4-key groups [g0[i], g0[i] + 4 ng[i]); group q of
        // the tile lands at s + 4 q
        long long g0[4];
        int first[5];                              // first group of each window
        first[0] = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            g0[i] = beg[i] & ~3ll;
            const int ng = len[i] > 0 ? (int)((((beg[i] + len[i] + 3) & ~3ll) - g0[i]) >> 2) : 0;
            first[i + 1] = first[i] + ng;
            pos[i] = 4 * first[i] + (int)(beg[i] - g0[i]);
        }
        const int groups = first[4];
        if (STAGE == STAGE_VEC) {
            constexpr int KMAX = (SV / 4 + NT - 1) / NT;
            U r[KMAX][4];
            uint4 rv[VALS ? KMAX : 1];
#pragma unroll
            for (int kk = 0; kk < KMAX; ++kk) {
                const int g = t + kk * NT;
                if (g < groups) {
                    const int i = g < first[1] ? 0 : g < first[2] ? 1 : g < first[3] ? 2 : 3;
                    const long long gb = pick4(i, g0[0], g0[1], g0[2], g0[3]) +
                                         4ll * (g - pick4(i, first[0], first[1], first[2], first[3]));
                    if (gb + 4 <= n) {
                        if (sizeof(T) == 4) {
                            const uint4 q = *reinterpret_cast<const uint4 *>(src_k + gb);
                            r[kk][0] = (U)q.x; r[kk][1] = (U)q.y; r[kk][2] = (U)q.z; r[kk][3] = (U)q.w;
                        } else {
                            const uint4 q0 = *reinterpret_cast<const uint4 *>(src_k + gb);
                            const uint4 q1 = *reinterpret_cast<const uint4 *>(src_k + gb + 2);
                            r[kk][0] = (U)(((unsigned long long)q0.y << 32) | q0.x);
                            r[kk][1] = (U)(((unsigned long long)q0.w << 32) | q0.z);
                            r[kk][2] = (U)(((unsigned long long)q1.y << 32) | q1.x);
                            r[kk][3] = (U)(((unsigned long long)q1.w << 32) | q1.z);
                        }
                        if (VALS) rv[kk] = *reinterpret_cast<const uint4 *>(src_v + gb);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) r[kk][e] = (gb + e < n) ? (U)src_k[gb + e] : U(0);
                        if (VALS) {
                            rv[kk].x = (gb + 0 < n) ? src_v[gb + 0] : 0u;
                            rv[kk].y = (gb + 1 < n) ? src_v[gb + 1] : 0u;
                            rv[kk].z = (gb + 2 < n) ? src_v[gb + 2] : 0u;
                            rv[kk].w = (gb + 3 < n) ? src_v[gb + 3] : 0u;
                        }
                    }
                }
            }
#pragma unroll
            for (int kk = 0; kk < KMAX; ++kk) {
                const int g = t + kk * NT;
                if (g < groups) {
                    if (sizeof(U) == 4) {
                        *reinterpret_cast<uint4 *>(s + 4 * g) =
                            make_uint4((uint32_t)K::ord((T)r[kk][0]), (uint32_t)K::ord((T)r[kk][1]),
                                       (uint32_t)K::ord((T)r[kk][2]), (uint32_t)K::ord((T)r[kk][3]));
                    } else {
                        *reinterpret_cast<ulonglong2 *>(s + 4 * g) = make_ulonglong2(
                            (unsigned long long)K::ord((T)r[kk][0]), (unsigned long long)K::ord((T)r[kk][1]));
                        *reinterpret_cast<ulonglong2 *>(s + 4 * g + 2) = make_ulonglong2(
                            (unsigned long long)K::ord((T)r[kk][2]), (unsigned long long)K::ord((T)r[kk][3]));
                    }
                    if (VALS) *reinterpret_cast<uint4 *>(sv + 4 * g) = rv[kk];
                }
            }
        } else {
            // bulk copies of every whole 16-byte stretch below n4; the few keys
            // of a window past the array's last 16-byte boundary by plain loads
            const long long n4 = n & ~3ll;
            if (t == 0) mbar_init(bar, 1);
            __syncthreads();
            if (t == 0) {
                unsigned bytes = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const long long ge = min(g0[i] + 4ll * (first[i + 1] - first[i]), n4);
                    if (ge > g0[i]) bytes += (unsigned)((ge - g0[i]) * (sizeof(T) + (VALS ? 4 : 0)));
                }
                mbar_arrive_expect(bar, bytes);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const long long ge = min(g0[i] + 4ll * (first[i + 1] - first[i]), n4);
                    if (ge > g0[i]) {
                        bulk_copy_g2s(s + 4 * first[i], src_k + g0[i], (unsigned)((ge - g0[i]) * sizeof(T)), bar);
                        if (VALS) bulk_copy_g2s(sv + 4 * first[i], src_v + g0[i], (unsigned)((ge - g0[i]) * 4), bar);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const long long e = beg[i] + len[i];
                if (len[i] > 0 && e > n4) {
                    const long long from = max(n4, g0[i]);
                    if (t < e - from) {
                        const long long g = from + t;
                        s[4 * first[i] + (g - g0[i])] = (U)src_k[g];
                        if (VALS) sv[4 * first[i] + (g - g0[i])] = src_v[g];
                    }
                }
            }
            const bool done = mbar_wait_bounded(bar, 0, BULK_WAIT_TRIES);
            if (!__syncthreads_and(done)) {
                if (t == 0 && status) atomicExch(status, (int)SR_ERR_TIMEOUT);
                mbar_wait_bounded(bar, 0, BULK_WAIT_TRIES);   // copies still in flight must land first
                return;
            }
            if (KT != SR_KEY_U32 && KT != SR_KEY_U64) {          // raw keys -> order images, in place
                for (int g = t; g < groups; g += NT) {
                    if (sizeof(U) == 4) {
                        uint4 q = *reinterpret_cast<uint4 *>(s + 4 * g);
                        q.x = (uint32_t)K::ord((T)q.x); q.y = (uint32_t)K::ord((T)q.y);
                        q.z = (uint32_t)K::ord((T)q.z); q.w = (uint32_t)K::ord((T)q.w);
                        *reinterpret_cast<uint4 *>(s + 4 * g) = q;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) s[4 * g + e] = K::ord((T)s[4 * g + e]);
                    }
                }
            }
        }
    }
    __syncthreads();
    // level 1: [AB | CD], IPT outputs per thread
    const int lab = len[0] + len[1];
    U k[IPT];
    int ix[IPT];
    {
        const int o = min(t * IPT, cnt);
        if (o + IPT <= lab) {
            const int sp = merge_path(s + pos[0], len[0], s + pos[1], len[1], o);
            serial_merge_slack<U, IPT>(s, pos[0] + sp, pos[0] + len[0], pos[1] + o - sp, pos[1] + len[1], k, ix);
        } else if (o >= lab) {
            const int oc = o - lab;
            const int sp = merge_path(s + pos[2], len[2], s + pos[3], len[3], oc);
            serial_merge_slack<U, IPT>(s, pos[2] + sp, pos[2] + len[2], pos[3] + oc - sp, pos[3] + len[3], k, ix);
        } else {
            const int sp = merge_path(s + pos[0], len[0], s + pos[1], len[1], o);
            serial_merge_switch<U, IPT>(s, pos[0] + sp, pos[0] + len[0], pos[1] + o - sp, pos[1] + len[1], lab - o,
                                        pos[2], pos[2] + len[2], pos[3], pos[3] + len[3], k, ix);
        }
    }
    uint32_t v[IPT];
    if (VALS) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) v[i] = sv[ix[i]];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        s[t * IPT + i] = k[i];
        if (VALS) sv[t * IPT + i] = v[i];
    }
    __syncthreads();
    // level 2: AB = s[0, lab) with CD = s[lab, cnt)
    const int diag = min(t * IPT, cnt);
    const int sp = merge_path(s, lab, s + lab, cnt - lab, diag);
    serial_merge_slack<U, IPT>(s, sp, lab, lab + diag - sp, cnt, k, ix);
    if (VALS) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) v[i] = sv[ix[i]];
    }
    write_tile<KT, NT, IPT, VALS, STAGE != STAGE_SCALAR>(k, v, s, sv, dst_k, dst_v, out0, cnt, samp, tile);
}

// One CTA per output tile of NT*IPT keys of a 4-way step: the tile's windows
// of A, B, C and D come from split4 (the runs' ends for a group's last tile).
template <int KT, int NT, int IPT, bool VALS, int STAGE>
__global__ void __launch_bounds__(NT, Shape<sizeof(typename Key<KT>::T), VALS>::MERGE4_MINB)
k_merge4(typename Key<KT>::T *uk, uint32_t *uv, typename Key<KT>::T *sk, uint32_t *svb, long long n,
         const long long *__restrict__ split4, const Ctrl *__restrict__ c, int step,
         typename Key<KT>::U *__restrict__ samp, long long smt, int *status) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int NV = NT * IPT;
    if (step >= steps_of(c)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long bar;
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + Merge4Cap<NV>::SV);
    const int cur = c->src_buf[step];
    const long long b = blockIdx.x;
    const long long out0 = b * NV;
    const long long out1 = min(out0 + NV, n);
    const bool last = out1 == split4[8 * b + 7];   // the group's last tile ends at its runs' ends
    long long beg[4];
    int len[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        beg[i] = split4[8 * b + i];
        const long long end = last ? split4[8 * b + 4 + i] : split4[8 * (b + 1) + i];
        len[i] = (int)(end - beg[i]);
    }
    merge_tile4<KT, NT, IPT, VALS, STAGE>(cur ? sk : uk, cur ? uk : sk, cur ? svb : uv, cur ? uv : svb, n, out0,
                                          (int)(out1 - out0), beg, len, s, sv, &bar, status,
                                          samp ? samp + (1 - cur) * smt : nullptr, b);
}

template <int KT, bool VALS>
__global__ void k_copy_back(typename Key<KT>::T *uk, uint32_t *uv, const typename Key<KT>::T *sk,
                            const uint32_t *svb, long long n, const Ctrl *__restrict__ c) {
    griddep_wait();
    if (call_mode(c, n) != MODE_SORT) return;
    if (c->src_buf[steps_of(c)] == 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uk[i] = sk[i];
        if (VALS) uv[i] = svb[i];
    }
}

}  // namespace sr
