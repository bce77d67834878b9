// sr_kernels.cuh -- the kernels of the plain sort (run detection, reversal,
// block sort, merge-path partition, merge pass, copy-back).  The launch
// sequence that drives them is described in sr_sort.cu.
#pragma once

#include "sr_device.cuh"

#ifndef SR_SPLIT_SAMPLES
#define SR_SPLIT_SAMPLES 1  // merge splits searched over recorded tile samples first
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
template <int KT, int NT, int IPT>
__global__ void __launch_bounds__(NT) k_detect(const typename Key<KT>::T *__restrict__ keys,
                                               long long n, Ctrl *__restrict__ c,
                                               const int *__restrict__ gate,
                                               typename Key<KT>::U *__restrict__ med, int mt) {
    griddep_wait();
    if (gate && *gate == 0) return;
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    constexpr int TS = NT * IPT;
    constexpr int VW = 16 / sizeof(T);             // keys per 16-byte vector
    __shared__ unsigned int red[4];
    const int t = threadIdx.x;
    const long long base = (long long)blockIdx.x * TS;
    const int cnt = (int)(n - base < (long long)TS ? n - base : (long long)TS);   // keys of the tile
    const bool more = base + cnt < n;              // a key follows the tile
    const bool vec = (((uintptr_t)(keys + base)) & 15) == 0;
    if (t < 4) red[t] = 0;
    __syncthreads();
    unsigned int d = 0, nd = 0, din = 0, ndin = 0;
    const int ng = (cnt + VW - 1) / VW;
    for (int g = t; g < ng; g += NT) {
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
    if ((t & 31) == 0) {
        if (d) atomicAdd(&red[0], d);
        if (nd) atomicAdd(&red[1], nd);
        if (din) atomicOr(&red[2], din);
        if (ndin) atomicOr(&red[3], ndin);
    }
    __syncthreads();
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

// Few distinct keys, step 1: FEW_SAMPLE keys spread over the whole array go
// into the call's set of distinct order images (until more than FEW_MAX
// appear); the last CTA to finish (a ticket after a fence) then, if the call
// would sort and the set is small, sorts the set into few_sorted as the
// candidate.  The counting pass checks every key against the set, so a
// sample that misses a key only costs that pass.  This is the k-way form of
// the fat (3-way) partition of the paper's quicksorts: keys equal to a pivot
// need no further comparisons.
enum { FEW_SAMPLE = 4096, FEW_NT = 256 };
static_assert(FEW_NT >= FEW_SLOTS, "one thread per set slot");
template <int KT>
__global__ void __launch_bounds__(FEW_NT) k_few_sample(const typename Key<KT>::T *__restrict__ keys, long long n,
                                                       Ctrl *__restrict__ c, const int *__restrict__ gate) {
    griddep_wait();
    __shared__ unsigned int s_v[FEW_MAX];
    __shared__ unsigned int s_k;
    __shared__ int s_last;
    __shared__ unsigned long long s_set[FEW_SLOTS];
    __shared__ unsigned int s_n;
    __shared__ int s_over;
    if (gate && *gate == 0) return;
    const int t = threadIdx.x;
    if (t < FEW_SLOTS) s_set[t] = 0ull;
    if (t == 0) { s_n = 0u; s_over = 0; }
    __syncthreads();
    // this CTA's samples go into a shared-memory set first; only a CTA that saw
    // at most FEW_MAX distinct keys touches the call's set in global memory
    const long long i = (long long)blockIdx.x * FEW_NT + t;
    if (i < FEW_SAMPLE && n > 0)
        few_insert(s_set, &s_n, &s_over, (unsigned int)Key<KT>::ord(__ldg(keys + (i * n) / FEW_SAMPLE)));
    __syncthreads();
    if (s_over) {
        if (t == 0) atomicExch(&c->few_over, 1);
    } else if (t < FEW_SLOTS && s_set[t] != 0ull && !((volatile int *)&c->few_over)[0]) {
        few_insert(c->few_slot, &c->few_n, &c->few_over, (unsigned int)(s_set[t] - 1ull));
    }
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(&c->few_ticket, 1u) == gridDim.x - 1;
        s_k = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (call_mode(c, n) != MODE_SORT) return;
    const int over = ((volatile int *)&c->few_over)[0];
    const unsigned int nd = ((volatile unsigned int *)&c->few_n)[0];
    if (over || nd == 0u || nd > (unsigned int)FEW_MAX) return;
    if (t < FEW_SLOTS) {
        const unsigned long long v = ((volatile unsigned long long *)c->few_slot)[t];
        if (v != 0ull) {
            const unsigned int q = atomicAdd(&s_k, 1u);
            if (q < (unsigned int)FEW_MAX) s_v[q] = (unsigned int)(v - 1ull);
        }
    }
    __syncthreads();
    const unsigned int k = s_k;
    if (k != nd) return;                           // cannot happen; the ordinary sort then runs
    if (t < (int)k) {
        unsigned int r = 0;
        for (unsigned int q = 0; q < k; ++q) r += s_v[q] < s_v[t];
        c->few_sorted[r] = s_v[t];
    }
    __syncthreads();
    if (t == 0) c->few_cand = 1;
}

// Few distinct keys, step 2: counts the keys equal to each candidate image (a
// binary search over at most FEW_MAX images per key, one shared-memory
// histogram per warp); a key outside the set raises few_miss and the ordinary
// sort runs instead.
template <int KT>
__global__ void __launch_bounds__(256) k_few_count(const typename Key<KT>::T *__restrict__ keys, long long n,
                                                   Ctrl *__restrict__ c) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::T T;
    constexpr int NW = 256 / 32;
    __shared__ unsigned int s_v[FEW_MAX];
    __shared__ unsigned int s_h[NW][FEW_MAX];    // one histogram per warp
    if (!c->few_cand) return;
    const int t = threadIdx.x;
    const int k = (int)c->few_n;
    if (t < FEW_MAX) s_v[t] = t < k ? c->few_sorted[t] : 0xffffffffu;
    for (int q = t; q < NW * FEW_MAX; q += 256) (&s_h[0][0])[q] = 0u;
    __syncthreads();
    unsigned int *h = s_h[t >> 5];
    bool miss = false;
    auto count = [&](T key) {
        const unsigned int u = (unsigned int)K::ord(key);
        int lo = 0, hi = k - 1;                    // the last image <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_v[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        if (s_v[lo] != u) miss = true;             // not in the sample's set
        else atomicAdd(&h[lo], 1u);
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
    if (t < k) {
        unsigned int sum = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) sum += s_h[w][t];
        if (sum) atomicAdd(&c->few_count[t], (unsigned long long)sum);
    }
}

// Few distinct keys, step 3: when every key was in the set, writes the sorted
// output, each distinct key repeated its count times (16-byte stores when the
// array is aligned), and switches the call to MODE_FEW: every later kernel of
// the ordinary sequence then returns at once.
template <int KT>
__global__ void __launch_bounds__(256) k_few_write(typename Key<KT>::T *__restrict__ keys, long long n,
                                                   Ctrl *__restrict__ c) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::T T;
    __shared__ unsigned long long s_start[FEW_MAX + 1];
    __shared__ T s_key[FEW_MAX];
    if (!c->few_cand || c->few_miss) return;
    const int t = threadIdx.x;
    if (blockIdx.x == 0 && t == 0) c->few_active = 1;
    const int k = (int)c->few_n;
    if (t == 0) {
        unsigned long long a = 0;
        for (int q = 0; q < k; ++q) { s_start[q] = a; a += c->few_count[q]; }
        for (int q = k; q <= FEW_MAX; ++q) s_start[q] = a;
    }
    if (t < k) s_key[t] = K::unord((typename K::U)c->few_sorted[t]);
    __syncthreads();
    // the last q with s_start[q] <= i
    auto which = [&](long long i) {
        int lo = 0, hi = k - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((long long)s_start[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + t;
    if ((((uintptr_t)keys) & 15) == 0) {
        const long long nv = n / 4;
        uint4 *q4 = reinterpret_cast<uint4 *>(keys);
        for (long long v = gtid; v < nv; v += stride) {
            const long long i = 4 * v;
            int j = which(i);
            uint32_t e[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                while (j + 1 < k && (long long)s_start[j + 1] <= i + m) ++j;
                e[m] = (uint32_t)s_key[j];
            }
            q4[v] = make_uint4(e[0], e[1], e[2], e[3]);
        }
        for (long long i = 4 * nv + gtid; i < n; i += stride) keys[i] = s_key[which(i)];
    } else {
        for (long long i = gtid; i < n; i += stride) keys[i] = s_key[which(i)];
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
__global__ void __launch_bounds__(NT)
k_block_sort(const typename Key<KT>::T *in_k, const uint32_t *in_v, typename Key<KT>::T *out_k,
             uint32_t *out_v, long long n, const Ctrl *__restrict__ c,
             typename Key<KT>::U *__restrict__ tile_lo, typename Key<KT>::U *__restrict__ tile_hi,
             typename Key<KT>::U *__restrict__ samp, int mv) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int NV = NT * IPT;
    if (c && call_mode(c, n) != MODE_SORT) return;
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + NV);
    const int t = threadIdx.x;
    const long long base = (long long)blockIdx.x * NV;
    const int cnt = (int)(n - base < (long long)NV ? n - base : (long long)NV);
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int idx = i * NT + t;
        s[idx] = idx < cnt ? K::ord(in_k[base + idx]) : umax_of<U>();
        if (VALS) sv[idx] = idx < cnt ? in_v[base + idx] : 0u;
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
    auto samples = [&](bool rev) {
        if (!samp) return;
        const int per = NV / mv;
        for (int q = t; q < per && q * mv < cnt; q += NT) {
            const int f = q * mv, l = min(f + mv, cnt) - 1;
            samp[2 * ((long long)blockIdx.x * per + q)] = rev ? s[cnt - 1 - f] : s[f];
            samp[2 * ((long long)blockIdx.x * per + q) + 1] = rev ? s[cnt - 1 - l] : s[l];
        }
    };
    if (!any_desc) {                       // already ascending
        if (t == 0 && tile_lo) { tile_lo[blockIdx.x] = s[0]; tile_hi[blockIdx.x] = s[cnt - 1]; }
        samples(false);
        if (out_k != in_k) {
            for (int idx = t; idx < cnt; idx += NT) {
                out_k[base + idx] = K::unord(s[idx]);
                if (VALS) out_v[base + idx] = sv[idx];
            }
        }
        return;
    }
    if (!any_nondesc) {                    // strictly descending: reverse
        if (t == 0 && tile_lo) { tile_lo[blockIdx.x] = s[cnt - 1]; tile_hi[blockIdx.x] = s[0]; }
        samples(true);
        for (int idx = t; idx < cnt; idx += NT) {
            out_k[base + idx] = K::unord(s[cnt - 1 - idx]);
            if (VALS) out_v[base + idx] = sv[cnt - 1 - idx];
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
    block_sort<U, NT, IPT, VALS>(k, v, s, sv);
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        s[t * IPT + i] = k[i];
        if (VALS) sv[t * IPT + i] = v[i];
    }
    __syncthreads();
    if (t == 0 && tile_lo) { tile_lo[blockIdx.x] = s[0]; tile_hi[blockIdx.x] = s[cnt - 1]; }
    samples(false);
    for (int idx = t; idx < cnt; idx += NT) {
        out_k[base + idx] = K::unord(s[idx]);
        if (VALS) out_v[base + idx] = sv[idx];
    }
}

// Pass planner (after the block sort): a merged run's smallest and largest
// keys are the smallest and largest of its tiles', so whether the two runs of a
// pair at pass p are already in order (A.last <= B.first) is known for every
// pass from the tile extremes alone.  Adds to c->unordered[p] the number of
// pairs of pass p that must be merged; a pass with none is skipped (technique
// (f) applied to whole passes).
//
// Each CTA reduces a chunk of PLAN_CHUNK tiles in shared memory, which settles
// every pass whose pairs lie inside one chunk; the last CTA to finish (a ticket
// taken after a fence) settles the remaining passes from the chunks' extremes.
enum { PLAN_CHUNK = 2048, PLAN_LEVELS = 11 };   // 2^11 tiles per chunk

// Once every unordered[p] is final: the buffer before each pass (and after
// the last), so later kernels read one byte instead of recounting flips.
__device__ __forceinline__ void record_buffers(Ctrl *c, int cur0, int passes) {
    int cur = cur0;
    for (int p = 0; p < passes; ++p) {
        c->src_buf[p] = (signed char)cur;
        cur ^= (((volatile int *)c->unordered)[p] != 0);
    }
    c->src_buf[passes] = (signed char)cur;
}

template <int KT>
__global__ void __launch_bounds__(1024)
k_plan(const typename Key<KT>::U *__restrict__ lo, const typename Key<KT>::U *__restrict__ hi,
       typename Key<KT>::U *__restrict__ chunk_lo, typename Key<KT>::U *__restrict__ chunk_hi,
       long long n, long long tiles, int passes, int cur0, Ctrl *__restrict__ c) {
    griddep_wait();
    typedef typename Key<KT>::U U;
    if (call_mode(c, n) != MODE_SORT) return;
    __shared__ U s_lo[PLAN_CHUNK], s_hi[PLAN_CHUNK];
    __shared__ unsigned int s_cnt;
    __shared__ int s_last;
    const int t = threadIdx.x;
    const long long base = (long long)blockIdx.x * PLAN_CHUNK;
    const int cnt = (int)min((long long)PLAN_CHUNK, tiles - base);
    for (int i = t; i < cnt; i += blockDim.x) { s_lo[i] = lo[base + i]; s_hi[i] = hi[base + i]; }
    // run r of pass p is kept at index r << p: the pair of runs starting at
    // ia = 2j << p and ib = ia + (1 << p) folds into ia
    const int inner = passes < PLAN_LEVELS ? passes : PLAN_LEVELS;
    for (int p = 0; p < inner; ++p) {
        if (t == 0) s_cnt = 0;
        __syncthreads();
        const int stride = 1 << p;
        unsigned int mine = 0;
        for (int ia = 2 * stride * t; ia < cnt; ia += 2 * stride * blockDim.x) {
            const int ib = ia + stride;
            if (ib < cnt) {
                mine += s_hi[ia] > s_lo[ib];
                s_lo[ia] = s_lo[ia] < s_lo[ib] ? s_lo[ia] : s_lo[ib];
                s_hi[ia] = s_hi[ia] > s_hi[ib] ? s_hi[ia] : s_hi[ib];
            }
        }
        mine = __reduce_add_sync(0xffffffffu, mine);
        if ((t & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
        __syncthreads();
        if (t == 0 && s_cnt) atomicAdd(&c->unordered[p], (int)s_cnt);
    }
    // the chunk is fully reduced into index 0
    if (t == 0) {
        chunk_lo[blockIdx.x] = s_lo[0];
        chunk_hi[blockIdx.x] = s_hi[0];
        __threadfence();
        s_last = atomicAdd(&c->plan_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (passes <= PLAN_LEVELS) {
        if (t == 0) record_buffers(c, cur0, passes);
        return;
    }
    const int chunks = (int)gridDim.x;            // at most PLAN_CHUNK chunks (2^22 tiles)
    for (int i = t; i < chunks; i += blockDim.x) {
        s_lo[i] = ((volatile U *)chunk_lo)[i];
        s_hi[i] = ((volatile U *)chunk_hi)[i];
    }
    for (int p = PLAN_LEVELS; p < passes; ++p) {
        if (t == 0) s_cnt = 0;
        __syncthreads();
        const int stride = 1 << (p - PLAN_LEVELS);
        unsigned int mine = 0;
        for (int ia = 2 * stride * t; ia < chunks; ia += 2 * stride * blockDim.x) {
            const int ib = ia + stride;
            if (ib < chunks) {
                mine += s_hi[ia] > s_lo[ib];
                s_lo[ia] = s_lo[ia] < s_lo[ib] ? s_lo[ia] : s_lo[ib];
                s_hi[ia] = s_hi[ia] > s_hi[ib] ? s_hi[ia] : s_hi[ib];
            }
        }
        mine = __reduce_add_sync(0xffffffffu, mine);
        if ((t & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
        __syncthreads();
        if (t == 0) c->unordered[p] = (int)s_cnt;
    }
    if (t == 0) record_buffers(c, cur0, passes);
}

// Merge-path split of every merge tile boundary of pass p, one group of
// 2^lg lanes per boundary (the host picks lg: wide groups take fewer
// dependent rounds, narrow ones fewer scattered loads when there are many
// boundaries).
// The merge-path split of output tile b (outputs from b*nv) of a merge pass
// over runs of w keys of src: the index in src where the tile's share of run
// A starts.  A group of 2^lg lanes computes it together (all lanes of the
// group get it).  samp (optional): the first and last key of every merge
// tile of src, as recorded when src was written; with it the search first
// narrows the split to one tile's stretch and then reads keys only there.
template <int KT>
__device__ __forceinline__ long long merge_split(const typename Key<KT>::T *__restrict__ src, long long n,
                                                 long long w, int nv, long long b, int lane, int lg,
                                                 const typename Key<KT>::U *__restrict__ samp) {
    typedef Key<KT> K;
    typedef typename K::U U;
    const long long out = min(b * (long long)nv, n);
    const long long pb = (out / (2 * w)) * (2 * w);
    const long long a_beg = pb, a_end = min(pb + w, n);
    const long long b_beg = a_end, b_end = min(pb + 2 * w, n);
    const long long na = a_end - a_beg, nb = b_end - b_beg, d = out - pb;
    long long lo = max(0ll, d - nb), hi = min(d, na);
    if (samp && out < n && hi > lo) {
        // Coarse: the merge-path test at the multiples m = j*nv uses only the
        // first key of A's tile j and the last key of B's tile d/nv - j - 1;
        // d, a_beg and b_beg are multiples of nv here.
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

// Splits of every output tile boundary of pass p, a group of 2^lg lanes per
// boundary.  The tile samples of the buffer a pass reads are at samp +
// smt * (that buffer: 0 the caller's, 1 the scratch copy).
template <int KT>
__global__ void __launch_bounds__(256)
k_partition(const typename Key<KT>::T *__restrict__ uk, const typename Key<KT>::T *__restrict__ sk,
            long long n, long long w, int nv, long long nbound, long long *__restrict__ splits,
            const Ctrl *__restrict__ c, int p, int lg, const typename Key<KT>::U *__restrict__ samp,
            long long smt) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> lg;
    if (b >= nbound) return;                       // uniform across the group
    if (c->unordered[p] == 0) return;             // also 0 for every pass unless the input needs sorting
    const int cur = c->src_buf[p];
    const long long sp = merge_split<KT>(cur ? sk : uk, n, w, nv, b, lane, lg, samp ? samp + cur * smt : nullptr);
    if ((lane & ((1 << lg) - 1)) == 0) splits[b] = sp;
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

// Dynamic shared memory that merge_tile needs: NT*IPT + 16 staged keys (and
// as many values), plus the key slack the one-load merge step reads into.
template <typename U, int NT, int IPT, bool VALS>
constexpr size_t merge_tile_smem() {
    return (size_t)(NT * IPT + 16) * (sizeof(U) + (VALS ? 4 : 0)) + (SR_MERGE_1LD ? (size_t)(IPT + 8) * sizeof(U) : 0);
}

// Merges one output tile: outputs [out0, out0 + cnt) of the stable merge of
// the sorted ranges A = src[a0 .. a1) and B = src[b0 .. b0 + cnt - (a1 - a0)),
// written to dst at out0.  All threads of the CTA call it; s / sv are shared
// buffers of NT*IPT + 16 keys / values, and with SR_MERGE_1LD the key buffer
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
template <int KT, int NT, int IPT, bool VALS, bool VEC>
__device__ __forceinline__ void merge_tile(const typename Key<KT>::T *__restrict__ src_k,
                                           typename Key<KT>::T *__restrict__ dst_k,
                                           const uint32_t *__restrict__ src_v, uint32_t *__restrict__ dst_v,
                                           long long n, long long out0, int cnt, long long a0, long long a1,
                                           long long b0, typename Key<KT>::U *s, uint32_t *sv,
                                           typename Key<KT>::U *samp = nullptr, long long tile = 0) {
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    constexpr int NV = NT * IPT;
    constexpr int SV = NV + 16;
    const int t = threadIdx.x;
    const int acnt = (int)(a1 - a0);
    const int bcnt = cnt - acnt;
    int sa, sb;                                    // staged positions of A[a0] and B[b0]
    if (VEC) {
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
    const int sp = merge_path(s + sa, acnt, s + sb, bcnt, diag);
    U k[IPT];
    int ix[IPT];
    if (SR_MERGE_1LD)
        serial_merge_slack<U, IPT>(s, sa + sp, sa + acnt, sb + diag - sp, sb + bcnt, k, ix);
    else
        serial_merge<U, IPT>(s, sa + sp, sa + acnt, sb + diag - sp, sb + bcnt, k, ix);
    uint32_t v[IPT];
    if (VALS) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) v[i] = (diag + i < cnt) ? sv[ix[i]] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        s[t * IPT + i] = k[i];
        if (VALS) sv[t * IPT + i] = v[i];
    }
    __syncthreads();
    if (samp && t == 0) {                          // the output tile's first and last key, for the next pass
        samp[2 * tile] = s[0];
        samp[2 * tile + 1] = s[cnt - 1];
    }
    if (VEC) {
        // keys before the first 4-key group boundary of the output go one by one
        const int head = min(cnt, (int)((4 - (out0 & 3)) & 3));
        if (t < head) {
            dst_k[out0 + t] = K::unord(s[t]);
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
                        make_uint4((uint32_t)K::unord((U)q.x), (uint32_t)K::unord((U)q.y),
                                   (uint32_t)K::unord((U)q.z), (uint32_t)K::unord((U)q.w));
                } else {
                    const ulonglong2 q0 = *reinterpret_cast<const ulonglong2 *>(s + j);
                    const ulonglong2 q1 = *reinterpret_cast<const ulonglong2 *>(s + j + 2);
                    const unsigned long long e0 = (unsigned long long)K::unord((U)q0.x);
                    const unsigned long long e1 = (unsigned long long)K::unord((U)q0.y);
                    const unsigned long long e2 = (unsigned long long)K::unord((U)q1.x);
                    const unsigned long long e3 = (unsigned long long)K::unord((U)q1.y);
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
                q.x = (uint32_t)K::unord(s[j + 0]);
                q.y = (uint32_t)K::unord(s[j + 1]);
                q.z = (uint32_t)K::unord(s[j + 2]);
                q.w = (uint32_t)K::unord(s[j + 3]);
                *reinterpret_cast<uint4 *>(dst_k + out0 + j) = q;
            } else {
                const unsigned long long e0 = (unsigned long long)K::unord(s[j + 0]);
                const unsigned long long e1 = (unsigned long long)K::unord(s[j + 1]);
                const unsigned long long e2 = (unsigned long long)K::unord(s[j + 2]);
                const unsigned long long e3 = (unsigned long long)K::unord(s[j + 3]);
                *reinterpret_cast<uint4 *>(dst_k + out0 + j) =
                    make_uint4((uint32_t)e0, (uint32_t)(e0 >> 32), (uint32_t)e1, (uint32_t)(e1 >> 32));
                *reinterpret_cast<uint4 *>(dst_k + out0 + j + 2) =
                    make_uint4((uint32_t)e2, (uint32_t)(e2 >> 32), (uint32_t)e3, (uint32_t)(e3 >> 32));
            }
            if (VALS)
                *reinterpret_cast<uint4 *>(dst_v + out0 + j) = make_uint4(sv[j], sv[j + 1], sv[j + 2], sv[j + 3]);
        }
        for (int i = head + 4 * full + t; i < cnt; i += NT) {
            dst_k[out0 + i] = K::unord(s[i]);
            if (VALS) dst_v[out0 + i] = sv[i];
        }
    } else {
        for (int i = t; i < cnt; i += NT) {
            dst_k[out0 + i] = K::unord(s[i]);
            if (VALS) dst_v[out0 + i] = sv[i];
        }
    }
}

// One CTA per output tile of NT*IPT keys of merge pass p.  The tile's A and B
// ranges come from the split table and are merged by merge_tile.  A run pair
// (2w keys) spans 2^lgt whole tiles.
template <int KT, int NT, int IPT, bool VALS, bool VEC>
__global__ void __launch_bounds__(NT, Shape<sizeof(typename Key<KT>::T), VALS>::MERGE_MINB)
k_merge(typename Key<KT>::T *uk, uint32_t *uv, typename Key<KT>::T *sk, uint32_t *svb, long long n,
        long long w, int lgt, const long long *__restrict__ splits, const Ctrl *__restrict__ c, int p,
        typename Key<KT>::U *__restrict__ samp, long long smt) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    constexpr int NV = NT * IPT;
    constexpr int SV = NV + 16;                    // staged keys, with room for window slack
    if (c->unordered[p] == 0) return;              // also 0 for every pass unless the input needs sorting
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + SV);
    const int cur = c->src_buf[p];
    const long long out0 = (long long)blockIdx.x * NV;
    const long long out1 = min(out0 + NV, n);
    const long long pb = (long long)(((unsigned long long)blockIdx.x >> lgt) << lgt) * NV;
    const long long a_beg = pb, a_end = min(pb + w, n);
    const long long b_beg = a_end, b_end = min(pb + 2 * w, n);
    const long long a0 = splits[blockIdx.x];
    const long long a1 = (out1 == b_end) ? a_end : splits[blockIdx.x + 1];
    const long long b0 = b_beg + (out0 - pb) - (a0 - a_beg);
    // the output's tile samples go with the buffer it lands in
    merge_tile<KT, NT, IPT, VALS, VEC>(cur ? sk : uk, cur ? uk : sk, cur ? svb : uv, cur ? uv : svb, n, out0,
                                       (int)(out1 - out0), a0, a1, b0, s, sv, samp ? samp + (1 - cur) * smt : nullptr,
                                       (long long)blockIdx.x);
}

template <int KT, bool VALS>
__global__ void k_copy_back(typename Key<KT>::T *uk, uint32_t *uv, const typename Key<KT>::T *sk,
                            const uint32_t *svb, long long n, const Ctrl *__restrict__ c, int passes) {
    griddep_wait();
    if (call_mode(c, n) != MODE_SORT) return;
    if (c->src_buf[passes] == 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uk[i] = sk[i];
        if (VALS) uv[i] = svb[i];
    }
}

}  // namespace sr
