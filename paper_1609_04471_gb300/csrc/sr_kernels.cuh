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

// Whether merge step s (binary levels [l0, l0 + nl)) has any run pair out of
// order; a step whose levels are all in order is skipped.
__device__ __forceinline__ bool step_needed(const Ctrl *c, int l0, int nl) {
    const volatile int *u = c->unordered;
    return u[l0] != 0 || (nl > 1 && u[l0 + 1] != 0);
}

// Once every unordered[level] is final: the buffer before each merge step (and
// after the last), so later kernels read one byte instead of recounting flips.
__device__ __forceinline__ void record_buffers(Ctrl *c, int cur0, int levels, bool fan4) {
    int cur = cur0;
    const int steps = merge_step_count(levels, fan4);
    for (int s = 0; s < steps; ++s) {
        int l0, nl;
        merge_step_levels(levels, fan4, s, &l0, &nl);
        c->src_buf[s] = (signed char)cur;
        cur ^= step_needed(c, l0, nl) ? 1 : 0;
    }
    c->src_buf[steps] = (signed char)cur;
}

template <int KT>
__global__ void __launch_bounds__(1024)
k_plan(const typename Key<KT>::U *__restrict__ lo, const typename Key<KT>::U *__restrict__ hi,
       typename Key<KT>::U *__restrict__ chunk_lo, typename Key<KT>::U *__restrict__ chunk_hi,
       long long n, long long tiles, int passes, int cur0, int fan4, Ctrl *__restrict__ c) {
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
        if (t == 0) record_buffers(c, cur0, passes, fan4 != 0);
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
    if (t == 0) record_buffers(c, cur0, passes, fan4 != 0);
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
            const Ctrl *__restrict__ c, int step, int l0, int nl, int lg,
            const typename Key<KT>::U *__restrict__ samp, long long smt) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> lg;
    if (b >= nbound) return;                       // uniform across the group
    if (!step_needed(c, l0, nl)) return;          // also skipped unless the input needs sorting
    const int cur = c->src_buf[step];
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
                                           long long out0, int cnt, typename Key<KT>::U *samp, long long tile) {
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    const int t = threadIdx.x;
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
    write_tile<KT, NT, IPT, VALS, VEC>(k, v, s, sv, dst_k, dst_v, out0, cnt, samp, tile);
}

// One CTA per output tile of NT*IPT keys of merge pass p.  The tile's A and B
// ranges come from the split table and are merged by merge_tile.  A run pair
// (2w keys) spans 2^lgt whole tiles.
template <int KT, int NT, int IPT, bool VALS, bool VEC>
__global__ void __launch_bounds__(NT, Shape<sizeof(typename Key<KT>::T), VALS>::MERGE_MINB)
k_merge(typename Key<KT>::T *uk, uint32_t *uv, typename Key<KT>::T *sk, uint32_t *svb, long long n,
        long long w, int lgt, const long long *__restrict__ splits, const Ctrl *__restrict__ c, int step,
        int l0, typename Key<KT>::U *__restrict__ samp, long long smt) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    constexpr int NV = NT * IPT;
    constexpr int SV = NV + 16;                    // staged keys, with room for window slack
    if (!step_needed(c, l0, 1)) return;            // also skipped unless the input needs sorting
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + SV);
    const int cur = c->src_buf[step];
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
// split1[t0 + j] is where P's tile j (outputs j*nv ..) starts in X.
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
    xs = split1[P.t0 + j];
    const long long o1 = min((j + 1) * (long long)nv, P.len);
    xe = o1 == P.len ? P.x_end : split1[P.t0 + j + 1];
    ys = P.x_end + j * (long long)nv - (xs - P.x_beg);
    ye = P.x_end + o1 - (xe - P.x_beg);
}

// The merge-path test of a 4-way boundary at m: whether AB[m] goes before
// CD[d - 1 - m] (!(CD[d-1-m] < AB[m])).  The two keys' inner searches run in
// one loop so their loads are in flight together.
template <int KT>
__device__ __forceinline__ bool probe_ab_cd(const typename Key<KT>::T *__restrict__ src,
                                            const long long *__restrict__ split1, const PairView &AB,
                                            const PairView &CD, int nv, long long d, long long m) {
    typedef Key<KT> K;
    typedef typename K::U U;
    const long long m2 = d - 1 - m;
    const long long j1 = m / nv, j2 = m2 / nv;
    long long xs1, xe1, ys1, ye1, xs2, xe2, ys2, ye2;
    pair_tile(split1, AB, nv, j1, xs1, xe1, ys1, ye1);
    pair_tile(split1, CD, nv, j2, xs2, xe2, ys2, ye2);
    const int r1 = (int)(m - j1 * nv), r2 = (int)(m2 - j2 * nv);
    const int ny1 = (int)(ye1 - ys1), ny2 = (int)(ye2 - ys2);
    int lo1 = max(0, r1 + 1 - ny1), hi1 = min(r1 + 1, (int)(xe1 - xs1));
    int lo2 = max(0, r2 + 1 - ny2), hi2 = min(r2 + 1, (int)(xe2 - xs2));
    while (lo1 < hi1 || lo2 < hi2) {
        if (lo1 < hi1) {
            const int mid = (lo1 + hi1) >> 1;
            if (!(K::ord(src[ys1 + r1 - mid]) < K::ord(src[xs1 + mid]))) lo1 = mid + 1;
            else hi1 = mid;
        }
        if (lo2 < hi2) {
            const int mid = (lo2 + hi2) >> 1;
            if (!(K::ord(src[ys2 + r2 - mid]) < K::ord(src[xs2 + mid]))) lo2 = mid + 1;
            else hi2 = mid;
        }
    }
    U a = 0, c = 0;                                // AB[m] and CD[m2]: the later of the two last keys taken
    if (lo1 > 0) a = K::ord(src[xs1 + lo1 - 1]);
    if (r1 - lo1 >= 0) {
        const U y = K::ord(src[ys1 + r1 - lo1]);
        a = a < y ? y : a;
    }
    if (lo2 > 0) c = K::ord(src[xs2 + lo2 - 1]);
    if (r2 - lo2 >= 0) {
        const U y = K::ord(src[ys2 + r2 - lo2]);
        c = c < y ? y : c;
    }
    return !(c < a);
}

// How many X keys are among the first x outputs of P (0 <= x <= P.len).
template <int KT>
__device__ __forceinline__ long long pair_split(const typename Key<KT>::T *__restrict__ src,
                                                const long long *__restrict__ split1, const PairView &P, int nv,
                                                long long x) {
    typedef Key<KT> K;
    if (x >= P.len) return P.x_end - P.x_beg;
    const long long j = x / nv;
    long long xs, xe, ys, ye;
    pair_tile(split1, P, nv, j, xs, xe, ys, ye);
    const int r = (int)(x - j * nv);
    const int nx = (int)(xe - xs), ny = (int)(ye - ys);
    int lo = max(0, r - ny), hi = min(r, nx);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!(K::ord(src[ys + r - 1 - mid]) < K::ord(src[xs + mid]))) lo = mid + 1;
        else hi = mid;
    }
    return xs + lo - P.x_beg;
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

// 4-way splits of every output tile boundary of step `step` (runs of w keys,
// groups of 4w), a group of 2^lg lanes per boundary: split4[4b + i] is where
// tile b's share of run i (A, B, C, D) starts in the source buffer.
template <int KT>
__global__ void __launch_bounds__(256)
k_partition4(const typename Key<KT>::T *__restrict__ uk, const typename Key<KT>::T *__restrict__ sk,
             long long n, long long w, int nv, long long nbound, const long long *__restrict__ split1,
             long long *__restrict__ split4, const Ctrl *__restrict__ c, int step, int l0, int lg) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> lg;
    if (b >= nbound) return;                       // uniform across the group
    if (!step_needed(c, l0, 2)) return;
    const bool leader = (lane & ((1 << lg) - 1)) == 0;
    if (b * (long long)nv >= n) {                  // the end of the array: never read as a tile start
        if (leader)
            for (int i = 0; i < 4; ++i) split4[4 * b + i] = n;
        return;
    }
    const typename Key<KT>::T *src = c->src_buf[step] ? sk : uk;
    const long long out = b * (long long)nv;
    const long long G0 = (out / (4 * w)) * (4 * w);
    long long e[5];                                // A = [e0, e1), B = [e1, e2), C = [e2, e3), D = [e3, e4)
#pragma unroll
    for (int i = 0; i < 5; ++i) e[i] = min(G0 + i * w, n);
    const PairView AB = pair_view(e[0], e[1], e[2], nv), CD = pair_view(e[2], e[3], e[4], nv);
    const long long d = out - G0;                  // a multiple of nv
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
        // fine: AB outputs among the first d outputs of merge(AB, CD)
        lo = group_search(lo, hi, lane, lg,
                          [&](long long m) { return probe_ab_cd<KT>(src, split1, AB, CD, nv, d, m); });
    }
    if (leader) {
        const long long x = lo;
        const long long a = pair_split<KT>(src, split1, AB, nv, x);
        const long long cc = pair_split<KT>(src, split1, CD, nv, d - x);
        split4[4 * b + 0] = e[0] + a;
        split4[4 * b + 1] = e[1] + (x - a);
        split4[4 * b + 2] = e[2] + cc;
        split4[4 * b + 3] = e[3] + (d - x - cc);
    }
}

// One of four values by a run-time index, without indexing a local array
// (which would live in local memory).
template <typename V>
__device__ __forceinline__ V pick4(int i, V a, V b, V c, V d) {
    return i == 0 ? a : i == 1 ? b : i == 2 ? c : d;
}

// Staging modes of a 4-way merge tile's four windows into shared memory.
enum { STAGE_SCALAR = 0, STAGE_VEC = 1, STAGE_BULK = 2 };

// Staged key capacity of a 4-way merge tile: NV keys plus, per window, up to
// 3 keys before its first and after its last 4-key group boundary.
template <int NV> struct Merge4Cap { enum { SV = NV + 32 }; };

// Dynamic shared memory of k_merge4: the staged keys (and values), plus the
// slack the one-load merge step reads into.
template <typename U, int NT, int IPT, bool VALS>
constexpr size_t merge4_smem() {
    return (size_t)Merge4Cap<NT * IPT>::SV * (sizeof(U) + (VALS ? 4 : 0)) + (size_t)(IPT + 8) * sizeof(U);
}

// Longest wait for a tile's bulk copies: tries of mbarrier.try_wait (each
// waits in hardware for a while); a tile that gives up reports
// SR_ERR_TIMEOUT in `status`.
enum { BULK_WAIT_TRIES = 1 << 22 };

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

// One CTA per output tile of NT*IPT keys of 4-way step `step` (runs of w
// keys): the tile's windows of A, B, C and D come from split4 (the run ends
// for a group's last tile).
template <int KT, int NT, int IPT, bool VALS, int STAGE>
__global__ void __launch_bounds__(NT, Shape<sizeof(typename Key<KT>::T), VALS>::MERGE4_MINB)
k_merge4(typename Key<KT>::T *uk, uint32_t *uv, typename Key<KT>::T *sk, uint32_t *svb, long long n,
         long long w, const long long *__restrict__ split4, const Ctrl *__restrict__ c, int step, int l0,
         typename Key<KT>::U *__restrict__ samp, long long smt, int *status) {
    griddep_wait();
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int NV = NT * IPT;
    if (!step_needed(c, l0, 2)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long bar;
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + Merge4Cap<NV>::SV);
    const int cur = c->src_buf[step];
    const long long b = blockIdx.x;
    const long long out0 = b * NV;
    const long long out1 = min(out0 + NV, n);
    const long long G0 = (out0 / (4 * w)) * (4 * w);
    const bool last = out1 == min(G0 + 4 * w, n);   // the group's last tile ends at its runs' ends
    long long beg[4];
    int len[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        beg[i] = split4[4 * b + i];
        const long long end = last ? min(G0 + (i + 1) * w, n) : split4[4 * (b + 1) + i];
        len[i] = (int)(end - beg[i]);
    }
    merge_tile4<KT, NT, IPT, VALS, STAGE>(cur ? sk : uk, cur ? uk : sk, cur ? svb : uv, cur ? uv : svb, n, out0,
                                          (int)(out1 - out0), beg, len, s, sv, &bar, status,
                                          samp ? samp + (1 - cur) * smt : nullptr, b);
}

template <int KT, bool VALS>
__global__ void k_copy_back(typename Key<KT>::T *uk, uint32_t *uv, const typename Key<KT>::T *sk,
                            const uint32_t *svb, long long n, const Ctrl *__restrict__ c, int steps) {
    griddep_wait();
    if (call_mode(c, n) != MODE_SORT) return;
    if (c->src_buf[steps] == 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uk[i] = sk[i];
        if (VALS) uv[i] = svb[i];
    }
}

}  // namespace sr
