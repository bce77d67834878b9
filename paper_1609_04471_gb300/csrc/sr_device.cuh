// sr_device.cuh -- device building blocks of the GB300 merge sort.
//
// Keys stay in their native bit patterns in global memory.  On load every key
// is mapped to an unsigned "order image" U whose unsigned order is the key
// order (two's-complement flip for signed types, IEEE-754 totalOrder for
// float32); every comparison is then one unsigned compare, and the inverse map
// is applied on store.
//
// The building blocks follow the merge structure of the paper's mergesort
// (Section 3): runs are merged pairwise, round after round (policy e1), and a
// merge never lets a B item pass an equal A item (stability, technique (a)).
// Where the paper's merge is one sequential loop, here a merge of two runs is
// cut along the diagonals of its merge matrix ("merge path") into pieces of
// IPT outputs, one per thread, each found by a binary search -- the parallel
// form of galloping (technique (g)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sortrace.h"

namespace sr {

// ------------------------------------------------------------ key images

template <int KT> struct Key;

template <> struct Key<SR_KEY_I32> {
    typedef uint32_t T;
    typedef uint32_t U;
    static __device__ __forceinline__ U ord(T x) { return x ^ 0x80000000u; }
    static __device__ __forceinline__ T unord(U u) { return u ^ 0x80000000u; }
};
template <> struct Key<SR_KEY_U32> {
    typedef uint32_t T;
    typedef uint32_t U;
    static __device__ __forceinline__ U ord(T x) { return x; }
    static __device__ __forceinline__ T unord(U u) { return u; }
};
// totalOrder: a clear sign bit maps above every set one; negative patterns
// are inverted so a larger magnitude orders lower.
template <> struct Key<SR_KEY_F32> {
    typedef uint32_t T;
    typedef uint32_t U;
    static __device__ __forceinline__ U ord(T x) {
        return x ^ ((uint32_t)((int32_t)x >> 31) | 0x80000000u);
    }
    static __device__ __forceinline__ T unord(U u) {
        return u ^ (((u >> 31) - 1u) | 0x80000000u);
    }
};
template <> struct Key<SR_KEY_U64> {
    typedef unsigned long long T;
    typedef unsigned long long U;
    static __device__ __forceinline__ U ord(T x) { return x; }
    static __device__ __forceinline__ T unord(U u) { return u; }
};
template <> struct Key<SR_KEY_I64> {
    typedef unsigned long long T;
    typedef unsigned long long U;
    static __device__ __forceinline__ U ord(T x) { return x ^ 0x8000000000000000ull; }
    static __device__ __forceinline__ T unord(U u) { return u ^ 0x8000000000000000ull; }
};

template <typename U> __device__ __forceinline__ U umax_of() { return ~U(0); }

// Programmatic dependent launch: every kernel first lets the next kernel on
// its stream be scheduled (its CTAs then wait in griddep_wait until this grid
// has finished and its writes are visible), then waits for the previous one.
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------- launch shapes
//
// IPT is odd so that thread t's IPT consecutive shared-memory words
// t*IPT .. t*IPT+IPT-1 fall in distinct banks across a warp (gcd(IPT, 32) = 1).
template <int KB, bool VALS> struct Shape;
// NT x IPT keys per merge CTA; SORT_NT x IPT keys per block-sort tile.  (A
// 1024-thread block sort saves one global pass but its extra shared-memory
// level costs more than that pass on GB300: 2.87 ms against 0.57 ms at 2^28.)
// Defaults measured on GB300 (plain int32 sort, 2^24 and 2^28 keys); each
// can be overridden at build time.  4-byte keys alone take 33 keys per thread:
// 16,896-key block-sort tiles need one merge step fewer than 12,800-key ones
// at 2^24 and at 2^28 (2^28: 7.68 -> 7.15 ms; 2^24: 0.539 -> 0.507 ms).
#ifndef SR_K4_IPT
#define SR_K4_IPT 33
#endif
#ifndef SR_K4V_IPT
#define SR_K4V_IPT 11
#endif
#ifndef SR_K8_IPT
#define SR_K8_IPT 17
#endif
#ifndef SR_K8V_IPT
#define SR_K8V_IPT 13
#endif
#ifndef SR_SORT_NT
#define SR_SORT_NT 512
#endif
#ifndef SR_MERGE_NT
#define SR_MERGE_NT 256
#endif
// MERGE_MINB: resident merge CTAs per SM the register allocator is held to
// (4-byte keys: 40 registers, six CTAs; the others keep the occupancy they
// reach unconstrained).
// MERGE4_MINB: the same for the 4-way merge kernel.
#ifndef SR_MERGE4_MINB4
#define SR_MERGE4_MINB4 5
#endif
// SORT_MINB: block-sort CTAs per SM the register allocator is held to (4-byte
// keys alone: two CTAs of 512 threads, 64 registers, with 33 keys a thread;
// three at 40 registers spilled).
// SR_BSORT_PP: how tiles are sorted -- 0: block_sort; 1: block_sort_pp (two
// shared buffers, end-marked runs; 4-byte keys alone); 2: block_sort_rs (one
// end-marked buffer, outputs through registers; every key shape).  Measured
// for 4-byte keys at 2^28 on GB300: 2.31, 2.11 and 2.02 ms.
#ifndef SR_BSORT_PP
#define SR_BSORT_PP 2
#endif
#ifndef SR_MERGE_MINB4
#define SR_MERGE_MINB4 6
#endif
#ifndef SR_SORT_MINB4
#define SR_SORT_MINB4 2
#endif
template <> struct Shape<4, false> { enum { NT = SR_MERGE_NT, IPT = SR_K4_IPT, SORT_NT = SR_SORT_NT, MERGE_MINB = SR_MERGE_MINB4, MERGE4_MINB = SR_MERGE4_MINB4, SORT_MINB = SR_SORT_MINB4 }; };
template <> struct Shape<4, true>  { enum { NT = SR_MERGE_NT, IPT = SR_K4V_IPT, SORT_NT = SR_SORT_NT, MERGE_MINB = 8, MERGE4_MINB = 6, SORT_MINB = 3 }; };
// SR_SORT_MINB8: block-sort CTAs per SM for 8-byte keys (with or without
// payloads): two, at 64 registers (block_sort_rs at 2^26: uint64 keys 1.49 ->
// 1.04 ms, pairs 2.13 -> 1.44 ms against one CTA unbounded).
#ifndef SR_SORT_MINB8
#define SR_SORT_MINB8 2
#endif
// MERGE4_MINB for 8-byte keys: five CTAs per SM for keys alone (48 registers;
// uint64 keys at 2^26: 4-way steps 2.30 -> 2.10 ms), four with payloads (five
// spill and ran slower).
#ifndef SR_MERGE4_MINB8
#define SR_MERGE4_MINB8 5
#endif
template <> struct Shape<8, false> { enum { NT = SR_MERGE_NT, IPT = SR_K8_IPT, SORT_NT = SR_SORT_NT, MERGE_MINB = 4, MERGE4_MINB = SR_MERGE4_MINB8, SORT_MINB = SR_SORT_MINB8 }; };
template <> struct Shape<8, true>  { enum { NT = SR_MERGE_NT, IPT = SR_K8V_IPT, SORT_NT = SR_SORT_NT, MERGE_MINB = 4, MERGE4_MINB = 4, SORT_MINB = SR_SORT_MINB8 }; };

// ------------------------------------------------------------- merge path

// Number of A items among the first `diag` outputs of the stable merge of
// sorted a[0..na) and b[0..nb): the largest i with a[i-1] <= b[diag-i]
// (an A item goes first on ties).
template <typename U>
__device__ __forceinline__ int merge_path(const U *a, int na, const U *b, int nb, int diag) {
    int lo = max(0, diag - nb), hi = min(diag, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!(b[diag - 1 - mid] < a[mid])) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The same split found over global memory by a group of G = 2^lg lanes of
// one warp (G = 1: plain binary search).  Each round the G lanes test G evenly
// spaced candidates m and a ballot counts those with the answer above m, which
// cuts the stretch holding the answer to 1/(G+1) of its length: about
// log_{G+1}(range) dependent rounds of 2G scattered loads.  Returns the number
// of A items among the first `diag` outputs of the stable merge of
// src[a_beg .. a_beg+na) and src[b_beg .. b_beg+nb).  All lanes of a group
// must call it with the same arguments; all of them return the answer.
template <typename K>
__device__ __forceinline__ long long group_split(const typename K::T *__restrict__ src, long long a_beg,
                                                 long long na, long long b_beg, long long nb,
                                                 long long diag, int lane, int lg) {
    typedef typename K::U U;
    const int G = 1 << lg;
    const int j = lane & (G - 1);
    const unsigned mask = lg == 5 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    long long lo = max(0ll, diag - nb), hi = min(diag, na);
    while (hi > lo) {
        const long long step = (hi - lo + G) / (G + 1);          // >= 1
        const long long m = lo + (long long)(j + 1) * step - 1;
        bool before = false;                                      // the answer is > m
        if (m < hi) {
            const U x = K::ord(src[a_beg + m]);
            const U y = K::ord(src[b_beg + diag - 1 - m]);
            before = !(y < x);
        }
        const int cnt = __popc(__ballot_sync(mask, before));
        const long long nhi = cnt == G ? hi : lo + (long long)(cnt + 1) * step - 1;
        lo = lo + (long long)cnt * step;
        hi = min(hi, nhi);
    }
    return lo;
}

// The smallest m in [lo, hi] with before(m) false, found by a group of
// 2^lg lanes (before(m) is true below the answer and false from it on; m = hi
// counts as false): the same (G+1)-ary search as group_split over any
// predicate.  All lanes of the group call it with the same lo, hi.
template <typename Pred>
__device__ __forceinline__ long long group_search(long long lo, long long hi, int lane, int lg, Pred before) {
    const int G = 1 << lg;
    const int j = lane & (G - 1);
    const unsigned mask = lg == 5 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    while (hi > lo) {
        const long long step = (hi - lo + G) / (G + 1);
        const long long m = lo + (long long)(j + 1) * step - 1;
        const bool b = m < hi && before(m);
        const int cnt = __popc(__ballot_sync(mask, b));
        const long long nhi = cnt == G ? hi : lo + (long long)(cnt + 1) * step - 1;
        lo = lo + (long long)cnt * step;
        hi = min(hi, nhi);
    }
    return lo;
}

template <typename K>
__device__ __forceinline__ long long warp_split(const typename K::T *__restrict__ src, long long a_beg,
                                                long long na, long long b_beg, long long nb,
                                                long long diag, int lane) {
    return group_split<K>(src, a_beg, na, b_beg, nb, diag, lane, 5);
}

// IPT outputs of the stable merge of s[a..a_end) and s[b..b_end) into
// registers; ix[i] is the shared-memory index each output came from.
// serial_merge for buffers with readable slack: one shared load per step (the
// next key of whichever side was taken), with no bounds test on the load.
// Reads reach index max(a_end, b_end) + IPT + 1 at most (a thread whose
// outputs run past the end keeps taking from an exhausted side), so s must be
// readable that far; keys read past a range's end are never selected.
template <typename U, int IPT>
__device__ __forceinline__ void serial_merge_slack(const U *s, int a, int a_end, int b, int b_end,
                                                   U (&k)[IPT], int (&ix)[IPT]) {
    U ak = s[a];
    U bk = s[b];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool take_a = (b >= b_end) || ((a < a_end) && !(bk < ak));
        k[i] = take_a ? ak : bk;
        ix[i] = take_a ? a : b;
        const int nx = (take_a ? a : b) + 1;
        const U nk = s[nx];
        if (take_a) { a = nx; ak = nk; }
        else        { b = nx; bk = nk; }
    }
}

// serial_merge_slack for ranges whose ends are marked: the key after each
// range is the largest image (umax) and neither range holds a umax key, so an
// exhausted side is never taken while the other has keys and a step is one
// comparison (ties still go to A).  A thread whose outputs run past both
// ranges keeps taking A past its mark: s must be readable IPT keys beyond it.
template <typename U, int IPT>
__device__ __forceinline__ void serial_merge_marked(const U *s, int a, int b, U (&k)[IPT], int (&ix)[IPT]) {
    U ak = s[a];
    U bk = s[b];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool take_a = !(bk < ak);
        k[i] = take_a ? ak : bk;
        ix[i] = take_a ? a : b;
        const int nx = (take_a ? a : b) + 1;
        const U nk = s[nx];
        if (take_a) { a = nx; ak = nk; }
        else        { b = nx; bk = nk; }
    }
}

// serial_merge_marked for keys alone, where equal keys cannot be told apart
// and no output needs its source index: the two heads are kept as (the head
// not taken, with its index) and (the key just loaded, with its index), so a
// step is the min and the max of the two heads and only the taken side's
// index moves (two selects fewer than tracking A's and B's heads).  The
// outputs are those of serial_merge_marked; the reads are the same keys, and
// a thread whose outputs run past both ranges keeps taking one side past its
// mark, so s must be readable IPT keys beyond the later mark.
template <typename U, int IPT>
__device__ __forceinline__ void serial_merge_marked_keys(const U *s, int a, int b, U (&k)[IPT]) {
    U x = s[a], y = s[b];
    int px = a, py = b;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool p = y < x;                      // take y's side
        k[i] = p ? y : x;
        const U o = p ? x : y;
        const int po = p ? px : py;
        const int pt = (p ? py : px) + 1;
        x = o;
        px = po;
        y = s[pt];
        py = pt;
    }
}

template <typename U, int IPT>
__device__ __forceinline__ void serial_merge(const U *s, int a, int a_end, int b, int b_end,
                                             U (&k)[IPT], int (&ix)[IPT]) {
    U ak = a < a_end ? s[a] : U(0);
    U bk = b < b_end ? s[b] : U(0);
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool take_a = (b >= b_end) || ((a < a_end) && !(bk < ak));
        k[i] = take_a ? ak : bk;
        ix[i] = take_a ? a : b;
        if (take_a) { ++a; if (a < a_end) ak = s[a]; }
        else        { ++b; if (b < b_end) bk = s[b]; }
    }
}

// IPT outputs of two stable merges in a row: the first `sw` outputs come from
// the merge of s[a..a_end) and s[b..b_end), the rest from the merge of
// s[c..c_end) and s[d..d_end) starting at their first keys.  For the one
// thread of a 4-way merge tile whose outputs straddle the end of the first
// pair's merged run.  Loads are guarded like serial_merge's.
template <typename U, int IPT>
__device__ __forceinline__ void serial_merge_switch(const U *s, int a, int a_end, int b, int b_end, int sw, int c,
                                                    int c_end, int d, int d_end, U (&k)[IPT], int (&ix)[IPT]) {
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        if (i == sw) { a = c; a_end = c_end; b = d; b_end = d_end; }
        const bool take_a = (b >= b_end) || ((a < a_end) && !(s[b] < s[a]));
        const int at = take_a ? a : b;
        k[i] = s[at];
        ix[i] = at;
        if (take_a) ++a;
        else ++b;
    }
}

// ------------------------------------------------ bulk copies into shared memory
//
// 1-D bulk copies (cp.async.bulk) from this GPU's global memory into the
// CTA's shared memory, completed on an mbarrier: one thread starts them and
// every thread waits for the barrier's phase.  Addresses and sizes must be
// multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One arrival that also announces `bytes` of copies still to land.
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for phase `parity` of the barrier, giving up after `limit` tries
// (each try itself waits a while in hardware).  Returns whether it completed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------- merge step schedule
//
// After the block sort the runs are one tile long at most; ceil(log2(tiles))
// binary merge levels remain.  Steps of fan-in 4 cover two levels each, so a
// call launches ceil(log_f(tiles)) steps; the run planner (k_runs) then tells
// each step whether the input's natural runs need it.
__host__ __device__ constexpr int merge_step_count(int levels, bool fan4) {
    return fan4 ? (levels + 1) / 2 : levels;
}

// Sort of a thread's IPT registers.  Keys alone: Batcher's odd-even merge
// sort network cut to IPT inputs, its pairs generated at compile time (246
// compare-exchanges for 33 keys against 528 for transposition; equal keys are
// indistinguishable, so stability does not arise).  Keys with values: odd-even
// transposition, which is stable (only neighbours swap, and only on a strict
// descent).
#ifndef SR_KEYS_NETWORK
#define SR_KEYS_NETWORK 1   // keys alone: Batcher's network as the register sort
#endif
// Batcher's odd-even merge sort network on N inputs: its compare-exchange
// pairs, generated at compile time.
struct NetPairs {
    int n;
    unsigned char a[1024], b[1024];     // enough for N <= 64
};
__host__ __device__ constexpr NetPairs batcher_pairs(int N) {
    NetPairs r{};
    r.n = 0;
    for (int p = 1; p < N; p <<= 1)
        for (int d = p; d >= 1; d >>= 1)
            for (int j = d % p; j + d <= N - 1; j += 2 * d)
                for (int i = 0; i < d && i + j + d <= N - 1; ++i)
                    if ((i + j) / (2 * p) == (i + j + d) / (2 * p)) {
                        r.a[r.n] = (unsigned char)(i + j);
                        r.b[r.n] = (unsigned char)(i + j + d);
                        ++r.n;
                    }
    return r;
}

template <typename U, int IPT, bool VALS>
__device__ __forceinline__ void thread_sort(U (&k)[IPT], uint32_t (&v)[IPT]) {
    if constexpr (!VALS && SR_KEYS_NETWORK) {
        static_assert(IPT <= 64, "network tables hold up to 64 inputs");
        constexpr NetPairs net = batcher_pairs(IPT);
#pragma unroll
        for (int c = 0; c < net.n; ++c) {
            const U x = k[net.a[c]], y = k[net.b[c]];
            k[net.a[c]] = x < y ? x : y;
            k[net.b[c]] = x < y ? y : x;
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
#pragma unroll
        for (int i = r & 1; i + 1 < IPT; i += 2) {
            if (k[i + 1] < k[i]) {
                const U tk = k[i]; k[i] = k[i + 1]; k[i + 1] = tk;
                if (VALS) { const uint32_t tv = v[i]; v[i] = v[i + 1]; v[i + 1] = tv; }
            }
        }
    }
}

// Sorts the NT*IPT items held blocked in registers (thread t holds items
// t*IPT .. t*IPT+IPT-1): a register sort, then log2(NT) rounds of stable
// pairwise merges through shared memory (sk: NT*IPT keys, sv: NT*IPT values).
// Rounds whose runs lie inside one warp synchronise that warp only.  On
// return the registers hold the sorted tile, blocked.
template <typename U, int NT, int IPT, bool VALS>
__device__ __forceinline__ void block_sort(U (&k)[IPT], uint32_t (&v)[IPT], U *sk, uint32_t *sv) {
    thread_sort<U, IPT, VALS>(k, v);
    const int t = threadIdx.x;
#pragma unroll 1
    for (int coop = 2; coop <= NT; coop <<= 1) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) sk[t * IPT + i] = k[i];
        if (VALS) {
#pragma unroll
            for (int i = 0; i < IPT; ++i) sv[t * IPT + i] = v[i];
        }
        if (coop <= 32) __syncwarp(); else __syncthreads();
        const int first = t & ~(coop - 1);
        const int run = (coop >> 1) * IPT;
        const int a0 = first * IPT, b0 = a0 + run;
        const int diag = (t - first) * IPT;
        const int sp = merge_path(sk + a0, run, sk + b0, run, diag);
        int ix[IPT];
        serial_merge<U, IPT>(sk, a0 + sp, b0, b0 + diag - sp, b0 + run, k, ix);
        if (VALS) {
#pragma unroll
            for (int i = 0; i < IPT; ++i) v[i] = sv[ix[i]];
        }
        if (coop <= 32) __syncwarp(); else __syncthreads();
    }
}

// IPT outputs of the merge of s[a..a_end) and s[b..b_end), written to
// out[0 .. IPT) in shared memory, for a thread whose IPT outputs all exist
// (the two ranges hold at least IPT keys from a and b on): it never takes from
// an exhausted side, so each step loads the next key of the side it took
// without a bounds test, reading s at most up to index max(a_end, b_end).
template <typename U, int IPT>
__device__ __forceinline__ void serial_merge_out(const U *s, int a, int a_end, int b, int b_end, U *out) {
    U ak = s[a];
    U bk = s[b];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool take_b = b < b_end && (a >= a_end || bk < ak);
        out[i] = take_b ? bk : ak;
        const int nx = (take_b ? b : a) + 1;
        const U nk = s[nx];
        if (take_b) { b = nx; bk = nk; }
        else        { a = nx; ak = nk; }
    }
}

// The same with the ranges' ends marked in s: the key after each range is the
// largest image (umax), and no key of either range is umax.  An exhausted
// side then shows umax and is never taken, so a step is one comparison.
template <typename U, int IPT>
__device__ __forceinline__ void serial_merge_out_marked(const U *s, int a, int b, U *out) {
    U ak = s[a];
    U bk = s[b];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const bool take_b = bk < ak;
        out[i] = take_b ? bk : ak;
        const int nx = (take_b ? b : a) + 1;
        const U nk = s[nx];
        if (take_b) { b = nx; bk = nk; }
        else        { a = nx; ak = nk; }
    }
}

// Shared keys one block-sort buffer holds: the tile and one end mark per run
// of the first merge round.
template <int NT, int IPT> constexpr int block_sort_pp_keys() { return NT * IPT + NT; }

// Keys alone: sorts the NT*IPT keys held blocked in registers (thread t holds
// items t*IPT ..), the merge rounds going from one shared buffer to the other
// (sa, sb: block_sort_pp_keys each), so no round holds its outputs in
// registers.  Every run of a round is followed by an end mark (umax).  Each
// warp owns W = 32*IPT + 32 keys of either buffer: the rounds that merge
// inside a warp (synchronised by the warp alone) keep their runs, L + 1 apart,
// in the warp's own stretch, so a warp never writes where another may still
// read; the later rounds (block barriers) place run q of L = c*IPT keys (c
// threads' worth) at q * (c/32) * W.  Tiles without a umax key merge with one
// comparison per step (serial_merge_out_marked), a tile holding umax keys (a
// key equal to the mark, or the last tile's padding) with the bounded steps.
// Keys are equal when their images are, so either merge gives the same sorted
// tile.  Returns the buffer that holds it, from index 0.
template <typename U, int NT, int IPT>
__device__ __forceinline__ U *block_sort_pp(U (&k)[IPT], U *sa, U *sb) {
    constexpr int W = 32 * IPT + 32;
    static_assert(NT % 32 == 0 && (NT / 32) * W == block_sort_pp_keys<NT, IPT>(), "warp stretches tile the buffer");
    uint32_t dv[IPT];
    thread_sort<U, IPT, false>(k, dv);
    const int t = threadIdx.x;
    const int w = t >> 5, lane = t & 31;
    const bool fast = !__syncthreads_or(k[IPT - 1] == umax_of<U>());
#pragma unroll
    for (int i = 0; i < IPT; ++i) sa[w * W + lane * (IPT + 1) + i] = k[i];
    sa[w * W + lane * (IPT + 1) + IPT] = umax_of<U>();
    U *src = sa, *dst = sb;
#pragma unroll 1
    for (int coop = 2; coop <= NT; coop <<= 1) {
        const int first = t & ~(coop - 1);
        const int run = (coop >> 1) * IPT;
        const int diag = (t - first) * IPT;
        int a0, b0, o0;                            // runs 2g and 2g + 1 of the round, and their merge
        if (coop <= 32) {
            __syncwarp();
            const int gl = (first & 31) / coop;    // the group's place in its warp
            a0 = w * W + 2 * gl * (run + 1);
            b0 = a0 + run + 1;
            o0 = w * W + gl * (2 * run + 1);
        } else {
            __syncthreads();
            const int rs = (coop / 64) * W;        // stride of this round's runs
            const int g = first / coop;
            a0 = 2 * g * rs;
            b0 = a0 + rs;
            o0 = 2 * g * rs;
        }
        const int sp = merge_path(src + a0, run, src + b0, run, diag);
        if (fast) serial_merge_out_marked<U, IPT>(src, a0 + sp, b0 + diag - sp, dst + o0 + diag);
        else      serial_merge_out<U, IPT>(src, a0 + sp, a0 + run, b0 + diag - sp, b0 + run, dst + o0 + diag);
        if (t - first == coop - 1) dst[o0 + 2 * run] = umax_of<U>();
        U *x = src; src = dst; dst = x;
    }
    __syncthreads();
    return src;
}

// block_sort_pp's rounds with one shared buffer (block_sort_pp_keys keys,
// and as many payloads in `va` when VALS): each round merges into registers,
// waits until its warp (or the block) has read the round's runs, then writes
// the merged runs back in the next round's layout.  Ties go to the earlier
// run, so with payloads the tile sort stays stable (the register sort is the
// stable transposition sort then).  Half the shared memory of block_sort_pp,
// for more resident CTAs.
template <typename U, int NT, int IPT, bool VALS>
__device__ __forceinline__ U *block_sort_rs(U (&k)[IPT], uint32_t (&v)[IPT], U *sa, uint32_t *va) {
    constexpr int W = 32 * IPT + 32;
    static_assert(NT % 32 == 0 && (NT / 32) * W == block_sort_pp_keys<NT, IPT>(), "warp stretches tile the buffer");
    thread_sort<U, IPT, VALS>(k, v);
    const int t = threadIdx.x;
    const int w = t >> 5, lane = t & 31;
    const bool fast = !__syncthreads_or(k[IPT - 1] == umax_of<U>());
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        sa[w * W + lane * (IPT + 1) + i] = k[i];
        if (VALS) va[w * W + lane * (IPT + 1) + i] = v[i];
    }
    sa[w * W + lane * (IPT + 1) + IPT] = umax_of<U>();
#pragma unroll 1
    for (int coop = 2; coop <= NT; coop <<= 1) {
        const int first = t & ~(coop - 1);
        const int run = (coop >> 1) * IPT;
        const int diag = (t - first) * IPT;
        int a0, b0, o0;
        if (coop <= 32) {
            __syncwarp();
            const int gl = (first & 31) / coop;
            a0 = w * W + 2 * gl * (run + 1);
            b0 = a0 + run + 1;
            o0 = w * W + gl * (2 * run + 1);
        } else {
            __syncthreads();
            const int rs = (coop / 64) * W;
            const int g = first / coop;
            a0 = 2 * g * rs;
            b0 = a0 + rs;
            o0 = 2 * g * rs;
        }
        const int sp = merge_path(sa + a0, run, sa + b0, run, diag);
        int ix[IPT];
        if (fast && !VALS) serial_merge_marked_keys<U, IPT>(sa, a0 + sp, b0 + diag - sp, k);
        else if (fast)     serial_merge_marked<U, IPT>(sa, a0 + sp, b0 + diag - sp, k, ix);
        else               serial_merge_slack<U, IPT>(sa, a0 + sp, a0 + run, b0 + diag - sp, b0 + run, k, ix);
        if (VALS) {
#pragma unroll
            for (int i = 0; i < IPT; ++i) v[i] = va[ix[i]];
        }
        if (coop <= 32) __syncwarp(); else __syncthreads();
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            sa[o0 + diag + i] = k[i];
            if (VALS) va[o0 + diag + i] = v[i];
        }
        if (t - first == coop - 1) sa[o0 + 2 * run] = umax_of<U>();
    }
    __syncthreads();
    return sa;
}

// ------------------------------------------------------- per-call control

enum { MODE_SORT = 0, MODE_SORTED = 1, MODE_REVERSE = 2, MODE_FEW = 3, MODE_REM = 4 };
enum { MAX_PASSES = 48 };
// Few distinct keys: at most FEW_MAX distinct order images (4-byte keys),
// found in a FEW_SAMPLE-key sample through a hash set of FEW_SLOTS slots.
enum { FEW_MAX = 4096, FEW_SLOTS_LOG2 = 14, FEW_SLOTS = 1 << FEW_SLOTS_LOG2 };

// The few-distinct-keys path's tables, in the call's scratch (zeroed at the
// start of every call): the set of sampled order images (image + 1 per slot,
// 0 = empty), the distinct images ascending, and the keys equal to each.
struct FewTables {
    unsigned long long slot[FEW_SLOTS];
    unsigned int sorted[FEW_MAX];
    unsigned long long count[FEW_MAX];
};

// Lives in the call's scratch; zeroed at the start of every call.
struct Ctrl {
    unsigned long long descents;        // pairs a[i] > a[i+1]
    unsigned long long nondescents;     // pairs a[i] <= a[i+1]
    unsigned long long tiles_ascending;
    unsigned long long tiles_descending;
    // written by the run planner (k_runs) after the block sort: the natural
    // runs of whole tiles, the merge steps they need, and which buffer (0 =
    // caller's, 1 = scratch) holds the data before step s (and after the last)
    int nruns;
    int nsteps;
    // Neighbour repair: after the block sort no tile's keys exceed those of
    // the tile two places on (repair), and no tile boundary's window of keys
    // out of order is larger than a merge tile (else repair_fail): then each
    // window is merged in place and no merge step runs.
    int tile_perm;                               // the block sort writes reversed chains of tiles reversed
    int repair;
    int repair_fail;
    unsigned long long repair_keys;              // keys in the merged windows
    int status;
    signed char src_buf[MAX_PASSES + 1];
    // Few distinct keys (4-byte keys, keys only): a sample of the keys goes
    // into a hash set of order images (FewTables) until more than FEW_MAX
    // appear (few_over); the counting pass then checks every key against it.
    int few_over;
    unsigned int few_n;                          // distinct images in the set
    unsigned int few_ticket;                     // CTAs of the sampling kernels that finished
    unsigned int few_ticket2;
    int few_cand;                                // the set is a candidate (sorted into FewTables::sorted)
    int few_miss;                                // some key is not in the set
    int few_active;                              // the call took MODE_FEW (output written)
    // Few displaced keys (keys only): the path was tried (rem_active), a
    // bucket overflowed (rem_over), or it wrote the output (rem_gate).
    int rem_active;
    int rem_over;
    int rem_gate;
    unsigned long long rem_dcount;               // keys that went through the buckets
};

// Merge steps the call runs: none after a neighbour repair, else the steps
// the natural runs need.
__device__ __forceinline__ int steps_of(const Ctrl *c) {
    return (c->repair && !c->repair_fail) ? 0 : c->nsteps;
}

__device__ __forceinline__ int call_mode(const Ctrl *c, long long n) {
    if (c->descents == 0) return MODE_SORTED;
    if (c->nondescents == 0 && n > 1) return MODE_REVERSE;
    if (c->few_active) return MODE_FEW;
    if (c->rem_gate) return MODE_REM;
    return MODE_SORT;
}

// Inserts order image u into the hash set `set` (2^LOG2 slots of image + 1,
// 0 = empty) shared by the threads that can see it; `cnt` counts distinct
// images and `over` is raised past `limit` of them (or after 32 probes, which
// at most a quarter of the slots used makes rare and only costs the fast
// path).  No waiting on other threads.
template <int LOG2>
__device__ __forceinline__ void few_insert(unsigned long long *set, unsigned int *cnt, int *over, unsigned int u,
                                           unsigned int limit) {
    const unsigned long long v = (unsigned long long)u + 1ull;
    const unsigned int h = (u * 2654435761u) >> (32 - LOG2);
    for (int probe = 0; probe < 32; ++probe) {               // a longer probe counts as "too many"
        const unsigned int i = (h + probe) & ((1u << LOG2) - 1u);
        const unsigned long long cur = ((volatile unsigned long long *)set)[i];
        if (cur == v) return;
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(set + i, 0ull, v);
            if (prev == 0ull) {
                if (atomicAdd(cnt, 1u) + 1u > limit) atomicExch(over, 1);
                return;
            }
            if (prev == v) return;
        }
    }
    atomicExch(over, 1);
}

}  // namespace sr
