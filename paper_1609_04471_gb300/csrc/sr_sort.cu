// sr_sort.cu -- the plain comparison sort: sr_sort_keys, sr_sort_pairs,
// sr_sort_keys_host and sr_detect_runs.
//
// One call is a fixed launch sequence on the caller's stream, with every
// data-dependent decision taken on the device (so a call can be captured in a
// CUDA graph):
//
//   k_detect     run-detection scan (Section 2's Run(A); Section 3 process 1):
//                counts descents and non-descents of neighbour pairs.
//   k_reverse    if every pair strictly descends, reverse the whole array in
//                one read + write (Section 3 technique (a); Section 4's remark
//                that sorted and reversely sorted lists take O(n)).
//   k_block_sort sort each tile of SORT_NT*IPT keys in shared memory; a tile
//                that is already ascending is left alone, a strictly
//                descending one is reversed (techniques (a), (b); Section 4 (f)).
//   per merge pass p (run width w = tile << p), policy e1 of Section 3:
//     k_partition  merge-path split of every output tile of NT*IPT keys, and a
//                  count of run pairs whose runs overlap (A.last > B.first);
//                  a pass where no pair overlaps is skipped -- nothing moves
//                  (technique (f) applied to whole passes).
//     k_merge      each CTA stages its A and B ranges in shared memory and
//                  merges them, IPT outputs per thread, stably.
//   k_copy_back  if skipped passes left the result in scratch, copy it home.
//
// If every pair is in order (the input is sorted) nothing after the scan moves
// any data.
#include <algorithm>
#include <cstring>

#include "sr_device.cuh"
#include "sr_runtime.cuh"

namespace sr {

// ------------------------------------------------------------- kernels

template <int KT, int NT, int IPT>
__global__ void __launch_bounds__(NT) k_detect(const typename Key<KT>::T *__restrict__ keys,
                                               long long n, Ctrl *__restrict__ c) {
    typedef Key<KT> K;
    typedef typename K::U U;
    constexpr int NV = NT * IPT;
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    __shared__ unsigned int red[4];
    const int t = threadIdx.x;
    const long long base = (long long)blockIdx.x * NV;
    const int cnt = (int)(n - base < (long long)NV + 1 ? n - base : (long long)NV + 1);   // one more for the pair across
    if (t < 4) red[t] = 0;
    for (int i = t; i < cnt; i += NT) s[i] = K::ord(keys[base + i]);
    __syncthreads();
    unsigned int d = 0, nd = 0, din = 0, ndin = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int j = t * IPT + i;
        if (j + 1 < cnt) {
            const bool de = s[j] > s[j + 1];
            d += de;
            nd += !de;
            if (j + 1 < NV) { din |= de; ndin |= !de; }
        }
    }
    d = __reduce_add_sync(0xffffffffu, d);
    nd = __reduce_add_sync(0xffffffffu, nd);
    din = __reduce_or_sync(0xffffffffu, din);
    ndin = __reduce_or_sync(0xffffffffu, ndin);
    if ((t & 31) == 0) {
        atomicAdd(&red[0], d);
        atomicAdd(&red[1], nd);
        atomicOr(&red[2], din);
        atomicOr(&red[3], ndin);
    }
    __syncthreads();
    if (t == 0) {
        if (red[0]) atomicAdd(&c->descents, (unsigned long long)red[0]);
        if (red[1]) atomicAdd(&c->nondescents, (unsigned long long)red[1]);
        if (!red[2]) atomicAdd(&c->tiles_ascending, 1ull);
        if (!red[3]) atomicAdd(&c->tiles_descending, 1ull);
    }
}

template <int KT, bool VALS>
__global__ void k_reverse(typename Key<KT>::T *__restrict__ k, uint32_t *__restrict__ v,
                          long long n, const Ctrl *__restrict__ c) {
    if (call_mode(c, n) != MODE_REVERSE) return;
    const long long half = n / 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < half; i += stride) {
        const long long j = n - 1 - i;
        const typename Key<KT>::T a = k[i], b = k[j];
        k[i] = b;
        k[j] = a;
        if (VALS) {
            const uint32_t x = v[i], y = v[j];
            v[i] = y;
            v[j] = x;
        }
    }
}

template <int KT, int NT, int IPT, bool VALS>
__global__ void __launch_bounds__(NT)
k_block_sort(const typename Key<KT>::T *in_k, const uint32_t *in_v, typename Key<KT>::T *out_k,
             uint32_t *out_v, long long n, const Ctrl *__restrict__ c) {
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
    if (!any_desc) {                       // already ascending
        if (out_k != in_k) {
            for (int idx = t; idx < cnt; idx += NT) {
                out_k[base + idx] = K::unord(s[idx]);
                if (VALS) out_v[base + idx] = sv[idx];
            }
        }
        return;
    }
    if (!any_nondesc) {                    // strictly descending: reverse
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
    for (int idx = t; idx < cnt; idx += NT) {
        out_k[base + idx] = K::unord(s[idx]);
        if (VALS) out_v[base + idx] = sv[idx];
    }
}

// One thread per merge-tile boundary b (0..tiles): splits[b] = the A index
// where output position b*nv falls, for the pair of runs that contains it.
template <int KT>
__global__ void k_partition(const typename Key<KT>::T *__restrict__ uk,
                            const typename Key<KT>::T *__restrict__ sk, long long n, long long w,
                            int nv, long long nbound, long long *__restrict__ splits,
                            Ctrl *__restrict__ c, int cur0, int p) {
    typedef Key<KT> K;
    typedef typename K::U U;
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbound) return;
    if (call_mode(c, n) != MODE_SORT) return;
    const typename K::T *src = buffer_before_pass(c, cur0, p) ? sk : uk;
    const long long out = min(b * (long long)nv, n);
    const long long pb = (out / (2 * w)) * (2 * w);
    const long long a_beg = pb, a_end = min(pb + w, n);
    const long long b_beg = a_end, b_end = min(pb + 2 * w, n);
    const long long diag = out - pb, na = a_end - a_beg, nb = b_end - b_beg;
    if (diag == 0 && nb > 0 && K::ord(src[a_end - 1]) > K::ord(src[b_beg]))
        atomicAdd(&c->unordered[p], 1);
    long long lo = max(0ll, diag - nb), hi = min(diag, na);
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        const U x = K::ord(src[a_beg + mid]);
        const U y = K::ord(src[b_beg + diag - 1 - mid]);
        if (!(y < x)) lo = mid + 1;
        else hi = mid;
    }
    splits[b] = a_beg + lo;
}

template <int KT, int NT, int IPT, bool VALS>
__global__ void __launch_bounds__(NT)
k_merge(typename Key<KT>::T *uk, uint32_t *uv, typename Key<KT>::T *sk, uint32_t *svb, long long n,
        long long w, const long long *__restrict__ splits, const Ctrl *__restrict__ c, int cur0,
        int p) {
    typedef Key<KT> K;
    typedef typename K::U U;
    typedef typename K::T T;
    constexpr int NV = NT * IPT;
    if (call_mode(c, n) != MODE_SORT || c->unordered[p] == 0) return;
    __shared__ int s_cur;
    if (threadIdx.x == 0) s_cur = buffer_before_pass(c, cur0, p);
    extern __shared__ __align__(16) unsigned char smem[];
    U *s = reinterpret_cast<U *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(s + NV);
    __syncthreads();
    const int cur = s_cur;
    const T *src_k = cur ? sk : uk;
    T *dst_k = cur ? uk : sk;
    const uint32_t *src_v = cur ? svb : uv;
    uint32_t *dst_v = cur ? uv : svb;
    const int t = threadIdx.x;
    const long long out0 = (long long)blockIdx.x * NV;
    const long long out1 = min(out0 + NV, n);
    const int cnt = (int)(out1 - out0);
    const long long pb = (out0 / (2 * w)) * (2 * w);
    const long long a_beg = pb, a_end = min(pb + w, n);
    const long long b_beg = a_end, b_end = min(pb + 2 * w, n);
    const long long a0 = splits[blockIdx.x];
    const long long a1 = (out1 == b_end) ? a_end : splits[blockIdx.x + 1];
    const long long b0 = b_beg + (out0 - pb) - (a0 - a_beg);
    const int acnt = (int)(a1 - a0);
    const int bcnt = cnt - acnt;
    for (int i = t; i < cnt; i += NT) {
        const long long g = i < acnt ? a0 + i : b0 + (i - acnt);
        s[i] = K::ord(src_k[g]);
        if (VALS) sv[i] = src_v[g];
    }
    __syncthreads();
    const int diag = min(t * IPT, cnt);
    const int sp = merge_path(s, acnt, s + acnt, bcnt, diag);
    U k[IPT];
    int ix[IPT];
    serial_merge<U, IPT>(s, sp, acnt, acnt + diag - sp, cnt, k, ix);
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
    for (int i = t; i < cnt; i += NT) {
        dst_k[out0 + i] = K::unord(s[i]);
        if (VALS) dst_v[out0 + i] = sv[i];
    }
}

template <int KT, bool VALS>
__global__ void k_copy_back(typename Key<KT>::T *uk, uint32_t *uv, const typename Key<KT>::T *sk,
                            const uint32_t *svb, long long n, const Ctrl *__restrict__ c,
                            int cur0, int passes) {
    if (call_mode(c, n) != MODE_SORT) return;
    if (buffer_before_pass(c, cur0, passes) == 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uk[i] = sk[i];
        if (VALS) uv[i] = svb[i];
    }
}

// --------------------------------------------------------------- host

static int grid_for(long long work, int per_block, int cap) {
    long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename F>
static sr_status allow_smem(F *kernel, size_t bytes) {
    if (bytes > 48 * 1024) {
        if (cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return launch_status();
    }
    return SR_OK;
}

template <int KT, bool VALS>
static sr_status sort_impl(void *d_keys, uint32_t *d_vals, size_t n, cudaStream_t s, int call) {
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    typedef Shape<sizeof(T), VALS> S;
    constexpr int NT = S::NT, IPT = S::IPT, SNT = S::SORT_NT;
    constexpr int NV = NT * IPT;    // keys per merge CTA
    constexpr int TS = SNT * IPT;   // keys per block-sort tile
    static_assert(TS % NV == 0, "sort tile must be a whole number of merge tiles");

    CallRecord &rec = call_record();
    rec = CallRecord();
    rec.host.call = call;
    rec.host.n = n;
    rec.host.key_type = KT;
    rec.host.tile = TS;
    rec.host.merge_tile = NV;
    rec.stream = s;
    rec.key_bytes = (int)sizeof(T);
    rec.val_bytes = VALS ? 4 : 0;
    if (n < 2) return SR_OK;

    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    const long long N = (long long)n;
    const long long tiles = (N + TS - 1) / TS;
    const int P = ceil_log2((unsigned long long)tiles);
    if (P > MAX_PASSES) return SR_ERR_UNSUPPORTED;
    const long long mtiles = (N + NV - 1) / NV;
    const size_t kbytes = align_up(n * sizeof(T), 256);
    const size_t vbytes = VALS ? align_up(n * 4, 256) : 0;
    const size_t sbytes = align_up((size_t)(mtiles + 1) * 8, 256);
    const size_t cbytes = align_up(sizeof(Ctrl), 256);
    void *scratch = nullptr;
    SR_TRY(scratch_alloc(ds, &scratch, (P > 0 ? kbytes + vbytes + sbytes : 0) + cbytes, s));
    unsigned char *sp = (unsigned char *)scratch;
    Ctrl *ctrl = (Ctrl *)sp;
    T *sk = (T *)(sp + cbytes);
    uint32_t *sv = (uint32_t *)(sp + cbytes + kbytes);
    long long *splits = (long long *)(sp + cbytes + kbytes + vbytes);
    T *uk = (T *)d_keys;
    uint32_t *uv = d_vals;
    const int cur0 = P & 1;          // the block sort writes where the last pass must not
    rec.cur0 = cur0;
    rec.host.passes_planned = P;

    sr_status st = SR_OK;
    do {
        if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) { st = launch_status(); break; }
        const size_t det_smem = (size_t)(TS + 1) * sizeof(U);
        if ((st = allow_smem(k_detect<KT, SNT, IPT>, det_smem)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT, det_smem, s,
                  uk, N, ctrl);
        SR_LAUNCH(SR_KERNEL_REVERSE, (k_reverse<KT, VALS>), grid_for(N / 2, 256, 152 * 16), 256, 0, s,
                  uk, uv, N, ctrl);
        const size_t bs_smem = (size_t)TS * (sizeof(U) + (VALS ? 4 : 0));
        if ((st = allow_smem(k_block_sort<KT, SNT, IPT, VALS>, bs_smem)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_BLOCK_SORT, (k_block_sort<KT, SNT, IPT, VALS>), (unsigned)tiles, SNT,
                  bs_smem, s, uk, uv, cur0 ? sk : uk, cur0 ? sv : uv, N, ctrl);
        const size_t m_smem = (size_t)NV * (sizeof(U) + (VALS ? 4 : 0));
        if ((st = allow_smem(k_merge<KT, NT, IPT, VALS>, m_smem)) != SR_OK) break;
        for (int p = 0; p < P; ++p) {
            const long long w = (long long)TS << p;
            const long long nb = mtiles + 1;
            SR_LAUNCH(SR_KERNEL_PARTITION, (k_partition<KT>), (unsigned)((nb + 255) / 256), 256, 0, s,
                      uk, sk, N, w, NV, nb, splits, ctrl, cur0, p);
            SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS>), (unsigned)mtiles, NT, m_smem, s,
                      uk, uv, sk, sv, N, w, splits, ctrl, cur0, p);
        }
        if (st != SR_OK) break;
        if (P > 0) {
            SR_LAUNCH(SR_KERNEL_COPY, (k_copy_back<KT, VALS>), grid_for(N, 256, 152 * 16), 256, 0, s,
                      uk, uv, sk, sv, N, ctrl, cur0, P);
        }
        if (cudaMemcpyAsync(ds->last_ctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess) {
            st = launch_status();
            break;
        }
        rec.has_ctrl = true;
    } while (0);
    scratch_free(scratch, s);
    return st;
}

template <bool VALS>
static sr_status dispatch_sort(void *d_keys, uint32_t *d_vals, size_t n, sr_key_type kt,
                               cudaStream_t s, int call) {
    switch (kt) {
    case SR_KEY_I32: return sort_impl<SR_KEY_I32, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_U32: return sort_impl<SR_KEY_U32, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_F32: return sort_impl<SR_KEY_F32, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_U64: return sort_impl<SR_KEY_U64, VALS>(d_keys, d_vals, n, s, call);
    case SR_KEY_I64: return sort_impl<SR_KEY_I64, VALS>(d_keys, d_vals, n, s, call);
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
        const size_t smem = (size_t)(TS + 1) * sizeof(typename K::U);
        if ((st = allow_smem(k_detect<KT, SNT, IPT>, smem)) != SR_OK) break;
        SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT, smem, s,
                  (const T *)d_keys, N, ctrl);
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
    return dispatch_sort<false>(d_keys, nullptr, n, kt, (cudaStream_t)stream, 1);
}

extern "C" sr_status sr_sort_pairs(void *d_keys, uint32_t *d_vals, size_t n, sr_key_type kt,
                                   sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && (!d_keys || !d_vals)) return SR_ERR_INVALID_ARG;
    if (n > 1 && (((uintptr_t)d_keys % key_bytes_of(kt)) != 0 || ((uintptr_t)d_vals % 4) != 0))
        return SR_ERR_INVALID_ARG;
    return dispatch_sort<true>(d_keys, d_vals, n, kt, (cudaStream_t)stream, 2);
}

extern "C" sr_status sr_sort_keys_host(void *h_keys, size_t n, sr_key_type kt, sr_stream stream) {
    if (!valid_key_type(kt)) return SR_ERR_INVALID_ARG;
    if (n > 1 && !h_keys) return SR_ERR_INVALID_ARG;
    if (n < 2) return SR_OK;
    DeviceState *ds = nullptr;
    SR_TRY(device_state(&ds));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = n * key_bytes_of(kt);
    void *d = nullptr;
    SR_TRY(scratch_alloc(ds, &d, bytes, s));
    sr_status st = SR_OK;
    if (cudaMemcpyAsync(d, h_keys, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) st = launch_status();
    if (st == SR_OK) st = dispatch_sort<false>(d, nullptr, n, kt, s, 1);
    if (st == SR_OK && cudaMemcpyAsync(h_keys, d, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = launch_status();
    scratch_free(d, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == SR_OK) st = launch_status();
    return st;
}

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
