// sr_plain.cuh -- the launch sequence of the plain sort over a given scratch
// area, shared by sr_sort_keys / sr_sort_pairs (pool scratch) and
// sr_sort_keys_noalloc (a fixed device array).
//
//   k_detect      run-detection scan: descents and non-descents (Run(A)).
//   k_few_sample  at most 64 distinct keys in a 4,096-key sample (4-byte
//                 keys only): k_few_count checks every key against them and
//                 counts each; if all were in the set, k_few_write writes the
//                 runs and nothing else runs.
//   k_reverse     strictly descending input: one reversal, nothing else runs.
//   k_rem_*       few displaced keys (keys only, when the plan asks for it;
//                 sr_rem.cuh): the keys left in order go straight to their
//                 block, the displaced ones through small per-tile buckets,
//                 and nothing else runs.
//   k_block_sort  tiles of SORT_NT*IPT keys sorted in shared memory (ascending
//                 tiles kept, strictly descending tiles reversed); records each
//                 tile's smallest and largest key.
//   k_plan        which merge passes have any run pair out of order.
//   per pass p    k_partition (merge-path splits of every output tile) and
//                 k_merge (policy e1); passes with every pair in order skip.
//                 The block sort and every merge record the first and last
//                 key of each merge tile they write; the next pass's split
//                 search runs over those samples first and reads keys only
//                 within one tile.
//   k_copy_back   if skipped passes left the result in scratch, copy it home.
#pragma once

#include "sr_device.cuh"
#include "sr_kernels.cuh"
#include "sr_rem.cuh"
#include "sr_runtime.cuh"

namespace sr {

template <int KT, bool VALS> struct PlainSort {
    typedef Key<KT> K;
    typedef typename K::T T;
    typedef typename K::U U;
    typedef Shape<sizeof(T), VALS> S;
    enum { NT = S::NT, IPT = S::IPT, SNT = S::SORT_NT, NV = S::NT * S::IPT, TS = S::SORT_NT * S::IPT };
    static_assert(TS % NV == 0, "sort tile must be a whole number of merge tiles");
    enum { LG_TS_NV = TS / NV == 1 ? 0 : TS / NV == 2 ? 1 : TS / NV == 4 ? 2 : TS / NV == 8 ? 3 : -1 };
    static_assert(LG_TS_NV >= 0, "merge tiles per sort tile must be a power of two up to 8");

    long long n = 0, tiles = 0, mtiles = 0;
    int passes = 0;
    bool rem = false;                  // the few-displaced-keys path is queued
    long long rem_dmax = 0;            // most descents for which it is tried
    long long rtiles = 0;              // its tiles of RT keys
    enum { RT = REM_TNT * IPT, RMIPT = IPT + (REM_CAP + REM_TNT - 1) / REM_TNT };
    static_assert((SNT * IPT) % RT == 0, "the scan's tile holds whole tiles of the displaced-keys path");
    static_assert(REM_TNT * RMIPT >= RT + REM_CAP, "a tile's block fits one merge tile");
    // byte offsets inside the scratch area
    size_t off_ctrl = 0, off_plan = 0, off_split = 0, off_samp = 0, off_keys = 0, off_vals = 0, bytes = 0;
    size_t off_rem_buck = 0, off_rem_bound = 0, off_rem_scount = 0, off_rem_bcount = 0, off_rem_blk = 0;

    // rem_: queue the few-displaced-keys path (keys only, at least
    // REM_MIN_TILES sort tiles).  Its tiles are RT = REM_TNT x IPT keys.
    enum { REM_MIN_TILES = 16 };
    explicit PlainSort(size_t n_, bool rem_ = false) {
        n = (long long)n_;
        tiles = (n + TS - 1) / TS;
        mtiles = (n + NV - 1) / NV;
        passes = ceil_log2((unsigned long long)(tiles > 0 ? tiles : 1));
        off_ctrl = 0;
        off_plan = align_up(sizeof(Ctrl), 256);
        const size_t plan_bytes = align_up((size_t)(2 * tiles + 2 * ((tiles + 1) / 2) + 2) * sizeof(U), 256);
        off_split = off_plan + plan_bytes;
        off_samp = off_split + align_up((size_t)(mtiles + 1) * 8, 256);
        // tile samples: one set per buffer (the caller's, the scratch copy)
        off_keys = off_samp + (SR_SPLIT_SAMPLES && passes > 0 ? align_up((size_t)(4 * mtiles) * sizeof(U), 256) : 0);
        const size_t kb = passes > 0 ? align_up((size_t)n * sizeof(T), 256) : 0;
        off_vals = off_keys + kb;
        const size_t vb = (VALS && passes > 0) ? align_up((size_t)n * 4, 256) : 0;
        bytes = off_vals + vb;
        rem = rem_ && !VALS && tiles >= REM_MIN_TILES && passes > 0;
        if (rem) {
            rem_dmax = n / 32;
            rtiles = (n + RT - 1) / RT;
            // the buckets follow the key buffer directly: one index space for the merge
            off_rem_buck = off_keys + kb;
            off_rem_bound = off_rem_buck + align_up((size_t)rtiles * REM_CAP * sizeof(T), 256);
            off_rem_scount = off_rem_bound + align_up((size_t)(rtiles + 1) * sizeof(U), 256);
            off_rem_bcount = off_rem_scount + align_up((size_t)rtiles * 4, 256);
            off_rem_blk = off_rem_bcount + align_up((size_t)rtiles * 4, 256);
            bytes = off_rem_blk + align_up((size_t)(rtiles + 1) * 8, 256);
        }
    }

    // Launches the whole sequence on stream s.  The block sort writes to the
    // scratch copy when the number of passes is odd, so the last merge lands in
    // the caller's buffer.
    // `gate` (optional device flag): when it is 0 at run time the whole
    // sequence does nothing.
    sr_status launch(T *uk, uint32_t *uv, unsigned char *scratch, cudaStream_t s,
                     const int *gate = nullptr) const {
        sr_status st = launch_prefix(uk, uv, scratch, s, gate);
        if (st == SR_OK) st = launch_sort(uk, uv, scratch, s);
        return st;
    }

    // The scan and the whole-input paths (sorted, strictly descending, few
    // distinct keys, few displaced keys): after them the call's mode is
    // final, and launch_sort's kernels all return at once unless it is
    // MODE_SORT.
    // Parts of the prefix, for a caller that routes between them on the device.
    enum { PART_SCAN = 1, PART_REVERSE = 2, PART_FEW = 4, PART_REM = 8, PART_ALL = 15 };
    sr_status launch_prefix(T *uk, uint32_t *uv, unsigned char *scratch, cudaStream_t s,
                            const int *gate = nullptr, int parts = PART_ALL) const {
        Ctrl *ctrl = (Ctrl *)(scratch + off_ctrl);
        T *sk = (T *)(scratch + off_keys);
        const bool vec = ((uintptr_t)uk % 16) == 0 && (!VALS || ((uintptr_t)uv % 16) == 0);
        sr_status st = SR_OK;
        do {
            U *rem_bound = rem ? (U *)(scratch + off_rem_bound) : nullptr;   // the scan records its medians
            constexpr bool FEW = sizeof(T) == 4 && !VALS && SR_FEW_KEYS;   // few distinct keys: written as runs
            if (parts & PART_SCAN) {
                if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) { st = launch_status(); break; }
                SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT, 0, s,
                          uk, n, ctrl, gate, rem_bound, (int)RT);
                if constexpr (FEW)
                    SR_LAUNCH(SR_KERNEL_DETECT, k_few_sample<KT>, FEW_SAMPLE / FEW_NT, FEW_NT, 0, s, uk, n, ctrl,
                              gate);
            }
            if (parts & PART_REVERSE)
                SR_LAUNCH(SR_KERNEL_REVERSE, (k_reverse<KT, VALS>), grid_for(n / 2, 256, 152 * 16), 256, 0, s,
                          uk, uv, n, ctrl);
            if constexpr (FEW) if (parts & PART_FEW) {
                SR_LAUNCH(SR_KERNEL_COPY, k_few_count<KT>, grid_for(n, 256, 152 * 8), 256, 0, s, uk, n, ctrl);
                SR_LAUNCH(SR_KERNEL_COPY, k_few_write<KT>, grid_for(n / 4 + 1, 256, 152 * 8), 256, 0, s, uk, n,
                          ctrl);
            }
            if constexpr (!VALS) if (rem && (parts & PART_REM)) {
                U *bound = rem_bound;
                unsigned int *scount = (unsigned int *)(scratch + off_rem_scount);
                unsigned int *bcount = (unsigned int *)(scratch + off_rem_bcount);
                long long *blk = (long long *)(scratch + off_rem_blk);
                T *buck = (T *)(scratch + off_rem_buck);
                const long long dofs = (long long)((off_rem_buck - off_keys) / sizeof(T));
                SR_LAUNCH(SR_KERNEL_DISPLACED, k_rem_bounds<KT>, 1, REM_NT, 0, s, n, rtiles, rem_dmax, ctrl, bound,
                          bcount);
                // grids of SR_REM_GRID CTAs per SM that loop over the tiles:
                // when the path is not taken, every CTA returns at once
                const unsigned rgrid = (unsigned)grid_for(rtiles, 1, 152 * SR_REM_GRID);
                const size_t sp_smem = (size_t)RT * (sizeof(U) + 1);
                SR_LAUNCH(SR_KERNEL_DISPLACED, (k_rem_split<KT, REM_TNT, IPT>), rgrid, REM_TNT, sp_smem, s, uk, n,
                          rtiles, ctrl, bound, sk, scount, buck, bcount);
                SR_LAUNCH(SR_KERNEL_DISPLACED, k_rem_bsort<KT>, rgrid + 1, REM_BSORT_NT, 0, s, buck, rtiles, ctrl,
                          scount, bcount, blk);
                const size_t rm_smem = merge_tile_smem<U, REM_TNT, RMIPT, false>();
                if ((st = allow_smem(k_rem_merge<KT, REM_TNT, RMIPT, true>, rm_smem)) != SR_OK) break;
                if ((st = allow_smem(k_rem_merge<KT, REM_TNT, RMIPT, false>, rm_smem)) != SR_OK) break;
                const long long n_src = dofs + rtiles * (long long)REM_CAP;
                if (vec) {
                    SR_LAUNCH(SR_KERNEL_DISPLACED, (k_rem_merge<KT, REM_TNT, RMIPT, true>), rgrid, REM_TNT, rm_smem,
                              s, uk, sk, n_src, dofs, (int)RT, rtiles, ctrl, scount, bcount, blk);
                } else {
                    SR_LAUNCH(SR_KERNEL_DISPLACED, (k_rem_merge<KT, REM_TNT, RMIPT, false>), rgrid, REM_TNT, rm_smem,
                              s, uk, sk, n_src, dofs, (int)RT, rtiles, ctrl, scount, bcount, blk);
                }
            }
        } while (0);
        (void)sk; (void)vec;
        return st;
    }

    // The block sort, the pass planner, the merge passes and the copy-back.
    sr_status launch_sort(T *uk, uint32_t *uv, unsigned char *scratch, cudaStream_t s) const {
        Ctrl *ctrl = (Ctrl *)(scratch + off_ctrl);
        U *plo = (U *)(scratch + off_plan);
        U *phi = plo + tiles;
        U *plo2 = phi + tiles;
        U *phi2 = plo2 + (tiles + 1) / 2 + 1;
        long long *splits = (long long *)(scratch + off_split);
        U *samp = SR_SPLIT_SAMPLES && passes > 0 ? (U *)(scratch + off_samp) : nullptr;
        T *sk = (T *)(scratch + off_keys);
        uint32_t *sv = (uint32_t *)(scratch + off_vals);
        const int P = passes;
        const int cur0 = P & 1;
        const bool vec = ((uintptr_t)uk % 16) == 0 && (!VALS || ((uintptr_t)uv % 16) == 0);
        sr_status st = SR_OK;
        do {
            const size_t bs_smem = (size_t)TS * (sizeof(U) + (VALS ? 4 : 0));
            if ((st = allow_smem(k_block_sort<KT, SNT, IPT, VALS>, bs_smem)) != SR_OK) break;
            SR_LAUNCH(SR_KERNEL_BLOCK_SORT, (k_block_sort<KT, SNT, IPT, VALS>), (unsigned)tiles, SNT,
                      bs_smem, s, uk, uv, cur0 ? sk : uk, cur0 ? sv : uv, n, ctrl, plo, phi,
                      samp ? samp + cur0 * 2 * mtiles : nullptr, (int)NV);
            if (P == 0) break;
            if ((tiles + PLAN_CHUNK - 1) / PLAN_CHUNK > PLAN_CHUNK) { st = SR_ERR_UNSUPPORTED; break; }
            SR_LAUNCH(SR_KERNEL_PARTITION, (k_plan<KT>), (unsigned)((tiles + PLAN_CHUNK - 1) / PLAN_CHUNK),
                      1024, 0, s, plo, phi, plo2, phi2, n, tiles, P, cur0, ctrl);
            const size_t m_smem = merge_tile_smem<U, NT, IPT, VALS>();
            if ((st = allow_smem(k_merge<KT, NT, IPT, VALS, true>, m_smem)) != SR_OK) break;
            if ((st = allow_smem(k_merge<KT, NT, IPT, VALS, false>, m_smem)) != SR_OK) break;
            for (int p = 0; p < P; ++p) {
                const long long w = (long long)TS << p;
                const int lgt = LG_TS_NV + 1 + p;          // merge tiles per run pair: 2w / NV
                const long long nb = mtiles + 1;
                const int lg = partition_lg(nb);
                SR_LAUNCH(SR_KERNEL_PARTITION, (k_partition<KT>), (unsigned)(((nb << lg) + 255) / 256), 256, 0,
                          s, uk, sk, n, w, NV, nb, splits, ctrl, p, lg, samp, 2 * mtiles);
                if (vec) {
                    SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS, true>), (unsigned)mtiles, NT,
                              m_smem, s, uk, uv, sk, sv, n, w, lgt, splits, ctrl, p, samp, 2 * mtiles);
                } else {
                    SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS, false>), (unsigned)mtiles, NT,
                              m_smem, s, uk, uv, sk, sv, n, w, lgt, splits, ctrl, p, samp, 2 * mtiles);
                }
            }
            if (st != SR_OK) break;
            SR_LAUNCH(SR_KERNEL_COPY, (k_copy_back<KT, VALS>), grid_for(n, 256, 152 * 16), 256, 0, s,
                      uk, uv, sk, sv, n, ctrl, P);
        } while (0);
        return st;
    }

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
};

}  // namespace sr
