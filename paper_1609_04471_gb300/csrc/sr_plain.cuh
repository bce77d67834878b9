// sr_plain.cuh -- the launch sequence of the plain sort over a given scratch
// area, shared by sr_sort_keys / sr_sort_pairs (pool scratch) and
// sr_sort_keys_noalloc (a fixed device array).
//
//   k_detect      run-detection scan: descents and non-descents (Run(A)).
//   k_few_sample  at most 4,096 distinct keys in a 65,536-key sample (4-byte
//                 keys only): k_few_count checks every key against them and
//                 counts each; if all were in the set, k_few_write writes the
//                 runs and nothing else runs.
//   k_reverse     strictly descending input: one reversal, nothing else runs.
//   k_rem_*       few displaced keys (keys only, when the plan asks for it;
//                 sr_rem.cuh): the keys left in order go straight to their
//                 block, the displaced ones through small per-tile buckets,
//                 and nothing else runs.
//   k_tile_order  chains of whole tiles in descending order (technique (a) at
//                 tile level, from the scan's per-tile extremes): the block
//                 sort writes them in reversed tile order.
//   k_block_sort  tiles of SORT_NT*IPT keys sorted in shared memory (ascending
//                 tiles kept, strictly descending tiles reversed); records each
//                 tile's smallest and largest key.
//   k_runs        the natural runs of whole tiles (a tile continues the run
//                 before it when that run's last key is <= its first) and the
//                 merge steps they need: ceil(log_f(runs)) for fan-in f.
//   k_repair_plan when only neighbouring tiles overlap (every tile's keys are
//   k_repair      <= those of the tile two places on): the window of keys out
//                 of order at each tile boundary, merged in place; then no
//                 merge step runs (a window larger than a merge tile cancels
//                 this and the steps run).
//   per step s    groups of f consecutive runs of the step before merged into
//                 one (policy e1 over the input's own runs).  2-way steps:
//                 k_partition (merge-path split of every output tile) and
//                 k_merge.  4-way steps: k_partition (2-way splits of every
//                 merge tile of the merged pairs AB and CD), k_partition4
//                 (4-way splits of every output tile) and k_merge4.  Steps past
//                 the ones the runs need return at once.  The block sort and
//                 every merge record the first and last key of each merge
//                 tile they write; the next step's split search runs over
//                 those samples first and reads keys only within one tile.
//   k_copy_back   if the last step left the result in scratch, copy it home.
#pragma once

#include <cstdlib>

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
    // few distinct keys: written as runs (4-byte keys alone)
    static constexpr bool FEW_PATH = sizeof(T) == 4 && !VALS && SR_FEW_KEYS;
    enum { LG_TS_NV = TS / NV == 1 ? 0 : TS / NV == 2 ? 1 : TS / NV == 4 ? 2 : TS / NV == 8 ? 3 : -1 };
    static_assert(LG_TS_NV >= 0, "merge tiles per sort tile must be a power of two up to 8");

    // Where each part of a call's scratch lies (byte offsets) and its size;
    // a compile-time function of n so that a fixed scratch area can be sized
    // and checked at build time.
    struct Layout {
        long long n, tiles, mtiles, rtiles, rem_dmax;
        int levels, steps;
        bool rem;
        size_t off_ctrl, off_plan, off_runs, off_win, off_split, off_split4, off_few, off_fewhist, off_samp, off_keys,
            off_vals;
        size_t off_rem_buck, off_rem_bound, off_rem_scount, off_rem_bcount, off_rem_blk, bytes;
    };
    static constexpr size_t up256(size_t x) { return (x + 255) / 256 * 256; }
    static constexpr int clog2(unsigned long long x) {
        int r = 0;
        while ((1ull << r) < x) ++r;
        return r;
    }
    static constexpr Layout layout(long long n_, bool rem_, bool fan4_) {
        Layout L{};
        L.n = n_;
        L.tiles = (n_ + TS - 1) / TS;
        L.mtiles = (n_ + NV - 1) / NV;
        L.levels = clog2((unsigned long long)(L.tiles > 0 ? L.tiles : 1));
        L.steps = merge_step_count(L.levels, fan4_);
        const bool merging = L.levels > 0;
        L.off_ctrl = 0;
        L.off_plan = up256(sizeof(Ctrl));
        const size_t plan_bytes = up256((size_t)(2 * L.tiles) * sizeof(U));
        L.off_runs = L.off_plan + plan_bytes;
        L.off_win = L.off_runs + up256((size_t)(L.tiles + 1) * 4);
        L.off_split = L.off_win + up256((size_t)(2 * L.tiles) * 4);
        L.off_split4 = L.off_split + up256((size_t)(L.mtiles + 1) * 32);
        const size_t split4_bytes = fan4_ && L.steps > 0 ? up256((size_t)(L.mtiles + 1) * 64) : 0;
        L.off_few = L.off_split4 + split4_bytes;
        L.off_fewhist = L.off_few + (FEW_PATH ? up256(sizeof(FewTables)) : 0);
        L.off_samp = L.off_fewhist + (FEW_PATH ? up256((size_t)FEW_COUNT_CTAS * FEW_MAX * 4) : 0);
        // tile samples: one set per buffer (the caller's, the scratch copy)
        L.off_keys = L.off_samp + (SR_SPLIT_SAMPLES && merging ? up256((size_t)(4 * L.mtiles) * sizeof(U)) : 0);
        const size_t kb = merging ? up256((size_t)n_ * sizeof(T)) : 0;
        L.off_vals = L.off_keys + kb;
        const size_t vb = (VALS && merging) ? up256((size_t)n_ * 4) : 0;
        L.bytes = L.off_vals + vb;
        L.rem = rem_ && !VALS && L.tiles >= REM_MIN_TILES && merging;
        if (L.rem) {
            L.rem_dmax = n_ / 32;
            L.rtiles = (n_ + RT - 1) / RT;
            // the buckets follow the key buffer directly: one index space for the merge
            L.off_rem_buck = L.off_keys + kb;
            L.off_rem_bound = L.off_rem_buck + up256((size_t)L.rtiles * REM_CAP * sizeof(T));
            L.off_rem_scount = L.off_rem_bound + up256((size_t)(L.rtiles + 1) * sizeof(U));
            L.off_rem_bcount = L.off_rem_scount + up256((size_t)L.rtiles * 4);
            L.off_rem_blk = L.off_rem_bcount + up256((size_t)L.rtiles * 4);
            L.bytes = L.off_rem_blk + up256((size_t)(L.rtiles + 1) * 8);
        }
        return L;
    }

    // Every region of the layout holds what the kernels write there: the tile
    // extremes (2 per tile), the run table (tiles + 1), the 2-way split table
    // (4 per boundary) and, when 4-way steps run, the 4-way one (8 per
    // boundary), the merge-tile samples (2 per merge tile and buffer), the
    // key and value copies; regions are in that order and do not overlap.
    static constexpr bool layout_ok(long long n_, bool rem_, bool fan4_) {
        const Layout L = layout(n_, rem_, fan4_);
        if (L.off_plan < sizeof(Ctrl)) return false;
        if (L.off_plan + (size_t)(2 * L.tiles) * sizeof(U) > L.off_runs) return false;
        if (L.off_runs + (size_t)(L.tiles + 1) * 4 > L.off_win) return false;
        if (L.off_win + (size_t)(2 * L.tiles) * 4 > L.off_split) return false;
        if (L.off_split + (size_t)(L.mtiles + 1) * 32 > L.off_split4) return false;
        if (fan4_ && L.steps > 0 && L.off_split4 + (size_t)(L.mtiles + 1) * 64 > L.off_few) return false;
        if (FEW_PATH && L.off_few + sizeof(FewTables) > L.off_fewhist) return false;
        if (FEW_PATH && L.off_fewhist + (size_t)FEW_COUNT_CTAS * FEW_MAX * 4 > L.off_samp) return false;
        if (SR_SPLIT_SAMPLES && L.levels > 0 && L.off_samp + (size_t)(4 * L.mtiles) * sizeof(U) > L.off_keys)
            return false;
        if (L.levels > 0 && L.off_keys + (size_t)n_ * sizeof(T) > L.off_vals) return false;
        if (VALS && L.levels > 0 && L.off_vals + (size_t)n_ * 4 > (L.rem ? L.off_rem_buck : L.bytes)) return false;
        return true;
    }
    static constexpr bool layouts_ok() {
        const long long ns[] = {2, NV - 1, NV + 1, TS - 1, TS, TS + 1, 2 * TS - 1, 2 * TS + 3, 3 * TS + 5,
                                4 * TS, 4 * TS + 1, 5 * TS + 7, 17 * TS + 1, 65 * TS + 3, 1000 * TS + 7};
        for (long long n_ : ns)
            for (int r = 0; r < 2; ++r)
                for (int f = 0; f < 2; ++f)
                    if (!layout_ok(n_, r == 1, f == 1)) return false;
        return true;
    }

    long long n = 0, tiles = 0, mtiles = 0;
    int passes = 0;                    // binary merge levels after the block sort
    int steps = 0;                     // merge steps that cover them
    bool fan4 = true;                  // 4-way steps
    bool rem = false;                  // the few-displaced-keys path is queued
    long long rem_dmax = 0;            // most descents for which it is tried
    long long rtiles = 0;              // its tiles of RT keys
    int sms = 152;                     // SMs of the device (grid sizes of grid-stride kernels)
    int *status = nullptr;             // device status word for errors found on the device
    enum { RT = REM_TNT * IPT, RMIPT = IPT + (REM_CAP + REM_TNT - 1) / REM_TNT };
    static_assert((SNT * IPT) % RT == 0, "the scan's tile holds whole tiles of the displaced-keys path");
    static_assert(REM_TNT * RMIPT >= RT + REM_CAP, "a tile's block fits one merge tile");
    // byte offsets inside the scratch area
    size_t off_ctrl = 0, off_plan = 0, off_runs = 0, off_win = 0, off_split = 0, off_split4 = 0, off_few = 0,
           off_fewhist = 0, off_samp = 0, off_keys = 0, off_vals = 0, bytes = 0;
    size_t off_rem_buck = 0, off_rem_bound = 0, off_rem_scount = 0, off_rem_bcount = 0, off_rem_blk = 0;

    // rem_: queue the few-displaced-keys path (keys only, at least
    // REM_MIN_TILES sort tiles).  Its tiles are RT = REM_TNT x IPT keys.
    // fan4_: merge four runs per step (else two).
    enum { REM_MIN_TILES = 16 };
    explicit PlainSort(size_t n_, bool rem_ = false, bool fan4_ = default_fan4()) {
        static_assert(layouts_ok(), "scratch layout regions too small or overlapping");
        const Layout L = layout((long long)n_, rem_, fan4_);
        n = L.n; tiles = L.tiles; mtiles = L.mtiles; passes = L.levels; steps = L.steps; fan4 = fan4_;
        rem = L.rem; rem_dmax = L.rem_dmax; rtiles = L.rtiles;
        off_ctrl = L.off_ctrl; off_plan = L.off_plan; off_runs = L.off_runs; off_win = L.off_win;
        off_split = L.off_split;
        off_split4 = L.off_split4; off_few = L.off_few; off_fewhist = L.off_fewhist;
        off_samp = L.off_samp; off_keys = L.off_keys; off_vals = L.off_vals; bytes = L.bytes;
        off_rem_buck = L.off_rem_buck; off_rem_bound = L.off_rem_bound; off_rem_scount = L.off_rem_scount;
        off_rem_bcount = L.off_rem_bcount; off_rem_blk = L.off_rem_blk;
        sms = device_sm_count();
    }

    // Merge fan-in per key shape, as measured on GB300: 4-way steps where a
    // step moves enough bytes per key to be bound by HBM (payloads, 8-byte
    // keys), 2-way steps for 4-byte keys alone, whose 2-way merge already runs
    // near the HBM roofline while the 4-way one is bound by instruction issue.
    // SORTRACE_MERGE_FANIN = "2" or "4" (read once) forces one for measuring.
    static bool default_fan4() {
        static const int forced = [] {
            const char *e = std::getenv("SORTRACE_MERGE_FANIN");
            return e && e[0] == '2' ? 2 : (e && e[0] == '4' ? 4 : 0);
        }();
        if (forced) return forced == 4;
        return VALS || sizeof(T) == 8;
    }
    // How a 2-way tile stages its windows when the arrays are 16-byte
    // aligned: 1-D bulk copies (measured faster on GB300: 2^28 int32 merge
    // steps 6.08 -> 5.81 ms), unless SORTRACE_MERGE2_STAGE is "vec" (16-byte
    // loads through registers).
    static int stage2() {
        static const int m = [] {
            const char *e = std::getenv("SORTRACE_MERGE2_STAGE");
            return (e && e[0] == 'v') ? (int)STAGE_VEC : (int)STAGE_BULK;
        }();
        return m;
    }
    // How a 4-way tile stages its windows when the arrays are 16-byte
    // aligned: 1-D bulk copies, unless SORTRACE_MERGE4_STAGE is "vec" (16-byte
    // loads through registers).
    static int stage4() {
        static const int m = [] {
            const char *e = std::getenv("SORTRACE_MERGE4_STAGE");
            return (e && e[0] == 'v') ? (int)STAGE_VEC : (int)STAGE_BULK;
        }();
        return m;
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
            constexpr bool FEW = FEW_PATH;
            FewTables *few = FEW ? (FewTables *)(scratch + off_few) : nullptr;
            if (parts & PART_SCAN) {
                if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) { st = launch_status(); break; }
                if (FEW && cudaMemsetAsync(few, 0, sizeof(FewTables), s) != cudaSuccess) {
                    st = launch_status();
                    break;
                }
                // the scan also records every tile's smallest and largest key
                // (for k_tile_order), where the block sort later puts its own
                U *plo = passes > 0 ? (U *)(scratch + off_plan) : nullptr;
                SR_LAUNCH(SR_KERNEL_DETECT, (k_detect<KT, SNT, IPT>), (unsigned)tiles, SNT, 0, s,
                          uk, n, ctrl, gate, rem_bound, (int)RT, plo, plo ? plo + tiles : nullptr);
                if constexpr (FEW) {
                    if ((st = allow_smem(k_few_sample<KT>, (size_t)FEW_A_SLOTS * 8)) != SR_OK) break;
                    SR_LAUNCH(SR_KERNEL_DETECT, k_few_sample<KT>, 1, FEW_NT2, (size_t)FEW_A_SLOTS * 8, s, uk, n, ctrl,
                              few, gate);
                    SR_LAUNCH(SR_KERNEL_DETECT, k_few_sample2<KT>, (FEW_SAMPLE - FEW_SAMPLE_A) / FEW_NT2, FEW_NT2, 0,
                              s, uk, n, ctrl, few, gate);
                }
            }
            if (parts & PART_REVERSE)
                SR_LAUNCH(SR_KERNEL_REVERSE, (k_reverse<KT, VALS>), grid_for(n / 2, 256, sms * 16), 256, 0, s,
                          uk, uv, n, ctrl);
            if constexpr (FEW) if (parts & PART_FEW) {
                unsigned int *hist = (unsigned int *)(scratch + off_fewhist);
                const int rows = grid_for(n / 4 + 1, FEW_COUNT_NT, sms < FEW_COUNT_CTAS ? sms : FEW_COUNT_CTAS);
                if ((st = allow_smem(k_few_count<KT>, few_count_smem())) != SR_OK) break;
                SR_LAUNCH(SR_KERNEL_COPY, k_few_count<KT>, rows, FEW_COUNT_NT, few_count_smem(), s, uk, n, ctrl, few,
                          hist);
                SR_LAUNCH(SR_KERNEL_COPY, k_few_reduce, FEW_MAX / 256, 256, 0, s, hist, rows, ctrl, few);
                SR_LAUNCH(SR_KERNEL_COPY, k_few_write<KT>, grid_for(n / 4 + 1, 256, sms * 4), 256, 0, s, uk, n,
                          ctrl, few);
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
                const unsigned rgrid = (unsigned)grid_for(rtiles, 1, sms * SR_REM_GRID);
                const size_t sp_smem = (size_t)RT * (sizeof(U) + 1);
                SR_LAUNCH(SR_KERNEL_DISPLACED, (k_rem_split<KT, REM_TNT, IPT>), rgrid, REM_TNT, sp_smem, s, uk, n,
                          rtiles, ctrl, bound, sk, scount, buck, bcount);
                SR_LAUNCH(SR_KERNEL_DISPLACED, k_rem_bsort<KT>, rgrid + 1, REM_BSORT_NT, 0, s, buck, rtiles, ctrl,
                          scount, bcount, blk);
                const size_t rm_smem = merge_tile_smem<U, REM_TNT, RMIPT, false>();
                if ((st = allow_smem(k_rem_merge<KT, REM_TNT, RMIPT, true>, rm_smem)) != SR_OK) break;
                if ((st = allow_smem(k_rem_merge<KT, REM_TNT, RMIPT, false>, rm_smem)) != SR_OK) break;
                const long long n_src = dofs + rtiles * (long long)REM_CAP;
                int *st_word = status ? status : &ctrl->status;
                if (vec) {
                    SR_LAUNCH(SR_KERNEL_DISPLACED, (k_rem_merge<KT, REM_TNT, RMIPT, true>), rgrid, REM_TNT, rm_smem,
                              s, uk, sk, n_src, dofs, (int)RT, rtiles, ctrl, scount, bcount, blk, st_word);
                } else {
                    SR_LAUNCH(SR_KERNEL_DISPLACED, (k_rem_merge<KT, REM_TNT, RMIPT, false>), rgrid, REM_TNT, rm_smem,
                              s, uk, sk, n_src, dofs, (int)RT, rtiles, ctrl, scount, bcount, blk, st_word);
                }
            }
        } while (0);
        (void)sk; (void)vec;
        return st;
    }

    // The block sort, the run planner, the merge steps and the copy-back.
    sr_status launch_sort(T *uk, uint32_t *uv, unsigned char *scratch, cudaStream_t s) const {
        Ctrl *ctrl = (Ctrl *)(scratch + off_ctrl);
        U *plo = (U *)(scratch + off_plan);
        U *phi = plo + tiles;
        int *runs = (int *)(scratch + off_runs);
        int *win = (int *)(scratch + off_win);
        long long *splits = (long long *)(scratch + off_split);
        long long *splits4 = (long long *)(scratch + off_split4);
        U *samp = SR_SPLIT_SAMPLES && passes > 0 ? (U *)(scratch + off_samp) : nullptr;
        T *sk = (T *)(scratch + off_keys);
        uint32_t *sv = (uint32_t *)(scratch + off_vals);
        const int cur0 = steps & 1;                 // when every step runs, the last lands in the caller's buffer
        const bool vec = ((uintptr_t)uk % 16) == 0 && (!VALS || ((uintptr_t)uv % 16) == 0);
        int *st_word = status ? status : &ctrl->status;
        sr_status st = SR_OK;
        do {
            int *dest = win;                        // free until the repair planner runs
            if (passes > 0)
                SR_LAUNCH(SR_KERNEL_PARTITION, (k_tile_order<KT>), 1, RUNS_NT, 0, s, plo, phi, n, (long long)TS,
                          tiles, VALS ? 1 : 0, dest, ctrl);
            const size_t bs_smem =
                SR_BSORT_PP == 2 ? (size_t)block_sort_pp_keys<SNT, IPT>() * (sizeof(U) + (VALS ? 4 : 0))
                : (!VALS && sizeof(U) == 4 && SR_BSORT_PP == 1) ? (size_t)2 * block_sort_pp_keys<SNT, IPT>() * sizeof(U)
                                                                : (size_t)TS * (sizeof(U) + (VALS ? 4 : 0));
            if ((st = allow_smem(k_block_sort<KT, SNT, IPT, VALS>, bs_smem)) != SR_OK) break;
            SR_LAUNCH(SR_KERNEL_BLOCK_SORT, (k_block_sort<KT, SNT, IPT, VALS>), (unsigned)tiles, SNT,
                      bs_smem, s, uk, uv, cur0 ? sk : uk, cur0 ? sv : uv, sk, sv, n, ctrl, plo, phi, samp,
                      (long long)2 * mtiles, (int)NV, passes > 0 ? dest : nullptr);
            if (passes == 0) break;
            const int fan = fan4 ? 4 : 2;
            SR_LAUNCH(SR_KERNEL_PARTITION, (k_runs<KT>), 1, RUNS_NT, 0, s, plo, phi, n, tiles, fan, cur0, runs, ctrl);
            if (tiles >= 3) {                       // neighbour repair, when only neighbouring tiles overlap
                SR_LAUNCH(SR_KERNEL_PARTITION, (k_repair_plan<KT>), (unsigned)((tiles + 255) / 256), 256, 0, s,
                          uk, sk, plo, phi, n, (long long)TS, tiles, (int)NV, win, ctrl);
                const size_t r_smem = merge_tile_smem<U, NT, IPT, VALS>();
                if ((st = allow_smem(k_repair<KT, NT, IPT, VALS>, r_smem)) != SR_OK) break;
                SR_LAUNCH(SR_KERNEL_DISPLACED, (k_repair<KT, NT, IPT, VALS>), (unsigned)(tiles - 1), NT, r_smem, s,
                          uk, uv, sk, sv, n, (long long)TS, tiles, win, ctrl);
            }
            const size_t m_smem = merge_tile_smem<U, NT, IPT, VALS>();
            const size_t m4_smem = merge4_smem<U, NT, IPT, VALS>();
            const int mode4 = vec ? stage4() : (int)STAGE_SCALAR;
            const long long nb = mtiles + 1;
            const int lg = partition_lg(nb);
            const int lg4 = partition4_lg(nb);
            long long span = 1;                     // natural runs per run of this step's input
            for (int step = 0; step < steps; ++step, span *= fan) {
                SR_LAUNCH(SR_KERNEL_PARTITION, (k_partition<KT>), (unsigned)(((nb << lg) + 255) / 256), 256, 0,
                          s, uk, sk, n, (long long)TS, tiles, NV, nb, splits, runs, span, ctrl, step, lg, samp,
                          2 * mtiles);
                if (!fan4) {
                    const int mode2 = vec ? stage2() : (int)STAGE_SCALAR;
                    if (mode2 == STAGE_BULK) {
                        if ((st = allow_smem(k_merge<KT, NT, IPT, VALS, STAGE_BULK>, m_smem)) != SR_OK) break;
                        SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS, STAGE_BULK>), (unsigned)mtiles, NT,
                                  m_smem, s, uk, uv, sk, sv, n, splits, ctrl, step, samp, 2 * mtiles, st_word);
                    } else if (mode2 == STAGE_VEC) {
                        if ((st = allow_smem(k_merge<KT, NT, IPT, VALS, STAGE_VEC>, m_smem)) != SR_OK) break;
                        SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS, STAGE_VEC>), (unsigned)mtiles, NT,
                                  m_smem, s, uk, uv, sk, sv, n, splits, ctrl, step, samp, 2 * mtiles, st_word);
                    } else {
                        if ((st = allow_smem(k_merge<KT, NT, IPT, VALS, STAGE_SCALAR>, m_smem)) != SR_OK) break;
                        SR_LAUNCH(SR_KERNEL_MERGE, (k_merge<KT, NT, IPT, VALS, STAGE_SCALAR>), (unsigned)mtiles, NT,
                                  m_smem, s, uk, uv, sk, sv, n, splits, ctrl, step, samp, 2 * mtiles, st_word);
                    }
                    continue;
                }
                SR_LAUNCH(SR_KERNEL_PARTITION, (k_partition4<KT>), (unsigned)(((nb << lg4) + 255) / 256), 256, 0,
                          s, uk, sk, n, (long long)TS, tiles, NV, nb, splits, splits4, runs, span, ctrl, step, lg4);
                if (mode4 == STAGE_BULK) {
                    if ((st = allow_smem(k_merge4<KT, NT, IPT, VALS, STAGE_BULK>, m4_smem)) != SR_OK) break;
                    SR_LAUNCH(SR_KERNEL_MERGE, (k_merge4<KT, NT, IPT, VALS, STAGE_BULK>), (unsigned)mtiles, NT,
                              m4_smem, s, uk, uv, sk, sv, n, splits4, ctrl, step, samp, 2 * mtiles, st_word);
                } else if (mode4 == STAGE_VEC) {
                    if ((st = allow_smem(k_merge4<KT, NT, IPT, VALS, STAGE_VEC>, m4_smem)) != SR_OK) break;
                    SR_LAUNCH(SR_KERNEL_MERGE, (k_merge4<KT, NT, IPT, VALS, STAGE_VEC>), (unsigned)mtiles, NT,
                              m4_smem, s, uk, uv, sk, sv, n, splits4, ctrl, step, samp, 2 * mtiles, st_word);
                } else {
                    if ((st = allow_smem(k_merge4<KT, NT, IPT, VALS, STAGE_SCALAR>, m4_smem)) != SR_OK) break;
                    SR_LAUNCH(SR_KERNEL_MERGE, (k_merge4<KT, NT, IPT, VALS, STAGE_SCALAR>), (unsigned)mtiles, NT,
                              m4_smem, s, uk, uv, sk, sv, n, splits4, ctrl, step, samp, 2 * mtiles, st_word);
                }
            }
            if (st != SR_OK) break;
            SR_LAUNCH(SR_KERNEL_COPY, (k_copy_back<KT, VALS>), grid_for(n, 256, sms * 16), 256, 0, s,
                      uk, uv, sk, sv, n, ctrl);
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
