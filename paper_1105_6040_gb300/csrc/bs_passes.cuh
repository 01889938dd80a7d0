// bs_passes.cuh -- host-side launch sequence of one sort (templated on the
// key code type and value type); instantiated per key width in bs_u32.cu /
// bs_u64.cu.  The sort phase's tile shape (THREADS x KPT keys) and the merge
// passes' tile shape (MT x MVT keys, at most the sort tile) are chosen
// independently.
#pragma once

#include <atomic>

#include "bs_internal.h"

namespace bs {

template <class Kern> static int resident_ctas(Kern kern, int threads, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

// Lets `kern` use `smem` bytes of dynamic shared memory and asks for the
// largest shared-memory carveout, so that as many CTAs are resident as the
// occupancy calculator (which the persistent grids are sized by) assumes.
template <class Kern> static bool allow_smem(Kern kern, size_t smem) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        cudaGetLastError();  // a hint only
    if (smem <= 48 * 1024) return true;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
           cudaSuccess;
}

static inline int64_t grid_for(int64_t work, int64_t resident) {
    int64_t g = work < resident ? work : resident;
    return g < 1 ? 1 : g;
}

// Shared memory a CTA may use while still leaving room for a second CTA.
constexpr size_t TMA_SMEM_AUTO_LIMIT = 112 * 1024;
constexpr int MERGE_STAGES = 2;  // stages of the TMA merge pipeline
constexpr size_t SMEM_OPT_IN_LIMIT = 227 * 1024;
constexpr int PART_THREADS = 256;  // partition threads per CTA

// The TMA merge pipeline at shape (MT consumer threads, MVT keys each):
// launches it and returns 1, or returns 0 when it cannot run here (shared
// memory, or above the automatic limit) so the caller runs the plain kernel.
template <class K, class V, int MT, int MVT>
int launch_merge_tma(const PassArgs &a, Launcher &L, const Level &lvl, int64_t tiles) {
    const int ci = a.merge_consumer == 1 ? 1 : 0;  // 1: warp bitonic consumers
    auto mt = ci ? merge_tma_kernel<K, V, MT, MVT, MERGE_STAGES, true>
                 : merge_tma_kernel<K, V, MT, MVT, MERGE_STAGES, false>;
    constexpr size_t msmem = tma_smem_bytes<K, V, MT, MVT, MERGE_STAGES, true>();
    static std::atomic<int> occ_mt[2] = {{0}, {0}};
    if (!occ_mt[ci].load()) {
        if (msmem <= SMEM_OPT_IN_LIMIT && allow_smem(mt, msmem))
            occ_mt[ci].store(resident_ctas(mt, MT + 32, msmem));
        else
            occ_mt[ci].store(-1);
    }
    if (occ_mt[ci].load() <= 0) return 0;
    if (a.merge_impl == MERGE_AUTO && msmem > TMA_SMEM_AUTO_LIMIT) return 0;
    const Geo &g = a.g;
    launch_overlapped(mt, (unsigned)grid_for(tiles, (int64_t)L.sms * occ_mt[ci]), MT + 32, msmem, L.stream, g,
                      lvl, (K *)a.k0, (K *)a.k1, (V *)a.v0, (V *)a.v1, a.codec, (const int64_t *)a.split,
                      a.ntiles_total);
    return 1;
}

// The plain merge kernel (any alignment, any item size) at shape (MT, MVT).
template <class K, class V, int MT, int MVT>
bool launch_merge_plain(const PassArgs &a, Launcher &L, const Level &lvl, int64_t tiles) {
    constexpr size_t smem = smem_bytes<K, V>(MT * MVT);
    auto mk = merge_kernel<K, V, MT, MVT>;
    static std::atomic<int> occ_mk{0};
    if (!occ_mk.load()) {
        if (!allow_smem(mk, smem)) return false;
        occ_mk.store(resident_ctas(mk, MT, smem));
    }
    const Geo &g = a.g;
    launch_overlapped(mk, (unsigned)grid_for(tiles, (int64_t)L.sms * occ_mk), MT, smem, L.stream, g, lvl,
                      (K *)a.k0, (K *)a.k1, (V *)a.v0, (V *)a.v1, a.codec, (const int64_t *)a.split,
                      a.ntiles_total);
    return true;
}

// Keys per consumer thread of the TMA merge: the option, else 32 for 32-bit
// keys alone and 16 for wider items (register budget).
template <class K, class V> int merge_vt_of(const PassArgs &a) {
    if (a.merge_vt) return a.merge_vt;
    return (sizeof(K) == 4 && !HasVal<V>::value) ? 32 : 16;
}

// Shared memory of the TMA merge pipeline for the shape merge_pass_any runs
// at merge tile 2^mlogT with vt keys per consumer thread.
template <class K, class V> size_t tma_bytes_at(int mlogT, int vt) {
    switch (mlogT) {
    case 11:
        return vt == 8    ? tma_smem_bytes<K, V, 256, 8, MERGE_STAGES, true>()
               : vt == 16 ? tma_smem_bytes<K, V, 128, 16, MERGE_STAGES, true>()
                          : tma_smem_bytes<K, V, 64, 32, MERGE_STAGES, true>();
    case 12:
        return vt == 8    ? tma_smem_bytes<K, V, 512, 8, MERGE_STAGES, true>()
               : vt == 16 ? tma_smem_bytes<K, V, 256, 16, MERGE_STAGES, true>()
                          : tma_smem_bytes<K, V, 128, 32, MERGE_STAGES, true>();
    default:
        return vt == 32 ? tma_smem_bytes<K, V, 256, 32, MERGE_STAGES, true>()
                        : tma_smem_bytes<K, V, 512, 16, MERGE_STAGES, true>();
    }
}

// One merge pass with merge tiles of 2^mlogT keys: merge-path splits, then
// the TMA pipeline (shape by keys per consumer thread: 8, 16 or 32; 8 is
// not offered for 8192-key tiles) where allowed and it fits, else the plain
// kernel at 16 keys per thread.
template <class K, class V>
bool merge_pass_any(const PassArgs &a, Launcher &L, const Level &lvl, int64_t tiles) {
    const Geo &g = a.g;
    L.begin(L.owner, CLS_PARTITION, L.stream);
    launch_overlapped(partition_kernel<K>,
                      (unsigned)grid_for((tiles + PART_THREADS - 1) / PART_THREADS, (int64_t)L.sms * 8),
                      PART_THREADS, 0, L.stream, g, lvl, (const K *)a.k0, (const K *)a.k1, a.split,
                      a.ntiles_total);
    if (!L.end(L.owner, CLS_PARTITION, L.stream)) return false;
    L.begin(L.owner, CLS_MERGE, L.stream);
    int done = 0;
    if (a.merge_impl != MERGE_SIMPLE) {
        const int vt = merge_vt_of<K, V>(a);
        switch (lvl.mlogT) {
        case 11:
            done = vt == 8    ? launch_merge_tma<K, V, 256, 8>(a, L, lvl, tiles)
                   : vt == 16 ? launch_merge_tma<K, V, 128, 16>(a, L, lvl, tiles)
                              : launch_merge_tma<K, V, 64, 32>(a, L, lvl, tiles);
            break;
        case 12:
            done = vt == 8    ? launch_merge_tma<K, V, 512, 8>(a, L, lvl, tiles)
                   : vt == 16 ? launch_merge_tma<K, V, 256, 16>(a, L, lvl, tiles)
                              : launch_merge_tma<K, V, 128, 32>(a, L, lvl, tiles);
            break;
        case 13:
            done = vt == 32 ? launch_merge_tma<K, V, 256, 32>(a, L, lvl, tiles)
                            : launch_merge_tma<K, V, 512, 16>(a, L, lvl, tiles);
            break;
        default: return false;
        }
    }
    if (!done) {
        bool ok;
        switch (lvl.mlogT) {
        case 11: ok = launch_merge_plain<K, V, 128, 16>(a, L, lvl, tiles); break;
        case 12: ok = launch_merge_plain<K, V, 256, 16>(a, L, lvl, tiles); break;
        case 13: ok = launch_merge_plain<K, V, 512, 16>(a, L, lvl, tiles); break;
        default: return false;
        }
        if (!ok) return false;
    }
    return L.end(L.owner, CLS_MERGE, L.stream);
}

// The persistent merge (every level in one launch) at shape (MT consumer
// threads, MVT keys each): launches it and returns 1, returns 0 when it cannot
// run here (shared memory, or above the automatic limit), -1 when the launch
// failed.
template <class K, class V, int MT, int MVT>
int launch_merge_persist_at(const PassArgs &a, Launcher &L, const PersistPlan &P, int64_t batches) {
    auto kern = merge_persist_kernel<K, V, MT, MVT, MERGE_STAGES>;
    constexpr size_t smem = persist_smem_bytes<K, V, MT, MVT, MERGE_STAGES>();
    static std::atomic<int> occ{0};
    if (!occ.load()) {
        int o = -1;
        if (smem <= SMEM_OPT_IN_LIMIT && allow_smem(kern, smem)) {
            o = resident_ctas(kern, persist_block<MT>(), smem);
            // the merge is latency-bound: fewer resident CTAs than the per-pass
            // TMA kernel would have costs more than the launches it saves
            auto mt = merge_tma_kernel<K, V, MT, MVT, MERGE_STAGES, false>;
            constexpr size_t msmem = tma_smem_bytes<K, V, MT, MVT, MERGE_STAGES, true>();
            if (msmem <= SMEM_OPT_IN_LIMIT && allow_smem(mt, msmem) && resident_ctas(mt, MT + 32, msmem) > o)
                o = -1;
        }
        occ.store(o);
    }
    if (occ.load() <= 0) return 0;
    if (a.merge_impl == MERGE_AUTO && smem > TMA_SMEM_AUTO_LIMIT) return 0;
    // A level is handed out as batches of PERSIST_BATCH tiles, each merged by
    // one CTA tile after tile, while the per-pass kernels merge every tile of
    // a level at once: unless a level holds a batch for every resident CTA,
    // the levels' chain of batches is slower than the per-pass launches
    // (2^20 int32 keys, p = 2: 0.33 against 0.10 ms; 2^24: 0.80 against
    // 0.56; 2^26: 1.74 against 1.87).  a.persistent == 2 forces it.
    const int64_t level_tiles = (a.g.n + (int64_t(1) << P.mlogT) - 1) >> P.mlogT;
    if (a.persistent != 2 && level_tiles < (int64_t)L.sms * occ.load() * PERSIST_BATCH) return 0;
    // every resident CTA (the queue balances the work), no more than there are batches
    const int64_t grid = grid_for(batches, (int64_t)L.sms * occ.load());
    PersistPlan Pm = P;
    Pm.ncw = 1;  // the producer counts each tile once
    L.begin(L.owner, CLS_MERGE, L.stream);
    launch_overlapped(kern, (unsigned)grid, persist_block<MT>(), smem, L.stream, a.g, Pm, (K *)a.k0, (K *)a.k1, (V *)a.v0,
                      (V *)a.v1, a.codec, a.ntiles_total);
    return L.end(L.owner, CLS_MERGE, L.stream) ? 1 : -1;
}

// Every merge level of the sort (nseg in-block levels, then the g.R
// cross-block rounds) in one persistent launch; the same return values.
// Runs only the default consumer (sequential merge) at the default keys per
// thread; other shapes take the per-pass path.
template <class K, class V>
int launch_merge_persist(const PassArgs &a, Launcher &L, int nseg, int mlogT) {
    const Geo &g = a.g;
    if (a.merge_consumer != 0 || (a.merge_vt && a.merge_vt != merge_vt_of<K, V>(PassArgs{})) || !a.pcnt)
        return 0;
    PersistPlan P{};
    P.nseg = nseg;
    P.nl = nseg + g.R;
    P.mlogT = mlogT;
    if (P.nl > PERSIST_MAX_LEVELS) return 0;
    if (P.nl == 0) return 1;  // nothing to merge
    if (persist_words(nseg, g.ntiles_ub, g.R, g.S) > a.pcnt_words) return 0;
    P.work = reinterpret_cast<unsigned long long *>(a.pcnt);
    P.cnt_seg = a.pcnt + 2;
    int64_t rows = 0;
    for (int lv = 0; lv < nseg; ++lv) {
        P.segrow[lv] = rows;
        rows += persist_seg_row(g.ntiles_ub, g.S, lv);
    }
    P.cnt_x = P.cnt_seg + rows;
    int64_t batches = 0, xoff = 0;
    const int64_t seg_tiles = a.ntiles_ub << (g.logT - mlogT);  // an upper bound (grid sizing only)
    batches += (int64_t)nseg * ((seg_tiles + PERSIST_BATCH - 1) / PERSIST_BATCH);
    for (int r = 0; r < g.R; ++r) {
        int64_t tpp = 0, nt = 0;
        const int64_t npairs = (g.S + (int64_t(2) << r) - 1) >> (r + 1);
        if (a.tpp_host) {
            tpp = a.tpp_host[r] << (g.logT - mlogT);
            nt = npairs * tpp;
        } else {
            nt = xblock_tiles(g.n, g.S, r, mlogT, &tpp);
        }
        P.xtiles[r] = nt;
        P.xtpp[r] = tpp;
        P.xcnt[r] = xoff;
        xoff += npairs;
        batches += (nt + PERSIST_BATCH - 1) / PERSIST_BATCH;
    }
    if constexpr (sizeof(K) == 4 && !HasVal<V>::value) {  // 32 keys per consumer thread
        switch (mlogT) {
        case 11: return launch_merge_persist_at<K, V, 64, 32>(a, L, P, batches);
        case 12: return launch_merge_persist_at<K, V, 128, 32>(a, L, P, batches);
        case 13: return launch_merge_persist_at<K, V, 256, 32>(a, L, P, batches);
        default: return 0;
        }
    } else {  // 16
        switch (mlogT) {
        case 11: return launch_merge_persist_at<K, V, 128, 16>(a, L, P, batches);
        case 12: return launch_merge_persist_at<K, V, 256, 16>(a, L, P, batches);
        case 13: return launch_merge_persist_at<K, V, 512, 16>(a, L, P, batches);
        default: return 0;
        }
    }
}

template <class K, class V, int THREADS, int KPT>
bs_status run_passes_t(const PassArgs &a, Launcher &L) {
    constexpr int T = THREADS * KPT;
    const size_t tsmem = tile_smem_bytes<K, V>(T);
    auto ts = tile_sort_kernel<K, V, THREADS, KPT>;
    static std::atomic<int> occ_ts{0};
    if (!occ_ts.load()) {
        if (!allow_smem(ts, tsmem)) return BS_ERR_CUDA;
        occ_ts.store(resident_ctas(ts, THREADS, tsmem));
    }
    const Geo &g = a.g;
    K *k0 = (K *)a.k0, *k1 = (K *)a.k1;
    V *v0 = (V *)a.v0, *v1 = (V *)a.v1;
    // merge tile: at most the sort tile (the plain kernel always uses the sort tile)
    int mlogT = a.merge_tile_log2 ? a.merge_tile_log2 : g.logT;
    if (mlogT > g.logT || mlogT < 11 || a.merge_impl == MERGE_SIMPLE) mlogT = g.logT;
    if (!a.merge_tile_log2 && a.merge_impl == MERGE_AUTO) {
        // wide items: shrink the merge tile until the TMA pipeline fits two CTAs per SM
        while (mlogT > 11 && tma_bytes_at<K, V>(mlogT, merge_vt_of<K, V>(a)) > TMA_SMEM_AUTO_LIMIT) --mlogT;
    }
    const int64_t TM = int64_t(1) << mlogT;

    if (a.merge_only) {
        // runs arrive sorted: encode them into the buffer the rounds start from
        L.begin(L.owner, CLS_SETUP, L.stream);
        launch_overlapped(encode_copy_kernel<K, V>, (unsigned)grid_for((g.n + 255) / 256, (int64_t)L.sms * 8),
                          256, 0, L.stream, (const K *)a.in_k, (const V *)a.in_v, (g.R & 1) ? k1 : k0,
                          (g.R & 1) ? v1 : v0, g.n, a.codec);
        if (!L.end(L.owner, CLS_SETUP, L.stream)) return BS_ERR_CUDA;
    } else if (!HasVal<V>::value && a.local_sort == 1) {
        // sort phase with Fig. 2's bubble sort (odd-even transposition per tile)
        auto kb = tile_bubble_kernel<K, THREADS, KPT>;
        const size_t sb = sizeof(K) * T;
        static std::atomic<int> occ_b{0};
        if (!occ_b.load()) occ_b.store(resident_ctas(kb, THREADS, sb));
        L.begin(L.owner, CLS_TILE_SORT, L.stream);
        launch_overlapped(kb, (unsigned)grid_for(a.ntiles_ub, (int64_t)L.sms * occ_b), THREADS, sb, L.stream,
                          g, (const K *)a.in_k, k0, k1, a.codec, a.ntiles_total);
        if (!L.end(L.owner, CLS_TILE_SORT, L.stream)) return BS_ERR_CUDA;
    } else if (!HasVal<V>::value && a.local_sort == 2) {
        // sort phase with Fig. 4's quick sort (CTA partition per tile)
        auto kq = tile_quick_kernel<K, THREADS, KPT>;
        constexpr size_t sq = quick_smem_bytes<K, THREADS, KPT>();
        static std::atomic<int> occ_q{0};
        if (!occ_q.load()) {
            if (!allow_smem(kq, sq)) return BS_ERR_CUDA;
            occ_q.store(resident_ctas(kq, THREADS, sq));
        }
        L.begin(L.owner, CLS_TILE_SORT, L.stream);
        launch_overlapped(kq, (unsigned)grid_for(a.ntiles_ub, (int64_t)L.sms * occ_q), THREADS, sq, L.stream,
                          g, (const K *)a.in_k, k0, k1, a.codec, a.ntiles_total);
        if (!L.end(L.owner, CLS_TILE_SORT, L.stream)) return BS_ERR_CUDA;
    } else {
        if constexpr (!HasVal<V>::value) {
            // sort phase, warp length class: the short segments, one warp each
            if (g.wmax > 0) {
                constexpr int WW = 4;
                const int64_t warps = g.S < (int64_t)L.sms * 32 ? g.S : (int64_t)L.sms * 32;
                L.begin(L.owner, CLS_TILE_SORT, L.stream);
                launch_overlapped(warp_class_kernel<K, KPT, WW>, (unsigned)grid_for((warps + WW - 1) / WW, warps),
                                  32 * WW, 0, L.stream, g, (const K *)a.in_k, k0, k1, a.codec);
                if (!L.end(L.owner, CLS_TILE_SORT, L.stream)) return BS_ERR_CUDA;
            }
        }
        // sort phase: every tile of every block
        if (!a.no_tiles) {
            L.begin(L.owner, CLS_TILE_SORT, L.stream);
            launch_overlapped(ts, (unsigned)grid_for(a.ntiles_ub, (int64_t)L.sms * occ_ts), THREADS, tsmem,
                              L.stream, g, (const K *)a.in_k, (const V *)a.in_v, k0, k1, v0, v1, a.codec,
                              a.ntiles_total);
            if (!L.end(L.owner, CLS_TILE_SORT, L.stream)) return BS_ERR_CUDA;
        }
    }

    // every merge level in one persistent launch, where it can run
    if (a.persistent && a.merge_impl != MERGE_SIMPLE && a.oddeven_rounds == 0) {
        const int pr = launch_merge_persist<K, V>(a, L, a.Lmax, mlogT);
        if (pr < 0) return BS_ERR_CUDA;
        if (pr > 0) return BS_OK;
    }

    // sort phase, continued: in-block merge levels
    for (int lv = 0; lv < a.Lmax; ++lv) {
        Level lvl{LEVEL_SEG, lv, 0, 0, 0, mlogT};
        if (!merge_pass_any<K, V>(a, L, lvl, a.ntiles_ub << (g.logT - mlogT))) return BS_ERR_CUDA;
    }

    // merge phase, odd-even form: compare-split rounds over equal blocks
    if (a.oddeven_rounds > 0) {
        const int64_t cap = g.n / g.S;
        const int64_t tpp = (2 * cap + TM - 1) / TM;
        for (int r = 0; r < a.oddeven_rounds; ++r) {
            Level lvl{LEVEL_ODDEVEN, 0, r, tpp, 0, mlogT};
            const int64_t npairs = (r & 1) ? 1 + g.S / 2 : (g.S + 1) / 2;
            lvl.ntiles = npairs * tpp;
            if (!merge_pass_any<K, V>(a, L, lvl, lvl.ntiles)) return BS_ERR_CUDA;
        }
        return BS_OK;
    }
    // merge phase: cross-block rounds, tiles aligned to each pair's start
    for (int r = 0; r < g.R; ++r) {
        Level lvl{LEVEL_XBLOCK, 0, r, 0, 0, mlogT};
        if (a.tpp_host) {
            // runs given by the caller: tiles per pair from their lengths (in sort tiles)
            lvl.tpp = a.tpp_host[r] << (g.logT - mlogT);
            lvl.ntiles = ((g.S + (int64_t(2) << r) - 1) >> (r + 1)) * lvl.tpp;
        } else {
            lvl.ntiles = xblock_tiles(g.n, g.S, r, mlogT, &lvl.tpp);
        }
        if (!merge_pass_any<K, V>(a, L, lvl, lvl.ntiles)) return BS_ERR_CUDA;
    }
    return BS_OK;
}

template <class K>
bs_status oddeven_scatter_t(const void *in, void *out, int64_t n, int64_t p, int64_t cap, int codec,
                            Launcher &L) {
    L.begin(L.owner, CLS_SETUP, L.stream);
    // about 8 CTAs per SM in all: chunks of a slot by (at most 65535) slots
    const int64_t ys = p < 65535 ? p : 65535;
    int64_t xs = ((int64_t)L.sms * 8 + ys - 1) / ys;
    const int64_t per_slot = (cap + 255) / 256;
    if (xs > per_slot) xs = per_slot;
    if (xs < 1) xs = 1;
    launch_overlapped(pad_scatter_kernel<K>, dim3((unsigned)xs, (unsigned)ys), 256, 0, L.stream, (const K *)in,
                      (K *)out, n, p, cap, codec);
    return L.end(L.owner, CLS_SETUP, L.stream) ? BS_OK : BS_ERR_CUDA;
}

template <class K>
bs_status oddeven_compact_t(const void *in, void *out, int64_t n, int codec, Launcher &L) {
    L.begin(L.owner, CLS_SETUP, L.stream);
    launch_overlapped(decode_copy_kernel<K>, (unsigned)grid_for((n + 255) / 256, (int64_t)L.sms * 8), 256, 0,
                      L.stream, (const K *)in, (K *)out, n, codec);
    return L.end(L.owner, CLS_SETUP, L.stream) ? BS_OK : BS_ERR_CUDA;
}

// Dispatch on the value width and the sort tile shape (T = 2^logT = THREADS*16).
// Sort-phase shapes (threads per CTA, keys per thread) by tile size: keys
// alone sort 32 per thread (a 191-comparator register network, then five
// warp-shuffle rounds reach 1024-key lists), pairs 16 per thread.
template <class K, class V> bs_status run_passes_v(const PassArgs &a, Launcher &L) {
    if constexpr (!HasVal<V>::value) {
        switch (a.g.logT) {
        case 12: return run_passes_t<K, V, 128, 32>(a, L);
        case 13: return run_passes_t<K, V, 256, 32>(a, L);
        default: break;
        }
    }
    switch (a.g.logT) {
    case 11: return run_passes_t<K, V, 128, 16>(a, L);
    case 12: return run_passes_t<K, V, 256, 16>(a, L);
    case 13: return run_passes_t<K, V, 512, 16>(a, L);
    default: return BS_ERR_INVALID_ARG;
    }
}

template <class K> bs_status run_passes_k(const PassArgs &a, Launcher &L) {
    switch (a.vbytes) {
    case 0: return run_passes_v<K, NoVal>(a, L);
    case 4: return run_passes_v<K, uint32_t>(a, L);
    case 8: return run_passes_v<K, uint64_t>(a, L);
    default: return BS_ERR_UNSUPPORTED_DTYPE;
    }
}

}  // namespace bs
