// bs_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "bs_device.cuh"
#include "bs_persist.cuh"
#include "bsort.h"

namespace bs {

// Launches `kern` with programmatic stream serialization: its CTAs may be
// scheduled, and run up to their griddepcontrol.wait, while the kernel before
// it on the stream drains, which hides most of the gap between two kernels.
// Only kernels that wait before touching global memory are launched so.
template <class... Params, class... Args>
inline cudaError_t launch_overlapped(void (*kern)(Params...), dim3 grid, unsigned block, size_t smem,
                                     cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, (Params)args...);
}

// Launch bookkeeping supplied by the C ABI layer: launch counting, optional
// CUDA-event timing per launch, and error capture.
struct Launcher {
    cudaStream_t stream;
    void *owner;  // the bs_handle
    int sms;      // multiprocessors of the device
    void (*begin)(void *owner, int cls, cudaStream_t s);
    bool (*end)(void *owner, int cls, cudaStream_t s);  // false: launch failed
};

// One complete sort: tile sort, in-segment merge levels, cross-block rounds.
struct PassArgs {
    Geo g;
    const void *in_k, *in_v;  // caller input (raw dtype bits)
    void *k0, *k1, *v0, *v1;  // buffer 0 = caller output, buffer 1 = scratch
    int codec;
    int vbytes;               // 0 (keys only), 4 or 8
    int Lmax;                 // in-segment merge levels to launch
    int64_t ntiles_ub;        // upper bound of the tile count (grid sizing)
    const int64_t *ntiles_total;  // device scalar: exact tile count
    int64_t *split;           // per tile merge-path split of the current pass
    int merge_impl;           // MERGE_SIMPLE or MERGE_TMA (the caller checked alignment)
    int merge_vt;             // keys per consumer thread in the TMA merge: 8, 16, 32 (0: by item size)
    bool merge_only;          // the blocks are caller-sorted runs: no sort phase
    const int64_t *tpp_host;  // merge_only: tiles per pair of each round (host array)
    int oddeven_rounds;       // > 0: after the sort phase, that many compare-split rounds
                              // instead of the cross-block tree (keys only, padded blocks)
    int local_sort;           // tile sort: 0 network + merges, 1 bubble (Fig. 2), 2 quick (Fig. 4)
    int merge_tile_log2;      // merge-pass tile (0: the sort tile; else 11 .. logT)
    int merge_consumer;       // TMA merge consumers: 0 per-thread sequential merge, 1 warp bitonic
    int persistent;           // every merge level in one persistent launch where it can run:
                              // 1 when a level holds a batch for every resident CTA, 2 always
    unsigned *pcnt;           // its pair counters and work queue (zeroed before the sort phase)
    int64_t pcnt_words;       // capacity of pcnt in 32-bit words
    bool no_tiles;            // every block is in the warp length class: no tile sort launch
};

// Longest segment of the warp length class for a keys-alone sort at tile
// 2^logT: 32 lanes x the tile sort's keys per thread (32, or 16 at 2048-key
// tiles).  Pair sorts and the alternative local sorts have no such class.
inline int64_t warp_class_max(int logT) { return logT >= 12 ? 32 * 32 : 32 * 16; }

// Words of the persistent merge's counter region for a sort whose in-block
// levels number `nseg` over `ntiles_ub` sort tiles in S blocks and whose
// merge phase has R rounds: the work-queue head (2 words), a row per
// in-block level lv of ntiles_ub / 2^(lv+1) + S + 2 pair counters, then one
// counter per pair of every cross-block round.
inline int64_t persist_seg_row(int64_t ntiles_ub, int64_t S, int lv) { return (ntiles_ub >> (lv + 1)) + S + 2; }
inline int64_t persist_words(int nseg, int64_t ntiles_ub, int R, int64_t S) {
    int64_t w = 2;
    for (int lv = 0; lv < nseg; ++lv) w += persist_seg_row(ntiles_ub, S, lv);
    for (int r = 0; r < R; ++r) w += (S + (int64_t(2) << r) - 1) >> (r + 1);
    return w;
}

enum : int { MERGE_AUTO = 0, MERGE_SIMPLE = 1, MERGE_TMA = 2 };

// Tiles of cross-block round r over S balanced blocks of n keys in total:
// every pair gets *tpp tiles (enough for the longest pair, ceil(G*n/S) keys
// with G = 2^(r+1) blocks per pair); returns npairs * tpp.
inline int64_t xblock_tiles(int64_t n, int64_t S, int r, int logT, int64_t *tpp) {
    const int64_t G = int64_t(2) << r;
    const int64_t npairs = (S + G - 1) / G;
    const unsigned __int128 gl = (unsigned __int128)(uint64_t)G * (uint64_t)n;
    int64_t maxpair = (int64_t)((gl + (uint64_t)S - 1) / (uint64_t)S);
    if (maxpair > n) maxpair = n;
    const int64_t T = int64_t(1) << logT;
    int64_t per = (maxpair + T - 1) / T;
    if (per < 1) per = 1;
    if (tpp) *tpp = per;
    return npairs * per;
}

// Largest tile count of any cross-block round (0 when S <= 1).
inline int64_t xblock_tiles_max(int64_t n, int64_t S, int logT) {
    int64_t m = 0;
    for (int r = 0; (int64_t(1) << r) < S; ++r) {
        const int64_t x = xblock_tiles(n, S, r, logT, nullptr);
        if (x > m) m = x;
    }
    return m;
}

bs_status run_passes_u32(const PassArgs &a, Launcher &L);
bs_status run_passes_u64(const PassArgs &a, Launcher &L);
// odd-even schedule helpers (keys only)
bs_status oddeven_scatter_u32(const void *in, void *out, int64_t n, int64_t p, int64_t cap, int codec,
                              Launcher &L);
bs_status oddeven_scatter_u64(const void *in, void *out, int64_t n, int64_t p, int64_t cap, int codec,
                              Launcher &L);
bs_status oddeven_compact_u32(const void *in, void *out, int64_t n, int codec, Launcher &L);
bs_status oddeven_compact_u64(const void *in, void *out, int64_t n, int codec, Launcher &L);

}  // namespace bs
