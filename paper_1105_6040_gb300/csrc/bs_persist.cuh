// bs_persist.cuh -- the whole merge phase of one sort in one persistent launch.
//
// The per-pass path runs every merge level of Fig. 1 (the in-block levels of
// the sort phase, then the cross-block rounds of the merge phase) as two
// kernels: a merge-path partition, then the TMA merge.  Here one persistent
// grid runs all levels.  Its work queue is a counter in device memory that
// hands out batches of PERSIST_BATCH consecutive merge tiles in level order
// (all tiles of level 0, then of level 1, ...).  A merge tile of level l may
// start once the two runs it reads are complete, i.e. once the level-(l-1)
// pairs that produced them have counted all their merge tiles as done; those
// tiles were handed out before it, so every wait is for work that some
// resident CTA already holds, and the queue cannot deadlock.  Low levels, with
// thousands of small pairs, flow without any grid-wide barrier; the top
// levels (a few large pairs) wait for their whole inputs, as the paper's
// merge rounds wait for their partners' messages.
//
// Each CTA is warp-specialised:
//   search warp    pops a batch, waits (bounded) on the counters of the pairs
//                  its tiles read, finds the merge-path split at the batch's
//                  PERSIST_BATCH + 1 tile boundaries (one group of lanes per
//                  boundary running a (group + 1)-way search over the runs in
//                  global memory), and hands the tiles' slices to the
//                  producer through a ring of batch slots;
//   producer warp  stages each tile's A and B slices into the stage ring by
//                  1-D bulk copies (TMA), as the per-pass TMA merge does;
//   consumers      merge the staged tile (the same consumer code as the
//                  per-pass kernel), store it and count their part stored in
//                  shared memory; whenever the search warp would wait, it
//                  releases the stored tiles at GPU scope and counts them done
//                  on their pairs' counters, which search warps read with
//                  acquire loads (a release waits for the stores to land, ~2 us,
//                  so it is kept off the warps that move data).
// Data written by one CTA's stores is read by another CTA's bulk copies and
// search loads: the writer releases after its stores, the reader acquires
// before its loads, search and tail loads bypass L1 (ld.global.cg), and the
// copying thread issues a generic-to-async proxy fence before its copies.
// Every wait is bounded by the handle's limit; a wait that runs out records
// BS_ERR_TIMEOUT and the warps leave (the producer first waits, bounded, for
// its copies in flight), so the context stays usable.
#pragma once

#include "bs_device.cuh"

namespace bs {

constexpr int PERSIST_MAX_LEVELS = 48;
constexpr int PERSIST_BATCH = 15;  // merge tiles per work item: 16 boundaries x 2 search lanes
constexpr int PERSIST_SLOTS = 2;  // batch slots between the search warp and the producer

// Everything the persistent merge needs besides Geo and the buffers.
struct PersistPlan {
    int nl;      // merge levels in all
    int nseg;    // levels 0 .. nseg-1 are in-block levels (LEVEL_SEG lv = l), the rest
                 // cross-block rounds (LEVEL_XBLOCK r = l - nseg)
    int mlogT;   // merge tile = 2^mlogT keys
    int ncw;     // increments a completed merge tile adds to its pair counter (1)
    int64_t xtiles[PERSIST_MAX_LEVELS];  // cross-block round r: its merge tiles
    int64_t xtpp[PERSIST_MAX_LEVELS];    // cross-block round r: merge tiles per pair
    int64_t xcnt[PERSIST_MAX_LEVELS];    // cross-block round r: first of its counters in cnt_x
    int64_t segrow[PERSIST_MAX_LEVELS];  // in-block level lv: first of its counters in cnt_seg
    unsigned *cnt_seg;          // in-block pair counters (slot: seg_pair_slot)
    unsigned *cnt_x;            // cross-block pair counters
    unsigned long long *work;   // batches handed out so far
};

// ---------------------------------------------------------------- memory-model helpers

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Global loads that skip L1: the data may have been written by another CTA
// of this grid after this SM last cached the line.
__device__ __forceinline__ uint32_t ld_cg(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint64_t ld_cg(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

// stage_window with the ragged end read through ld_cg.
template <class T>
__device__ __forceinline__ int stage_window_cg(T *dst, const T *a, int64_t n, int64_t lo, int64_t hi,
                                               uint64_t *bar, uint32_t *tx) {
    constexpr int64_t E = 16 / sizeof(T);
    const int64_t ws = lo & ~(E - 1);
    if (hi <= lo) return (int)(lo - ws);
    int64_t we = (hi + E - 1) & ~(E - 1);
    const int64_t nfull = n & ~(E - 1);
    if (we > nfull) we = nfull;
    if (we > ws) {
        const uint32_t bytes = (uint32_t)((we - ws) * (int64_t)sizeof(T));
        tma_load_1d(dst, a + ws, bytes, bar);
        *tx += bytes;
    } else {
        we = ws;
    }
    for (int64_t x = we; x < hi; ++x) dst[x - ws] = ld_cg(a + x);
    return (int)(lo - ws);
}

// ---------------------------------------------------------------- plan helpers

__device__ __forceinline__ Level persist_level(const PersistPlan &P, int l) {
    Level L{};
    L.mlogT = P.mlogT;
    if (l < P.nseg) {
        L.kind = LEVEL_SEG;
        L.lv = l;
    } else {
        L.kind = LEVEL_XBLOCK;
        L.r = l - P.nseg;
        L.tpp = P.xtpp[L.r];
        L.ntiles = P.xtiles[L.r];
    }
    return L;
}

__device__ __forceinline__ int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Counter slot of pair c of segment s at in-block level lv (the pair covers
// sort tiles tprefix[s] + c*2^(lv+1) ..): floor(tprefix[s] / 2^(lv+1)) + s + c.
// Distinct for distinct (s, c) -- segment s's last pair stays below segment
// s+1's first, since its start tile is at least tprefix[s] + tiles of s --
// and below ntiles / 2^(lv+1) + S + 2, so level lv needs a row that long.
__device__ __forceinline__ int64_t seg_pair_slot(const Geo &g, int64_t s, int64_t c, int lv) {
    return (g.tprefix[s] >> (lv + 1)) + s + c;
}

// Where a merge tile's completion is counted, and the two counters (with the
// count each must reach) of the pairs that produced the runs it reads; a run
// produced by the sort phase (or handed in sorted) has none.
struct PairDeps {
    unsigned *ctr;
    const unsigned *dep0, *dep1;
    unsigned need0, need1;
};

__device__ __forceinline__ PairDeps pair_deps(const Geo &g, const PersistPlan &P, const Level &L,
                                              const TilePair &p, int64_t t) {
    PairDeps d{nullptr, nullptr, nullptr, 0u, 0u};
    const int64_t TM = int64_t(1) << P.mlogT;
    const unsigned ncw = (unsigned)P.ncw;
    if (L.kind == LEVEL_SEG) {
        const int sh = g.logT - L.mlogT;
        const int64_t ts = t >> sh;
        const int64_t s = g.tseg[ts];
        const int64_t c = (ts - g.tprefix[s]) >> (L.lv + 1);  // this pair of the segment
        d.ctr = P.cnt_seg + P.segrow[L.lv] + seg_pair_slot(g, s, c, L.lv);
        if (L.lv > 0) {
            // runs A and B are pairs 2c and 2c+1 of level lv-1
            const unsigned *prev = P.cnt_seg + P.segrow[L.lv - 1];
            d.dep0 = prev + seg_pair_slot(g, s, 2 * c, L.lv - 1);
            d.need0 = ncw * (unsigned)ceil_div64(p.pm - p.ps, TM);
            if (p.pe > p.pm) {
                d.dep1 = prev + seg_pair_slot(g, s, 2 * c + 1, L.lv - 1);
                d.need1 = ncw * (unsigned)ceil_div64(p.pe - p.pm, TM);
            }
        }
    } else {
        const int64_t k = t / L.tpp;
        d.ctr = P.cnt_x + P.xcnt[L.r] + k;
        if (L.r > 0) {
            const unsigned *prev = P.cnt_x + P.xcnt[L.r - 1];
            d.dep0 = prev + 2 * k;
            d.need0 = ncw * (unsigned)ceil_div64(p.pm - p.ps, TM);
            if (p.pe > p.pm) {
                d.dep1 = prev + 2 * k + 1;
                d.need1 = ncw * (unsigned)ceil_div64(p.pe - p.pm, TM);
            }
        } else if (P.nseg > 0) {
            // round 0 reads blocks 2k and 2k+1 as their last in-block level left them
            for (int h = 0; h < 2; ++h) {
                const int64_t b = 2 * k + h;
                if (b >= g.S) break;
                int64_t lo, hi;
                seg_bounds(g, b, lo, hi);
                const int Lb = seg_levels(hi - lo, g.logT);
                if (Lb == 0) continue;  // the sort phase produced it
                const unsigned *c = P.cnt_seg + P.segrow[Lb - 1] + seg_pair_slot(g, b, 0, Lb - 1);
                const unsigned need = ncw * (unsigned)ceil_div64(hi - lo, TM);
                if (h == 0) d.dep0 = c, d.need0 = need;
                else d.dep1 = c, d.need1 = need;
            }
        }
    }
    return d;
}

__device__ __forceinline__ bool deps_done(const PairDeps &d) {
    return (!d.dep0 || ld_acquire_u32(d.dep0) >= d.need0) && (!d.dep1 || ld_acquire_u32(d.dep1) >= d.need1);
}

// One tile's slices as the search warp hands them to the producer (kept
// small: the slots' shared memory decides whether a third CTA fits per SM for
// wide items).
struct BatchRec {
    int64_t a_lo, b_lo, x0;
    int na, nb;
    unsigned ctr;  // its pair counter: cnt_seg + ctr
    int flags;     // bit0 active, bit1 src parity, bit2 dst parity, bit3 final pass
};
struct BatchSlot {
    BatchRec rec[PERSIST_BATCH];
    int count;  // >= 0: records; -1: no more work
    int pad[3];
};

constexpr int STAGE_STOP = 8;  // StageDesc flag: no more tiles

constexpr int PERSIST_PEND = 32;  // tiles staged but not yet counted done, at most

// Shared state between the consumers, the producer and the signal thread.
struct SignalRing {
    unsigned ctr[PERSIST_PEND];   // pair counter of staged tile j (cnt_seg + ctr), at j % PERSIST_PEND
    unsigned done[32];            // tiles consumer warp w has stored (monotone)
    unsigned retired;             // tiles counted done
    unsigned final_tiles;         // tiles staged in all, once the producer stops (~0u before)
};

template <class K, class V, int THREADS, int VT, int STAGES>
__host__ __device__ constexpr size_t persist_smem_bytes() {
    return STAGES * TmaLayout<K, V, THREADS * VT>::stage + (THREADS / 32) * WarpScratch<K, V, VT>::bytes +
           PERSIST_SLOTS * sizeof(BatchSlot) + (2 * STAGES + 2 * PERSIST_SLOTS) * sizeof(uint64_t) +
           sizeof(SignalRing) + 128;
}

__device__ __forceinline__ void red_release_cta_add(unsigned *p, unsigned v) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cta(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(unsigned *p, unsigned v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// Threads of a persistent-merge CTA: consumers, then the producer and search
// warps.
template <int THREADS> constexpr int persist_block() { return THREADS + 64; }

template <class K, class V, int THREADS, int VT, int STAGES> constexpr int persist_min_ctas() {
    const int by_smem = (int)((228 * 1024) / (persist_smem_bytes<K, V, THREADS, VT, STAGES>() + 1024));
    const int regs = 64;
    const int by_regs = 65536 / (persist_block<THREADS>() * regs);
    const int m = by_smem < by_regs ? by_smem : by_regs;
    return m < 1 ? 1 : m;
}

// ---------------------------------------------------------------- the kernel

template <class K, class V, int THREADS, int VT, int STAGES>
__global__ void __launch_bounds__(persist_block<THREADS>(), (persist_min_ctas<K, V, THREADS, VT, STAGES>()))
merge_persist_kernel(Geo g, const __grid_constant__ PersistPlan P, K *buf_k0, K *buf_k1, V *buf_v0, V *buf_v1, int codec,
                     const int64_t *__restrict__ ntiles_total) {
    constexpr int TT = THREADS * VT;
    constexpr bool HV = HasVal<V>::value;
    constexpr int NB = PERSIST_BATCH + 1;  // boundaries per batch
    constexpr int GS = 32 / NB;            // search lanes per boundary
    static_assert(GS >= 1 && NB * GS <= 32, "batch boundaries fit one warp");
    using LY = TmaLayout<K, V, TT>;
    using WS = WarpScratch<K, V, VT>;
    constexpr size_t SCRATCH = (THREADS / 32) * WS::bytes;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BatchSlot *slots = reinterpret_cast<BatchSlot *>(smem_raw + STAGES * LY::stage + SCRATCH);
    constexpr int NCW = THREADS / 32;
    static_assert(NCW <= 32, "consumer warps fit the signal ring");
    uint64_t *full = reinterpret_cast<uint64_t *>(slots + PERSIST_SLOTS);
    uint64_t *empty = full + STAGES;
    uint64_t *sfull = empty + STAGES;
    uint64_t *sempty = sfull + PERSIST_SLOTS;
    SignalRing *ring = reinterpret_cast<SignalRing *>(sempty + PERSIST_SLOTS);
    auto stage_k = [&](int s) { return reinterpret_cast<K *>(smem_raw + s * LY::stage); };
    auto stage_v = [&](int s) { return reinterpret_cast<V *>(smem_raw + s * LY::stage + LY::keys); };
    auto stage_desc = [&](int s) {
        return reinterpret_cast<StageDesc *>(smem_raw + s * LY::stage + LY::keys + LY::vals);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], THREADS);
        }
        for (int w = 0; w < 32; ++w) ring->done[w] = 0;
        ring->retired = 0;
        ring->final_tiles = ~0u;
        for (int s = 0; s < PERSIST_SLOTS; ++s) {
            mbar_init(&sfull[s], 1);
            mbar_init(&sempty[s], 1);
        }
        mbar_fence_init();
    }
    __syncthreads();
    griddep_wait();  // the sorted tiles (or encoded runs) come from the kernel before

    const uint64_t WAIT_LIMIT = g.wait_ns ? g.wait_ns : WAIT_LIMIT_DEFAULT;
    const int64_t n = g.n;
    // tiles per level, padded to whole batches, and the total
    const int64_t seg_tiles =
        ntiles_total ? (min(*ntiles_total, g.ntiles_ub) << (g.logT - P.mlogT)) : int64_t(0);

    if (threadIdx.x >= THREADS + 32) {
        // ================================================================ search warp
        const int lane = threadIdx.x - (THREADS + 32);
        const unsigned FULL = 0xffffffffu;
        const int grp = lane / GS, sub = lane % GS;
        int slot = 0;
        uint32_t sph = 0;  // phase of the slot's "empty" barrier we wait for
        uint64_t nbatch = 0;
        // Counting the CTA's stored tiles done (lane 0), whenever the warp would
        // otherwise wait: a GPU-scope fence (the consumers' stores, acquired
        // through their counts, before anything after it) and the pair
        // counters' increments.  The fence waits for the stores to land (~2 us),
        // so it is kept off the warps that move data.  Returns true if any tile
        // was counted.
        unsigned retired = 0;
        auto signal = [&]() -> bool {
            bool any = false;
            if (lane == 0) {
                unsigned m = ~0u;
                for (int w = 0; w < NCW; ++w) {
                    const unsigned d = ld_acquire_cta(&ring->done[w]);
                    m = d < m ? d : m;
                }
                if (m != retired) {
                    __threadfence();
                    fence_proxy_async_global();
                    for (; retired != m; ++retired) atomicAdd(P.cnt_seg + ring->ctr[retired % PERSIST_PEND], 1u);
                    st_release_cta(&ring->retired, retired);
                    any = true;
                }
            }
            return __shfl_sync(FULL, (int)any, 0) != 0;
        };
        // after the last batch: count every tile the producer staged, then leave
        auto finish = [&]() {
            uint64_t t0 = global_ns();
            for (uint32_t i = 1;; ++i) {
                if (signal()) t0 = global_ns();
                const bool all = __shfl_sync(FULL, (int)(ld_acquire_cta(&ring->final_tiles) == retired), 0) != 0;
                if (all) return;
                if ((i & 15) == 0 &&
                    __shfl_sync(FULL, (int)(global_ns() - t0 > WAIT_LIMIT), 0) != 0) {
                    if (lane == 0 && g.err) atomicCAS(g.err, 0, (int)BS_ERR_TIMEOUT);
                    return;
                }
                __nanosleep(200);
            }
        };
        for (;;) {
            // ---- pop a batch and find its level
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(P.work, 1ull);
            b = __shfl_sync(FULL, b, 0);
            int64_t i0 = (int64_t)b * PERSIST_BATCH;
            int l = 0;
            int64_t nt = 0;
            for (; l < P.nl; ++l) {
                nt = l < P.nseg ? seg_tiles : P.xtiles[l - P.nseg];
                const int64_t np = ceil_div64(nt, PERSIST_BATCH) * PERSIST_BATCH;
                if (i0 < np) break;
                i0 -= np;
            }
            const bool stop = l >= P.nl;
            // ---- the batch's tiles: lane u <= PERSIST_BATCH takes tile i0 + u
            TilePair p{};
            PairDeps dp{nullptr, nullptr, nullptr, 0u, 0u};
            Level L{};
            bool act = false;
            if (!stop) {
                L = persist_level(P, l);
                const int64_t t = i0 + lane;
                if (lane <= PERSIST_BATCH && t < nt) {
                    p = tile_pair(g, L, t);
                    act = p.active;
                    if (act && lane < PERSIST_BATCH) dp = pair_deps(g, P, L, p, t);
                }
                // ---- wait (bounded) until the runs these tiles read are complete
                bool ok = !(act && lane < PERSIST_BATCH) || deps_done(dp);
                if (!__all_sync(FULL, ok)) {
                    const uint64_t t0 = global_ns();
                    bool timed_out = false;
                    for (uint32_t it = 1; !__all_sync(FULL, ok); ++it) {
                        signal();  // this CTA's own tiles may be among those awaited
                        if (!ok) ok = deps_done(dp);
                        if ((it & 15) == 0) {
                            timed_out = __shfl_sync(FULL, (int)(global_ns() - t0 > WAIT_LIMIT), 0) != 0;
                            if (timed_out) break;
                        }
                    }
                    if (timed_out) {
                        if (lane == 0 && g.err) atomicCAS(g.err, 0, (int)BS_ERR_TIMEOUT);
                        l = P.nl;  // hand over "no more work" and leave
                    }
                }
            }
            const bool done = l >= P.nl;
            // ---- merge-path splits at the batch's boundaries: boundary q is the
            // start of tile i0 + q; the last one only when it continues the
            // pair of the tile before it
            int64_t split = 0;
            if (!done) {
                const int q = grp < NB ? grp : 0;
                const int64_t ps = __shfl_sync(FULL, p.ps, q), pm = __shfl_sync(FULL, p.pm, q);
                const int64_t pe = __shfl_sync(FULL, p.pe, q), x0 = __shfl_sync(FULL, p.x0, q);
                const int srcp = __shfl_sync(FULL, p.src, q);
                const bool qact = __shfl_sync(FULL, (int)act, q) != 0;
                const int64_t prev_ps = __shfl_sync(FULL, p.ps, PERSIST_BATCH - 1);
                const bool prev_act = __shfl_sync(FULL, (int)act, PERSIST_BATCH - 1) != 0;
                bool need = grp < NB && qact && (grp < PERSIST_BATCH || (prev_act && prev_ps == ps));
                const K *src = srcp ? buf_k1 : buf_k0;
                const int64_t na = pm - ps, nb = pe - pm, dg = x0 - ps;
                int64_t lo = need ? (dg > nb ? dg - nb : 0) : 0;
                int64_t hi = need ? (dg < na ? dg : na) : 0;
                const unsigned gmask = ((1u << GS) - 1u) << (grp < NB ? grp * GS : 0);
                while (__any_sync(FULL, lo < hi)) {
                    const bool live = lo < hi;
                    const int64_t mid = lo + ((int64_t)(sub + 1) * (hi - lo)) / (GS + 1);
                    bool test = false;
                    if (live) test = ld_cg(src + pm + (dg - 1 - mid)) < ld_cg(src + ps + mid);
                    const unsigned yes = (__ballot_sync(FULL, test) & gmask) >> (grp < NB ? grp * GS : 0);
                    const int f = yes ? __ffs(yes) - 1 : GS;
                    const int base = grp < NB ? grp * GS : 0;
                    const int64_t mprev = __shfl_sync(FULL, mid, base + (f > 0 ? f - 1 : 0));
                    const int64_t mf = __shfl_sync(FULL, mid, base + (f < GS ? f : GS - 1));
                    if (live) {
                        if (f > 0) lo = mprev + 1;
                        if (f < GS) hi = mf;
                    }
                }
                split = ps + lo;
            }
            // ---- hand the batch to the producer
            if (nbatch >= PERSIST_SLOTS && !mbar_try_wait(&sempty[slot], sph ^ 1u)) {
                const uint64_t t0 = global_ns();
                bool timed_out = false;
                for (uint32_t i = 1; !mbar_try_wait(&sempty[slot], sph ^ 1u); ++i) {
                    signal();
                    if ((i & 15) == 0 &&
                        __shfl_sync(FULL, (int)(global_ns() - t0 > WAIT_LIMIT), 0) != 0) {
                        timed_out = true;
                        break;
                    }
                }
                if (timed_out) {
                    if (lane == 0 && g.err) atomicCAS(g.err, 0, (int)BS_ERR_TIMEOUT);
                    finish();
                    return;  // the producer is gone or stuck: it times out on its own
                }
            }
            const int64_t s_lo = __shfl_sync(FULL, split, (lane < PERSIST_BATCH ? lane : 0) * GS);
            const int64_t s_hi = __shfl_sync(FULL, split, (lane < PERSIST_BATCH ? lane + 1 : 0) * GS);
            BatchSlot &bs = slots[slot];
            if (lane < PERSIST_BATCH) {
                BatchRec r{};
                if (!done && act) {
                    const int64_t len = p.x1 - p.x0;
                    r.a_lo = clamp64(s_lo, p.ps, p.pm);
                    const int64_t a_hi = (p.x1 == p.pe) ? p.pm : s_hi;
                    const int64_t ahc = clamp64(a_hi, r.a_lo, min(p.pm, r.a_lo + len));
                    r.b_lo = clamp64(p.pm + (p.x0 - p.ps) - (r.a_lo - p.ps), p.pm, p.pe);
                    const int64_t nbk = min(len - (ahc - r.a_lo), p.pe - r.b_lo);
                    r.na = (int)(ahc - r.a_lo);
                    r.nb = (int)(nbk > 0 ? nbk : 0);
                    r.x0 = p.x0;
                    r.ctr = (unsigned)(dp.ctr - P.cnt_seg);
                    r.flags = 1 | (p.src << 1) | (p.dst << 2) | (p.fin ? 8 : 0);
                }
                bs.rec[lane] = r;
            }
            if (lane == 0) bs.count = done ? -1 : PERSIST_BATCH;
            __syncwarp();
            if (lane == 0) mbar_arrive(&sfull[slot]);
            ++nbatch;
            sph ^= (slot == PERSIST_SLOTS - 1);
            slot = (slot == PERSIST_SLOTS - 1) ? 0 : slot + 1;
            if (done) {
                finish();
                return;
            }
            signal();
        }
    }

    if (threadIdx.x >= THREADS) {
        // ================================================================ producer warp (lane 0)
        // Stages each tile as the per-pass kernel does, and records its pair
        // counter in the signal ring (at most PERSIST_PEND tiles ahead of the
        // tiles counted done).
        if (threadIdx.x != THREADS) return;
        int slot = 0;
        uint32_t sph = 0;
        int64_t it = 0;        // stage uses so far
        unsigned issued = 0;   // tiles staged
        int stg = 0;
        uint32_t ph = 0;
        auto drain = [&]() {  // wait (bounded) for this CTA's copies still in flight
            for (int64_t jt = (it > STAGES ? it - STAGES : 0); jt < it; ++jt)
                mbar_wait(&full[jt % STAGES], (uint32_t)((jt / STAGES) & 1), WAIT_LIMIT);
        };
        auto fail = [&]() {
            if (g.err) atomicCAS(g.err, 0, (int)BS_ERR_TIMEOUT);
            drain();
        };
        auto claim = [&]() -> bool {  // the next stage is free
            if (it >= STAGES && !mbar_wait(&empty[stg], ph ^ 1u, WAIT_LIMIT)) {
                fail();
                return false;
            }
            return true;
        };
        auto ring_room = [&]() -> bool {  // the signal ring has a free entry
            if (issued - ld_acquire_cta(&ring->retired) < (unsigned)PERSIST_PEND) return true;
            const uint64_t t0 = global_ns();
            for (uint32_t i = 1; issued - ld_acquire_cta(&ring->retired) >= (unsigned)PERSIST_PEND; ++i)
                if ((i & 63) == 0 && global_ns() - t0 > WAIT_LIMIT) {
                    fail();
                    return false;
                }
            return true;
        };
        auto advance = [&]() {
            ++it;
            ph ^= (stg == STAGES - 1);
            stg = (stg == STAGES - 1) ? 0 : stg + 1;
        };
        for (;;) {
            if (!mbar_wait(&sfull[slot], sph, WAIT_LIMIT)) {
                fail();
                break;
            }
            const BatchSlot &bs = slots[slot];
            if (bs.count < 0) {
                // tell the consumers there is no more work
                if (!claim()) break;
                StageDesc d{};
                d.flags = STAGE_STOP;
                *stage_desc(stg) = d;
                mbar_arrive_expect_tx(&full[stg], 0);
                advance();
                drain();
                break;
            }
            bool ok = true;
            for (int u = 0; u < bs.count && ok; ++u) {
                const BatchRec r = bs.rec[u];
                if (!(r.flags & 1)) continue;
                if (!claim() || !ring_room()) {
                    ok = false;
                    break;
                }
                if (!(g.withhold && blockIdx.x == 0 && it == 0)) {  // test hook: nothing arrives
                    // the consumers' reads of this stage, and (through the search
                    // warp's acquire) other CTAs' stores of the runs, before the copies
                    proxy_fence_async_smem();
                    fence_proxy_async_global();
                    const int s = stg;
                    const K *src = (r.flags & 2) ? buf_k1 : buf_k0;
                    StageDesc d{};
                    uint32_t tx = 0;
                    d.o_lo = r.x0;
                    d.na = r.na;
                    d.nb = r.nb;
                    d.flags = 1 | (((r.flags >> 2) & 1) << 1) | ((r.flags & 8) ? 4 : 0);
                    const int64_t a_hi = r.a_lo + r.na, b_hi = r.b_lo + r.nb;
                    const int ak = window_span<K>(r.a_lo, a_hi);
                    d.a_off = stage_window_cg(stage_k(s), src, n, r.a_lo, a_hi, &full[s], &tx);
                    d.b_off = ak + stage_window_cg(stage_k(s) + ak, src, n, r.b_lo, b_hi, &full[s], &tx);
                    if constexpr (HV) {
                        const V *srcv = (r.flags & 2) ? buf_v1 : buf_v0;
                        const int av = window_span<V>(r.a_lo, a_hi);
                        d.av_off = stage_window_cg(stage_v(s), srcv, n, r.a_lo, a_hi, &full[s], &tx);
                        d.bv_off = av + stage_window_cg(stage_v(s) + av, srcv, n, r.b_lo, b_hi, &full[s], &tx);
                    }
                    *stage_desc(s) = d;
                    ring->ctr[issued % PERSIST_PEND] = r.ctr;  // published by the arrive below
                    ++issued;
                    mbar_arrive_expect_tx(&full[s], tx);
                }
                advance();
            }
            if (!ok) break;
            mbar_arrive(&sempty[slot]);
            sph ^= (slot == PERSIST_SLOTS - 1);
            slot = (slot == PERSIST_SLOTS - 1) ? 0 : slot + 1;
        }
        st_release_cta(&ring->final_tiles, issued);  // the search warp may finish counting
        return;
    }

    // ==================================================================== consumers
    const int tid = threadIdx.x, lane = tid & 31;
    int stg = 0;
    uint32_t ph = 0;
    // A warp counts its part of a tile stored (release at CTA scope) just
    // before it stores the next tile, or before it waits for one: the release
    // then finds the tile's stores long complete instead of waiting for them.
    bool pend = false;
    unsigned *my_done = &ring->done[tid >> 5];
    auto release_prev = [&]() {
        if (pend) {
            __syncwarp();
            if (lane == 0) red_release_cta_add(my_done, 1u);
            pend = false;
        }
    };
    for (;; ph ^= (stg == STAGES - 1), stg = (stg == STAGES - 1) ? 0 : stg + 1) {
        const int s = stg;
        if (pend && !mbar_try_wait(&full[s], ph)) release_prev();  // about to wait
        if (!mbar_wait(&full[s], ph, WAIT_LIMIT)) {
            if (g.err) atomicCAS(g.err, 0, (int)BS_ERR_TIMEOUT);
            return;
        }
        const StageDesc d = *stage_desc(s);
        if (d.flags & STAGE_STOP) {
            release_prev();
            return;
        }
        const K *sa = stage_k(s) + d.a_off;
        K *sb = stage_k(s) + d.b_off;
        const int na = d.na, nb = d.nb;
        unsigned char *ws = smem_raw + STAGES * LY::stage + (tid >> 5) * WS::bytes;
        const bool fin = (d.flags & 4) != 0;
        K *dk = out_buf<K>(fin, g.fin_k, (d.flags >> 1) & 1, buf_k0, buf_k1);
        V *dv = out_buf<V>(fin, g.fin_v, (d.flags >> 1) & 1, buf_v0, buf_v1);
        thread_merge_tile<K, V, VT>(sa, sb, stage_v(s) + d.av_off, stage_v(s) + d.bv_off, na, nb, dk, dv, d.o_lo,
                                    fin, codec, &empty[s], tid, reinterpret_cast<K *>(ws),
                                    reinterpret_cast<uint32_t *>(ws + WS::keys), release_prev);
        // this warp's part of the tile is stored; it says so later (release_prev),
        // and the search warp counts the tile done once every consumer warp has
        pend = true;
        if (tid == 0) count_bytes(g, CLS_MERGE, 2ull * (sizeof(K) + (HV ? sizeof(V) : 0)) * (na + nb));
    }
}

}  // namespace bs
