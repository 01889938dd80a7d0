// bs_api.cu -- C ABI, planner and set-up kernels of the block-decomposed sort.
//
// Planner (El-Nashar 2011, Fig. 1): for bs_sort_keys / bs_sort_pairs the p
// blocks of the scatter phase are the balanced bounds b_i = floor(i*n/p)
// (Fig. 1, scatter phase), written to device memory by one small kernel; for
// bs_sort_segmented the caller's offsets are the blocks.  Every block is cut
// into tiles of T keys from its start; an exclusive scan of the per-block
// tile counts gives each tile its block.  Then:
//   sort phase   1 tile-sort pass + ceil(log2(tiles per block)) merge passes
//   merge phase  ceil(log2 p) cross-block rounds (none for segmented sorts)
// Buffers ping-pong between the caller's output and the scratch copy; each
// block's tile sort writes to the buffer that makes its last pass land in the
// output, so no copy pass is needed.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <algorithm>
#include <vector>

#include "bs_internal.h"

using namespace bs;

// ====================================================================== set-up kernels

// Scatter bounds b_i = floor(i*n/p), i = 0..p (Fig. 1, scatter phase).
__global__ void balanced_offsets_kernel(int64_t *off, int64_t n, int64_t p) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= p;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned __int128 v = (unsigned __int128)(uint64_t)i * (uint64_t)n;
        off[i] = (int64_t)(v / (uint64_t)p);
    }
}

// Zeroes n 32-bit words (the persistent merge's queue head and pair
// counters).  A kernel rather than cudaMemsetAsync: a memset may be carried
// out by a copy engine, and would then queue behind large host copies.
__global__ void zero_words_kernel(unsigned *p, int64_t n) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

// Order keys: the order-preserving code of every key as a signed 64-bit
// integer -- 4-byte codes zero-extended, 8-byte codes with the top bit
// flipped -- so that a signed comparison gives the sort order.
template <class K>
__global__ void order_keys_kernel(const K *__restrict__ in, int64_t *out, int64_t n, int codec) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const K c = enc_code(in[i], codec);
        out[i] = sizeof(K) == 4 ? (int64_t)(uint64_t)c : (int64_t)((uint64_t)c ^ 0x8000000000000000ull);
    }
}

// ---------------------------------------------------------------- device checkers

// The two 64-bit mixes of the multiset hashes: MurmurHash3's fmix64
// finaliser, and an add-xorshift-multiply mix (shifts 29, 32, 29), as
// bsort.h defines them.
__device__ __forceinline__ uint64_t check_mix_a(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}
__device__ __forceinline__ uint64_t check_mix_b(uint64_t x) {
    x += 0x632be59bd9b4e019ull;
    x ^= x >> 29;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 32;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 29;
    return x;
}

// Device-side accumulators of bs_check_keys: the smallest offending
// positions (all ones = none) and the two hash sums.
struct CheckAcc {
    unsigned long long first_unsorted, first_unstable, hash_a, hash_b;
};

// Whether position i (0 < i < n) starts a segment: some off[s] == i.  A
// binary search for the largest s with off[s] <= i (off[0] = 0 <= i and
// off[S] = n > i bracket it); it runs only where the keys drop or tie.
__device__ __forceinline__ bool check_seg_start(const int64_t *off, int64_t S, int64_t i) {
    int64_t lo = 0, hi = S;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return off[lo] == i;
}

// One pass over the keys: each key's code into both hash sums; at every
// position whose key is below its predecessor's (a drop), or equal to it
// with a payload index not above the predecessor's (stability), the
// position unless it starts a segment.  Index payloads are compared as
// signed (isigned) or unsigned 64-bit integers.  One atomic per warp.
template <class K>
__global__ void check_keys_kernel(const K *__restrict__ keys, int64_t n, int codec, const int64_t *off,
                                  int64_t S, const void *idx, int iw, int isigned, CheckAcc *acc) {
    griddep_wait();
    uint64_t ha = 0, hb = 0;
    unsigned long long bad = ~0ull, unst = ~0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t c = (uint64_t)enc_code(keys[i], codec);
        ha += check_mix_a(c);
        hb += check_mix_b(c);
        if (i == 0) continue;
        const uint64_t pc = (uint64_t)enc_code(keys[i - 1], codec);
        if (pc > c) {
            if (!(off && check_seg_start(off, S, i)) && (unsigned long long)i < bad) bad = (unsigned long long)i;
        } else if (pc == c && idx) {
            uint64_t a, b;
            if (iw == 4) {
                const uint32_t *x = static_cast<const uint32_t *>(idx);
                a = isigned ? (uint64_t)(int64_t)(int32_t)x[i - 1] : (uint64_t)x[i - 1];
                b = isigned ? (uint64_t)(int64_t)(int32_t)x[i] : (uint64_t)x[i];
            } else {
                const uint64_t *x = static_cast<const uint64_t *>(idx);
                a = x[i - 1];
                b = x[i];
            }
            if (isigned) {  // signed order as unsigned: flip the sign bits
                a ^= 0x8000000000000000ull;
                b ^= 0x8000000000000000ull;
            }
            if (a >= b && !(off && check_seg_start(off, S, i)) && (unsigned long long)i < unst)
                unst = (unsigned long long)i;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        ha += __shfl_xor_sync(0xffffffffu, ha, d);
        hb += __shfl_xor_sync(0xffffffffu, hb, d);
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bad, d);
        const unsigned long long ou = __shfl_xor_sync(0xffffffffu, unst, d);
        bad = ob < bad ? ob : bad;
        unst = ou < unst ? ou : unst;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc->hash_a, (unsigned long long)ha);
        atomicAdd(&acc->hash_b, (unsigned long long)hb);
        if (bad != ~0ull) atomicMin(&acc->first_unsorted, bad);
        if (unst != ~0ull) atomicMin(&acc->first_unstable, unst);
    }
}

// Caller offsets must start at 0, end at n, never decrease, and (when a
// bound is given) hold no segment longer than max_len.
__global__ void validate_offsets_kernel(const int64_t *off, int64_t S, int64_t n, int64_t max_len,
                                        int *err) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = off[i], hi = off[i + 1];
        bool bad = hi < lo || lo < 0 || hi > n || (max_len > 0 && hi - lo > max_len);
        if (i == 0 && lo != 0) bad = true;
        if (i == S - 1 && hi != n) bad = true;
        if (bad) atomicCAS(err, 0, (int)BS_ERR_INVALID_ARG);
    }
}

// Gathered segments: segment s reads len_s items from src_off[s] of an input
// array of n_in items.
__global__ void validate_gather_kernel(const int64_t *off, const int64_t *src_off, int64_t S,
                                       int64_t n_in, int *err) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = off[i + 1] - off[i], so = src_off[i];
        if (so < 0 || len < 0 || so > n_in - len) atomicCAS(err, 0, (int)BS_ERR_INVALID_ARG);
    }
}

constexpr int SCAN_TH = 256, SCAN_IT = 16, SCAN_BLOCK = SCAN_TH * SCAN_IT;

__device__ __forceinline__ int64_t tiles_of(const int64_t *off, int64_t s, int64_t n, int logT) {
    int64_t lo = clamp64(off[s], 0, n), hi = clamp64(off[s + 1], lo, n);
    return (hi - lo + (int64_t(1) << logT) - 1) >> logT;
}

// Block-local inclusive scan of the per-segment tile counts.
__global__ void __launch_bounds__(SCAN_TH)
tile_scan_block_kernel(const int64_t *off, int64_t S, int64_t n, int logT, int64_t *tprefix,
                       int64_t *bsum) {
    __shared__ int64_t warp_tot[SCAN_TH / 32];
    griddep_wait();
    const int64_t base = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x * (int64_t)SCAN_IT;
    int64_t v[SCAN_IT];
    int64_t run = 0;
#pragma unroll
    for (int u = 0; u < SCAN_IT; ++u) {
        int64_t i = base + u;
        run += (i < S) ? tiles_of(off, i, n, logT) : 0;
        v[u] = run;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    int64_t wprefix = 0;
    for (int w = 0; w < wid; ++w) wprefix += warp_tot[w];
    const int64_t excl = wprefix + x - run;
#pragma unroll
    for (int u = 0; u < SCAN_IT; ++u) {
        int64_t i = base + u;
        if (i < S) tprefix[i + 1] = excl + v[u];
    }
    if (threadIdx.x == SCAN_TH - 1) bsum[blockIdx.x] = excl + run;
    if (blockIdx.x == 0 && threadIdx.x == 0) tprefix[0] = 0;
}

// Exclusive scan of the block totals in place (one CTA, chunked with carry).
__global__ void tile_scan_top_kernel(int64_t *bsum, int64_t nb) {
    griddep_wait();
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
        int64_t i = c0 + threadIdx.x;
        int64_t val = i < nb ? bsum[i] : 0;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int64_t x = val;
        for (int d = 1; d < 32; d <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        int64_t wprefix = 0;
        for (int w = 0; w < wid; ++w) wprefix += warp_tot[w];
        const int64_t base = carry;
        if (i < nb) bsum[i] = base + wprefix + x - val;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = base + wprefix + x;
        __syncthreads();
    }
}

__global__ void tile_scan_add_kernel(int64_t *tprefix, const int64_t *bsum, int64_t S) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S;
         i += (int64_t)gridDim.x * blockDim.x)
        tprefix[i + 1] += bsum[i / SCAN_BLOCK];
}

// The plan of a sort in one kernel, for up to PLAN_MAX_CHUNKS chunks of
// SCAN_BLOCK blocks: the block bounds -- balanced ones b_i = floor(i*n/p)
// written to off_w (Fig. 1, scatter phase), or the caller's offsets (and
// gathered sources) checked, as validate_offsets_kernel and
// validate_gather_kernel do --, each block's tile count and their exclusive
// scan into tprefix, and `nzero` words (the persistent merge's counters)
// zeroed.  Blocks of at most wmax keys get no tiles (the tile sort's warp
// length class sorts them).  CTA c < nsb scans chunk c on its own (tprefix[i+1] = the tiles of
// the chunk's blocks up to i); every CTA zeroes a share of the words; the
// last CTA to finish, found by a ticket it then resets to zero, turns the
// chunk totals into offsets and adds them to the later chunks' entries.  No
// CTA waits for another, so the kernel needs no co-resident grid.
constexpr int PLAN_MAX_CHUNKS = 64;

__global__ void __launch_bounds__(SCAN_TH)
plan_scan_kernel(int64_t *off_w, const int64_t *off_r, int64_t S, int64_t n, int64_t p, int logT,
                 int64_t wmax, int64_t max_len, const int64_t *src_off, int64_t n_in, int *err,
                 int64_t *tprefix, int64_t *bsum, unsigned *ticket, unsigned *zero, int64_t nzero) {
    __shared__ int64_t warp_tot[SCAN_TH / 32];
    __shared__ int64_t chunk_base[PLAN_MAX_CHUNKS];
    __shared__ int last;
    griddep_wait();
    const int64_t nsb = (S + SCAN_BLOCK - 1) / SCAN_BLOCK;
    for (int64_t i = blockIdx.x * (int64_t)SCAN_TH + threadIdx.x; i < nzero; i += (int64_t)gridDim.x * SCAN_TH)
        zero[i] = 0u;
    if (blockIdx.x < nsb) {
        const int64_t base = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x * (int64_t)SCAN_IT;
        int64_t v[SCAN_IT];
        int64_t run = 0;
#pragma unroll
        for (int u = 0; u < SCAN_IT; ++u) {
            const int64_t i = base + u;
            int64_t t = 0;
            if (i < S) {
                int64_t lo, hi;
                if (off_w) {
                    lo = (int64_t)(((unsigned __int128)(uint64_t)i * (uint64_t)n) / (uint64_t)p);
                    hi = (int64_t)(((unsigned __int128)(uint64_t)(i + 1) * (uint64_t)n) / (uint64_t)p);
                    off_w[i] = lo;
                    if (i == S - 1) off_w[S] = hi;
                } else {
                    lo = off_r[i];
                    hi = off_r[i + 1];
                    bool bad = hi < lo || lo < 0 || hi > n || (max_len > 0 && hi - lo > max_len);
                    if (i == 0 && lo != 0) bad = true;
                    if (i == S - 1 && hi != n) bad = true;
                    if (src_off) {
                        const int64_t so = src_off[i], len = hi - lo;
                        if (so < 0 || len < 0 || so > n_in - len) bad = true;
                    }
                    if (bad) atomicCAS(err, 0, (int)BS_ERR_INVALID_ARG);
                    lo = clamp64(lo, 0, n);
                    hi = clamp64(hi, lo, n);
                }
                // a segment of the warp length class has no tiles
                t = hi - lo <= wmax ? 0 : (hi - lo + (int64_t(1) << logT) - 1) >> logT;
            }
            run += t;
            v[u] = run;
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int64_t x = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        int64_t wprefix = 0;
        for (int w = 0; w < wid; ++w) wprefix += warp_tot[w];
        const int64_t excl = wprefix + x - run;
#pragma unroll
        for (int u = 0; u < SCAN_IT; ++u) {
            const int64_t i = base + u;
            if (i < S) tprefix[i + 1] = excl + v[u];
        }
        if (threadIdx.x == SCAN_TH - 1) bsum[blockIdx.x] = excl + run;
        if (blockIdx.x == 0 && threadIdx.x == 0) tprefix[0] = 0;
    }
    // the last CTA to finish adds the earlier chunks' totals
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's writes, before its ticket
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();  // every CTA's writes (their tickets came first)
    if (nsb > 1) {
        if (threadIdx.x == 0) {
            int64_t acc = 0;
            for (int64_t c = 0; c < nsb; ++c) {
                chunk_base[c] = acc;
                acc += __ldcg(bsum + c);
            }
        }
        __syncthreads();
        for (int64_t i = SCAN_BLOCK + threadIdx.x; i < S; i += SCAN_TH)
            tprefix[i + 1] = __ldcg(tprefix + i + 1) + chunk_base[i / SCAN_BLOCK];
    }
    if (threadIdx.x == 0) *ticket = 0u;  // ready for the next sort
}

// tseg[t] = the segment owning tile t (t < total tiles).
__global__ void tile_map_kernel(const int64_t *tprefix, int64_t S, int32_t *tseg, int64_t ub) {
    griddep_wait();
    const int64_t total = tprefix[S];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ub && t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = S;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (tprefix[mid] <= t) lo = mid;
            else hi = mid;
        }
        tseg[t] = (int32_t)lo;
    }
}

// ====================================================================== handle

// Most slots of bs_sort_keys_host_async (BS_OPT_HOST_SLOTS: 2 or 3, default
// 3): with three the copy out of call k-3, not of call k-2, gates the sort of
// call k, so a copy out that runs a little longer than one sort (the host
// link shared with the copy in) does not stall the sorts.
constexpr int HOST_SLOTS = 3;

struct bs_handle {
    int device = 0;
    int sms = 1;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int *d_err = nullptr;
    unsigned long long *d_counters = nullptr;
    unsigned *d_ticket = nullptr;  // plan_scan_kernel's ticket: zero between sorts
    int64_t launches[BS_KERNEL_CLASSES] = {0, 0, 0, 0};
    int logT = 12;
    int merge_impl = MERGE_AUTO;
    int merge_vt = 0;         // 0: 32 for 32-bit keys alone, 16 for wider items
    uint64_t wait_ns = 0;  // 0: the kernels' default limit
    int withhold = 0;      // test hook (BS_OPT_TEST_WITHHOLD)
    int schedule = BS_SCHEDULE_TREE;
    int local_sort = BS_LOCAL_MERGE;
    int merge_tile_log2 = 0;  // 0: the sort tile
    int merge_consumer = 0;   // 0 per-thread sequential merge, 1 warp bitonic merger
    int host_direct = 1;      // bs_sort_keys_host: address page-locked host buffers directly
    int count_bytes = 0;      // kernels count algorithmic bytes (BS_OPT_COUNT_BYTES)
    int persistent = 1;       // every merge level in one persistent launch: 1 when large enough,
                              // 2 always, 0 never (BS_OPT_MERGE_PERSISTENT)
    int length_classes = 1;   // warp length class for short segments (BS_OPT_LENGTH_CLASSES)
    cudaStream_t last_stream = nullptr;
    // per-launch timing
    bool timing = false;
    struct Ev {
        cudaEvent_t a, b;
        int cls;
    };
    std::vector<Ev> evs;
    std::vector<cudaEvent_t> spare;
    // host-buffer entry point
    cudaStream_t own_stream = nullptr;
    void *hb = nullptr;
    size_t hb_bytes = 0;
    // bs_sort_keys_host_async: HOST_SLOTS slots used in turn, each an input
    // and an output device buffer; a stream for the copies in and one for
    // the copies out, and per slot the events "copied in", "sorted",
    // "copied out"
    void *ab[HOST_SLOTS] = {}, *ob[HOST_SLOTS] = {};
    size_t ab_bytes[HOST_SLOTS] = {}, ob_bytes[HOST_SLOTS] = {};
    cudaStream_t cp_in = nullptr, cp_out = nullptr;
    cudaEvent_t ev_in[HOST_SLOTS] = {}, ev_sorted[HOST_SLOTS] = {}, ev_out[HOST_SLOTS] = {};
    unsigned long long async_calls = 0;
    int host_slots = HOST_SLOTS;  // slots in use (BS_OPT_HOST_SLOTS)
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

cudaEvent_t take_event(bs_handle *h) {
    if (!h->spare.empty()) {
        cudaEvent_t e = h->spare.back();
        h->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void launch_begin(void *owner, int cls, cudaStream_t s) {
    bs_handle *h = (bs_handle *)owner;
    if (!h->timing) return;
    bs_handle::Ev ev{take_event(h), take_event(h), cls};
    if (ev.a && ev.b) {
        cudaEventRecord(ev.a, s);
        h->evs.push_back(ev);
    }
}

bool launch_end(void *owner, int cls, cudaStream_t s) {
    bs_handle *h = (bs_handle *)owner;
    if (cudaGetLastError() != cudaSuccess) return false;
    h->launches[cls]++;
    if (h->timing && !h->evs.empty() && h->evs.back().cls == cls) cudaEventRecord(h->evs.back().b, s);
    return true;
}

struct WsLayout {
    size_t tmp_k, tmp_v, off, tprefix, bsum, tseg, split, pcnt, total;
    int64_t pcnt_words;
};

constexpr int64_t MIN_TILE = 2048;

WsLayout ws_layout(int64_t n, int64_t S, size_t ks, size_t vs, int64_t extra_tiles = 0) {
    WsLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += (bytes + 255) & ~size_t(255);
        return at;
    };
    const int64_t gt = (n + MIN_TILE - 1) / MIN_TILE;
    const int64_t ub = gt + S + 1;
    L.tmp_k = take((size_t)n * ks);
    L.tmp_v = take((size_t)n * vs);
    L.off = take((size_t)(S + 1) * 8);
    L.tprefix = take((size_t)(S + 1) * 8);
    L.bsum = take((size_t)((S + 1) / SCAN_BLOCK + 2) * 8);
    int64_t xt = xblock_tiles_max(n, S, 11);
    if (extra_tiles > xt) xt = extra_tiles;
    // in-block levels launch (n / T + S + 1) << (logT - mlogT) merge tiles, with
    // 2^11 <= 2^mlogT <= T <= 2^13: at most n / 2^11 + 4 (S + 1)
    const int64_t seg_merge_tiles = (n + MIN_TILE - 1) / MIN_TILE + 4 * (S + 1);
    if (seg_merge_tiles > xt) xt = seg_merge_tiles;
    L.tseg = take((size_t)ub * 4);
    L.split = take((size_t)((ub > xt ? ub : xt) + 1) * 8);
    // persistent merge: work queue + pair counters, for the largest in-block
    // level count any tile size gives (levels of 2^11-key tiles)
    int lv = 0, R = 0;
    while ((int64_t(MIN_TILE) << lv) < n) ++lv;
    while ((int64_t(1) << R) < S) ++R;
    L.pcnt_words = persist_words(lv, ub, R, S);
    L.pcnt = take((size_t)L.pcnt_words * 4);
    L.total = o;
    return L;
}

bs_status ensure_ws(bs_handle *h, size_t bytes) {
    if (bytes <= h->ws_bytes) return BS_OK;
    if (h->ws) {
        cudaDeviceSynchronize();  // the old workspace may still be in use
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_OUT_OF_MEMORY;
    }
    h->ws_bytes = bytes;
    return BS_OK;
}

int key_width(bs_dtype t) {
    switch (t) {
    case BS_INT32:
    case BS_UINT32:
    case BS_FLOAT32: return 4;
    case BS_INT64:
    case BS_UINT64:
    case BS_FLOAT64: return 8;
    default: return 0;
    }
}

int key_codec(bs_dtype t) {
    switch (t) {
    case BS_INT32:
    case BS_INT64: return CODEC_SIGNED;
    case BS_FLOAT32:
    case BS_FLOAT64: return CODEC_FLOAT;
    default: return CODEC_IDENT;
    }
}

int levels_for(int64_t len, int logT) {
    if (len <= (int64_t(1) << logT)) return 0;
    int64_t tiles = (len + (int64_t(1) << logT) - 1) >> logT;
    int l = 0;
    while ((int64_t(1) << l) < tiles) ++l;
    return l;
}

int ceil_log2(int64_t p) {
    int r = 0;
    while ((int64_t(1) << r) < p) ++r;
    return r;
}

inline unsigned blocks_for(int64_t work, int threads, int cap) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// The whole method for one call.  balanced: blocks are floor(i*n/p); else
// user_off holds S+1 segment offsets (no cross-block rounds).
// fin_k (nullable): where the decoded keys go instead of kout, which then
// only serves as ping-pong buffer 0 (pinned host memory the GPU addresses).
bs_status do_sort(bs_handle *h, const void *kin, void *kout, const void *vin, void *vout, int64_t n,
                  bs_dtype kt, int vbytes, bool balanced, int64_t p, const int64_t *user_off,
                  int64_t S, int64_t max_len, cudaStream_t stream, const int64_t *src_off = nullptr,
                  int64_t n_in = 0, bool oddeven = false, void *fin_k = nullptr) {
    const int kw = key_width(kt);
    const int64_t blocks = balanced ? p : S;
    if (blocks > INT32_MAX) return BS_ERR_INVALID_ARG;
    // odd-even schedule: the sort runs on p padded blocks of cap keys each
    const int64_t slot_cap = oddeven ? (n + p - 1) / p : 0;
    const int64_t n_user = n;
    const void *kout_user = fin_k ? fin_k : kout;
    if (oddeven) n = slot_cap * p;
    const WsLayout W = ws_layout(n, blocks, (size_t)kw, (size_t)vbytes);
    const size_t pad_bytes = oddeven ? (((size_t)n * kw + 255) & ~size_t(255)) : 0;
    bs_status st = ensure_ws(h, W.total + pad_bytes);
    if (st != BS_OK) return st;
    char *ws = (char *)h->ws;
    h->last_stream = stream;

    Geo g{};
    g.S = blocks;
    g.n = n;
    g.logT = h->logT;
    g.tprefix = (const int64_t *)(ws + W.tprefix);
    g.tseg = (const int32_t *)(ws + W.tseg);
    g.counters = h->count_bytes ? h->d_counters : nullptr;
    g.err = h->d_err;
    g.wait_ns = h->wait_ns;
    g.withhold = h->withhold;
    g.R = balanced ? ceil_log2(p) : 0;
    g.fin_k = oddeven ? nullptr : fin_k;  // the odd-even form decodes in its compaction

    Launcher L{stream, h, h->sms, launch_begin, launch_end};
    int codec = key_codec(kt);
    // the persistent merge's queue head and pair counters start at zero
    const int64_t T0 = int64_t(1) << g.logT;
    const int64_t ub0 = (n + T0 - 1) / T0 + blocks;
    int64_t Lmax0 = 0;
    if (balanced) {
        Lmax0 = levels_for((n + p - 1) / p, g.logT);
    } else {
        const int64_t lim = (max_len > 0 && max_len < n) ? max_len : n;
        Lmax0 = levels_for(lim, g.logT);
    }
    const bool persist = h->persistent && !oddeven;
    const int64_t pwords = persist_words((int)Lmax0, ub0, g.R, blocks);
    const int64_t nzero = (persist && pwords <= W.pcnt_words) ? pwords : 0;
    if (oddeven) {
        // scatter + encode into the padded buffer A; then sort A in place
        void *A = ws + W.total;
        st = kw == 4 ? oddeven_scatter_u32(kin, A, n_user, p, slot_cap, codec, L)
                     : oddeven_scatter_u64(kin, A, n_user, p, slot_cap, codec, L);
        if (st != BS_OK) return st;
        kin = A;
        kout = A;
        codec = CODEC_IDENT;
        g.R = 0;
    }
    const int cap = h->sms * 8;
    int64_t *tprefix = (int64_t *)(ws + W.tprefix);
    int64_t *bsum = (int64_t *)(ws + W.bsum);
    const int64_t nsb = (blocks + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (!balanced) {
        g.off = user_off;
        if (src_off) {
            g.src_off = src_off;
            g.n_in = n_in;
        }
    }
    // the warp length class: keys alone, the default tile sort, tree schedule
    // (balanced blocks: only when they are that short)
    if (h->length_classes && vbytes == 0 && h->local_sort == BS_LOCAL_MERGE && !oddeven &&
        nsb <= PLAN_MAX_CHUNKS && (!balanced || (n + p - 1) / p <= warp_class_max(g.logT)))
        g.wmax = warp_class_max(g.logT);
    if (nsb <= PLAN_MAX_CHUNKS) {
        // bounds or their checks, tile scan and counter zeroing in one kernel
        int64_t *off_w = balanced ? (int64_t *)(ws + W.off) : nullptr;
        if (balanced) g.off = off_w;
        int64_t zc = (nzero + SCAN_TH * 16 - 1) / (SCAN_TH * 16);
        if (zc > 2 * (int64_t)h->sms) zc = 2 * (int64_t)h->sms;
        const int64_t grid = nsb > zc ? nsb : zc;
        launch_begin(h, CLS_SETUP, stream);
        launch_overlapped(plan_scan_kernel, (unsigned)(grid > 0 ? grid : 1), SCAN_TH, 0, stream, off_w,
                          balanced ? nullptr : user_off, blocks, n, balanced ? p : int64_t(1), g.logT,
                          g.wmax, balanced ? int64_t(0) : max_len, balanced ? nullptr : src_off, n_in, h->d_err,
                          tprefix, bsum, h->d_ticket, (unsigned *)(ws + W.pcnt), nzero);
        if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
    } else {
        if (nzero) {
            launch_begin(h, CLS_SETUP, stream);
            launch_overlapped(zero_words_kernel, blocks_for(nzero, 256, h->sms * 8), 256, 0, stream,
                              (unsigned *)(ws + W.pcnt), nzero);
            if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
        }
        if (balanced) {
            int64_t *off = (int64_t *)(ws + W.off);
            launch_begin(h, CLS_SETUP, stream);
            launch_overlapped(balanced_offsets_kernel, blocks_for(p + 1, 256, cap), 256, 0, stream, off, n, p);
            if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
            g.off = off;
        } else {
            launch_begin(h, CLS_SETUP, stream);
            launch_overlapped(validate_offsets_kernel, blocks_for(S, 256, cap), 256, 0, stream, user_off, S, n,
                              max_len, h->d_err);
            if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
            if (src_off) {
                launch_begin(h, CLS_SETUP, stream);
                launch_overlapped(validate_gather_kernel, blocks_for(S, 256, cap), 256, 0, stream, user_off,
                                  src_off, S, n_in, h->d_err);
                if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
            }
        }
        // exclusive scan of tiles per block
        launch_begin(h, CLS_SETUP, stream);
        launch_overlapped(tile_scan_block_kernel, (unsigned)nsb, SCAN_TH, 0, stream, g.off, blocks, n, g.logT,
                          tprefix, bsum);
        if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
        launch_begin(h, CLS_SETUP, stream);
        launch_overlapped(tile_scan_top_kernel, 1, 1024, 0, stream, bsum, nsb);
        if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
        launch_begin(h, CLS_SETUP, stream);
        launch_overlapped(tile_scan_add_kernel, blocks_for(blocks, 256, cap), 256, 0, stream, tprefix, bsum,
                          blocks);
        if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
    }

    // tile map: tile -> block (none when every block is in the warp length
    // class: balanced blocks that short, or segments bounded by max_len; a
    // longer segment is flagged by the plan)
    const int64_t T = int64_t(1) << g.logT;
    const int64_t ub = (n + T - 1) / T + blocks;
    const bool no_tiles = g.wmax > 0 && (balanced || (max_len > 0 && max_len <= g.wmax));
    g.ntiles_ub = ub;
    if (!no_tiles) {
        launch_begin(h, CLS_SETUP, stream);
        launch_overlapped(tile_map_kernel, blocks_for(ub, 256, cap), 256, 0, stream, tprefix, blocks,
                          (int32_t *)g.tseg, ub);
        if (!launch_end(h, CLS_SETUP, stream)) return BS_ERR_CUDA;
    }

    PassArgs a{};
    a.g = g;  // g.ntiles_ub is set above, before the tile map launch
    a.in_k = kin;
    a.in_v = vin;
    a.k0 = kout;
    a.k1 = ws + W.tmp_k;
    a.v0 = vout;
    a.v1 = vbytes ? (void *)(ws + W.tmp_v) : nullptr;
    a.codec = codec;
    a.vbytes = vbytes;
    if (balanced) {
        a.Lmax = levels_for((n + p - 1) / p, g.logT);
    } else {
        int64_t lim = (max_len > 0 && max_len < n) ? max_len : n;
        a.Lmax = levels_for(lim, g.logT);
    }
    a.ntiles_ub = ub;
    a.ntiles_total = tprefix + blocks;
    a.split = (int64_t *)(ws + W.split);
    const uintptr_t al = (uintptr_t)kout | (uintptr_t)a.k1 | (uintptr_t)vout | (uintptr_t)a.v1 |
                         (uintptr_t)g.fin_k;
    a.merge_impl = (al & 15) ? MERGE_SIMPLE : h->merge_impl;
    a.merge_vt = h->merge_vt;
    a.oddeven_rounds = oddeven ? (int)p : 0;
    a.local_sort = h->local_sort;
    a.merge_tile_log2 = h->merge_tile_log2;
    a.merge_consumer = h->merge_consumer;
    a.persistent = (persist && pwords <= W.pcnt_words) ? h->persistent : 0;
    a.pcnt = (unsigned *)(ws + W.pcnt);
    a.pcnt_words = pwords;
    a.no_tiles = no_tiles;
    st = kw == 4 ? run_passes_u32(a, L) : run_passes_u64(a, L);
    if (st != BS_OK || !oddeven) return st;
    // after p rounds the keys are in buffer (p & 1): decode the first n
    const void *res = (p & 1) ? a.k1 : a.k0;
    return kw == 4 ? oddeven_compact_u32(res, (void *)kout_user, n_user, key_codec(kt), L)
                   : oddeven_compact_u64(res, (void *)kout_user, n_user, key_codec(kt), L);
}

int value_width(bs_dtype vt) {
    if (vt == BS_NONE) return 0;
    return key_width(vt);
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

bs_status bs_create(bs_handle **out, int device) {
    if (!out) return BS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return BS_ERR_INVALID_ARG;
    DevGuard dg(device);
    bs_handle *h = new (std::nothrow) bs_handle();
    if (!h) return BS_ERR_OUT_OF_MEMORY;
    h->device = device;
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) h->sms = 1;
    if (cudaMalloc(&h->d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->d_counters, sizeof(unsigned long long) * BS_KERNEL_CLASSES) != cudaSuccess ||
        cudaMalloc(&h->d_ticket, sizeof(unsigned)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        bs_destroy(h);
        return BS_ERR_OUT_OF_MEMORY;
    }
    cudaMemset(h->d_err, 0, sizeof(int));
    cudaMemset(h->d_counters, 0, sizeof(unsigned long long) * BS_KERNEL_CLASSES);
    cudaMemset(h->d_ticket, 0, sizeof(unsigned));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        bs_destroy(h);
        return BS_ERR_CUDA;
    }
    *out = h;
    return BS_OK;
}

bs_status bs_destroy(bs_handle *h) {
    if (!h) return BS_OK;
    DevGuard dg(h->device);
    cudaDeviceSynchronize();
    for (auto &e : h->evs) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (auto e : h->spare) cudaEventDestroy(e);
    if (h->ws) cudaFree(h->ws);
    if (h->hb) cudaFree(h->hb);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_counters) cudaFree(h->d_counters);
    if (h->d_ticket) cudaFree(h->d_ticket);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    for (int j = 0; j < HOST_SLOTS; ++j) {
        if (h->ab[j]) cudaFree(h->ab[j]);
        if (h->ob[j]) cudaFree(h->ob[j]);
        if (h->ev_in[j]) cudaEventDestroy(h->ev_in[j]);
        if (h->ev_sorted[j]) cudaEventDestroy(h->ev_sorted[j]);
        if (h->ev_out[j]) cudaEventDestroy(h->ev_out[j]);
    }
    if (h->cp_in) cudaStreamDestroy(h->cp_in);
    if (h->cp_out) cudaStreamDestroy(h->cp_out);
    delete h;
    return BS_OK;
}

bs_status bs_sort_keys(bs_handle *h, const void *d_in, void *d_out, int64_t n, bs_dtype kt, int64_t p,
                       void *stream) {
    if (!h || n < 0 || p < 0) return BS_ERR_INVALID_ARG;
    if (!key_width(kt)) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0) return BS_OK;
    if (!d_in || !d_out) return BS_ERR_INVALID_ARG;
    if (p == 0) p = 1;
    if (p > n) p = n;
    DevGuard dg(h->device);
    if (h->schedule == BS_SCHEDULE_ODDEVEN && p >= 2)
        return do_sort(h, d_in, d_out, nullptr, nullptr, n, kt, 0, true, p, nullptr, p, 0,
                       (cudaStream_t)stream, nullptr, 0, true);
    return do_sort(h, d_in, d_out, nullptr, nullptr, n, kt, 0, true, p, nullptr, p, 0,
                   (cudaStream_t)stream);
}

bs_status bs_sort_pairs(bs_handle *h, const void *d_kin, void *d_kout, const void *d_vin, void *d_vout,
                        int64_t n, bs_dtype kt, bs_dtype vt, int64_t p, void *stream) {
    if (!h || n < 0 || p < 0) return BS_ERR_INVALID_ARG;
    if (!key_width(kt) || !value_width(vt)) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0) return BS_OK;
    if (!d_kin || !d_kout || !d_vin || !d_vout) return BS_ERR_INVALID_ARG;
    if (p == 0) p = 1;
    if (p > n) p = n;
    DevGuard dg(h->device);
    return do_sort(h, d_kin, d_kout, d_vin, d_vout, n, kt, value_width(vt), true, p, nullptr, p, 0,
                   (cudaStream_t)stream);
}

bs_status bs_sort_segmented(bs_handle *h, const void *d_kin, void *d_kout, const void *d_vin,
                            void *d_vout, int64_t n, const int64_t *d_offsets, int64_t S,
                            int64_t max_seg_len, bs_dtype kt, bs_dtype vt, void *stream) {
    if (!h || n < 0 || S < 0 || max_seg_len < 0) return BS_ERR_INVALID_ARG;
    if (!key_width(kt)) return BS_ERR_UNSUPPORTED_DTYPE;
    const bool has_v = (vt != BS_NONE);
    if (has_v && !value_width(vt)) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0 && S == 0) return BS_OK;
    if (S == 0 || !d_offsets) return BS_ERR_INVALID_ARG;  // offsets must cover [0, n)
    if (n > 0 && (!d_kin || !d_kout)) return BS_ERR_INVALID_ARG;
    if (has_v && n > 0 && (!d_vin || !d_vout)) return BS_ERR_INVALID_ARG;
    if (!has_v && (d_vin || d_vout)) return BS_ERR_INVALID_ARG;
    DevGuard dg(h->device);
    if (n == 0) {
        // still check the offsets (all must be 0)
        h->last_stream = (cudaStream_t)stream;
        launch_begin(h, CLS_SETUP, (cudaStream_t)stream);
        launch_overlapped(validate_offsets_kernel, blocks_for(S, 256, h->sms * 8), 256, 0,
                          (cudaStream_t)stream, d_offsets, S, 0, 0, h->d_err);
        return launch_end(h, CLS_SETUP, (cudaStream_t)stream) ? BS_OK : BS_ERR_CUDA;
    }
    return do_sort(h, d_kin, d_kout, has_v ? d_vin : nullptr, has_v ? d_vout : nullptr, n, kt,
                   has_v ? value_width(vt) : 0, false, 0, d_offsets, S, max_seg_len,
                   (cudaStream_t)stream);
}

bs_status bs_sort_segmented_gather(bs_handle *h, const void *d_kin, int64_t n_in,
                                   const int64_t *d_src_offsets, void *d_kout, const void *d_vin,
                                   void *d_vout, int64_t n, const int64_t *d_offsets, int64_t S,
                                   int64_t max_seg_len, bs_dtype kt, bs_dtype vt, void *stream) {
    if (!h || n < 0 || n_in < 0 || S < 0 || max_seg_len < 0) return BS_ERR_INVALID_ARG;
    if (!key_width(kt)) return BS_ERR_UNSUPPORTED_DTYPE;
    const bool has_v = (vt != BS_NONE);
    if (has_v && !value_width(vt)) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0 && S == 0) return BS_OK;
    if (S == 0 || !d_offsets || !d_src_offsets) return BS_ERR_INVALID_ARG;
    if (n > 0 && (!d_kin || !d_kout)) return BS_ERR_INVALID_ARG;
    if (has_v && n > 0 && (!d_vin || !d_vout)) return BS_ERR_INVALID_ARG;
    if (!has_v && (d_vin || d_vout)) return BS_ERR_INVALID_ARG;
    if (n == 0) return bs_sort_segmented(h, d_kin, d_kout, d_vin, d_vout, 0, d_offsets, S, 0, kt, vt, stream);
    DevGuard dg(h->device);
    return do_sort(h, d_kin, d_kout, has_v ? d_vin : nullptr, has_v ? d_vout : nullptr, n, kt,
                   has_v ? value_width(vt) : 0, false, 0, d_offsets, S, max_seg_len,
                   (cudaStream_t)stream, d_src_offsets, n_in);
}

bs_status bs_merge_runs(bs_handle *h, const void *d_kin, void *d_kout, const void *d_vin,
                        void *d_vout, int64_t n, const int64_t *h_run_offsets, int64_t runs,
                        bs_dtype kt, bs_dtype vt, void *stream) {
    if (!h || n < 0 || runs < 1 || !h_run_offsets) return BS_ERR_INVALID_ARG;
    const int kw = key_width(kt);
    if (!kw) return BS_ERR_UNSUPPORTED_DTYPE;
    const bool has_v = (vt != BS_NONE);
    const int vw = has_v ? value_width(vt) : 0;
    if (has_v && !vw) return BS_ERR_UNSUPPORTED_DTYPE;
    if (h_run_offsets[0] != 0 || h_run_offsets[runs] != n) return BS_ERR_INVALID_ARG;
    for (int64_t i = 0; i < runs; ++i)
        if (h_run_offsets[i + 1] < h_run_offsets[i]) return BS_ERR_INVALID_ARG;
    if (runs > INT32_MAX) return BS_ERR_INVALID_ARG;
    if (n == 0) return BS_OK;
    if (!d_kin || !d_kout || (has_v && (!d_vin || !d_vout))) return BS_ERR_INVALID_ARG;
    DevGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    if (runs == 1) {
        if (d_kin != d_kout &&
            cudaMemcpyAsync(d_kout, d_kin, (size_t)n * kw, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return BS_ERR_CUDA;
        if (has_v && d_vin != d_vout &&
            cudaMemcpyAsync(d_vout, d_vin, (size_t)n * vw, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return BS_ERR_CUDA;
        return BS_OK;
    }
    // tiles per pair of every round, from the real run lengths
    const int R = ceil_log2(runs);
    const int64_t T = int64_t(1) << h->logT;
    std::vector<int64_t> tpp(R);
    int64_t need = 0;
    for (int r = 0; r < R; ++r) {
        const int64_t G = int64_t(2) << r;
        int64_t longest = 0;
        for (int64_t k = 0; k * G < runs; ++k) {
            const int64_t a = h_run_offsets[k * G], b = h_run_offsets[std::min(k * G + G, runs)];
            longest = std::max(longest, b - a);
        }
        tpp[r] = std::max<int64_t>(1, (longest + T - 1) / T);
        // merge tiles may be up to 4x smaller than sort tiles
        need = std::max(need, ((runs + G - 1) / G) * tpp[r] * 4);
    }
    const WsLayout W = ws_layout(n, runs, (size_t)kw, (size_t)vw, need);
    bs_status st = ensure_ws(h, W.total);
    if (st != BS_OK) return st;
    char *ws = (char *)h->ws;
    int64_t *off = (int64_t *)(ws + W.off);
    if (cudaMemcpyAsync(off, h_run_offsets, sizeof(int64_t) * (runs + 1), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return BS_ERR_CUDA;
    const int64_t pwords = persist_words(0, 0, R, runs);
    const bool persist = h->persistent && pwords <= W.pcnt_words;
    if (persist) {
        launch_begin(h, CLS_SETUP, s);
        launch_overlapped(zero_words_kernel, blocks_for(pwords, 256, h->sms * 8), 256, 0, s,
                          (unsigned *)(ws + W.pcnt), pwords);
        if (!launch_end(h, CLS_SETUP, s)) return BS_ERR_CUDA;
    }
    Geo g{};
    g.off = off;
    g.S = runs;
    g.n = n;
    g.logT = h->logT;
    g.R = R;
    g.ntiles_ub = 0;
    g.counters = h->count_bytes ? h->d_counters : nullptr;
    g.err = h->d_err;
    g.wait_ns = h->wait_ns;
    g.withhold = h->withhold;
    Launcher L{s, h, h->sms, launch_begin, launch_end};
    PassArgs a{};
    a.g = g;
    a.in_k = d_kin;
    a.in_v = has_v ? d_vin : nullptr;
    a.k0 = d_kout;
    a.k1 = ws + W.tmp_k;
    a.v0 = has_v ? d_vout : nullptr;
    a.v1 = has_v ? (void *)(ws + W.tmp_v) : nullptr;
    a.codec = key_codec(kt);
    a.vbytes = vw;
    a.Lmax = 0;
    a.ntiles_ub = 0;
    a.ntiles_total = nullptr;
    a.split = (int64_t *)(ws + W.split);
    const uintptr_t al = (uintptr_t)d_kout | (uintptr_t)a.k1 | (uintptr_t)a.v0 | (uintptr_t)a.v1;
    a.merge_impl = (al & 15) ? MERGE_SIMPLE : h->merge_impl;
    a.merge_vt = h->merge_vt;
    a.merge_only = true;
    a.tpp_host = tpp.data();
    a.oddeven_rounds = 0;
    a.local_sort = 0;
    a.merge_tile_log2 = h->merge_tile_log2;
    a.merge_consumer = h->merge_consumer;
    a.persistent = persist ? h->persistent : 0;
    a.pcnt = (unsigned *)(ws + W.pcnt);
    a.pcnt_words = pwords;
    return kw == 4 ? run_passes_u32(a, L) : run_passes_u64(a, L);
}

// Device address of host memory the GPU can access directly (page-locked
// or registered, mapped into the unified address space), else nullptr.
static void *host_device_ptr(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// A device buffer of the handle, grown to `bytes` (a growing buffer waits
// for the device first: the old one may still be in use on some stream).
static bs_status ensure_buf(void *&buf, size_t &have, size_t bytes) {
    if (bytes <= have) return BS_OK;
    if (buf) {
        cudaDeviceSynchronize();
        cudaFree(buf);
        buf = nullptr;
        have = 0;
    }
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_OUT_OF_MEMORY;
    }
    have = bytes;
    return BS_OK;
}

// Call k of bs_sort_keys_host_async uses slot j = k % HOST_SLOTS (input
// buffer in_j, output buffer out_j); call k - HOST_SLOTS used it before:
//   copy-in stream:  wait "sorted"[j] (that call has read in_j), copy h_in ->
//                    in_j, record "copied in"[j];
//   caller's stream: wait "copied in"[j], "copied out"[j] (that call's copy
//                    out has read out_j) and "sorted" of call k-1's slot (the
//                    workspace is shared), sort in_j -> out_j, record
//                    "sorted"[j];
//   copy-out stream: wait "sorted"[j], copy out_j -> h_out, record
//                    "copied out"[j].
// So call k+1's copy in and call k-1's copy out run on the copy engines while
// call k sorts, and neither copy waits for the other: a slot's next copy in
// needs only its last sort, not its copy out (one buffer per slot made the
// two copies chain behind each sort).  An event not yet recorded counts as
// complete.
bs_status bs_sort_keys_host_async(bs_handle *h, const void *h_in, void *h_out, int64_t n, bs_dtype kt,
                                  int64_t p, void *stream) {
    if (!h || n < 0 || p < 0) return BS_ERR_INVALID_ARG;
    const int kw = key_width(kt);
    if (!kw) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0) return BS_OK;
    if (!h_in || !h_out) return BS_ERR_INVALID_ARG;
    DevGuard dg(h->device);
    if (!h->cp_in) {
        if (cudaStreamCreateWithFlags(&h->cp_in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h->cp_out, cudaStreamNonBlocking) != cudaSuccess)
            return BS_ERR_CUDA;
        for (int j = 0; j < HOST_SLOTS; ++j)
            if (cudaEventCreateWithFlags(&h->ev_in[j], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_sorted[j], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_out[j], cudaEventDisableTiming) != cudaSuccess)
                return BS_ERR_CUDA;
    }
    const int ns = h->host_slots;
    const int j = (int)(h->async_calls % ns), prev = (j + ns - 1) % ns;
    const size_t bytes = (size_t)n * kw;
    bs_status st = ensure_buf(h->ab[j], h->ab_bytes[j], bytes);
    if (st == BS_OK) st = ensure_buf(h->ob[j], h->ob_bytes[j], bytes);
    if (st != BS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamWaitEvent(h->cp_in, h->ev_sorted[j], 0) != cudaSuccess ||
        cudaMemcpyAsync(h->ab[j], h_in, bytes, cudaMemcpyHostToDevice, h->cp_in) != cudaSuccess ||
        cudaEventRecord(h->ev_in[j], h->cp_in) != cudaSuccess ||
        cudaStreamWaitEvent(s, h->ev_in[j], 0) != cudaSuccess ||
        cudaStreamWaitEvent(s, h->ev_out[j], 0) != cudaSuccess ||
        cudaStreamWaitEvent(s, h->ev_sorted[prev], 0) != cudaSuccess)
        return BS_ERR_CUDA;
    st = bs_sort_keys(h, h->ab[j], h->ob[j], n, kt, p, (void *)s);
    if (st != BS_OK) return st;
    if (cudaEventRecord(h->ev_sorted[j], s) != cudaSuccess ||
        cudaStreamWaitEvent(h->cp_out, h->ev_sorted[j], 0) != cudaSuccess ||
        cudaMemcpyAsync(h_out, h->ob[j], bytes, cudaMemcpyDeviceToHost, h->cp_out) != cudaSuccess ||
        cudaEventRecord(h->ev_out[j], h->cp_out) != cudaSuccess)
        return BS_ERR_CUDA;
    h->async_calls++;
    h->last_stream = h->cp_out;  // bs_sync_status waits for the last copy out (and all before it)
    return BS_OK;
}

bs_status bs_sort_keys_host(bs_handle *h, const void *h_in, void *h_out, int64_t n, bs_dtype kt,
                            int64_t p) {
    if (!h || n < 0 || p < 0) return BS_ERR_INVALID_ARG;
    const int kw = key_width(kt);
    if (!kw) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0) return BS_OK;
    if (!h_in || !h_out) return BS_ERR_INVALID_ARG;
    DevGuard dg(h->device);
    const size_t bytes = (size_t)n * kw;
    bs_status st0 = ensure_buf(h->hb, h->hb_bytes, bytes);
    if (st0 != BS_OK) return st0;
    cudaStream_t s = h->own_stream;
    void *din = h->host_direct ? host_device_ptr(h_in) : nullptr;
    void *dout = h->host_direct ? host_device_ptr(h_out) : nullptr;
    if (din && dout) {
        // the sort phase reads h_in and the last pass writes h_out across the
        // host link; every other pass stays in HBM (hb and the workspace)
        if (p == 0) p = 1;
        if (p > n) p = n;
        const bool oe = h->schedule == BS_SCHEDULE_ODDEVEN && p >= 2;
        bs_status st = do_sort(h, din, h->hb, nullptr, nullptr, n, kt, 0, true, p, nullptr, p, 0, s,
                               nullptr, 0, oe, dout);
        if (st != BS_OK) return st;
    } else {
        if (cudaMemcpyAsync(h->hb, h_in, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return BS_ERR_CUDA;
        bs_status st = bs_sort_keys(h, h->hb, h->hb, n, kt, p, (void *)s);
        if (st != BS_OK) return st;
        if (cudaMemcpyAsync(h_out, h->hb, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return BS_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return BS_ERR_CUDA;
    return BS_OK;
}

bs_status bs_workspace_bytes(int64_t n, int64_t S, bs_dtype kt, bs_dtype vt, size_t *bytes) {
    if (!bytes || n < 0 || S < 0) return BS_ERR_INVALID_ARG;
    if (!key_width(kt) || (vt != BS_NONE && !value_width(vt))) return BS_ERR_UNSUPPORTED_DTYPE;
    if (S < 1) S = 1;
    *bytes = ws_layout(n, S, (size_t)key_width(kt), (size_t)value_width(vt)).total;
    return BS_OK;
}

bs_status bs_order_keys(const void *d_in, int64_t *d_out, int64_t n, bs_dtype kt, void *stream) {
    if (n < 0) return BS_ERR_INVALID_ARG;
    const int kw = key_width(kt);
    if (!kw) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0) return BS_OK;
    if (!d_in || !d_out) return BS_ERR_INVALID_ARG;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    const unsigned grid = blocks_for(n, 256, sms * 8);
    const cudaStream_t s = (cudaStream_t)stream;
    if (kw == 4)
        launch_overlapped(order_keys_kernel<uint32_t>, grid, 256, 0, s, (const uint32_t *)d_in, d_out, n, key_codec(kt));
    else
        launch_overlapped(order_keys_kernel<uint64_t>, grid, 256, 0, s, (const uint64_t *)d_in, d_out, n, key_codec(kt));
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_check_keys(const void *d_keys, int64_t n, bs_dtype kt, const int64_t *d_offsets, int64_t S,
                        const void *d_idx, bs_dtype it, bs_check_result *result, void *stream) {
    if (!result || n < 0 || (d_offsets && S < 1)) return BS_ERR_INVALID_ARG;
    const int kw = key_width(kt);
    if (!kw) return BS_ERR_UNSUPPORTED_DTYPE;
    int iw = 0, isigned = 0;
    if (d_idx) {
        switch (it) {
        case BS_INT32: iw = 4, isigned = 1; break;
        case BS_UINT32: iw = 4; break;
        case BS_INT64: iw = 8, isigned = 1; break;
        case BS_UINT64: iw = 8; break;
        default: return BS_ERR_UNSUPPORTED_DTYPE;
        }
    }
    if (n > 0 && !d_keys) return BS_ERR_INVALID_ARG;
    result->first_unsorted = -1;
    result->first_unstable = -1;
    result->hash_a = result->hash_b = 0;
    if (n == 0) return BS_OK;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    CheckAcc *acc = nullptr;
    if (cudaMallocAsync((void **)&acc, sizeof(CheckAcc), s) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_OUT_OF_MEMORY;
    }
    CheckAcc host{};
    bool ok = cudaMemsetAsync(acc, 0xff, 2 * sizeof(unsigned long long), s) == cudaSuccess &&
              cudaMemsetAsync(&acc->hash_a, 0, 2 * sizeof(unsigned long long), s) == cudaSuccess;
    if (ok) {
        const unsigned grid = blocks_for(n, 256, sms * 8);
        const int codec = key_codec(kt);
        if (kw == 4)
            launch_overlapped(check_keys_kernel<uint32_t>, grid, 256, 0, s, (const uint32_t *)d_keys, n, codec,
                              d_offsets, S, d_idx, iw, isigned, acc);
        else
            launch_overlapped(check_keys_kernel<uint64_t>, grid, 256, 0, s, (const uint64_t *)d_keys, n, codec,
                              d_offsets, S, d_idx, iw, isigned, acc);
        ok = cudaGetLastError() == cudaSuccess &&
             cudaMemcpyAsync(&host, acc, sizeof(CheckAcc), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    }
    cudaFreeAsync(acc, s);
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    result->first_unsorted = host.first_unsorted == ~0ull ? -1 : (int64_t)host.first_unsorted;
    result->first_unstable = host.first_unstable == ~0ull ? -1 : (int64_t)host.first_unstable;
    result->hash_a = host.hash_a;
    result->hash_b = host.hash_b;
    return BS_OK;
}

bs_status bs_reserve_workspace(bs_handle *h, int64_t n, int64_t S, bs_dtype kt, bs_dtype vt, size_t *bytes) {
    if (!h || n < 0 || S < 0) return BS_ERR_INVALID_ARG;
    if (!key_width(kt) || (vt != BS_NONE && !value_width(vt))) return BS_ERR_UNSUPPORTED_DTYPE;
    if (S < 1) S = 1;
    DevGuard dg(h->device);
    const bs_status st = ensure_ws(h, ws_layout(n, S, (size_t)key_width(kt), (size_t)value_width(vt)).total);
    if (bytes) *bytes = h->ws_bytes;
    return st;
}

bs_status bs_sync_status(bs_handle *h) {
    if (!h) return BS_ERR_INVALID_ARG;
    DevGuard dg(h->device);
    // the last stream, and the copies out of asynchronous host sorts (each
    // waits for its sort), whichever stream the handle was used on last
    if (cudaStreamSynchronize(h->last_stream) != cudaSuccess ||
        (h->cp_out && cudaStreamSynchronize(h->cp_out) != cudaSuccess)) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    int err = 0;
    if (cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return BS_ERR_CUDA;
    if (err) {
        cudaMemset(h->d_err, 0, sizeof(int));
        return (bs_status)err;
    }
    if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;
    return BS_OK;
}

const char *bs_status_str(bs_status s) {
    switch (s) {
    case BS_OK: return "BS_OK";
    case BS_ERR_INVALID_ARG: return "BS_ERR_INVALID_ARG";
    case BS_ERR_UNSUPPORTED_DTYPE: return "BS_ERR_UNSUPPORTED_DTYPE";
    case BS_ERR_OUT_OF_MEMORY: return "BS_ERR_OUT_OF_MEMORY";
    case BS_ERR_CUDA: return "BS_ERR_CUDA";
    case BS_ERR_TIMEOUT: return "BS_ERR_TIMEOUT";
    case BS_ERR_TOO_LARGE: return "BS_ERR_TOO_LARGE";
    default: return "BS_ERR_UNKNOWN";
    }
}

bs_status bs_launch_stats(bs_handle *h, int64_t *counts, double *bytes, int reset) {
    if (!h) return BS_ERR_INVALID_ARG;
    DevGuard dg(h->device);
    if (counts)
        for (int k = 0; k < BS_KERNEL_CLASSES; ++k) counts[k] = h->launches[k];
    if (bytes) {
        unsigned long long c[BS_KERNEL_CLASSES];
        if (cudaDeviceSynchronize() != cudaSuccess) return BS_ERR_CUDA;
        if (cudaMemcpy(c, h->d_counters, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
            return BS_ERR_CUDA;
        for (int k = 0; k < BS_KERNEL_CLASSES; ++k) bytes[k] = (double)c[k];
    }
    if (reset) {
        for (int k = 0; k < BS_KERNEL_CLASSES; ++k) h->launches[k] = 0;
        cudaDeviceSynchronize();
        cudaMemset(h->d_counters, 0, sizeof(unsigned long long) * BS_KERNEL_CLASSES);
    cudaMemset(h->d_ticket, 0, sizeof(unsigned));
        cudaDeviceSynchronize();
    }
    return BS_OK;
}

bs_status bs_set_kernel_timing(bs_handle *h, int enable) {
    if (!h) return BS_ERR_INVALID_ARG;
    h->timing = enable != 0;
    return BS_OK;
}

bs_status bs_kernel_times(bs_handle *h, double *ms, int64_t *n) {
    if (!h) return BS_ERR_INVALID_ARG;
    DevGuard dg(h->device);
    double acc[BS_KERNEL_CLASSES] = {0, 0, 0, 0};
    int64_t cnt[BS_KERNEL_CLASSES] = {0, 0, 0, 0};
    bs_status st = BS_OK;
    for (auto &e : h->evs) {
        float t = 0.f;
        if (cudaEventSynchronize(e.b) != cudaSuccess || cudaEventElapsedTime(&t, e.a, e.b) != cudaSuccess) {
            cudaGetLastError();
            st = BS_ERR_CUDA;
        } else {
            acc[e.cls] += t;
            cnt[e.cls] += 1;
        }
        h->spare.push_back(e.a);
        h->spare.push_back(e.b);
    }
    h->evs.clear();
    for (int k = 0; k < BS_KERNEL_CLASSES; ++k) {
        if (ms) ms[k] = acc[k];
        if (n) n[k] = cnt[k];
    }
    return st;
}

bs_status bs_set_option(bs_handle *h, bs_option opt, int64_t value) {
    if (!h) return BS_ERR_INVALID_ARG;
    switch (opt) {
    case BS_OPT_TILE_LOG2:
        return bs_set_tile_log2(h, (int)value);
    case BS_OPT_MERGE_KERNEL:
        if (value < BS_MERGE_AUTO || value > BS_MERGE_TMA) return BS_ERR_INVALID_ARG;
        h->merge_impl = (int)value;
        return BS_OK;
    case BS_OPT_WAIT_LIMIT_MS:
        if (value < 0 || value > 60000) return BS_ERR_INVALID_ARG;
        h->wait_ns = (uint64_t)value * 1000000ull;
        return BS_OK;
    case BS_OPT_TEST_WITHHOLD:
        h->withhold = value != 0;
        return BS_OK;
    case BS_OPT_LOCAL_SORT:
        if (value < BS_LOCAL_MERGE || value > BS_LOCAL_QUICK) return BS_ERR_INVALID_ARG;
        h->local_sort = (int)value;
        return BS_OK;
    case BS_OPT_MERGE_TILE_LOG2:
        if (value != 0 && (value < 11 || value > 13)) return BS_ERR_INVALID_ARG;
        h->merge_tile_log2 = (int)value;
        return BS_OK;
    case BS_OPT_HOST_DIRECT:
        if (value != 0 && value != 1) return BS_ERR_INVALID_ARG;
        h->host_direct = (int)value;
        return BS_OK;
    case BS_OPT_MERGE_CONSUMER:
        if (value != 0 && value != 1) return BS_ERR_INVALID_ARG;
        h->merge_consumer = (int)value;
        return BS_OK;
    case BS_OPT_MERGE_SCHEDULE:
        if (value != BS_SCHEDULE_TREE && value != BS_SCHEDULE_ODDEVEN) return BS_ERR_INVALID_ARG;
        h->schedule = (int)value;
        return BS_OK;
    case BS_OPT_MERGE_VT:
        if (value != 0 && value != 8 && value != 16 && value != 32) return BS_ERR_INVALID_ARG;
        h->merge_vt = (int)value;
        return BS_OK;
    case BS_OPT_COUNT_BYTES:
        if (value != 0 && value != 1) return BS_ERR_INVALID_ARG;
        h->count_bytes = (int)value;
        return BS_OK;
    case BS_OPT_MERGE_PERSISTENT:
        if (value < 0 || value > 2) return BS_ERR_INVALID_ARG;
        h->persistent = (int)value;
        return BS_OK;
    case BS_OPT_LENGTH_CLASSES:
        if (value != 0 && value != 1) return BS_ERR_INVALID_ARG;
        h->length_classes = (int)value;
        return BS_OK;
    case BS_OPT_HOST_SLOTS: {
        if (value != 0 && value != 2 && value != 3) return BS_ERR_INVALID_ARG;
        const int v = value ? (int)value : HOST_SLOTS;
        if (v != h->host_slots) {
            // the slot sequence restarts: wait for the calls in flight first
            const bs_status st = bs_sync_status(h);
            h->host_slots = v;
            h->async_calls = 0;
            return st;
        }
        return BS_OK;
    }
    default:
        return BS_ERR_INVALID_ARG;
    }
}

bs_status bs_set_tile_log2(bs_handle *h, int tile_log2) {
    if (!h) return BS_ERR_INVALID_ARG;
    if (tile_log2 == 0) tile_log2 = 12;
    if (tile_log2 < 11 || tile_log2 > 13) return BS_ERR_INVALID_ARG;
    h->logT = tile_log2;
    return BS_OK;
}

// ====================================================================== CUDA graphs

}  // extern "C"

struct bs_graph {
    bs_handle *h = nullptr;  // private handle: owns the workspace the graph refers to
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last = nullptr;
};

namespace {

// Capture one call (run by `body` on the capture stream) into a graph that
// owns a private handle with the workspace pre-sized to `ws_bytes`.
template <class Body>
bs_status capture_graph(bs_handle *h, size_t ws_bytes, Body body, bs_graph **out) {
    *out = nullptr;
    bs_graph *g = new (std::nothrow) bs_graph();
    if (!g) return BS_ERR_OUT_OF_MEMORY;
    bs_status st = bs_create(&g->h, h->device);
    if (st != BS_OK) {
        delete g;
        return st;
    }
    g->h->logT = h->logT;
    g->h->merge_impl = h->merge_impl;
    g->h->merge_vt = h->merge_vt;
    g->h->schedule = h->schedule;
    g->h->local_sort = h->local_sort;
    g->h->merge_tile_log2 = h->merge_tile_log2;
    g->h->merge_consumer = h->merge_consumer;
    g->h->count_bytes = h->count_bytes;
    g->h->persistent = h->persistent;
    g->h->length_classes = h->length_classes;
    DevGuard dg(h->device);
    st = ensure_ws(g->h, ws_bytes);  // allocate before capture: nothing allocates inside it
    if (st == BS_OK && cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess)
        st = BS_ERR_CUDA;
    if (st == BS_OK) {
        if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            st = BS_ERR_CUDA;
        } else {
            st = body(g->h, g->cap);
            cudaGraph_t graph = nullptr;
            const cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
            g->graph = graph;
            if (st == BS_OK && (e != cudaSuccess || !graph)) st = BS_ERR_CUDA;
            if (st == BS_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
                st = BS_ERR_CUDA;
        }
    }
    if (st != BS_OK) {
        cudaGetLastError();
        bs_graph_destroy(g);
        return st;
    }
    *out = g;
    return BS_OK;
}

}  // namespace

extern "C" {

bs_status bs_graph_capture_segmented(bs_handle *h, const void *d_kin, void *d_kout,
                                     const void *d_vin, void *d_vout, int64_t n,
                                     const int64_t *d_offsets, int64_t S, int64_t max_seg_len,
                                     bs_dtype kt, bs_dtype vt, bs_graph **out) {
    if (!h || !out || n <= 0 || S <= 0 || max_seg_len < 0 || !d_offsets || !d_kin || !d_kout)
        return BS_ERR_INVALID_ARG;
    if (!key_width(kt) || (vt != BS_NONE && !value_width(vt))) return BS_ERR_UNSUPPORTED_DTYPE;
    const size_t ws = ws_layout(n, S, (size_t)key_width(kt), (size_t)value_width(vt)).total;
    return capture_graph(
        h, ws,
        [&](bs_handle *gh, cudaStream_t s) {
            return bs_sort_segmented(gh, d_kin, d_kout, d_vin, d_vout, n, d_offsets, S, max_seg_len,
                                     kt, vt, (void *)s);
        },
        out);
}

bs_status bs_graph_capture_keys(bs_handle *h, const void *d_in, void *d_out, int64_t n, bs_dtype kt,
                                int64_t p, bs_graph **out) {
    if (!h || !out || n <= 0 || p < 0 || !d_in || !d_out) return BS_ERR_INVALID_ARG;
    if (!key_width(kt)) return BS_ERR_UNSUPPORTED_DTYPE;
    const int64_t pp = p == 0 ? 1 : (p > n ? n : p);
    const size_t ws = ws_layout(n, pp, (size_t)key_width(kt), 0).total;
    return capture_graph(
        h, ws,
        [&](bs_handle *gh, cudaStream_t s) { return bs_sort_keys(gh, d_in, d_out, n, kt, p, (void *)s); },
        out);
}

bs_status bs_graph_launch(bs_graph *g, void *stream) {
    if (!g || !g->exec) return BS_ERR_INVALID_ARG;
    DevGuard dg(g->h->device);
    if (cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    g->last = (cudaStream_t)stream;
    g->h->last_stream = (cudaStream_t)stream;
    return BS_OK;
}

bs_status bs_graph_sync_status(bs_graph *g) {
    if (!g) return BS_ERR_INVALID_ARG;
    return bs_sync_status(g->h);
}

bs_status bs_graph_destroy(bs_graph *g) {
    if (!g) return BS_OK;
    if (g->h) {
        DevGuard dg(g->h->device);
        if (g->last) cudaStreamSynchronize(g->last);
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->cap) cudaStreamDestroy(g->cap);
        bs_destroy(g->h);
    }
    delete g;
    return BS_OK;
}

}  // extern "C"
