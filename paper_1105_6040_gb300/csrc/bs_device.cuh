// bs_device.cuh -- device code of the GB300 block-decomposed sort.
//
// The paper's paradigm (El-Nashar 2011, Sec. 3.2, Fig. 1) mapped to one GPU:
//   scatter (Fig. 1, scatter phase): block bounds are an offsets array in device
//     memory; nothing moves.
//   sort phase (Fig. 1): every block is cut into tiles of T keys
//     aligned to the block start; one CTA sorts one tile in registers and
//     shared memory (tile_sort_kernel), then merge passes in HBM join the
//     sorted tiles of each block pairwise (in-block levels) until the block
//     is one sorted run.
//   merge phase (Fig. 1): pairs of sorted blocks are merged, round after
//     round (cross-block levels), until one run remains.
// Every merge pass splits its output into merge tiles; the start of each
// output tile inside its pair of runs is found by a merge-path search
// (Odeh, Green, Mwassi, Shmueli, Birk: "Merge Path", IPDPSW 2012:
// partition_kernel), so each CTA merges an independent slice, staged into
// shared memory by TMA bulk copies (merge_tma_kernel; merge_kernel for
// unaligned buffers).  Ties go to the left run, which makes all merges
// stable.
//
// Keys travel as order-preserving unsigned codes (encoded when the tile sort
// loads them, decoded by the pass that writes the final output), so every
// comparison is an unsigned integer one.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "bsort.h"

namespace bs {

// ---------------------------------------------------------------- key codes

enum Codec : int { CODEC_IDENT = 0, CODEC_SIGNED = 1, CODEC_FLOAT = 2 };

__device__ __forceinline__ uint32_t enc_code(uint32_t x, int c) {
    if (c == CODEC_SIGNED) return x ^ 0x80000000u;
    if (c == CODEC_FLOAT) return (x & 0x80000000u) ? ~x : (x | 0x80000000u);
    return x;
}
__device__ __forceinline__ uint32_t dec_code(uint32_t x, int c) {
    if (c == CODEC_SIGNED) return x ^ 0x80000000u;
    if (c == CODEC_FLOAT) return (x & 0x80000000u) ? (x & 0x7fffffffu) : ~x;
    return x;
}
__device__ __forceinline__ uint64_t enc_code(uint64_t x, int c) {
    const uint64_t s = 0x8000000000000000ull;
    if (c == CODEC_SIGNED) return x ^ s;
    if (c == CODEC_FLOAT) return (x & s) ? ~x : (x | s);
    return x;
}
__device__ __forceinline__ uint64_t dec_code(uint64_t x, int c) {
    const uint64_t s = 0x8000000000000000ull;
    if (c == CODEC_SIGNED) return x ^ s;
    if (c == CODEC_FLOAT) return (x & s) ? (x & ~s) : ~x;
    return x;
}

template <class K> __device__ __forceinline__ K max_code() { return ~K(0); }

// Payload-less sorts use this empty value type.
struct NoVal {};
template <class V> struct HasVal { static constexpr bool value = true; };
template <> struct HasVal<NoVal> { static constexpr bool value = false; };

// Shared-memory index with one padding slot per 128 bytes, so that a warp
// writing KPT consecutive elements per thread hits distinct banks.
template <class T> __device__ __forceinline__ int spad(int x) {
    return sizeof(T) == 8 ? x + (x >> 4) : x + (x >> 5);
}
template <class T> __host__ __device__ constexpr int spad_size(int n) {
    return sizeof(T) == 8 ? n + (n >> 4) + 1 : n + (n >> 5) + 1;
}
// Dynamic shared memory of a CTA staging T keys (and values): keys first,
// values at the next 16-byte boundary.
template <class K> __host__ __device__ constexpr size_t smem_val_offset(int T) {
    return (sizeof(K) * (size_t)spad_size<K>(T) + 15) & ~size_t(15);
}
template <class K, class V> __host__ __device__ constexpr size_t smem_bytes(int T) {
    return smem_val_offset<K>(T) + (sizeof(V) > 1 ? sizeof(V) * (size_t)spad_size<V>(T) : 0);
}

// ---------------------------------------------------------------- geometry

// Everything a kernel needs to know about the decomposition.
struct Geo {
    const int64_t *off;      // S+1 block/segment bounds (device)
    int64_t S;               // number of blocks/segments
    int64_t n;               // total keys
    const int64_t *tprefix;  // S+1: first tile of each segment (exclusive scan)
    const int32_t *tseg;     // per tile: its segment
    int64_t ntiles_ub;       // capacity of the tile arrays (bounds every tile loop)
    int logT;                // tile = 2^logT keys
    int R;                   // number of cross-block merge rounds
    unsigned long long *counters;  // algorithmic bytes per kernel class (nullable: no counting)
    int *err;                      // device status flag (nullable): first error wins
    const int64_t *src_off;        // gathered input: segment s reads in[src_off[s] ..] (nullable)
    int64_t n_in;                  // length of the input array when src_off is set
    uint64_t wait_ns;              // limit of every bounded wait (0: the default)
    int withhold;                  // test hook: CTA 0's producer withholds its first stage
    void *fin_k, *fin_v;           // final (decoded) outputs go here when set, else to
                                   // buffer 0 (e.g. pinned host memory the GPU addresses)
    int64_t wmax;                  // length class: segments of 1..wmax keys have no tiles
                                   // and one warp sorts each (0: every segment has tiles)
};

// Destination of a pass's output: the final buffers when this is the last
// pass of its run and they are set, else ping-pong buffer `parity`.
template <class T>
__device__ __forceinline__ T *out_buf(bool fin, void *fin_buf, int parity, T *buf0, T *buf1) {
    return (fin && fin_buf) ? static_cast<T *>(fin_buf) : (parity ? buf1 : buf0);
}

// kernel classes of the statistics counters (same order as the C ABI's)
enum : int { CLS_TILE_SORT = 0, CLS_MERGE = 1, CLS_PARTITION = 2, CLS_SETUP = 3 };

// Adds a launch's algorithmic bytes to its class counter, when counting is on
// (g.counters set); a sort that does not count pays nothing for it.
__device__ __forceinline__ void count_bytes(const Geo &g, int cls, unsigned long long bytes) {
    if (g.counters) atomicAdd(g.counters + cls, bytes);
}

// Kernels launched with programmatic stream serialization may start while
// the previous kernel on their stream finishes: they call this before
// touching anything it wrote (a no-op for a plain launch).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int64_t clamp64(int64_t x, int64_t lo, int64_t hi) {
    return x < lo ? lo : (x > hi ? hi : x);
}

// Bounds of segment s, clamped into [0, n] and made non-decreasing so that
// malformed offsets can never address memory outside the arrays.
__device__ __forceinline__ void seg_bounds(const Geo &g, int64_t s, int64_t &lo, int64_t &hi) {
    lo = clamp64(g.off[s], 0, g.n);
    hi = clamp64(g.off[s + 1], lo, g.n);
}

// Number of in-segment merge levels a segment of `len` keys needs:
// ceil(log2(number of its tiles)).
__device__ __forceinline__ int seg_levels(int64_t len, int logT) {
    if (len <= (int64_t(1) << logT)) return 0;
    int64_t tiles = (len + (int64_t(1) << logT) - 1) >> logT;
    return 64 - __clzll((unsigned long long)(tiles - 1));
}

// Largest s in [0, S) with off[s] <= x: the (non-empty) segment holding x.
__device__ __forceinline__ int64_t seg_of(const Geo &g, int64_t x) {
    int64_t lo = 0, hi = g.S;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (g.off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- merge path

// Number of A items among the first `diag` outputs of the merge of sorted
// A[0, na) and B[0, nb), where b_less_a(ia, ib) says B[ib] goes strictly
// before A[ia] (so an A item wins a tie and the merge is stable).
template <class I, class BLessA>
__device__ __forceinline__ I merge_path_pred(I na, I nb, I diag, BLessA b_less_a) {
    I lo = diag > nb ? diag - nb : I(0);
    I hi = diag < na ? diag : na;
    while (lo < hi) {
        I mid = (lo + hi) >> 1;
        if (!b_less_a(mid, diag - 1 - mid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The same on plain codes through accessors A(i), B(i) (shared or global).
template <class K, class I, class AccA, class AccB>
__device__ __forceinline__ I merge_path(AccA A, I na, AccB B, I nb, I diag) {
    return merge_path_pred<I>(na, nb, diag, [&](I ia, I ib) {
        K a = A(ia), b = B(ib);
        return b < a;
    });
}

// ---------------------------------------------------------------- in-register networks

// Keys with a tie-breaking index: (code, index) pairs are all distinct, so
// any network sorts them into one order, and it is the stable order when the
// index follows the input order.
template <class K> __device__ __forceinline__ bool ki_less(K ak, uint32_t ai, K bk, uint32_t bi) {
    return ak < bk || (ak == bk && ai < bi);
}

template <class K> __device__ __forceinline__ void cas_keys(K &a, K &b) {
    K lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

template <class K>
__device__ __forceinline__ void cas_pairs(K &a, uint32_t &ai, K &b, uint32_t &bi) {
    const bool sw = ki_less(b, bi, a, ai);
    const K k = a;
    const uint32_t i = ai;
    a = sw ? b : a;
    ai = sw ? bi : ai;
    b = sw ? k : b;
    bi = sw ? i : bi;
}

// Odd-even merge sorting network over N registers, ascending (Batcher 1968),
// in Knuth's iterative form: for each merge size 2p and comparator distance
// q = p, p/2, .., 1, compare i+j with i+j+q when both lie in the same block
// of 2p.  63 comparators for N = 16 (bitonic sorting takes 80).  The list
// is built at compile time, so the unrolled network indexes registers only.
template <int N> struct OddEvenNet {
    int a[N * N], b[N * N], n;
    constexpr OddEvenNet() : a(), b(), n(0) {
        for (int p = 1; p < N; p <<= 1)
            for (int q = p; q >= 1; q >>= 1)
                for (int j = q % p; j + q < N; j += 2 * q)
                    for (int i = 0; i < q && i < N - j - q; ++i)
                        if ((i + j) / (2 * p) == (i + j + q) / (2 * p)) {
                            a[n] = i + j;
                            b[n] = i + j + q;
                            ++n;
                        }
    }
};

// Applies comparator C and the ones after it, one template instance each,
// so every register index is a compile-time constant (no local memory).
template <int N, int C> struct OddEvenApply {
    static constexpr OddEvenNet<N> net{};
    template <class K> static __device__ __forceinline__ void keys(K (&k)[N]) {
        if constexpr (C < net.n) {
            cas_keys(k[net.a[C]], k[net.b[C]]);
            OddEvenApply<N, C + 1>::keys(k);
        }
    }
    template <class K> static __device__ __forceinline__ void pairs(K (&k)[N], uint32_t (&x)[N]) {
        if constexpr (C < net.n) {
            cas_pairs(k[net.a[C]], x[net.a[C]], k[net.b[C]], x[net.b[C]]);
            OddEvenApply<N, C + 1>::pairs(k, x);
        }
    }
};

template <int N, class K> __device__ __forceinline__ void reg_sort_keys(K (&k)[N]) {
    OddEvenApply<N, 0>::keys(k);
}

template <int N, class K> __device__ __forceinline__ void reg_sort_pairs(K (&k)[N], uint32_t (&x)[N]) {
    OddEvenApply<N, 0>::pairs(k, x);
}

// Ascending bitonic merge of a bitonic sequence held in N registers.
template <int N, class K> __device__ __forceinline__ void bitonic_merge_keys(K (&k)[N]) {
#pragma unroll
    for (int s = N >> 1; s > 0; s >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((i & s) == 0) cas_keys(k[i], k[i + s]);
}

template <int N, class K>
__device__ __forceinline__ void bitonic_merge_pairs(K (&k)[N], uint32_t (&x)[N]) {
#pragma unroll
    for (int s = N >> 1; s > 0; s >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((i & s) == 0) cas_pairs(k[i], x[i], k[i + s], x[i + s]);
}

// ---------------------------------------------------------------- warp-level bitonic merge

// One merge round inside a warp, keys only.  Each lane holds N sorted keys;
// groups of 2^r lanes hold sorted lists of N << r keys, and this round
// merges adjacent pairs of such groups into lists of N << (r+1) keys, by a
// bitonic merger written with register shuffles: a "flip" stage compares
// element e of the first list with element 2m-1-e of the pair (partner lane
// l ^ (2^(r+1)-1), register N-1-u); then half-cleaners with lane strides
// 2^(r-1) .. 1 (shuffles) and register strides N/2 .. 1 (in-thread) finish
// it.  Every stage sends the lower key of a compared pair to the lower
// position, so the merged list is ascending in (lane, register) order.
template <int N, class K> __device__ __forceinline__ K shfl_xor_k(K v, int mask) {
    if constexpr (sizeof(K) == 4) {
        return (K)__shfl_xor_sync(0xffffffffu, (uint32_t)v, mask);
    } else {
        const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, mask);
        const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), mask);
        return (K)(((uint64_t)hi << 32) | lo);
    }
}

template <int N, class K> __device__ __forceinline__ void warp_merge_round(K (&k)[N], int r, int lane) {
    const bool upper = (lane >> r) & 1;
    K t[N];
#pragma unroll
    for (int u = 0; u < N; ++u) t[u] = shfl_xor_k<N>(k[N - 1 - u], (2 << r) - 1);
    // the lower lane keeps the smaller key, the upper the larger: take the
    // partner's key when (partner < own) differs from "upper" (one compare
    // and one select per key)
#pragma unroll
    for (int u = 0; u < N; ++u) k[u] = ((t[u] < k[u]) != upper) ? t[u] : k[u];
    for (int ls = (1 << r) >> 1; ls > 0; ls >>= 1) {
        const bool up = lane & ls;
#pragma unroll
        for (int u = 0; u < N; ++u) {
            const K p = shfl_xor_k<N>(k[u], ls);
            k[u] = ((p < k[u]) != up) ? p : k[u];
        }
    }
    bitonic_merge_keys<N>(k);
}

// ---------------------------------------------------------------- candidate merge

// The VT smallest items of the merge of sorted lists A = S[a0, a0+na) and
// B = S[b0, b0+nb) in shared memory (padded indices), from the merge-path
// split (i, j).  With A' = A[i, i+VT) and B' = B[j, j+VT), the sequence
// A' ++ reverse(B') is bitonic; one half-cleaner step (min of A'[u] and
// B'[VT-1-u]) keeps its VT smallest items and a bitonic merge sorts them
// (Batcher's bitonic merger).  The 2*VT shared loads are independent of one
// another, so no load waits on a comparison.  Items past a list end read as
// the largest code, so they never displace a real item.
template <class K, int VT>
__device__ __forceinline__ void cand_merge_keys(const K *sk, int a0, int na, int b0, int nb, int i,
                                                int j, K (&out)[VT]) {
#pragma unroll
    for (int u = 0; u < VT; ++u) {
        const int ia = i + u, ib = j + VT - 1 - u;
        const K x = ia < na ? sk[spad<K>(a0 + ia)] : max_code<K>();
        const K y = ib < nb ? sk[spad<K>(b0 + ib)] : max_code<K>();
        out[u] = x < y ? x : y;
    }
    bitonic_merge_keys<VT>(out);
}

// Pairs: each item carries a tie-breaking index -- sx[position] when sx is
// given (original input positions), else the shared-memory position itself
// (A before B, each in input order).  Missing items are (largest code,
// largest index).  oi[] receives the indices of the outputs.
template <class K, int VT>
__device__ __forceinline__ void cand_merge_pairs(const K *sk, const uint32_t *sx, int a0, int na,
                                                 int b0, int nb, int i, int j, K (&out)[VT],
                                                 uint32_t (&oi)[VT]) {
#pragma unroll
    for (int u = 0; u < VT; ++u) {
        const int ia = i + u, ib = j + VT - 1 - u;
        K x = max_code<K>(), y = max_code<K>();
        uint32_t xi = 0xffffffffu, yi = 0xffffffffu;
        if (ia < na) {
            x = sk[spad<K>(a0 + ia)];
            xi = sx ? sx[spad<uint32_t>(a0 + ia)] : (uint32_t)(a0 + ia);
        }
        if (ib < nb) {
            y = sk[spad<K>(b0 + ib)];
            yi = sx ? sx[spad<uint32_t>(b0 + ib)] : (uint32_t)(b0 + ib);
        }
        const bool tx = ki_less(x, xi, y, yi);
        out[u] = tx ? x : y;
        oi[u] = tx ? xi : yi;
    }
    bitonic_merge_pairs<VT>(out, oi);
}

// Sequential merge of KPT outputs from two sorted lists in padded shared
// memory, A = S[a0, a0+m) and B = S[b0, b0+m), starting at the merge-path
// split (i, j): each step takes the smaller head (A's on a tie) and loads
// the next item of that list -- one shared load per output.  A head past
// its list's end reads as the largest code, so a step needs one compare:
// while the other list has real items below the largest code they win, and
// once its head is the largest code too every output left is that value
// (keys only: which list supplies an equal key does not matter).  Reads stay
// inside the two lists.
template <class K, int KPT>
__device__ __forceinline__ void seq_merge_keys(const K *sk, int a0, int b0, int m, int i, int j, K (&out)[KPT]) {
    K a = i < m ? sk[spad<K>(a0 + i)] : max_code<K>();
    K b = j < m ? sk[spad<K>(b0 + j)] : max_code<K>();
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
        const bool tb = b < a;  // take B's head
        out[u] = tb ? b : a;
        i += tb ? 0 : 1;
        j += tb ? 1 : 0;
        const int li = tb ? j : i;
        const K nxt = li < m ? sk[spad<K>((tb ? b0 : a0) + li)] : max_code<K>();
        a = tb ? a : nxt;
        b = tb ? nxt : b;
    }
}

// The same for pairs whose lists cover consecutive ranges of original
// positions (the left list's first): the left item on a tie is the stable
// order, so only codes are compared; each output's staging index is kept
// and its position fetched after the loop (independent loads).
template <class K, int KPT>
__device__ __forceinline__ void seq_merge_carry(const K *sk, const uint32_t *sx, int a0, int b0, int m, int i,
                                                int j, K (&out)[KPT], uint32_t (&oi)[KPT]) {
    K a = sk[spad<K>(a0 + i)], b = sk[spad<K>(b0 + j)];
    int from[KPT];
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
        const bool tb = i >= m || (j < m && b < a);  // take B's head
        out[u] = tb ? b : a;
        from[u] = tb ? b0 + j : a0 + i;
        i += tb ? 0 : 1;
        j += tb ? 1 : 0;
        const K nxt = sk[spad<K>(tb ? b0 + j : a0 + i)];
        a = tb ? a : nxt;
        b = tb ? nxt : b;
    }
#pragma unroll
    for (int u = 0; u < KPT; ++u) oi[u] = sx[spad<uint32_t>(from[u])];
}

// ---------------------------------------------------------------- tile sort

// A 16-byte vector of keys: N keys, element e read by get, every element
// replaced by map.
template <class K> struct Vec16;
template <> struct Vec16<uint32_t> {
    using T = uint4;
    static constexpr int N = 4;
    static __device__ __forceinline__ uint32_t get(const uint4 &v, int e) {
        return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
    }
    template <class F> static __device__ __forceinline__ void map(uint4 &v, F f) {
        v.x = f(v.x), v.y = f(v.y), v.z = f(v.z), v.w = f(v.w);
    }
};
template <> struct Vec16<uint64_t> {
    using T = ulonglong2;
    static constexpr int N = 2;
    static __device__ __forceinline__ uint64_t get(const ulonglong2 &v, int e) {
        return e == 0 ? (uint64_t)v.x : (uint64_t)v.y;
    }
    template <class F> static __device__ __forceinline__ void map(ulonglong2 &v, F f) {
        v.x = f((uint64_t)v.x), v.y = f((uint64_t)v.y);
    }
};

// Shared memory of the tile sort: codes, then (pairs) original positions and
// values, each at a 16-byte boundary.
// Keys alone: two ping-pong buffers of keys_round_buf(T) keys each (see
// tile_smem_rounds).
__host__ __device__ constexpr int keys_round_buf(int T) {
    // T keys, the first round's padding (one slot per 32), a sentinel per pair
    // of runs of at least 512 keys, slack; rounded to 16 bytes of 8-byte keys
    return ((T + T / 32 + T / 512 + 64) + 1) & ~1;
}
template <class K, class V> __host__ __device__ constexpr size_t tile_smem_bytes(int T) {
    return sizeof(V) > 1 ? smem_val_offset<K>(T) + smem_val_offset<uint32_t>(T) + sizeof(V) * (size_t)spad_size<V>(T)
                         : 2 * sizeof(K) * (size_t)keys_round_buf(T);
}

// The shared-memory merge rounds of the keys-only tile sort.  On entry every
// warp holds one sorted run of M0 = 32*KPT keys, lane l the keys
// [KPT*l, KPT*l + KPT) of it; each round merges pairs of runs (m -> 2m) until
// the tile is one run, and the function returns where it lies (plain layout,
// T keys), after a barrier.
//
// Layout.  A round reads pair q of runs A = [0, m), B = [m, 2m) from a region
// of its source buffer and writes the merged run to the destination buffer,
// ping-pong: pair q of a round's input lies at q*(2m+1), A first, then B,
// then one slot holding the largest code (B's sentinel).  The first round's
// input comes from registers: element e of pair q is at q*R1 + e + e/32
// (R1 = 2*M0 + 2*M0/32 + 1), so that the 32 lanes writing KPT consecutive keys
// each hit distinct banks; its sentinel is the region's last slot.
//
// Merge.  Warp w produces the outputs [w*M0, (w+1)*M0) of the round (one run
// of 2m >= 2*M0 holds them all); lane l produces S = KPT+1 of them from
// w*M0 + S*l on (the last lanes fewer), so lanes that write their outputs in
// step sit an odd distance apart, in distinct banks.  A lane finds its
// merge-path split by a binary search, then merges sequentially: each step
// takes B's head when A is exhausted or B's head is smaller (A wins ties:
// keys alone, either is right), stores it, and loads the next key of that
// run.  B's sentinel stops B without a test; A's end is tested, because
// A's successor is B's first key.  Keys equal to the largest code need no
// special case: B's sentinel then ties with A's head and A is taken.  A lane
// never consumes more than the 2m - diag keys left in its pair, so no read
// passes B's sentinel, whatever the keys.
//
// Short tiles.  Keys at positions >= nreal (the tile's key count) are
// padding: the largest code.  They stay at positions >= nreal after every
// round (each run's real keys sort to its front), so a warp whose outputs
// all lie there writes the largest code without merging, and in the last
// round, whose positions >= nreal are never stored, nothing at all.
template <class K, int THREADS, int KPT>
__device__ __forceinline__ const K *tile_smem_rounds(K (&k)[KPT], K *x, K *y, int tid, int nreal) {
    constexpr int T = THREADS * KPT;
    constexpr int M0 = 32 * KPT;  // run length after the warp rounds
    constexpr int WO = M0;        // outputs per warp per round
    constexpr int S = KPT + 1;    // outputs per lane (odd)
    constexpr int R1 = 2 * M0 + (2 * M0) / 32 + 1;
    static_assert(T >= 2 * M0, "at least one shared-memory round");
    const int lane = tid & 31, w = tid >> 5;
    {
        const int q = w >> 1, h = w & 1;
        K *pr = x + q * R1;
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
            const int e = h * M0 + lane * KPT + u;
            pr[e + (e >> 5)] = k[u];
        }
        if (h == 1 && lane == 0) pr[R1 - 1] = max_code<K>();
    }
    __syncthreads();
    const int start = min(S * lane, WO), cnt = min(S, WO - start);
    const K *src = x;
    K *dst = y;
#pragma unroll 1
    for (int m = M0; 2 * m <= T; m *= 2) {
        const bool first = (m == M0), last = (2 * m == T);
        const int p = (w * WO) / (2 * m);      // output run = input pair
        const int diag = (w * WO) % (2 * m) + start;
        // where output e of run p goes: the last round's plain layout, or the
        // next round's pair layout (and this run's half of that pair)
        K *out = last ? dst + p * (2 * m) : dst + (p >> 1) * (4 * m + 1) + (p & 1) * (2 * m);
        if (!last && (p & 1) && (w * WO) % (2 * m) + WO == 2 * m && lane == 31)
            out[2 * m] = max_code<K>();  // the next round's B sentinel
        out += diag;
        if (w * WO >= nreal) {
            if (!last)
                for (int u = 0; u < cnt; ++u) out[u] = max_code<K>();
        } else if (first) {
            const K *pb0 = src + p * R1;
            auto at = [&](int e) { return pb0[e + (e >> 5)]; };
            int lo = diag > m ? diag - m : 0, hi = diag < m ? diag : m;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (at(m + diag - 1 - mid) < at(mid)) hi = mid;
                else lo = mid + 1;
            }
            int ia = lo, ib = m + diag - lo;
            K a = at(ia), b = at(ib);
            if (cnt == S) {
#pragma unroll
                for (int u = 0; u < S; ++u) {
                    const bool tb = ia >= m || b < a;
                    out[u] = tb ? b : a;
                    ia += tb ? 0 : 1;
                    ib += tb ? 1 : 0;
                    const K nxt = at(tb ? ib : ia);
                    a = tb ? a : nxt;
                    b = tb ? nxt : b;
                }
            } else {
                for (int u = 0; u < cnt; ++u) {
                    const bool tb = ia >= m || b < a;
                    out[u] = tb ? b : a;
                    ia += tb ? 0 : 1;
                    ib += tb ? 1 : 0;
                    const K nxt = at(tb ? ib : ia);
                    a = tb ? a : nxt;
                    b = tb ? nxt : b;
                }
            }
        } else {
            const K *base = src + p * (2 * m + 1);
            int lo = diag > m ? diag - m : 0, hi = diag < m ? diag : m;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (base[m + diag - 1 - mid] < base[mid]) hi = mid;
                else lo = mid + 1;
            }
            const K *pa = base + lo, *pb = base + m + (diag - lo);
            const K *const a_end = base + m;
            K a = *pa, b = *pb;
            if (cnt == S) {
#pragma unroll
                for (int u = 0; u < S; ++u) {
                    const bool tb = pa >= a_end || b < a;
                    out[u] = tb ? b : a;
                    pa += tb ? 0 : 1;
                    pb += tb ? 1 : 0;
                    const K nxt = *(tb ? pb : pa);
                    a = tb ? a : nxt;
                    b = tb ? nxt : b;
                }
            } else {
                for (int u = 0; u < cnt; ++u) {
                    const bool tb = pa >= a_end || b < a;
                    out[u] = tb ? b : a;
                    pa += tb ? 0 : 1;
                    pb += tb ? 1 : 0;
                    const K nxt = *(tb ? pb : pa);
                    a = tb ? a : nxt;
                    b = tb ? nxt : b;
                }
            }
        }
        __syncthreads();
        src = dst;
        dst = (dst == y) ? x : y;
    }
    return src;
}

// The warp length class of the sort phase: every segment of 1..g.wmax keys
// (wmax <= 32*KPT; the plan gave these segments no tiles) is sorted whole by
// one warp -- KPT keys per lane through the register network, then the five
// shuffle rounds leave lane l holding outputs l*KPT .. l*KPT+KPT-1 -- and
// stored through the warp's own shared-memory buffer `wb` (33*KPT keys,
// padded so that neither the blocked write nor the striped read conflicts)
// as coalesced rows.  Warp gw of nw takes segments gw, gw+nw, gw+2nw, ..;
// its lanes read 32 candidates' bounds at a time and the warp sorts the ones
// in the class one after another.  A segment of this class is never merged
// afterwards, so its result is final (or, with cross-block rounds, the
// buffer the first round reads).  Returns the bytes it moved.  It runs as a
// launch of its own: inside the tile sort kernel it changed that kernel's
// register allocation.
template <class K, int KPT>
__device__ __forceinline__ unsigned long long warp_class_sort(const Geo &g, const K *__restrict__ in_k,
                                                              K *buf_k0, K *buf_k1, int codec, K *wb,
                                                              int lane, int64_t gw, int64_t nw) {
    unsigned long long bytes = 0;
    const bool fin = g.R == 0;
    K *dst = out_buf<K>(fin, g.fin_k, g.R & 1, buf_k0, buf_k1);
    for (int64_t i0 = 0; gw + nw * i0 < g.S; i0 += 32) {
        const int64_t s = gw + nw * (i0 + lane);
        int64_t lo = 0, hi = 0;
        if (s < g.S) seg_bounds(g, s, lo, hi);
        unsigned m = __ballot_sync(0xffffffffu, hi > lo && hi - lo <= g.wmax);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const int64_t ss = __shfl_sync(0xffffffffu, s, src);
            const int64_t slo = __shfl_sync(0xffffffffu, lo, src);
            const int len = (int)(__shfl_sync(0xffffffffu, hi, src) - slo);
            int64_t ibase = slo;
            int lcnt = len;
            if (g.src_off) {
                if (len <= g.n_in) ibase = clamp64(g.src_off[ss], 0, g.n_in - len);
                else lcnt = 0;  // malformed request (flagged by the offset check): load nothing
            }
            K k[KPT];
#pragma unroll
            for (int u = 0; u < KPT; ++u) {
                const int pos = lane + 32 * u;
                k[u] = pos < lcnt ? enc_code(in_k[ibase + pos], codec) : max_code<K>();
            }
            reg_sort_keys<KPT>(k);
#pragma unroll 1
            for (int r = 0; r < 5; ++r) warp_merge_round<KPT>(k, r, lane);
#pragma unroll
            for (int u = 0; u < KPT; ++u) {
                const int e = lane * KPT + u;
                wb[e + (e >> 5)] = k[u];
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < KPT; ++u) {
                const int pos = lane + 32 * u;
                if (pos < len) {
                    const K c = wb[pos + (pos >> 5)];
                    dst[slo + pos] = fin ? dec_code(c, codec) : c;
                }
            }
            __syncwarp();  // the buffer is free for the next segment
            bytes += 2ull * sizeof(K) * (unsigned)len;
        }
    }
    return bytes;
}

// The warp length class as its own launch (before the tile sort, which
// never sees these segments): WARPS warps per CTA, each with its buffer.
template <class K, int KPT, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
warp_class_kernel(Geo g, const K *__restrict__ in_k, K *buf_k0, K *buf_k1, int codec) {
    __shared__ K wb[WARPS][33 * KPT];
    griddep_wait();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long b =
        warp_class_sort<K, KPT>(g, in_k, buf_k0, buf_k1, codec, wb[w], lane,
                                (int64_t)blockIdx.x * WARPS + w, (int64_t)gridDim.x * WARPS);
    if (lane == 0 && b) count_bytes(g, CLS_TILE_SORT, b);
}

// Tile sort (the sort phase of Fig. 1 at CTA scale).  Tile t covers
// keys [s + j*T, min(s + (j+1)*T, e)) of segment [s, e).  Each thread sorts
// KPT keys in registers; keys-only tiles then merge pairs of lists with five
// warp-shuffle rounds (one sorted run of 32*KPT keys per warp) and the
// remaining rounds in shared memory (tile_smem_rounds); pairs merge every
// round through shared memory (merge-path split + sequential merge of KPT
// outputs per thread; rounds whose lists live inside one warp synchronise
// only that warp).  Pairs sort
// (code, original position), which is the stable order; values move once,
// at the final store.  The sorted tile is written -- decoded if this is the
// segment's last pass -- to the buffer its merge schedule starts from.
// Resident CTAs per SM the keys-alone tile sort of 32-bit keys is compiled
// for: as many as its shared memory allows (3 at 8192-key tiles, 6 at 4096;
// 8 at 2048), so that the register allocation does not lower them.
template <class K, class V, int THREADS, int KPT> constexpr int tile_min_ctas() {
    return (sizeof(K) == 4 && !HasVal<V>::value) ? (THREADS * KPT == 8192 ? 3 : THREADS * KPT == 4096 ? 6 : 8)
                                                 : 1;
}

template <class K, class V, int THREADS, int KPT>
__global__ void __launch_bounds__(THREADS, (tile_min_ctas<K, V, THREADS, KPT>()))
tile_sort_kernel(Geo g, const K *__restrict__ in_k, const V *__restrict__ in_v,
                 K *buf_k0, K *buf_k1, V *buf_v0, V *buf_v1, int codec,
                 const int64_t *__restrict__ ntiles_total) {
    constexpr int T = THREADS * KPT;
    constexpr bool HV = HasVal<V>::value;
    griddep_wait();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    K *sk = reinterpret_cast<K *>(smem_raw);
    uint32_t *sx = reinterpret_cast<uint32_t *>(smem_raw + smem_val_offset<K>(T));
    V *sv = reinterpret_cast<V *>(smem_raw + smem_val_offset<K>(T) + smem_val_offset<uint32_t>(T));

    const int64_t total = min(*ntiles_total, g.ntiles_ub);
    const int tid = threadIdx.x;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int64_t s = g.tseg[t];
        int64_t slo, shi;
        seg_bounds(g, s, slo, shi);
        const int64_t j = t - g.tprefix[s];
        const int64_t base = slo + (j << g.logT);
        const int cnt = (int)(shi - base < (int64_t)T ? shi - base : (int64_t)T);
        const int L = seg_levels(shi - slo, g.logT);
        const int par = (L + g.R) & 1;
        const bool fin = (L + g.R) == 0;
        K *dst_k = out_buf<K>(fin, g.fin_k, par, buf_k0, buf_k1);
        V *dst_v = out_buf<V>(fin, g.fin_v, par, buf_v0, buf_v1);
        // where this tile's keys come from: in place, or (gathered segments)
        // from the segment's own offset in the input array, kept inside it
        int64_t ibase = base;
        int lcnt = cnt;
        if (g.src_off) {
            const int64_t len = shi - slo;
            if (len <= g.n_in) ibase = clamp64(g.src_off[s], 0, g.n_in - len) + (base - slo);
            else lcnt = 0;  // malformed request (flagged by the offset check): load nothing
        }

        // striped, coalesced load; padding slots get the largest code (and,
        // for pairs, positions past every real one)
        K k[KPT];
        uint32_t x[KPT];
        if constexpr (HV) {
            // pairs: thread t takes positions KPT*t .. KPT*t + KPT-1 (through
            // shared memory), so every list the rounds merge covers one range
            // of positions and the left list's items all come first: taking
            // the left item on a tie is then the stable order, and only the
            // register network compares (code, position)
#pragma unroll
            for (int u = 0; u < KPT; ++u) {
                const int pos = tid + u * THREADS;
                sk[spad<K>(pos)] = pos < lcnt ? enc_code(in_k[ibase + pos], codec) : max_code<K>();
                if (pos < lcnt) sv[spad<V>(pos)] = in_v[ibase + pos];
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < KPT; ++u) {
                k[u] = sk[spad<K>(tid * KPT + u)];
                x[u] = (uint32_t)(tid * KPT + u);
            }
            __syncthreads();  // the first round overwrites sk
            reg_sort_pairs<KPT>(k, x);
        } else {
            // warp w loads positions [w*32*KPT, (w+1)*32*KPT): a full tile
            // starting on a 16-byte boundary as 16-byte vectors (512 bytes per
            // warp and step), else 32 consecutive keys per step; a warp past
            // the last key holds padding alone, already in order, and skips
            // the network and the shuffle rounds
            const int lane = tid & 31, w0 = (tid >> 5) * 32 * KPT;
            using VK = Vec16<K>;
            if (lcnt == T && ((uintptr_t)(in_k + ibase) & 15) == 0) {
#pragma unroll
                for (int q = 0; q < KPT / VK::N; ++q) {
                    const typename VK::T v = *reinterpret_cast<const typename VK::T *>(
                        in_k + ibase + w0 + VK::N * (lane + 32 * q));
#pragma unroll
                    for (int e = 0; e < VK::N; ++e) k[VK::N * q + e] = enc_code(VK::get(v, e), codec);
                }
            } else {
#pragma unroll
                for (int u = 0; u < KPT; ++u) {
                    const int pos = w0 + lane + 32 * u;
                    k[u] = pos < lcnt ? enc_code(in_k[ibase + pos], codec) : max_code<K>();
                }
            }
            if (w0 < cnt) {
                reg_sort_keys<KPT>(k);
                // the first merges inside a warp: register shuffles, no shared memory
#pragma unroll 1
                for (int r = 0; r < 5; ++r) warp_merge_round<KPT>(k, r, lane);
            }
        }

        if constexpr (!HV) {
            // then the shared-memory rounds, and the coalesced striped store
            // (16-byte vectors for a full tile starting on a 16-byte boundary)
            const K *res = tile_smem_rounds<K, THREADS, KPT>(k, sk, sk + keys_round_buf(T), tid, cnt);
            using VK = Vec16<K>;
            static_assert((keys_round_buf(T) * sizeof(K)) % 16 == 0, "both buffers 16-byte aligned");
            if (cnt == T && ((uintptr_t)(dst_k + base) & 15) == 0) {
#pragma unroll
                for (int q = 0; q < KPT / VK::N; ++q) {
                    const int vpos = VK::N * (tid + THREADS * q);
                    typename VK::T v = *reinterpret_cast<const typename VK::T *>(res + vpos);
                    if (fin) VK::map(v, [&](K c) { return dec_code(c, codec); });
                    *reinterpret_cast<typename VK::T *>(dst_k + base + vpos) = v;
                }
            } else {
#pragma unroll
                for (int u = 0; u < KPT; ++u) {
                    const int pos = tid + u * THREADS;
                    if (pos < cnt) {
                        const K c = res[pos];
                        dst_k[base + pos] = fin ? dec_code(c, codec) : c;
                    }
                }
            }
            if (tid == 0) count_bytes(g, CLS_TILE_SORT, 2ull * sizeof(K) * cnt);
            __syncthreads();  // the buffers are free for the next tile
            continue;
        }
#pragma unroll 1
        for (int r = 0; (KPT << r) < T; ++r) {
            const bool warp_round = (2 << r) <= 32;  // both lists inside one warp
#pragma unroll
            for (int u = 0; u < KPT; ++u) {
                sk[spad<K>(tid * KPT + u)] = k[u];
                if constexpr (HV) sx[spad<uint32_t>(tid * KPT + u)] = x[u];
            }
            if (warp_round) __syncwarp();
            else __syncthreads();
            const int m = KPT << r;
            const int a0 = (tid >> (r + 1)) * 2 * m, b0 = a0 + m;
            const int diag = (tid & ((2 << r) - 1)) * KPT;
            if constexpr (HV) {
                const int i = merge_path_pred<int>(m, m, diag, [&](int ia, int ib) {
                    return sk[spad<K>(b0 + ib)] < sk[spad<K>(a0 + ia)];
                });
                seq_merge_carry<K, KPT>(sk, sx, a0, b0, m, i, diag - i, k, x);
            } else {
                const int i = merge_path_pred<int>(m, m, diag, [&](int ia, int ib) {
                    return sk[spad<K>(b0 + ib)] < sk[spad<K>(a0 + ia)];
                });
                seq_merge_keys<K, KPT>(sk, a0, b0, m, i, diag - i, k);
            }
            if (warp_round) __syncwarp();
            else __syncthreads();
        }

        // blocked registers -> shared -> coalesced striped store
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
            sk[spad<K>(tid * KPT + u)] = k[u];
            if constexpr (HV) sx[spad<uint32_t>(tid * KPT + u)] = x[u];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
            const int pos = tid + u * THREADS;
            if (pos < cnt) {
                const K c = sk[spad<K>(pos)];
                dst_k[base + pos] = fin ? dec_code(c, codec) : c;
                if constexpr (HV) dst_v[base + pos] = sv[spad<V>((int)sx[spad<uint32_t>(pos)])];
            }
        }
        if (tid == 0) count_bytes(g, CLS_TILE_SORT, 2ull * (sizeof(K) + (HV ? sizeof(V) : 0)) * cnt);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- tile sorts after Figs. 2 and 4

// Tile bookkeeping shared by the alternative tile sorts (keys only).
struct TileInfo {
    int64_t base, ibase;
    int cnt, lcnt;
    bool fin;
    int par;
};
__device__ __forceinline__ TileInfo tile_info(const Geo &g, int64_t t, int T) {
    TileInfo ti;
    const int64_t s = g.tseg[t];
    int64_t slo, shi;
    seg_bounds(g, s, slo, shi);
    const int64_t j = t - g.tprefix[s];
    ti.base = slo + j * T;
    ti.cnt = (int)(shi - ti.base < (int64_t)T ? shi - ti.base : (int64_t)T);
    const int L = seg_levels(shi - slo, g.logT);
    ti.par = (L + g.R) & 1;
    ti.fin = (L + g.R) == 0;
    ti.ibase = ti.base;
    ti.lcnt = ti.cnt;
    if (g.src_off) {
        const int64_t len = shi - slo;
        if (len <= g.n_in) ti.ibase = clamp64(g.src_off[s], 0, g.n_in - len) + (ti.base - slo);
        else ti.lcnt = 0;
    }
    return ti;
}

// Fig. 2 on a GPU: bubble sort's adjacent exchange, run as odd-even
// transposition over the tile in shared memory -- cnt rounds, each
// comparing the pairs (i, i+1) with i of the round's parity and exchanging
// them on a strict '>'.  O(T^2) work per tile, like the paper's O(s^2).
template <class K, int THREADS, int KPT>
__global__ void __launch_bounds__(THREADS)
tile_bubble_kernel(Geo g, const K *__restrict__ in_k, K *buf_k0, K *buf_k1, int codec,
                   const int64_t *__restrict__ ntiles_total) {
    constexpr int T = THREADS * KPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    K *sk = reinterpret_cast<K *>(smem_raw);
    griddep_wait();
    const int64_t total = min(*ntiles_total, g.ntiles_ub);
    const int tid = threadIdx.x;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const TileInfo ti = tile_info(g, t, T);
        for (int pos = tid; pos < T; pos += THREADS)
            sk[pos] = pos < ti.lcnt ? enc_code(in_k[ti.ibase + pos], codec) : max_code<K>();
        __syncthreads();
        for (int rd = 0; rd < ti.cnt; ++rd) {
            for (int i = 2 * tid + (rd & 1); i + 1 < ti.cnt; i += 2 * THREADS) {
                const K a = sk[i], b = sk[i + 1];
                if (b < a) sk[i] = b, sk[i + 1] = a;
            }
            __syncthreads();
        }
        K *dst = out_buf<K>(ti.fin, g.fin_k, ti.par, buf_k0, buf_k1);
        for (int pos = tid; pos < ti.cnt; pos += THREADS) {
            const K c = sk[pos];
            dst[ti.base + pos] = ti.fin ? dec_code(c, codec) : c;
        }
        if (tid == 0) count_bytes(g, CLS_TILE_SORT, 2ull * sizeof(K) * ti.cnt);
        __syncthreads();
    }
}

// Block-wide exclusive scan of one int per thread; returns the total.
template <int THREADS>
__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int &excl) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    int before = 0, total = 0;
    for (int i = 0; i < THREADS / 32; ++i) {
        const int ws = warp_sums[i];
        if (i < w) before += ws;
        total += ws;
    }
    excl = before + x - v;
    __syncthreads();
    return total;
}

// Fig. 4 on a GPU: quick sort of the tile in shared memory.  A segment
// [lo, hi) longer than QS_SMALL is partitioned around its middle element
// (the pivot choice of Fig. 4): keys '< pivot' first, then the pivot, then
// the rest -- in parallel, by block scans of the per-thread counts -- and
// its two sides are pushed on a stack; shorter segments are finished by one
// thread each with insertion sort.  Keys equal to the pivot all go right, as
// in Fig. 4, so heavy duplicates make it quadratic like the original.
constexpr int QS_SMALL = 32;

template <class K, int THREADS, int KPT>
__global__ void __launch_bounds__(THREADS)
tile_quick_kernel(Geo g, const K *__restrict__ in_k, K *buf_k0, K *buf_k1, int codec,
                  const int64_t *__restrict__ ntiles_total) {
    constexpr int T = THREADS * KPT;
    constexpr int MAXSTACK = T / QS_SMALL + 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    griddep_wait();
    K *sk = reinterpret_cast<K *>(smem_raw);
    K *tmp = sk + T;
    int2 *stack = reinterpret_cast<int2 *>(tmp + T);
    int2 *small = stack + MAXSTACK;                  // up to T short segments
    int *warp_sums = reinterpret_cast<int *>(small + T);
    __shared__ int top, nsmall, seg_lo, seg_hi;
    const int64_t total = min(*ntiles_total, g.ntiles_ub);
    const int tid = threadIdx.x;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const TileInfo ti = tile_info(g, t, T);
        for (int pos = tid; pos < T; pos += THREADS)
            sk[pos] = pos < ti.lcnt ? enc_code(in_k[ti.ibase + pos], codec) : max_code<K>();
        if (tid == 0) {
            top = 0;
            nsmall = 0;
            if (ti.cnt > QS_SMALL) stack[top++] = make_int2(0, ti.cnt);
            else if (ti.cnt > 1) small[nsmall++] = make_int2(0, ti.cnt);
        }
        __syncthreads();
        for (;;) {
            // thread 0 pops the next segment (or -1 when none is left) and
            // publishes it; every thread reads it after the barrier, and
            // thread 0 writes it again only after the body's last barrier
            if (tid == 0) {
                if (top > 0) {
                    const int2 sg = stack[--top];
                    seg_lo = sg.x;
                    seg_hi = sg.y;
                } else {
                    seg_lo = -1;
                }
            }
            __syncthreads();
            if (seg_lo < 0) break;
            const int lo = seg_lo, hi = seg_hi, len = hi - lo, mid = lo + len / 2;
            const K pivot = sk[mid];
            // this thread's chunk of the segment
            const int per = (len + THREADS - 1) / THREADS;
            const int c0 = min(lo + tid * per, hi), c1 = min(c0 + per, hi);
            int nl = 0, nr = 0;
            for (int x = c0; x < c1; ++x) {
                if (x == mid) continue;
                if (sk[x] < pivot) ++nl;
                else ++nr;
            }
            int el, er;
            const int tl = block_excl_scan<THREADS>(nl, warp_sums, el);
            block_excl_scan<THREADS>(nr, warp_sums, er);
            int wl = lo + el, wr = lo + tl + 1 + er;
            for (int x = c0; x < c1; ++x) {
                if (x == mid) continue;
                const K v = sk[x];
                if (v < pivot) tmp[wl++] = v;
                else tmp[wr++] = v;
            }
            if (tid == 0) tmp[lo + tl] = pivot;
            __syncthreads();
            for (int x = lo + tid; x < hi; x += THREADS) sk[x] = tmp[x];
            if (tid == 0) {
                const int2 sides[2] = {make_int2(lo, lo + tl), make_int2(lo + tl + 1, hi)};
                for (int q = 0; q < 2; ++q) {
                    // the pending segments are disjoint, so neither list can
                    // overflow; the bounds are checked all the same
                    const int sl = sides[q].y - sides[q].x;
                    if (sl > QS_SMALL && top < MAXSTACK) stack[top++] = sides[q];
                    else if (sl > 1 && nsmall < T) small[nsmall++] = sides[q];
                }
            }
            __syncthreads();
        }
        // short segments: insertion sort, one thread each
        for (int q = tid; q < nsmall; q += THREADS) {
            const int lo = small[q].x, hi = small[q].y;
            for (int i = lo + 1; i < hi; ++i) {
                const K v = sk[i];
                int j = i - 1;
                while (j >= lo && v < sk[j]) {
                    sk[j + 1] = sk[j];
                    --j;
                }
                sk[j + 1] = v;
            }
        }
        __syncthreads();
        K *dst = out_buf<K>(ti.fin, g.fin_k, ti.par, buf_k0, buf_k1);
        for (int pos = tid; pos < ti.cnt; pos += THREADS) {
            const K c = sk[pos];
            dst[ti.base + pos] = ti.fin ? dec_code(c, codec) : c;
        }
        if (tid == 0) count_bytes(g, CLS_TILE_SORT, 2ull * sizeof(K) * ti.cnt);
        __syncthreads();
    }
}

template <class K, int THREADS, int KPT> __host__ __device__ constexpr size_t quick_smem_bytes() {
    return 2 * sizeof(K) * THREADS * KPT + sizeof(int2) * (THREADS * KPT / QS_SMALL + 2) +
           sizeof(int2) * THREADS * KPT + sizeof(int) * (THREADS / 32) + 16;
}

// ---------------------------------------------------------------- CTA merge of a slice

// Merge src[a_lo, a_lo+na) with src[b_lo, b_lo+nb) into dst[o_lo ..), with
// na + nb <= THREADS*VT, staged through shared memory.
template <class K, class V, int THREADS, int VT>
__device__ __forceinline__ void cta_merge(const K *__restrict__ src_k, const V *__restrict__ src_v,
                                          int64_t a_lo, int na, int64_t b_lo, int nb,
                                          K *__restrict__ dst_k, V *__restrict__ dst_v, int64_t o_lo,
                                          bool fin, int codec, K *sk, V *sv) {
    constexpr bool HV = HasVal<V>::value;
    const int tid = threadIdx.x;
    const int total = na + nb;
    K k[VT];
    V v[VT];
    uint32_t idx[VT];
#pragma unroll
    for (int u = 0; u < VT; ++u) {
        int x = tid + u * THREADS;
        if (x < total) {
            int64_t gi = x < na ? a_lo + x : b_lo + (x - na);
            k[u] = src_k[gi];
            if constexpr (HV) v[u] = src_v[gi];
        }
    }
#pragma unroll
    for (int u = 0; u < VT; ++u) {
        int x = tid + u * THREADS;
        if (x < total) {
            sk[spad<K>(x)] = k[u];
            if constexpr (HV) sv[spad<V>(x)] = v[u];
        }
    }
    __syncthreads();
    const int diag = min(tid * VT, total);
    // shared positions order A before B, so "ties to A" is the stable order
    const int i = merge_path_pred<int>(na, nb, diag, [&](int ia, int ib) {
        return sk[spad<K>(na + ib)] < sk[spad<K>(ia)];
    });
    const int count = min(VT, total - diag);
    if constexpr (HV) {
        cand_merge_pairs<K, VT>(sk, nullptr, 0, na, na, nb, i, diag - i, k, idx);
#pragma unroll
        for (int u = 0; u < VT; ++u)
            if (u < count) v[u] = sv[spad<V>((int)idx[u])];
    } else {
        cand_merge_keys<K, VT>(sk, 0, na, na, nb, i, diag - i, k);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < VT; ++u) {
        if (u < count) {
            sk[spad<K>(diag + u)] = k[u];
            if constexpr (HV) sv[spad<V>(diag + u)] = v[u];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < VT; ++u) {
        int x = tid + u * THREADS;
        if (x < total) {
            K c = sk[spad<K>(x)];
            dst_k[o_lo + x] = fin ? dec_code(c, codec) : c;
            if constexpr (HV) dst_v[o_lo + x] = sv[spad<V>(x)];
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- merge levels

// One merge pass.  kind LEVEL_SEG: level `lv` of the in-block schedule --
// inside segment [s, e) the runs are [s + q*W, s + (q+1)*W), W = T << lv, and
// runs 2c, 2c+1 merge into one; a segment is active while lv < its level
// count.  kind LEVEL_XBLOCK: round `r` of the merge phase -- groups of 2^r
// consecutive blocks are runs and pair k merges groups 2k and 2k+1 (an
// unpaired last group is copied).  Every pair is cut into output tiles of T
// keys from its start (tpp tiles per pair for cross-block rounds, enough for
// the longest pair; tiles past a pair's end are inactive), so an output tile
// always lies inside one pair.
enum : int { LEVEL_SEG = 0, LEVEL_XBLOCK = 1, LEVEL_ODDEVEN = 2 };
struct Level {
    int kind;
    int lv;          // LEVEL_SEG: level
    int r;           // LEVEL_XBLOCK / LEVEL_ODDEVEN: round
    int64_t tpp;     // LEVEL_XBLOCK / LEVEL_ODDEVEN: tiles per pair
    int64_t ntiles;  // LEVEL_XBLOCK / LEVEL_ODDEVEN: npairs * tpp (LEVEL_SEG reads the tile count)
    int mlogT;       // merge tile = 2^mlogT keys (<= the sort tile; LEVEL_SEG cuts every sort
                     // tile into 2^(logT - mlogT) merge tiles)
};

struct TilePair {
    int64_t ps, pm, pe;  // A = [ps, pm), B = [pm, pe)
    int64_t x0, x1;      // this tile's output range
    int src, dst;        // buffer parities
    bool fin, active;
};

__device__ __forceinline__ TilePair tile_pair(const Geo &g, const Level &L, int64_t t) {
    TilePair p;
    const int64_t T = int64_t(1) << g.logT;
    const int64_t TM = int64_t(1) << L.mlogT;
    if (L.kind == LEVEL_SEG) {
        const int sh = g.logT - L.mlogT;
        const int64_t ts = t >> sh, h = t & ((int64_t(1) << sh) - 1);
        const int64_t s = g.tseg[ts];
        int64_t slo, shi;
        seg_bounds(g, s, slo, shi);
        const int Ls = seg_levels(shi - slo, g.logT);
        const int64_t j = ts - g.tprefix[s];
        const int64_t W = T << L.lv;
        p.x0 = slo + j * T + h * TM;
        p.x1 = min(p.x0 + TM, shi);
        p.active = L.lv < Ls && p.x0 < shi;
        p.ps = slo + (j >> (L.lv + 1)) * 2 * W;
        p.pm = min(p.ps + W, shi);
        p.pe = min(p.ps + 2 * W, shi);
        p.src = (Ls - L.lv + g.R) & 1;
        p.dst = (Ls - L.lv - 1 + g.R) & 1;
        p.fin = (L.lv == Ls - 1) && g.R == 0;
    } else if (L.kind == LEVEL_ODDEVEN) {
        // compare-split round r: even rounds pair blocks (0,1),(2,3)..; odd
        // rounds leave block 0 alone and pair (1,2),(3,4)..; a block without
        // a partner is copied.  Merging a pair in place is the compare-split:
        // the lower block keeps the first |block| keys, the upper the rest.
        const int64_t k = t / L.tpp, j = t - k * L.tpp;
        const int64_t first = (L.r & 1) ? (k == 0 ? 0 : 2 * k - 1) : 2 * k;
        const int64_t nblk = ((L.r & 1) && k == 0) ? 1 : 2;
        const int64_t last = min(first + nblk, g.S);
        p.ps = clamp64(g.off[min(first, g.S)], 0, g.n);
        p.pe = clamp64(g.off[last], p.ps, g.n);
        p.pm = last - first >= 2 ? clamp64(g.off[first + 1], p.ps, p.pe) : p.pe;
        p.x0 = p.ps + j * TM;
        p.x1 = min(p.x0 + TM, p.pe);
        p.active = p.x0 < p.pe;
        p.src = L.r & 1;
        p.dst = (L.r + 1) & 1;
        p.fin = false;
    } else {
        const int64_t k = t / L.tpp, j = t - k * L.tpp;
        const int64_t G = int64_t(2) << L.r, H = int64_t(1) << L.r;
        p.ps = clamp64(g.off[min(k * G, g.S)], 0, g.n);
        p.pm = clamp64(g.off[min(k * G + H, g.S)], p.ps, g.n);
        p.pe = clamp64(g.off[min(k * G + G, g.S)], p.pm, g.n);
        p.x0 = p.ps + j * TM;
        p.x1 = min(p.x0 + TM, p.pe);
        p.active = p.x0 < p.pe;
        p.src = (g.R - L.r) & 1;
        p.dst = (g.R - L.r - 1) & 1;
        p.fin = (L.r == g.R - 1);
    }
    return p;
}

__device__ __forceinline__ int64_t level_tiles(const Geo &g, const Level &L,
                                               const int64_t *ntiles_total) {
    return L.kind == LEVEL_SEG ? min(*ntiles_total, g.ntiles_ub) << (g.logT - L.mlogT) : L.ntiles;
}

// Merge-path split (absolute A index) at the start of every active tile, one
// thread per tile (a binary search).  On 2^28 keys this beat both wider
// searches tried: 4, 8 or 32 lanes per tile running a (lanes+1)-way search
// (0.065 to 0.13 ms a pass against 0.047 ms) and one thread probing three
// quartiles per step (0.053 ms): fewer rounds of dependent loads do not pay
// for the extra loads.
template <class K>
__global__ void partition_kernel(Geo g, Level L, const K *buf0, const K *buf1, int64_t *split,
                                 const int64_t *__restrict__ ntiles_total) {
    griddep_wait();
    const int64_t total = level_tiles(g, L, ntiles_total);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const TilePair p = tile_pair(g, L, t);
        if (!p.active) continue;
        const K *src = p.src ? buf1 : buf0;
        auto A = [&](int64_t i) { return src[p.ps + i]; };
        auto B = [&](int64_t i) { return src[p.pm + i]; };
        split[t] = p.ps + merge_path<K, int64_t>(A, p.pm - p.ps, B, p.pe - p.pm, p.x0 - p.ps);
    }
}

// The A and B slices of tile t: A[a_lo, a_hi), B[b_lo, b_hi) -> out[x0, x1).
// For sorted runs the splits are monotone and these are exact.  Runs that
// are not sorted (a caller's bad input, or malformed segment offsets) make
// the splits arbitrary; the clamps then keep both slices inside their runs
// and their total within the tile (x1 - x0), so the output is undefined but
// no memory outside the arrays or the staging buffers is touched.
struct Slice {
    int64_t a_lo, a_hi, b_lo, b_hi;
};
__device__ __forceinline__ Slice tile_slice(const TilePair &p, const int64_t *split, int64_t t) {
    Slice q;
    const int64_t len = p.x1 - p.x0;
    q.a_lo = clamp64(split[t], p.ps, p.pm);
    const int64_t a_hi = (p.x1 == p.pe) ? p.pm : split[t + 1];
    q.a_hi = clamp64(a_hi, q.a_lo, min(p.pm, q.a_lo + len));
    q.b_lo = clamp64(p.pm + (p.x0 - p.ps) - (q.a_lo - p.ps), p.pm, p.pe);
    const int64_t nb = min(len - (q.a_hi - q.a_lo), p.pe - q.b_lo);
    q.b_hi = q.b_lo + (nb > 0 ? nb : 0);
    return q;
}

// Merge pass staged through padded shared memory with plain loads (any key
// and value type, any alignment).
template <class K, class V, int THREADS, int VT>
__global__ void __launch_bounds__(THREADS)
merge_kernel(Geo g, Level L, K *buf_k0, K *buf_k1, V *buf_v0, V *buf_v1, int codec,
             const int64_t *__restrict__ split, const int64_t *__restrict__ ntiles_total) {
    constexpr int TT = THREADS * VT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    K *sk = reinterpret_cast<K *>(smem_raw);
    V *sv = reinterpret_cast<V *>(smem_raw + smem_val_offset<K>(TT));
    griddep_wait();
    const int64_t total = level_tiles(g, L, ntiles_total);
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const TilePair p = tile_pair(g, L, t);
        if (!p.active) continue;
        const Slice q = tile_slice(p, split, t);
        cta_merge<K, V, THREADS, VT>(p.src ? buf_k1 : buf_k0, p.src ? buf_v1 : buf_v0, q.a_lo,
                                     (int)(q.a_hi - q.a_lo), q.b_lo, (int)(q.b_hi - q.b_lo),
                                     out_buf<K>(p.fin, g.fin_k, p.dst, buf_k0, buf_k1),
                                     out_buf<V>(p.fin, g.fin_v, p.dst, buf_v0, buf_v1), p.x0, p.fin,
                                     codec, sk, sv);
        if (threadIdx.x == 0)
            count_bytes(g, CLS_MERGE, 2ull * (sizeof(K) + (HasVal<V>::value ? sizeof(V) : 0)) * (p.x1 - p.x0));
    }
}

// Encode a whole array into codes (and copy its values): the first step of
// merging caller-sorted runs, whose keys arrive in their dtype.
template <class K, class V>
__global__ void encode_copy_kernel(const K *__restrict__ in_k, const V *__restrict__ in_v, K *out_k,
                                   V *out_v, int64_t n, int codec) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        out_k[i] = enc_code(in_k[i], codec);
        if constexpr (HasVal<V>::value) out_v[i] = in_v[i];
    }
}

// Odd-even schedule: scatter the n keys of p balanced blocks (bounds
// floor(i*n/p)) into p slots of `cap` keys each, encoded; the slots past a
// block's keys hold the largest code (+infinity sentinels).  Grid: x chunks
// of a slot by y slots, so every thread computes its slot's bounds once.
template <class K>
__global__ void pad_scatter_kernel(const K *__restrict__ in, K *out, int64_t n, int64_t p, int64_t cap,
                                   int codec) {
    griddep_wait();
    for (int64_t i = blockIdx.y; i < p; i += gridDim.y) {
        const int64_t b0 = (int64_t)(((unsigned __int128)(uint64_t)i * (uint64_t)n) / (uint64_t)p);
        const int64_t b1 = (int64_t)(((unsigned __int128)(uint64_t)(i + 1) * (uint64_t)n) / (uint64_t)p);
        K *o = out + i * cap;
        for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < cap; l += (int64_t)gridDim.x * blockDim.x)
            o[l] = l < b1 - b0 ? enc_code(in[b0 + l], codec) : max_code<K>();
    }
}

// Odd-even schedule, last step: the first n slots hold the sorted keys.
template <class K>
__global__ void decode_copy_kernel(const K *__restrict__ in, K *out, int64_t n, int codec) {
    griddep_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dec_code(in[i], codec);
}

// ---------------------------------------------------------------- TMA pipeline helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on an mbarrier phase: gives up (false) once `limit_ns` of
// global time has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0 && global_ns() - t0 > limit_ns) return false;
    }
}
// Cross-proxy fence: orders this thread's (and, by cumulativity, what it has
// acquired of other threads') generic-proxy shared-memory accesses before its
// later async-proxy ones (bulk copies).
__device__ __forceinline__ void proxy_fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 1-D bulk copy global -> shared (TMA), completing `bytes` on the mbarrier.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

constexpr uint64_t WAIT_LIMIT_DEFAULT = 2000000000ull;  // 2 s

// Stage a[lo, hi) of a 16-byte aligned array of `n` items into shared memory
// dst[0 ..): the 16-byte chunks by TMA, the ragged end past the array's last
// full chunk by plain loads.  Returns the index in dst of item lo; adds the
// TMA bytes to *tx.
template <class T>
__device__ __forceinline__ int stage_window(T *dst, const T *a, int64_t n, int64_t lo, int64_t hi,
                                            uint64_t *bar, uint32_t *tx) {
    constexpr int64_t E = 16 / sizeof(T);
    const int64_t ws = lo & ~(E - 1);
    if (hi <= lo) return (int)(lo - ws);
    int64_t we = (hi + E - 1) & ~(E - 1);
    const int64_t nfull = n & ~(E - 1);
    if (we > nfull) we = nfull;  // never read past the array
    if (we > ws) {
        const uint32_t bytes = (uint32_t)((we - ws) * (int64_t)sizeof(T));
        tma_load_1d(dst, a + ws, bytes, bar);
        *tx += bytes;
    } else {
        we = ws;
    }
    for (int64_t x = we; x < hi; ++x) dst[x - ws] = a[x];  // at most E-1 items
    return (int)(lo - ws);
}

// Items that stage_window(.., lo, hi, ..) occupies in shared memory, rounded
// up to 16 bytes: where the next window may start.
template <class T> __device__ __forceinline__ int window_span(int64_t lo, int64_t hi) {
    constexpr int64_t E = 16 / sizeof(T);
    if (hi <= lo) return 0;
    return (int)(((hi - (lo & ~(E - 1))) + E - 1) & ~(E - 1));
}

// Descriptor of one staged tile, written by the producer next to its data.
struct StageDesc {
    int64_t o_lo;
    int a_off, na, b_off, nb;  // key windows
    int av_off, bv_off;        // value windows
    int flags;                 // bit0 active, bit1 dst parity, bit2 final pass (bit3: no more tiles)
    int pad;
    unsigned *ctr;             // persistent merge: the pair counter that counts this tile done
};

// One stage holds the tile's A and B windows back to back (B's starts at the
// next 16-byte boundary after A's), so it needs the tile's size plus the
// rounding of four window ends: TT + 6 * (16 / item size) items; the key
// window has 32 more, which a thread consumer's run-ahead reads past the end
// of B may touch (their values are never used).
template <class K, class V, int TT> struct TmaLayout {
    static constexpr int EK = 16 / (int)sizeof(K);
    static constexpr int EV = sizeof(V) > 1 ? 16 / (int)sizeof(V) : 1;
    static constexpr size_t keys = ((size_t)(TT + 6 * EK + 32) * sizeof(K) + 127) & ~size_t(127);
    static constexpr size_t vals =
        sizeof(V) > 1 ? (((size_t)(TT + 6 * EV) * sizeof(V) + 127) & ~size_t(127)) : 0;
    static constexpr size_t stage = keys + vals + 128;  // windows + descriptor
};

// Per-warp scratch of the warp consumer: the warp's 32*VT keys (and, for
// pairs, their staging indices), in 16-byte chunks of keys stored at the
// XOR-swizzled chunk position c ^ ((c >> 3) & 7), which keeps the striped
// scalar writes and the 16-byte chunk reads and writes of both transposes
// free of bank conflicts.
template <class K, class V, int VT> struct WarpScratch {
    static constexpr size_t keys = ((size_t)32 * VT * sizeof(K) + 127) & ~size_t(127);
    static constexpr size_t idx = HasVal<V>::value ? (((size_t)32 * VT * 4 + 127) & ~size_t(127)) : 0;
    static constexpr size_t bytes = keys + idx;
};
__device__ __forceinline__ int swz_chunk(int c) { return c ^ ((c >> 3) & 7); }

// N items of T (8 or 16 bytes in all) moved as one shared-memory access.
template <class T, int N> __device__ __forceinline__ void ld_chunk(const T *p, T *v) {
    static_assert(sizeof(T) * N == 16 || sizeof(T) * N == 8, "chunk of 8 or 16 bytes");
    if constexpr (sizeof(T) * N == 16) {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        memcpy(v, &u, 16);
    } else {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        memcpy(v, &u, 8);
    }
}
template <class T, int N> __device__ __forceinline__ void st_chunk(T *p, const T *v) {
    static_assert(sizeof(T) * N == 16 || sizeof(T) * N == 8, "chunk of 8 or 16 bytes");
    if constexpr (sizeof(T) * N == 16) {
        uint4 u;
        memcpy(&u, v, 16);
        *reinterpret_cast<uint4 *>(p) = u;
    } else {
        uint2 u;
        memcpy(&u, v, 8);
        *reinterpret_cast<uint2 *>(p) = u;
    }
}

template <class K, class V, int THREADS, int VT, int STAGES, bool WARPMERGE>
__host__ __device__ constexpr size_t tma_smem_bytes() {
    return STAGES * TmaLayout<K, V, THREADS * VT>::stage + (THREADS / 32) * WarpScratch<K, V, VT>::bytes +
           2 * STAGES * sizeof(uint64_t) + 128;
}

// The merge-path splits of a tile at the warp's output range [d0, d1):
// lanes 0-15 search diagonal d0, lanes 16-31 diagonal d1.  Each half-warp
// tests 16 evenly spaced points of the interval holding its split (the
// predicate B[d-1-i] < A[i] is false then true) and keeps the piece between
// the last false and the first true test: a 17-way search, 3 rounds for a
// 4096-key tile.  Returns the A index of both splits in every lane.
template <class K>
__device__ __forceinline__ void warp_splits(const K *sa, const K *sb, int na, int nb, int d0, int d1, int lane,
                                            int &i0, int &i1) {
    const int half = lane >> 4, sub = lane & 15;
    const int dd = half ? d1 : d0;
    int lo = dd > nb ? dd - nb : 0, hi = dd < na ? dd : na;
    while (__any_sync(0xffffffffu, lo < hi)) {
        const bool live = lo < hi;
        const int mid = lo + ((sub + 1) * (hi - lo)) / 17;  // lo <= mid < hi
        const bool test = live && sb[dd - 1 - mid] < sa[mid];
        const unsigned yes = (__ballot_sync(0xffffffffu, test) >> (16 * half)) & 0xffffu;
        const int f = yes ? __ffs(yes) - 1 : 16;  // first point whose test holds
        const int mprev = __shfl_sync(0xffffffffu, mid, 16 * half + (f > 0 ? f - 1 : 0));
        const int mf = __shfl_sync(0xffffffffu, mid, 16 * half + (f < 16 ? f : 15));
        if (live) {
            if (f > 0) lo = mprev + 1;
            if (f < 16) hi = mf;
        }
    }
    i0 = __shfl_sync(0xffffffffu, lo, 0);
    i1 = __shfl_sync(0xffffffffu, lo, 16);
}

// Emits a warp's 32*VT merged outputs held chunk-striped: lane l has the
// 16-byte chunks l, l+32, .. (chunk m of the lane in registers m*E ..
// m*E + E-1; for pairs x[] holds their staging indices, A's first, then
// B's from na), so every store instruction writes 512 contiguous bytes.
// Pairs fetch their values from the stage by index and then release it
// (keys-only callers release it before).  cnt = valid outputs, o = global
// index of the first.
template <class K, class V, int VT>
__device__ __forceinline__ void emit_chunk_striped(K (&v)[VT], const uint32_t (&x)[VT], const V *sav,
                                                   const V *sbv, int na, K *dk, V *dv, int64_t o, int cnt,
                                                   bool fin, int codec, uint64_t *empty_bar, int lane) {
    constexpr bool HV = HasVal<V>::value;
    constexpr int E = 16 / (int)sizeof(K);  // keys per 16-byte chunk
    constexpr int C = VT / E;               // chunks per lane
    V vals[VT];
    if constexpr (HV) {
#pragma unroll
        for (int m = 0; m < C; ++m)
#pragma unroll
            for (int p = 0; p < E; ++p) {
                const int i = m * E + p;
                if ((32 * m + lane) * E + p < cnt) vals[i] = (int)x[i] < na ? sav[x[i]] : sbv[x[i] - na];
            }
        mbar_arrive(empty_bar);
    }
    if (fin) {
#pragma unroll
        for (int i = 0; i < VT; ++i) v[i] = dec_code(v[i], codec);
    }
    const bool aligned = (o % E) == 0;
#pragma unroll
    for (int m = 0; m < C; ++m) {
        const int eb = (32 * m + lane) * E;  // first output of this chunk
        if (aligned && eb + E <= cnt) {
            st_chunk<K, E>(dk + o + eb, v + m * E);
        } else {
#pragma unroll
            for (int p = 0; p < E; ++p)
                if (eb + p < cnt) dk[o + eb + p] = v[m * E + p];
        }
        if constexpr (HV) {
#pragma unroll
            for (int p = 0; p < E; ++p)
                if (eb + p < cnt) dv[o + eb + p] = vals[m * E + p];
        }
    }
}

// Stores a warp's 32*VT merged outputs held lane-blocked (lane l has
// outputs VT*l .. VT*l + VT - 1): a transpose through the warp's XOR-swizzled
// scratch makes them chunk-striped, then emit_chunk_striped stores them.
template <class K, class V, int VT>
__device__ __forceinline__ void store_warp_outputs(K (&v)[VT], uint32_t (&x)[VT], const V *sav, const V *sbv,
                                                   int na, K *dk, V *dv, int64_t o, int cnt, bool fin, int codec,
                                                   uint64_t *empty_bar, int lane, K *wk, uint32_t *wx) {
    constexpr bool HV = HasVal<V>::value;
    constexpr int E = 16 / (int)sizeof(K);
    constexpr int C = VT / E;
    static_assert(C >= 1 && VT % E == 0, "whole chunks per lane");
#pragma unroll
    for (int r = 0; r < C; ++r) {
        const int at = swz_chunk(C * lane + r) * E;
        st_chunk<K, E>(wk + at, v + r * E);
        if constexpr (HV) st_chunk<uint32_t, E>(wx + at, x + r * E);
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < C; ++m) {
        const int at = swz_chunk(32 * m + lane) * E;
        ld_chunk<K, E>(wk + at, v + m * E);
        if constexpr (HV) ld_chunk<uint32_t, E>(wx + at, x + m * E);
    }
    __syncwarp();  // the scratch is free for the warp's next tile
    emit_chunk_striped<K, V, VT>(v, x, sav, sbv, na, dk, dv, o, cnt, fin, codec, empty_bar, lane);
}

// The same for outputs held S apart (S odd, S = VT + 1): lane l has outputs
// S*l .. S*l + S - 1 below 32*VT (the last lane the remainder).  The odd
// stride makes the scalar scratch writes conflict-free without a swizzle;
// the chunk reads are contiguous across lanes.
template <class K, class V, int VT, int S>
__device__ __forceinline__ void store_warp_outputs_spaced(const K (&v)[S], const uint32_t (&x)[S], const V *sav,
                                                          const V *sbv, int na, K *dk, V *dv, int64_t o, int cnt,
                                                          bool fin, int codec, uint64_t *empty_bar, int lane,
                                                          K *wk, uint32_t *wx) {
    constexpr bool HV = HasVal<V>::value;
    constexpr int WO = 32 * VT;
    constexpr int E = 16 / (int)sizeof(K);
    constexpr int C = VT / E;
    static_assert(S % 2 == 1 && 31 * S <= WO, "odd spacing, the last lane keeps at least nothing");
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const int e = lane * S + q;
        if (e < WO) {
            wk[e] = v[q];
            if constexpr (HV) wx[e] = x[q];
        }
    }
    __syncwarp();
    K c[VT];
    uint32_t cx[VT];
#pragma unroll
    for (int m = 0; m < C; ++m) {
        ld_chunk<K, E>(wk + (32 * m + lane) * E, c + m * E);
        if constexpr (HV) ld_chunk<uint32_t, E>(wx + (32 * m + lane) * E, cx + m * E);
    }
    __syncwarp();  // the scratch is free for the warp's next tile
    emit_chunk_striped<K, V, VT>(c, cx, sav, sbv, na, dk, dv, o, cnt, fin, codec, empty_bar, lane);
}

// Warp consumer of one staged tile (bitonic): warp w produces outputs
// [d0, d1) of the tile (32*VT of them).  After its two merge-path splits it
// reads its A slice followed by its B slice reversed -- a bitonic sequence,
// padded in the middle with the largest key -- striped across lanes
// (element e at lane e%32, register e/32: conflict-free shared loads) and
// sorts it with a bitonic merger: the strides of 32 and more are register
// compare-exchanges in this layout; a transpose through the warp's scratch
// then gives each lane VT consecutive elements, so that of the strides
// below 32 only those of VT and more cross lanes (shuffles) and the rest are
// register compare-exchanges again.  Pairs compare (key, staging index).
template <class K, class V, int VT>
__device__ __forceinline__ void warp_merge_tile(const K *sa, const K *sb, const V *sav, const V *sbv,
                                                int na, int nb, K *dk, V *dv, int64_t o_lo, bool fin,
                                                int codec, uint64_t *empty_bar, int tid, K *wk,
                                                uint32_t *wx) {
    constexpr bool HV = HasVal<V>::value;
    constexpr int WO = 32 * VT;
    constexpr int E = 16 / (int)sizeof(K);
    constexpr int C = VT / E;
    const int lane = tid & 31, w = tid >> 5;
    const int total = na + nb;
    const int d0 = min(w * WO, total), d1 = min(d0 + WO, total);
    int i0, i1;
    warp_splits<K>(sa, sb, na, nb, d0, d1, lane, i0, i1);
    const int naw = i1 - i0, j0 = d0 - i0, nbw = (d1 - d0) - naw;
    K v[VT];
    uint32_t x[VT];
    if (naw + nbw == WO) {
        // a full warp: every element is A's or B's
        const K *pa = sa + i0, *pb = sb + (j0 + WO - 1);
#pragma unroll
        for (int k = 0; k < VT; ++k) {
            const int e = lane + 32 * k;
            const bool in_a = e < naw;
            v[k] = *(in_a ? pa + e : pb - e);
            x[k] = in_a ? (uint32_t)(i0 + e) : (uint32_t)(na + j0 + WO - 1 - e);
        }
    } else {
#pragma unroll
        for (int k = 0; k < VT; ++k) {
            const int e = lane + 32 * k;
            if (e < naw) {
                v[k] = sa[i0 + e];
                x[k] = (uint32_t)(i0 + e);
            } else if (e >= WO - nbw) {
                const int bi = j0 + (WO - 1 - e);
                v[k] = sb[bi];
                x[k] = (uint32_t)(na + bi);
            } else {
                v[k] = max_code<K>();
                x[k] = 0xffffffffu;
            }
        }
    }
    if constexpr (!HV) mbar_arrive(empty_bar);  // every shared read of this stage is done
    // strides WO/2 .. 32: registers k and k + r of the same lane
#pragma unroll
    for (int r = VT >> 1; r > 0; r >>= 1) {
#pragma unroll
        for (int k = 0; k < VT; ++k) {
            if ((k & r) == 0) {
                if constexpr (HV) cas_pairs(v[k], x[k], v[k + r], x[k + r]);
                else cas_keys(v[k], v[k + r]);
            }
        }
    }
    // transpose: element e = lane + 32k -> lane e / VT, register e % VT
#pragma unroll
    for (int k = 0; k < VT; ++k) {
        const int e = lane + 32 * k;
        const int at = swz_chunk(e / E) * E + e % E;
        wk[at] = v[k];
        if constexpr (HV) wx[at] = x[k];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < C; ++r) {
        const int at = swz_chunk(C * lane + r) * E;
        ld_chunk<K, E>(wk + at, v + r * E);
        if constexpr (HV) ld_chunk<uint32_t, E>(wx + at, x + r * E);
    }
    __syncwarp();
    // now lane l holds elements VT*l + q; strides 16 .. VT cross lanes
#pragma unroll
    for (int s = 16; s >= VT; s >>= 1) {
        const int ls = s / VT;
        const bool up = lane & ls;
#pragma unroll
        for (int q = 0; q < VT; ++q) {
            const K pk = shfl_xor_k<VT>(v[q], ls);
            if constexpr (HV) {
                const uint32_t px = __shfl_xor_sync(0xffffffffu, x[q], ls);
                const bool take = up ? ki_less(v[q], x[q], pk, px) : ki_less(pk, px, v[q], x[q]);
                v[q] = take ? pk : v[q];
                x[q] = take ? px : x[q];
            } else {
                v[q] = ((pk < v[q]) != up) ? pk : v[q];
            }
        }
    }
    // strides below VT (and below 32): registers q and q + r
#pragma unroll
    for (int r = (VT < 32 ? VT : 32) >> 1; r > 0; r >>= 1) {
#pragma unroll
        for (int q = 0; q < VT; ++q) {
            if ((q & r) == 0) {
                if constexpr (HV) cas_pairs(v[q], x[q], v[q + r], x[q + r]);
                else cas_keys(v[q], v[q + r]);
            }
        }
    }
    store_warp_outputs<K, V, VT>(v, x, sav, sbv, na, dk, dv, o_lo + d0, d1 - d0, fin, codec, empty_bar, lane, wk,
                                 wx);
}

// Thread consumer of one staged tile (sequential merge): lane l of warp w
// produces outputs [d, d + VT) of the tile, d = 32*VT*w + VT*l.  Its
// merge-path split comes from a binary search over the tile; then VT steps
// of the sequential merge each take the smaller head (A's on a tie, which is
// the stable order, so pairs need no index compares) and load the next item
// of that run: one shared load and a few integer ops per output.  The warp
// first writes the largest key just past B's last item (stage slack, past
// what the copies delivered), so an exhausted B never wins; A's end is
// tested explicitly.
// A hook that does nothing (thread_merge_tile's default before_store).
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

template <class K, class V, int VT, class Hook = NoHook>
__device__ __forceinline__ void thread_merge_tile(const K *sa, K *sb, const V *sav, const V *sbv,
                                                  int na, int nb, K *dk, V *dv, int64_t o_lo, bool fin,
                                                  int codec, uint64_t *empty_bar, int tid, K *wk,
                                                  uint32_t *wx, Hook before_store = Hook()) {
    constexpr bool HV = HasVal<V>::value;
    constexpr int WO = 32 * VT;
    const int lane = tid & 31, w = tid >> 5;
    const int total = na + nb;
    const int d0 = min(w * WO, total), d1 = min(d0 + WO, total);
    if (lane == 0) sb[nb] = max_code<K>();  // every warp writes the same sentinel
    __syncwarp();
    // outputs per lane: VT, or VT + 1 (odd) when VT >= 31 -- lanes whose
    // sequential reads advance in step then sit an odd distance apart, in
    // distinct banks (the last lane takes the remainder)
    constexpr int S = VT >= 31 ? VT + 1 : VT;
    const int diag = min(d0 + lane * S, d1);
    const int i_split = merge_path_pred<int>(na, nb, diag, [&](int ia, int ib) { return sb[ib] < sa[ia]; });
    // A warp whose outputs all come from one run (sorted or reversed input,
    // long runs of equal keys) copies them instead: its lanes' sequential
    // reads would sit VT items apart, all in one or two shared-memory banks.
    {
        const int i0 = __shfl_sync(0xffffffffu, i_split, 0), j0 = d0 - i0, wn = d1 - d0;
        const bool all_a = wn > 0 && i0 + wn <= na && (j0 >= nb || !(sb[j0] < sa[i0 + wn - 1]));
        const bool all_b = wn > 0 && !all_a && j0 + wn <= nb && (i0 >= na || sb[j0 + wn - 1] < sa[i0]);
        if (all_a || all_b) {
            before_store();
            const K *src = all_a ? sa + i0 : sb + j0;
            const V *srcv = all_a ? sav + i0 : sbv + j0;
            K *out = dk + o_lo + d0;
            V *outv = dv + o_lo + d0;
            if (fin) {
#pragma unroll 4
                for (int e = lane; e < wn; e += 32) {
                    out[e] = dec_code(src[e], codec);
                    if constexpr (HV) outv[e] = srcv[e];
                }
            } else {
#pragma unroll 4
                for (int e = lane; e < wn; e += 32) {
                    out[e] = src[e];
                    if constexpr (HV) outv[e] = srcv[e];
                }
            }
            mbar_arrive(empty_bar);  // every shared read of this stage is done
            return;
        }
    }
    const K *pa = sa + i_split, *pb = sb + (diag - i_split);
    const K *const a_end = sa + na;
    K a = *pa, b = *pb;  // a is not used once A is exhausted
    K v[S];
    uint32_t x[S];
#pragma unroll
    for (int u = 0; u < S; ++u) {
        const bool tb = pa >= a_end || b < a;  // take B's head
        v[u] = tb ? b : a;
        if constexpr (HV) x[u] = tb ? (uint32_t)(na + (pb - sb)) : (uint32_t)(pa - sa);
        pa += tb ? 0 : 1;
        pb += tb ? 1 : 0;
        const K nxt = *(tb ? pb : pa);
        a = tb ? a : nxt;
        b = tb ? nxt : b;
    }
    if constexpr (!HV) mbar_arrive(empty_bar);  // every shared read of this stage is done
    before_store();
    if constexpr (S == VT)
        store_warp_outputs<K, V, VT>(v, x, sav, sbv, na, dk, dv, o_lo + d0, d1 - d0, fin, codec, empty_bar, lane,
                                     wk, wx);
    else
        store_warp_outputs_spaced<K, V, VT, S>(v, x, sav, sbv, na, dk, dv, o_lo + d0, d1 - d0, fin, codec,
                                               empty_bar, lane, wk, wx);
}

// Merge pass with a TMA pipeline (warp specialised, persistent).  The last
// warp produces: its lanes compute the A and B slices of 32 of this CTA's
// tiles at a time and stage them by 1-D bulk copies into a ring of STAGES
// shared-memory stages (full/empty mbarriers).  THREADS consumer threads
// take each stage; every warp produces 32*VT outputs, either with the warp
// bitonic merger (WARPMERGE) or with one sequential merge of VT outputs per
// thread, and stores them as 512-byte runs.  All waits are bounded; a
// timeout records BS_ERR_TIMEOUT and ends the CTA.  Needs 16-byte aligned
// buffers.
// CTAs per SM the merge pipeline is compiled for (a register cap): as many
// as its shared memory lets reside (228 KB per SM, 1 KB reserved per CTA),
// but no more than leave each thread 56 registers (32-bit keys alone) or 64
// (otherwise).  Its speed follows the resident warps.
template <class K, class V, int THREADS, int VT, int STAGES, bool WARPMERGE> constexpr int merge_min_ctas() {
    const int by_smem = (int)((228 * 1024) / (tma_smem_bytes<K, V, THREADS, VT, STAGES, WARPMERGE>() + 1024));
    const int regs = (sizeof(K) == 4 && !HasVal<V>::value) ? 56 : 64;
    const int by_regs = 65536 / ((THREADS + 32) * regs);
    const int m = by_smem < by_regs ? by_smem : by_regs;
    return m < 1 ? 1 : m;
}

template <class K, class V, int THREADS, int VT, int STAGES, bool WARPMERGE>
__global__ void __launch_bounds__(THREADS + 32, (merge_min_ctas<K, V, THREADS, VT, STAGES, WARPMERGE>()))
merge_tma_kernel(Geo g, Level L, K *buf_k0, K *buf_k1, V *buf_v0, V *buf_v1, int codec,
                 const int64_t *__restrict__ split, const int64_t *__restrict__ ntiles_total) {
    constexpr int TT = THREADS * VT;
    constexpr bool HV = HasVal<V>::value;
    using LY = TmaLayout<K, V, TT>;
    using WS = WarpScratch<K, V, VT>;
    constexpr size_t SCRATCH = (THREADS / 32) * WS::bytes;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + STAGES * LY::stage + SCRATCH);
    uint64_t *empty = full + STAGES;
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
        mbar_fence_init();
    }
    __syncthreads();
    griddep_wait();  // the splits and the runs come from the kernels before

    const int64_t total = level_tiles(g, L, ntiles_total);
    const int64_t n = g.n;
    const uint64_t WAIT_LIMIT = g.wait_ns ? g.wait_ns : WAIT_LIMIT_DEFAULT;

    if (threadIdx.x >= THREADS) {
        // ---------------- producer warp
        // The 32 lanes compute the slices of the CTA's next 32 tiles at once
        // (their index loads overlap), then take turns, in tile order, to
        // claim a free stage and issue that tile's copies.
        const int lane = threadIdx.x - THREADS;
        int64_t it = 0;
        int stg = 0;          // it % STAGES
        uint32_t ph = 0;      // (it / STAGES) & 1
        for (int64_t base = blockIdx.x; base < total; base += 32 * (int64_t)gridDim.x) {
            const int64_t t = base + (int64_t)lane * gridDim.x;
            TilePair p{};
            Slice q{};
            if (t < total) {
                p = tile_pair(g, L, t);
                if (p.active) q = tile_slice(p, split, t);
            }
            const int64_t left = (total - base + gridDim.x - 1) / gridDim.x;
            const int cnt = left < 32 ? (int)left : 32;
            for (int j = 0; j < cnt; ++j, ++it, ph ^= (stg == STAGES - 1), stg = (stg == STAGES - 1) ? 0 : stg + 1) {
                bool ok = true;
                if (lane == j) {
                    const int s = stg;
                    if (it >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT)) {
                        if (g.err) atomicCAS(g.err, 0, (int)BS_ERR_TIMEOUT);
                        // drain: wait (bounded) for this CTA's copies still in flight
                        for (int64_t jt = (it > STAGES ? it - STAGES : 0); jt < it; ++jt)
                            mbar_wait(&full[jt % STAGES], (uint32_t)((jt / STAGES) & 1), WAIT_LIMIT);
                        ok = false;
                    } else if (!(g.withhold && blockIdx.x == 0 && it == 0)) {  // test hook: nothing arrives
                        // the consumers' shared-memory reads of this stage (generic
                        // proxy), acquired through the empty barrier, are ordered
                        // before the bulk copies (async proxy) that overwrite it
                        proxy_fence_async_smem();
                        StageDesc d{};
                        uint32_t issued = 0;
                        if (p.active) {
                            const K *src = p.src ? buf_k1 : buf_k0;
                            d.o_lo = p.x0;
                            d.na = (int)(q.a_hi - q.a_lo);
                            d.nb = (int)(q.b_hi - q.b_lo);
                            d.flags = 1 | (p.dst << 1) | (p.fin ? 4 : 0);
                            // bulk copies first (they may complete before the expect
                            // below: the transaction count may go negative within a
                            // phase), then the plain writes, then the releasing
                            // arrive that publishes them
                            const int ak = window_span<K>(q.a_lo, q.a_hi);
                            d.a_off = stage_window(stage_k(s), src, n, q.a_lo, q.a_hi, &full[s], &issued);
                            d.b_off = ak + stage_window(stage_k(s) + ak, src, n, q.b_lo, q.b_hi, &full[s], &issued);
                            if constexpr (HV) {
                                const V *srcv = p.src ? buf_v1 : buf_v0;
                                const int av = window_span<V>(q.a_lo, q.a_hi);
                                d.av_off = stage_window(stage_v(s), srcv, n, q.a_lo, q.a_hi, &full[s], &issued);
                                d.bv_off = av + stage_window(stage_v(s) + av, srcv, n, q.b_lo, q.b_hi, &full[s], &issued);
                            }
                        }
                        *stage_desc(s) = d;
                        mbar_arrive_expect_tx(&full[s], issued);
                    }
                }
                if (!__shfl_sync(0xffffffffu, (int)ok, j)) return;
            }
        }
        return;
    }

    // ---------------- consumers
    const int tid = threadIdx.x;
    int stg = 0;      // tile number % STAGES
    uint32_t ph = 0;  // (tile number / STAGES) & 1
    for (int64_t t = blockIdx.x; t < total;
         t += gridDim.x, ph ^= (stg == STAGES - 1), stg = (stg == STAGES - 1) ? 0 : stg + 1) {
        const int s = stg;
        if (!mbar_wait(&full[s], ph, WAIT_LIMIT)) {
            if (g.err) atomicCAS(g.err, 0, (int)BS_ERR_TIMEOUT);
            return;
        }
        const StageDesc d = *stage_desc(s);
        if (d.flags & 1) {
            const K *sa = stage_k(s) + d.a_off;
            K *sb = stage_k(s) + d.b_off;
            const int na = d.na, nb = d.nb, total_out = na + nb;
            unsigned char *ws = smem_raw + STAGES * LY::stage + (tid >> 5) * WS::bytes;
            const bool fin = (d.flags & 4) != 0;
            K *dk = out_buf<K>(fin, g.fin_k, (d.flags >> 1) & 1, buf_k0, buf_k1);
            V *dv = out_buf<V>(fin, g.fin_v, (d.flags >> 1) & 1, buf_v0, buf_v1);
            if constexpr (WARPMERGE)
                warp_merge_tile<K, V, VT>(sa, sb, stage_v(s) + d.av_off, stage_v(s) + d.bv_off, na, nb, dk, dv,
                                          d.o_lo, fin, codec, &empty[s], tid, reinterpret_cast<K *>(ws),
                                          reinterpret_cast<uint32_t *>(ws + WS::keys));
            else
                thread_merge_tile<K, V, VT>(sa, sb, stage_v(s) + d.av_off, stage_v(s) + d.bv_off, na, nb, dk, dv,
                                            d.o_lo, fin, codec, &empty[s], tid, reinterpret_cast<K *>(ws),
                                            reinterpret_cast<uint32_t *>(ws + WS::keys));
            if (tid == 0) count_bytes(g, CLS_MERGE, 2ull * (sizeof(K) + (HV ? sizeof(V) : 0)) * total_out);
        } else {
            mbar_arrive(&empty[s]);
        }
    }
}

}  // namespace bs
