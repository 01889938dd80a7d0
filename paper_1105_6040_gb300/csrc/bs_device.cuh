// bs_device.cuh -- device code of the GB300 block-decomposed sort.
//
// The paper's paradigm (El-Nashar 2011, Sec. 3.2, Fig. 1) mapped to one GPU:
//   scatter (Fig. 1, scatter phase): block bounds are an offsets array in device
//     memory; nothing moves.
//   sort phase (Fig. 1): every block is cut into tiles of T keys
//     aligned to the block start; one CTA sorts one tile in registers and
//     shared memory (tile_sort_kernel), then merge passes in HBM join the
//     sorted tiles of each block pairwise (seg_merge_kernel) until the block
//     is one sorted run.
//   merge phase (Fig. 1): pairs of sorted blocks are merged,
//     round after round (xblock_merge_kernel), until one run remains.
// Every merge pass splits its output into tiles of T keys; the start of each
// output tile inside its pair of runs is found by a merge-path search
// (Odeh, Green, Mwassi, Shmueli, Birk: "Merge Path", IPDPSW 2012), so each
// CTA merges an independent slice.  Ties go to the left run, which makes all
// merges stable.
//
// Keys travel as order-preserving unsigned codes (encoded when the tile sort
// loads them, decoded by the pass that writes the final output), so every
// comparison is an unsigned integer one.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

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
    unsigned long long *counters;  // algorithmic bytes per kernel class (stats)
};

// kernel classes of the statistics counters (same order as the C ABI's)
enum : int { CLS_TILE_SORT = 0, CLS_MERGE = 1, CLS_PARTITION = 2, CLS_SETUP = 3 };

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

// Bitonic sorting network over N registers, ascending (Batcher 1968).
template <int N, class K> __device__ __forceinline__ void reg_sort_keys(K (&k)[N]) {
#pragma unroll
    for (int size = 2; size <= N; size <<= 1)
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int j = i ^ stride;
                if (j > i) {
                    if ((i & size) == 0) cas_keys(k[i], k[j]);
                    else cas_keys(k[j], k[i]);
                }
            }
}

template <int N, class K> __device__ __forceinline__ void reg_sort_pairs(K (&k)[N], uint32_t (&x)[N]) {
#pragma unroll
    for (int size = 2; size <= N; size <<= 1)
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int j = i ^ stride;
                if (j > i) {
                    if ((i & size) == 0) cas_pairs(k[i], x[i], k[j], x[j]);
                    else cas_pairs(k[j], x[j], k[i], x[i]);
                }
            }
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

// ---------------------------------------------------------------- tile sort

// Shared memory of the tile sort: codes, then (pairs) original positions and
// values, each at a 16-byte boundary.
template <class K, class V> __host__ __device__ constexpr size_t tile_smem_bytes(int T) {
    return smem_val_offset<K>(T) +
           (sizeof(V) > 1 ? smem_val_offset<uint32_t>(T) + sizeof(V) * (size_t)spad_size<V>(T) : 0);
}

// Tile sort (the sort phase of Fig. 1 at CTA scale).  Tile t covers
// keys [s + j*T, min(s + (j+1)*T, e)) of segment [s, e).  Each thread sorts
// KPT keys in registers, then log2(THREADS) rounds merge pairs of sorted
// lists through shared memory (merge-path split + candidate merge); rounds
// whose lists live inside one warp synchronise only that warp.  Pairs sort
// (code, original position), which is the stable order; values move once,
// at the final store.  The sorted tile is written -- decoded if this is the
// segment's last pass -- to the buffer its merge schedule starts from.
template <class K, class V, int THREADS, int KPT>
__global__ void __launch_bounds__(THREADS)
tile_sort_kernel(Geo g, const K *__restrict__ in_k, const V *__restrict__ in_v,
                 K *buf_k0, K *buf_k1, V *buf_v0, V *buf_v1, int codec,
                 const int64_t *__restrict__ ntiles_total) {
    constexpr int T = THREADS * KPT;
    constexpr bool HV = HasVal<V>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
        K *dst_k = par ? buf_k1 : buf_k0;
        V *dst_v = par ? buf_v1 : buf_v0;

        // striped, coalesced load; padding slots get the largest code (and,
        // for pairs, positions past every real one)
        K k[KPT];
        uint32_t x[KPT];
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
            const int pos = tid + u * THREADS;
            k[u] = pos < cnt ? enc_code(in_k[base + pos], codec) : max_code<K>();
            if constexpr (HV) {
                x[u] = (uint32_t)pos;
                if (pos < cnt) sv[spad<V>(pos)] = in_v[base + pos];
            }
        }
        if constexpr (HV) reg_sort_pairs<KPT>(k, x);
        else reg_sort_keys<KPT>(k);

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
                    return ki_less(sk[spad<K>(b0 + ib)], sx[spad<uint32_t>(b0 + ib)],
                                   sk[spad<K>(a0 + ia)], sx[spad<uint32_t>(a0 + ia)]);
                });
                cand_merge_pairs<K, KPT>(sk, sx, a0, m, b0, m, i, diag - i, k, x);
            } else {
                const int i = merge_path_pred<int>(m, m, diag, [&](int ia, int ib) {
                    return sk[spad<K>(b0 + ib)] < sk[spad<K>(a0 + ia)];
                });
                cand_merge_keys<K, KPT>(sk, a0, m, b0, m, i, diag - i, k);
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
        if (tid == 0) atomicAdd(g.counters + CLS_TILE_SORT, 2ull * (sizeof(K) + (HV ? sizeof(V) : 0)) * cnt);
        __syncthreads();
    }
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

// ---------------------------------------------------------------- in-segment merge level

// Level L of the in-block merge schedule: inside segment [s, e) the runs are
// [s + q*W, s + (q+1)*W) with W = T << L; runs 2c and 2c+1 merge into one.
// A segment is active at level L while L < its level count.  The pair holding
// tile t of the segment and the buffer parities follow from (s, e, L).
struct SegPair {
    int64_t ps, pm, pe;  // A = [ps, pm), B = [pm, pe)
    int64_t x0, x1;      // this tile's output range
    int src, dst;        // buffer parities
    bool fin, active;
};

__device__ __forceinline__ SegPair seg_pair(const Geo &g, int64_t t, int level) {
    SegPair p;
    const int64_t s = g.tseg[t];
    int64_t slo, shi;
    seg_bounds(g, s, slo, shi);
    const int Ls = seg_levels(shi - slo, g.logT);
    p.active = level < Ls;
    const int64_t j = t - g.tprefix[s];
    p.x0 = slo + (j << g.logT);
    p.x1 = min(p.x0 + (int64_t(1) << g.logT), shi);
    const int64_t W = int64_t(1) << (g.logT + level);
    const int64_t cell = (j << g.logT) / (2 * W);
    p.ps = slo + cell * 2 * W;
    p.pm = min(p.ps + W, shi);
    p.pe = min(p.ps + 2 * W, shi);
    p.src = (Ls - level + g.R) & 1;
    p.dst = (Ls - level - 1 + g.R) & 1;
    p.fin = (level == Ls - 1) && g.R == 0;
    return p;
}

// Merge-path split (absolute A index) at the start of every active tile.
template <class K>
__global__ void seg_partition_kernel(Geo g, int level, const K *buf0, const K *buf1,
                                     int64_t *split, const int64_t *__restrict__ ntiles_total) {
    const int64_t total = min(*ntiles_total, g.ntiles_ub);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        SegPair p = seg_pair(g, t, level);
        if (!p.active) continue;
        const K *src = p.src ? buf1 : buf0;
        const int64_t na = p.pm - p.ps, nb = p.pe - p.pm;
        auto A = [&](int64_t i) { return src[p.ps + i]; };
        auto B = [&](int64_t i) { return src[p.pm + i]; };
        split[t] = p.ps + merge_path<K, int64_t>(A, na, B, nb, p.x0 - p.ps);
    }
}

template <class K, class V, int THREADS, int VT>
__global__ void __launch_bounds__(THREADS)
seg_merge_kernel(Geo g, int level, K *buf_k0, K *buf_k1, V *buf_v0, V *buf_v1, int codec,
                 const int64_t *__restrict__ split, const int64_t *__restrict__ ntiles_total) {
    constexpr int TT = THREADS * VT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sk = reinterpret_cast<K *>(smem_raw);
    V *sv = reinterpret_cast<V *>(smem_raw + smem_val_offset<K>(TT));
    const int64_t total = min(*ntiles_total, g.ntiles_ub);
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        SegPair p = seg_pair(g, t, level);
        if (!p.active) continue;
        const int64_t a_lo = split[t];
        const int64_t a_hi = (p.x1 == p.pe) ? p.pm : split[t + 1];
        const int64_t b_lo = p.pm + (p.x0 - p.ps) - (a_lo - p.ps);
        const int64_t b_hi = p.pm + (p.x1 - p.ps) - (a_hi - p.ps);
        cta_merge<K, V, THREADS, VT>(p.src ? buf_k1 : buf_k0, p.src ? buf_v1 : buf_v0, a_lo,
                                     (int)(a_hi - a_lo), b_lo, (int)(b_hi - b_lo),
                                     p.dst ? buf_k1 : buf_k0, p.dst ? buf_v1 : buf_v0, p.x0, p.fin,
                                     codec, sk, sv);
        if (threadIdx.x == 0)
            atomicAdd(g.counters + CLS_MERGE,
                      2ull * (sizeof(K) + (HasVal<V>::value ? sizeof(V) : 0)) * (p.x1 - p.x0));
    }
}

// ---------------------------------------------------------------- cross-block rounds

// Round r of the merge phase: groups of 2^r consecutive blocks are sorted
// runs; pair k merges groups 2k and 2k+1 (the last group may be unpaired and
// is copied).  Output tiles of T keys lie on a global grid, so one tile may
// span several pairs.
struct XPair {
    int64_t ps, pm, pe;
};
__device__ __forceinline__ XPair x_pair(const Geo &g, int r, int64_t k) {
    const int64_t G = int64_t(2) << r, H = int64_t(1) << r;
    XPair p;
    p.ps = clamp64(g.off[min(k * G, g.S)], 0, g.n);
    p.pm = clamp64(g.off[min(k * G + H, g.S)], p.ps, g.n);
    p.pe = clamp64(g.off[min(k * G + G, g.S)], p.pm, g.n);
    return p;
}

struct XSplit {
    int64_t k;  // pair holding the boundary (npairs for the end boundary)
    int64_t a;  // absolute A index of the merge-path split
};

template <class K>
__global__ void x_partition_kernel(Geo g, int r, const K *buf0, const K *buf1, XSplit *xs,
                                   int64_t nbound) {
    const K *src = ((g.R - r) & 1) ? buf1 : buf0;
    const int64_t npairs = (g.S + (int64_t(2) << r) - 1) >> (r + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nbound;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = min(t << g.logT, g.n);
        XSplit out;
        if (d >= g.n) {
            out.k = npairs;
            out.a = g.n;
        } else {
            const int64_t blk = seg_of(g, d);
            out.k = blk >> (r + 1);
            XPair p = x_pair(g, r, out.k);
            auto A = [&](int64_t i) { return src[p.ps + i]; };
            auto B = [&](int64_t i) { return src[p.pm + i]; };
            out.a = p.ps + merge_path<K, int64_t>(A, p.pm - p.ps, B, p.pe - p.pm, d - p.ps);
        }
        xs[t] = out;
    }
}

template <class K, class V, int THREADS, int VT>
__global__ void __launch_bounds__(THREADS)
xblock_merge_kernel(Geo g, int r, K *buf_k0, K *buf_k1, V *buf_v0, V *buf_v1, int codec,
                    const XSplit *__restrict__ xs, int64_t ntiles) {
    constexpr int TT = THREADS * VT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *sk = reinterpret_cast<K *>(smem_raw);
    V *sv = reinterpret_cast<V *>(smem_raw + smem_val_offset<K>(TT));
    const int src = (g.R - r) & 1, dst = (g.R - r - 1) & 1;
    const bool fin = (r == g.R - 1);
    const int64_t npairs = (g.S + (int64_t(2) << r) - 1) >> (r + 1);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t d0 = t << g.logT, d1 = min(d0 + (int64_t(1) << g.logT), g.n);
        const XSplit s0 = xs[t], s1 = xs[t + 1];
        const int64_t klast = min(s1.k, npairs - 1);
        for (int64_t kk = s0.k; kk <= klast; ++kk) {
            XPair p = x_pair(g, r, kk);
            const int64_t x_lo = max(p.ps, d0), x_hi = min(p.pe, d1);
            if (x_hi <= x_lo) continue;
            const int64_t a_lo = (kk == s0.k) ? s0.a : p.ps;
            const int64_t a_hi = (kk == s1.k) ? s1.a : p.pm;
            const int64_t b_lo = p.pm + (x_lo - p.ps) - (a_lo - p.ps);
            const int64_t b_hi = p.pm + (x_hi - p.ps) - (a_hi - p.ps);
            cta_merge<K, V, THREADS, VT>(src ? buf_k1 : buf_k0, src ? buf_v1 : buf_v0, a_lo,
                                         (int)(a_hi - a_lo), b_lo, (int)(b_hi - b_lo),
                                         dst ? buf_k1 : buf_k0, dst ? buf_v1 : buf_v0, x_lo, fin,
                                         codec, sk, sv);
        }
        if (threadIdx.x == 0)
            atomicAdd(g.counters + CLS_MERGE,
                      2ull * (sizeof(K) + (HasVal<V>::value ? sizeof(V) : 0)) * (d1 - d0));
    }
}

}  // namespace bs
