// bs_noalloc.cu -- bs_sort_keys_noalloc: a key sort that allocates nothing.
//
// Who needs this.  Some code that wants to sort cannot call cudaMalloc at
// that moment: a real-time or latency-critical path where cudaMalloc/cudaFree
// would stall (they can synchronise the whole device), a plug-in or callback
// running inside another framework that owns every byte of device memory
// through its own pool and forbids stray allocations, or code running under
// a fixed memory budget decided once at start-up.  bs_sort_keys needs a
// handle, whose scratch grows with cudaMalloc; this entry point runs the same
// passes with every scratch byte taken from one fixed array compiled into the
// library's device image instead.
//
// The array.  `bs_noalloc_scratch` below is a file-scope static __device__
// array of BS_NOALLOC_SCRATCH_BYTES.  Every GPU that loads this library holds
// it until the process exits, whether or not this entry point is called.  In
// host code the name of the array is only a host-side stand-in, not a device
// address, so the host looks the real address up once per device with
// cudaGetSymbolAddress (with that device current) and passes it to the
// kernels.  That look-up happens inside the first call made on each device,
// so make the first call on a device before any stream capture.
//
// Sharing.  All calls in the process share the one array and it keeps the
// contents of the previous call.  Nothing in it has to start at zero: every
// call writes each index array before reading it, and the kernels are given
// no statistics counters (they count bytes only when handed a counter array).
// Two calls whose GPU work overlaps in time (different streams, or different
// host threads, on the same device) race on the array and corrupt each
// other's results: serialise them, e.g. by issuing them on one stream.
//
// The cached address is only valid for the CUDA context it was looked up in:
// after cudaDeviceReset the library's device image may load elsewhere, so do
// not use this entry point across a cudaDeviceReset.
//
// Errors the GPU could find.  The merge kernels bound every wait (2 s by
// default); a wait that runs out ends them early.  This entry point returns
// before the GPU work runs and keeps no state a caller can query, so such a
// timeout -- only possible on a GPU stalled for seconds -- leaves an
// incomplete output with no error reported.  Callers that need it reported
// use bs_sort_keys with a handle and bs_sync_status.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "bs_internal.h"

// Set-up kernels of the regular path (defined in bs_api.cu).
__global__ void balanced_offsets_kernel(int64_t *off, int64_t n, int64_t p);
__global__ void tile_scan_block_kernel(const int64_t *off, int64_t S, int64_t n, int logT,
                                       int64_t *tprefix, int64_t *bsum);
__global__ void tile_map_kernel(const int64_t *tprefix, int64_t S, int32_t *tseg, int64_t ub);

namespace {

constexpr size_t AUX_BYTES = 64 * 1024;  // index arrays (59 KiB at p = 1024, n = 2^20)
constexpr size_t SCRATCH_BYTES = (size_t)BS_NOALLOC_MAX_KEY_BYTES + AUX_BYTES;
constexpr int LOGT = 12;                 // tile of 4096 keys
constexpr int SCAN_THREADS = 256;        // block size of tile_scan_block_kernel
constexpr int MAX_DEVICES = 64;

}  // namespace

static __device__ __align__(256) unsigned char bs_noalloc_scratch[SCRATCH_BYTES];

namespace {

std::mutex g_mu;
void *g_scratch[MAX_DEVICES] = {};
int g_sms[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once.
bs_status scratch_of_current_device(unsigned char **ptr, int *sms) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, bs_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return BS_ERR_CUDA;
        }
        int s = 1;
        if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            s = 1;
        }
        g_scratch[dev] = p;
        g_sms[dev] = s;
    }
    *ptr = (unsigned char *)g_scratch[dev];
    *sms = g_sms[dev];
    return BS_OK;
}

void no_begin(void *, int, cudaStream_t) {}
bool check_end(void *, int, cudaStream_t) { return cudaGetLastError() == cudaSuccess; }

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

int key_bytes(bs_dtype t) {
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

int codec_of(bs_dtype t) {
    if (t == BS_INT32 || t == BS_INT64) return bs::CODEC_SIGNED;
    if (t == BS_FLOAT32 || t == BS_FLOAT64) return bs::CODEC_FLOAT;
    return bs::CODEC_IDENT;
}

int ceil_log2(int64_t x) {
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
}

}  // namespace

extern "C" bs_status bs_sort_keys_noalloc(const void *d_in, void *d_out, int64_t n, bs_dtype kt,
                                          int64_t p, void *stream) {
    if (n < 0 || p < 0) return BS_ERR_INVALID_ARG;
    const int kw = key_bytes(kt);
    if (!kw) return BS_ERR_UNSUPPORTED_DTYPE;
    if (n == 0) return BS_OK;
    if (!d_in || !d_out) return BS_ERR_INVALID_ARG;
    if (p == 0) p = 1;
    if (p > n) p = n;
    if ((uint64_t)n * (uint64_t)kw > (uint64_t)BS_NOALLOC_MAX_KEY_BYTES || p > BS_NOALLOC_MAX_BLOCKS)
        return BS_ERR_TOO_LARGE;

    unsigned char *base = nullptr;
    int sms = 1;
    bs_status st = scratch_of_current_device(&base, &sms);
    if (st != BS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // carve the array: scratch keys, then the small index arrays
    const int64_t T = int64_t(1) << LOGT;
    const int64_t gtiles = (n + T - 1) / T;
    const int64_t ub = gtiles + p;
    size_t at = BS_NOALLOC_MAX_KEY_BYTES;
    auto take = [&](size_t bytes) {
        unsigned char *q = base + at;
        at += up256(bytes);
        return q;
    };
    int64_t *off = (int64_t *)take(sizeof(int64_t) * (p + 1));
    int64_t *tprefix = (int64_t *)take(sizeof(int64_t) * (p + 1));
    int64_t *bsum = (int64_t *)take(sizeof(int64_t) * 2);
    int32_t *tseg = (int32_t *)take(sizeof(int32_t) * ub);
    // one merge-path split per merge tile (+1): merge tiles may be as small as
    // 2^11 keys (the pass planner shrinks them when a shape's stages do not fit),
    // so size for that -- the cross-block rounds' tiles, and the in-block levels'
    // (n / 2^11 + 4 (p + 1)) -- as the handle's workspace does
    int64_t xt = bs::xblock_tiles_max(n, p, 11);
    const int64_t seg_merge_tiles = (n + 2047) / 2048 + 4 * (p + 1);
    if (seg_merge_tiles > xt) xt = seg_merge_tiles;
    int64_t *split = (int64_t *)take(sizeof(int64_t) * ((ub > xt ? ub : xt) + 1));
    if (at > SCRATCH_BYTES) return BS_ERR_TOO_LARGE;  // cannot happen within the limits above

    bs::Geo g{};
    g.off = off;
    g.S = p;
    g.n = n;
    g.tprefix = tprefix;
    g.tseg = tseg;
    g.ntiles_ub = ub;
    g.logT = LOGT;
    g.R = ceil_log2(p);
    g.counters = nullptr;  // no byte counting
    g.err = nullptr;       // no status word: see "Errors the GPU could find" above

    // scatter bounds, tiles per block (p <= 1024 fits one scan block), tile map
    const unsigned pb = (unsigned)((p + 1 + 255) / 256);
    bs::launch_overlapped(balanced_offsets_kernel, pb, 256, 0, s, off, n, p);
    if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;
    bs::launch_overlapped(tile_scan_block_kernel, 1, SCAN_THREADS, 0, s, off, p, n, LOGT, tprefix, bsum);
    if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;
    unsigned mb = (unsigned)((ub + 255) / 256);
    if (mb > (unsigned)sms * 8) mb = (unsigned)sms * 8;
    bs::launch_overlapped(tile_map_kernel, mb, 256, 0, s, tprefix, p, tseg, ub);
    if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;

    bs::PassArgs a{};
    a.g = g;
    a.in_k = d_in;
    a.in_v = nullptr;
    a.k0 = d_out;
    a.k1 = base;  // scratch keys at the start of the array
    a.v0 = nullptr;
    a.v1 = nullptr;
    a.codec = codec_of(kt);
    a.vbytes = 0;
    const int64_t largest_block = (n + p - 1) / p;
    a.Lmax = largest_block <= T ? 0 : ceil_log2((largest_block + T - 1) / T);
    a.ntiles_ub = ub;
    a.ntiles_total = tprefix + p;
    a.split = split;
    a.merge_impl = (((uintptr_t)d_out | (uintptr_t)base) & 15) ? bs::MERGE_SIMPLE : bs::MERGE_AUTO;
    a.merge_vt = 0;  // the default shape
    a.merge_only = false;
    a.tpp_host = nullptr;
    a.oddeven_rounds = 0;
    a.local_sort = 0;
    a.merge_tile_log2 = 0;
    a.merge_consumer = 0;
    bs::Launcher L{s, nullptr, sms, no_begin, check_end};
    return kw == 4 ? bs::run_passes_u32(a, L) : bs::run_passes_u64(a, L);
}
