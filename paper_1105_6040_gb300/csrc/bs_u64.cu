// Sort passes for 8-byte key codes (int64, uint64, float64 keys).
#include "bs_passes.cuh"

namespace bs {
bs_status run_passes_u64(const PassArgs &a, Launcher &L) { return run_passes_k<uint64_t>(a, L); }
bs_status oddeven_scatter_u64(const void *in, void *out, int64_t n, int64_t p, int64_t cap, int codec,
                           Launcher &L) {
    return oddeven_scatter_t<uint64_t>(in, out, n, p, cap, codec, L);
}
bs_status oddeven_compact_u64(const void *in, void *out, int64_t n, int codec, Launcher &L) {
    return oddeven_compact_t<uint64_t>(in, out, n, codec, L);
}
}  // namespace bs
