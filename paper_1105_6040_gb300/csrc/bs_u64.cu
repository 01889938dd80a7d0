// Sort passes for 8-byte key codes (int64, uint64, float64 keys).
#include "bs_passes.cuh"

namespace bs {
bs_status run_passes_u64(const PassArgs &a, Launcher &L) { return run_passes_k<uint64_t>(a, L); }
}  // namespace bs
