// Sort passes for 4-byte key codes (int32, uint32, float32 keys).
#include "bs_passes.cuh"

namespace bs {
bs_status run_passes_u32(const PassArgs &a, Launcher &L) { return run_passes_k<uint32_t>(a, L); }
}  // namespace bs
