// bs_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "bs_device.cuh"
#include "bsort.h"

namespace bs {

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
    int64_t *split;           // per tile merge-path split (in-segment levels)
    XSplit *xs;               // per global boundary split (cross-block rounds)
};

bs_status run_passes_u32(const PassArgs &a, Launcher &L);
bs_status run_passes_u64(const PassArgs &a, Launcher &L);

}  // namespace bs
