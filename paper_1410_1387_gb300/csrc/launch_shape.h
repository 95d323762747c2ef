// Default launch shape of the isotropic sweep: the z chunk fitted to whole
// waves of resident CTAs.  Host code only.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "fd_internal.h"

namespace fdk {

// Streaming multiprocessors of the current device (cached per device, atomically:
// host threads may ask at once; 152, a GB300's count, if the query fails).
inline int device_sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

// z chunk that fits the launch to the GPU: with `slots` CTAs resident at a time
// and each CTA's time taken as (its planes + P), P the planes it loads before its
// first output (2R), the step takes about waves x (zchunk + P).  Among the even
// splits of nz into chunks of 32 to `hi` planes, the cheapest (ties: the longer
// chunk).  At 512^3 on 304 slots this picks 7 chunks of 74 planes (5.9 waves)
// over 8 of 64 (6.7 waves, the last one three-quarters full).  Longer chunks
// measured slower than the model says (fewer CTAs to overlap each one's start),
// hence the cap: 96 planes for the isotropic sweep, 64 for the VTI sweep, whose
// 512^3 step measured fastest at 64 planes and slowest at 74 of 43-74.
inline int wave_zchunk(const Launch &L, int nx, int ny, int nz, long slots, int P, int hi = 96)
{
    const long tiles = (long)((nx + L.tx - 1) / L.tx) * ((ny + L.ty - 1) / L.ty);
    const int lo = nz < 32 ? nz : 32;
    if (hi < lo) hi = lo;
    if (slots < 1) slots = 1;
    int best = lo;
    long best_cost = -1;
    for (long c = (nz + hi - 1) / hi; c <= nz; ++c) {
        const int zc = (int)((nz + c - 1) / c);
        if (zc < lo) break;
        const long chunks = (nz + zc - 1) / zc;
        const long waves = (tiles * chunks + slots - 1) / slots;
        const long cost = waves * (zc + P);
        if (best_cost < 0 || cost < best_cost) {   // c grows, zc shrinks: ties keep the longer chunk
            best = zc;
            best_cost = cost;
        }
    }
    return best > kMaxChunk ? kMaxChunk : best;
}

}  // namespace fdk
