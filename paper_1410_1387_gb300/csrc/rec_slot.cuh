// Receiver slot of one thread's 4 x points of one row: where the fused receiver
// lattice takes their values.  A full-rate lattice (stride 1 in x) with aligned
// rows takes each thread's 4 values as one 16-byte store; other lattices take one
// 4-byte store per receiver point.
#pragma once

#include <stdint.h>

#include "fd_internal.h"

namespace fdk {

// off: column of the first receiver point in a trace row; flags: bit e set when
// point e is a receiver, bit 4 when all four are, at consecutive columns that a
// 16-byte store reaches.  flags = 0: no receiver here (or receivers off).
struct RecSlot {
    int off;
    int flags;
};

__device__ __forceinline__ RecSlot rec_slot(const RecLattice &r, const int gxi, const int gyi, const int nx)
{
    RecSlot s{0, 0};
    if (!r.on) return s;
    const int ry = gyi - r.ry0;
    if (ry < 0 || ry % r.rsy != 0 || ry / r.rsy >= r.rny) return s;
    int first = -1, mask = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int rx = gxi + e - r.rx0;
        if (gxi + e < nx && rx >= 0 && rx % r.rsx == 0 && rx / r.rsx < r.rnx) {
            if (first < 0) first = rx / r.rsx;
            mask |= 1 << e;
        }
    }
    if (!mask) return s;
    s.off = (ry / r.rsy) * r.rnx + first;
    const bool vec = mask == 0xF && (s.off & 3) == 0 && (r.nrec & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(r.trace) & 15) == 0;
    s.flags = mask | (vec ? 16 : 0);
    return s;
}

// Writes the receiver values of plane k (the lattice's plane) at time index n:
// row n - t0 of the trace, the receiver points of o in x order.
__device__ __forceinline__ void rec_store(const RecLattice &r, const RecSlot &s, const int n, const float (&o)[4])
{
    const int row = n - r.t0;
    if (row < 0 || row >= r.cap) return;
    float *trow = r.trace + (long long)row * r.nrec + s.off;
    if (s.flags & 16) {
        *reinterpret_cast<float4 *>(trow) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if ((s.flags >> e) & 1) trow[__popc(s.flags & ((1 << e) - 1))] = o[e];
    }
}

}  // namespace fdk
