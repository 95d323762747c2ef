// Default launch of the isotropic sweep for a grid: the sweep's own default
// (iso_default_launch), except that a radius-4 grid too small to fill the GPU's
// CTA slots with 32 x 32 CTAs even at the shortest z chunks (32 planes) runs the
// one-row 64 x 16 form.  Such a grid leaves SMs idle whichever form runs, and the
// one-row form's 288 threads per 1024 columns then finish a CTA sooner than the
// two-row form's 160.  Host code only.
#pragma once

#include "fd_internal.h"
#include "launch_shape.h"

namespace fdk {

inline Launch iso_grid_launch(int R, int nx, int ny, int nz)
{
    Launch L = iso_default_launch(R, nx, ny, nz);
    if (R == 4 && L.tx == 32 && L.ty == 32) {
        const long slots = (long)device_sm_count() * 3;   // three 32 x 32, lookahead-3 CTAs per SM
        const long most = (long)((nx + 31) / 32) * ((ny + 31) / 32) * ((nz + 31) / 32);
        if (most < slots) {
            L.tx = 64;
            L.ty = 16;
            L.lookahead = 3;
            // two CTAs of 64 x 16 (288 threads) per SM
            L.zchunk = wave_zchunk(L, nx, ny, nz, (long)device_sm_count() * 2, 2 * R);
        }
    }
    return L;
}

}  // namespace fdk
