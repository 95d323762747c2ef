// Internal declarations shared by the host side (fd_api.cpp) and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdk {

constexpr int kMaxR = 12;          // largest stencil radius compiled in

// Device-resident status block (64 bytes, library-allocated).
struct DevState {
    int step;               // time index n of the level u^n the next launch reads
    unsigned int done;      // CTAs of the current launch that have read `step`
    int err;                // bit flags, see kErr*
    int err_info;           // 1 + linear CTA index of the first error
    float vmax;             // model statistics written by the model kernels
    float kxmax;
    unsigned int bad;       // count of invalid model values
    unsigned int eps_lt_delta;
    int pad[8];
};
static_assert(sizeof(DevState) == 64, "status block size");
constexpr int kErrTmaTimeout = 1;

// Fused receiver lattice: a row-major rnx x rny lattice on plane rk.
struct RecLattice {
    float *trace;           // device, rows of nrec floats
    long long nrec;         // rnx * rny
    int on;                 // 1 when sampled inside the stencil kernel
    int rk, rx0, ry0, rsx, rsy, rnx, rny;
    int t0;                 // time index at which row 0 was defined
    int cap;                // rows available
};

struct Source {
    const float *tab;       // tab[n] = dt^2 * s(n) / V (float), n < len
    int len;
    int sx, sy, sz;         // cell; sx < 0 = no source
    int into_q;             // VTI: add to q as well
};

// Arguments of the isotropic sweep (Eq. 3 with the Laplacian of Eq. 4 on all axes).
struct alignas(16) IsoArgs {
    float *prev;            // stored older level in, u^{n+1} out (in place)
    const float *cur;       // u^n (plain loads for the first planes of a z chunk)
    const float *kappa;     // (v dt)^2
    const float *gx, *gy, *gz;  // damping factors per axis (1 outside the layer)
    long long pitch;        // floats per row
    long long plane;        // floats per plane
    int nx, ny, nz;
    int zchunk;             // planes per CTA
    float w0;               // centre weight c0 (2/h^2 + 1/dz^2)
    float wxy[kMaxR + 1];   // c_l / h^2
    float wz[kMaxR + 1];    // c_l / dz^2
    float2 wxy2[kMaxR + 1]; // (c_l / h^2, c_l / h^2): operands of packed f32x2 FMAs
    float2 wz2[kMaxR + 1];
    Source src;
    RecLattice rec;
    RecLattice inj;         // additive sources on a lattice: row n - t0 of inj.trace at step n
    DevState *st;
    unsigned int ncta;
    float c2dt;             // 2 dt: the gradient sweep's factor
    int skip_plane1;        // test hook: 1 + a plane whose u^n copy CTA (0,0,0) withholds (0 = none)
    // Part of a step (all zero: the whole step): planes [zb, nz - ztop) are
    // updated; hold = 1 leaves the time index for a later part to advance.
    int zb, ztop, hold;
};

// Arguments of the VTI sweep (Eqs. 1-2, 4-5).
struct VtiArgs {
    float *pprev, *qprev;   // stored older levels in, new levels out (in place)
    const float *p, *q;     // p^n, q^n
    const float *kx, *kn, *kz;
    const float *gx, *gy, *gz;
    const float *ztab;      // nz rows of vti_zrow(R_z) floats: paired z weights, then G_z(k)
    long long pitch, plane;
    int nx, ny, nz;
    int zchunk;
    float w0;               // 2 c0 / h^2
    float wxy[kMaxR + 1];   // c_l / h^2
    float2 wxy2[kMaxR + 1]; // (c_l / h^2, c_l / h^2) for packed f32x2 FMAs
    Source src;
    RecLattice rec;
    DevState *st;
    unsigned int ncta;
    int zb, ztop, hold;     // part of a step, as in IsoArgs (all zero: the whole step)
    int skip_plane1;        // test hook: 1 + a plane whose p^n copy CTA (0,0,0) withholds (0 = none)
};

// fd_debug_skip_copy(NULL, plane) arms the hook for the next fd_iso_step_static()
// call on the calling host thread (-1 = none).
extern thread_local int t_static_skip;

// Launch configuration of one sweep.
struct Launch {
    int tx, ty;             // tile (x multiple of 4)
    int zchunk;             // planes per CTA
    int lookahead;          // TMA planes in flight ahead of use
};

// Largest z chunk of one CTA (its damping factors are staged in shared memory).
constexpr int kMaxChunk = 1024;

// Planes per CTA: enough CTAs (about `target`, 2048 by default) for several
// waves over 152 SMs, at least 32 planes per chunk (measured: shorter chunks lose
// more to priming the z queue and filling the pipeline than they gain in
// waves), at most kMaxChunk.
inline int default_zchunk(const Launch &L, int nx, int ny, int nz, long target = 2048)
{
    const long tiles = (long)((nx + L.tx - 1) / L.tx) * ((ny + L.ty - 1) / L.ty);
    long chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int zc = (int)((nz + chunks - 1) / chunks);
    const int lo = nz < 32 ? nz : 32;
    zc = zc < lo ? lo : zc;
    return zc > kMaxChunk ? kMaxChunk : zc;
}

// Tensor maps of one isotropic launch: u^n with the R halo, u^{n-1} and kappa tiles.
struct IsoMaps {
    CUtensorMap cur, prev, kappa;
    CUtensorMap cur_tile;   // u^n with the tile box (radius 8 streams its z-queue entries through it)
};

// 3D tensor map over a pitched nx x ny x nz float field, box (bx, by, 1).
// Returns 0 or a CUresult / cudaError_t code.
int encode_field_map(CUtensorMap *m, const float *base, int nx, int ny, int nz, long long pitch, int bx,
                     int by);

// Kernel launchers (iso_sweep.cu, vti_sweep.cu, aux_kernels.cu).  Return a cudaError_t.
cudaError_t launch_iso(int R, const Launch &L, const IsoMaps &tm, const IsoArgs &a, cudaStream_t s);
// One member shot of a batched isotropic launch (device array, one per shot).
// The shot's time index n (its status block) picks the buffer holding u^n:
// buf[cur0 ^ ((n - n0) & 1)]; launches stop advancing it once n reaches n_end.
struct alignas(128) BatchShot {
    CUtensorMap halo[2];    // u buffers with the R halo (box tile + 2R)
    CUtensorMap tile[2];    // u buffers, box tile
    CUtensorMap kappa;      // box tile
    IsoArgs a;              // a.prev / a.cur unused
    float *buf[2];
    int n0, cur0, n_end;
    unsigned ncta;          // CTAs of this shot per launch
};
cudaError_t launch_iso_batch(int R, const Launch &L, const int4 *items, int nitems, const BatchShot *shots,
                             int max_zchunk, cudaStream_t s);

// Floats per plane row of the VTI z table: the 2 R_z + 1 weights each twice,
// then the plane's damping factor, padded to 16 bytes.
constexpr int vti_zrow(int rz) { return (2 * (2 * rz + 1) + 1 + 3) / 4 * 4; }

// Tensor maps of one VTI launch: p^n with the R_xy halo, tiles of q^n, p_prev,
// q_prev and the three kappa arrays.
struct VtiMaps {
    CUtensorMap p, q, pp, qp, kx, kn, kz;
};
cudaError_t launch_vti(int rxy, int rz, const Launch &L, const VtiMaps &tm, const VtiArgs &a, cudaStream_t s);
Launch iso_default_launch(int R, int nx, int ny, int nz);
Launch vti_default_launch(int rxy, int rz, int nx, int ny, int nz);
bool iso_supported(int R);
bool iso_config_built(int R, const Launch &L);
bool vti_config_built(int rxy, int rz, const Launch &L);
bool vti_supported(int rxy, int rz);

cudaError_t launch_model_iso(const float *v, long long src_pitch, float *kappa, int nx, int ny,
                             int nz, long long pitch, double dt, DevState *st, cudaStream_t s);
cudaError_t launch_model_vti(const float *vz, const float *eps, const float *delta,
                             long long src_pitch, float *kx, float *kn, float *kz, int nx, int ny,
                             int nz, long long pitch, double dt, DevState *st, cudaStream_t s);
cudaError_t launch_gather(const float *field, long long pitch, long long plane, const int *idx,
                          int nrec, float *trace, int t0, int cap, const DevState *st,
                          cudaStream_t s);
// Gradient sweep: a.prev = grad (in/out), a.cur = the forward level, a.c2dt = 2 dt;
// tm.cur = that level with the R halo, tm.prev = z, tm.kappa = kappa, tm_grad =
// grad (tile boxes of L).  grad += 2 dt z (L a) / sqrt(kappa).
Launch iso_grad_launch(int R, int nx, int ny, int nz);
cudaError_t launch_iso_grad(int R, const Launch &L, const IsoMaps &tm, const CUtensorMap &tm_grad, const IsoArgs &a,
                            cudaStream_t s);
// inj[m][r] = kappa(x_r) (tr - dobs)[nt-1-m][r] on the lattice `rec`; misfit += 1/2 sum (tr - dobs)^2.
cudaError_t launch_adjoint_source(const RecLattice &rec, const float *kappa, long long pitch, long long plane,
                                  const float *tr, const float *dobs, int nt, float *inj, double *misfit,
                                  cudaStream_t s);

}  // namespace fdk
