// fd_iso_step_static(): one isotropic step that allocates no device memory.
//
// Who needs it: some callers cannot call cudaMalloc.  A serving process may
// hand all of the GPU's memory to its own pool allocator and forbid any other
// allocation; a latency-critical loop may not afford the implicit device-wide
// synchronisation that cudaMalloc and cudaFree can cause.  The grid API
// (fd_create_grid) allocates small tables and a status block, so it is closed
// to them.  This entry point runs the same isotropic sweep kernel with every
// piece of scratch it needs -- the 64-byte status block, the three damping
// profiles and the source sample -- placed in one file-scope __device__ array
// of fixed size, g_scratch below.  The caller passes only the inputs and the
// output (u^n, the stored older level that becomes u^{n+1}, kappa) and, if it
// wants the outcome, one device int for the status.
//
// Limits and behaviour:
//   * nx, ny, nz <= FD_STATIC_MAX_AXIS (8192) and a damping layer of at most
//     FD_STATIC_MAX_SPONGE (512) cells; larger descriptions are rejected with
//     FD_ERR_OUT_OF_RANGE before anything is enqueued.
//   * g_scratch (about 97 KiB) exists on every GPU that loads the library and
//     stays allocated until the process exits.
//   * Every call rewrites g_scratch on the caller's stream before its sweep: a
//     small kernel clears the status block and fills the damping tables and the
//     source sample from values passed as kernel arguments, so a call makes the
//     host wait for nothing.  Calls whose work can overlap on the GPU -- on
//     different streams without ordering between them, or on different host
//     threads -- race on the array; order them on one stream.
//   * The first call on a device looks up g_scratch's device address with
//     cudaGetSymbolAddress (host code cannot use the symbol itself: on the host
//     it names a stand-in, not device memory).  Make that first call before any
//     stream capture on that device.
//   * A device-side wait that runs out sets a flag in the status block; after
//     the sweep a one-thread kernel copies the outcome (FD_OK or FD_ERR_TIMEOUT)
//     into the caller's status word, when one is given.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "coeffs.h"
#include "fd.h"
#include "fd_internal.h"
#include "launch_policy.h"

namespace fdk {
int set_last_error(int code, const char *msg);

// fd_debug_skip_copy(NULL, plane): the next static call on this host thread
// has CTA (0,0,0) withhold that plane's copy (the failure-detection test hook).
thread_local int t_static_skip = -1;
}  // namespace fdk

namespace {

using namespace fdk;

constexpr int kMaxAxis = FD_STATIC_MAX_AXIS;
constexpr int kMaxSponge = FD_STATIC_MAX_SPONGE;
constexpr size_t kOffState = 0;                                   // DevState (64 B)
constexpr size_t kOffGx = 256;                                    // kMaxAxis floats
constexpr size_t kOffGy = kOffGx + sizeof(float) * kMaxAxis;
constexpr size_t kOffGz = kOffGy + sizeof(float) * kMaxAxis;
constexpr size_t kOffSrc = kOffGz + sizeof(float) * kMaxAxis;     // one source sample
constexpr size_t kScratchBytes = kOffSrc + 256;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Everything one call writes into g_scratch, passed by value as the fill
// kernel's argument (about 2 KiB): the Cerjan factor exp(-(a d)^2) for each
// depth d = 0..width into the layer (prof[0] = 1), the axis lengths and the
// source sample.
struct StaticFill {
    float prof[kMaxSponge + 1];
    int nx, ny, nz, pitch, width;
    float src;
};

// Depth into the damping layer of index i on an axis of n points: the same
// case analysis as the grid API's host-side profile (coeffs.cpp, cerjan()).
__device__ __forceinline__ int layer_depth(int i, int n, int width)
{
    if (width <= 0) return 0;
    if (i < width) return width - i;
    if (i >= n - width) return i - (n - width - 1);
    return 0;
}

__global__ void static_fill_kernel(const __grid_constant__ StaticFill f)
{
    float *gx = reinterpret_cast<float *>(g_scratch + kOffGx);
    float *gy = reinterpret_cast<float *>(g_scratch + kOffGy);
    float *gz = reinterpret_cast<float *>(g_scratch + kOffGz);
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < f.pitch; i += stride)
        gx[i] = i < f.nx ? f.prof[layer_depth(i, f.nx, f.width)] : 1.f;   // padded to the pitch
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < f.ny; j += stride)
        gy[j] = f.prof[layer_depth(j, f.ny, f.width)];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < f.nz; k += stride)
        gz[k] = f.prof[layer_depth(k, f.nz, f.width)];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // time index 0, CTA counter 0, no error
        int *st = reinterpret_cast<int *>(g_scratch + kOffState);
        for (int w = 0; w < (int)(sizeof(DevState) / sizeof(int)); ++w) st[w] = 0;
        *reinterpret_cast<float *>(g_scratch + kOffSrc) = f.src;
    }
}

// The outcome of the sweep that preceded it on the stream.
__global__ void static_status_kernel(int *status)
{
    const DevState *st = reinterpret_cast<const DevState *>(g_scratch + kOffState);
    *status = (st->err & kErrTmaTimeout) ? FD_ERR_TIMEOUT : FD_OK;
}

constexpr int kMaxDevices = 64;
// device address of g_scratch per device (looked up on a device's first call;
// atomic because host threads may make their first calls at the same time)
std::atomic<unsigned char *> g_scratch_dev[kMaxDevices];

int err(int code, const char *msg) { return set_last_error(code, msg); }

int cuda_err(cudaError_t e, const char *what)
{
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return set_last_error(FD_ERR_CUDA, buf);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int fd_iso_step_static(const fd_desc *d, const float *u_cur, float *u_prev, const float *kappa,
                                  int n, int src_ix, int src_iy, int src_iz, double freq_hz, double t0,
                                  double amp, int *status, void *stream)
{
    const int skip = t_static_skip;   // the hook covers the next call only, whatever its outcome
    t_static_skip = -1;
    fd_layout_t lay;
    int rc = fd_layout(d, &lay);   // validates the description
    if (rc) return rc;
    if (d->mode != FD_MODE_ISO) return err(FD_ERR_INVALID_ARG, "fd_iso_step_static takes an isotropic description");
    if (d->nx > kMaxAxis || d->ny > kMaxAxis || d->nz > kMaxAxis) {
        char buf[160];
        snprintf(buf, sizeof buf, "grid %d x %d x %d exceeds the static scratch limit of %d points per axis", d->nx,
                 d->ny, d->nz, kMaxAxis);
        return err(FD_ERR_OUT_OF_RANGE, buf);
    }
    if (d->sponge_width > kMaxSponge) {
        char buf[160];
        snprintf(buf, sizeof buf, "damping layer of %d cells exceeds the static limit of %d", d->sponge_width,
                 kMaxSponge);
        return err(FD_ERR_OUT_OF_RANGE, buf);
    }
    if (!u_cur || !u_prev || !kappa) return err(FD_ERR_INVALID_ARG, "NULL field pointer");
    if (!aligned16(u_cur) || !aligned16(u_prev) || !aligned16(kappa))
        return err(FD_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (n < 0) return err(FD_ERR_INVALID_ARG, "negative time index");
    const bool has_src = src_ix >= 0;
    if (has_src && (src_ix >= d->nx || src_iy < 0 || src_iy >= d->ny || src_iz < 0 || src_iz >= d->nz))
        return err(FD_ERR_INVALID_ARG, "source cell outside the grid");
    if (has_src && (!(freq_hz > 0.0) || !std::isfinite(freq_hz) || !std::isfinite(t0) || !std::isfinite(amp)))
        return err(FD_ERR_INVALID_ARG, "bad Ricker parameters");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return err(FD_ERR_UNSUPPORTED, "device ordinal above 63");
    unsigned char *scr = g_scratch_dev[dev].load(std::memory_order_acquire);
    if (!scr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return cuda_err(e, "cudaGetSymbolAddress(g_scratch)");
        scr = static_cast<unsigned char *>(p);
        g_scratch_dev[dev].store(scr, std::memory_order_release);   // every thread finds the same address
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // this call's tables, as the grid API builds them (Eq. 4 on every axis, the
    // Cerjan layer, the Ricker sample of step n scaled by dt^2 / V)
    const int R = d->r_xy;
    double c[kMaxR + 1];
    central_d2(R, c);
    StaticFill f;
    const int width = d->sponge_width > 0 ? d->sponge_width : 0;
    f.prof[0] = 1.f;
    for (int dd = 1; dd <= width; ++dd)   // cerjan() at depth dd of a layer of `width` cells
        f.prof[dd] = (float)cerjan(width - dd, 2 * width + 1, width, d->sponge_a);
    f.nx = d->nx;
    f.ny = d->ny;
    f.nz = d->nz;
    f.pitch = lay.pitch;
    f.width = width;
    const double scale = d->dt * d->dt / (d->h * d->h * d->dz);
    f.src = has_src ? (float)(amp * ricker(n * d->dt - t0, freq_hz) * scale) : 0.f;
    const int longest = std::max(lay.pitch, std::max(d->ny, d->nz));
    static_fill_kernel<<<(longest + 255) / 256, 256, 0, s>>>(f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "scratch fill launch");

    const Launch L = iso_grid_launch(R, d->nx, d->ny, d->nz);
    IsoMaps tm;
    int cr = encode_field_map(&tm.cur, u_cur, d->nx, d->ny, d->nz, lay.pitch, L.tx + 2 * R, L.ty + 2 * R);
    if (!cr) cr = encode_field_map(&tm.prev, u_prev, d->nx, d->ny, d->nz, lay.pitch, L.tx, L.ty);
    if (!cr) cr = encode_field_map(&tm.kappa, kappa, d->nx, d->ny, d->nz, lay.pitch, L.tx, L.ty);
    if (!cr) cr = encode_field_map(&tm.cur_tile, u_cur, d->nx, d->ny, d->nz, lay.pitch, L.tx, L.ty);
    if (cr) return err(FD_ERR_CUDA, "tensor map encoding failed");

    IsoArgs a{};
    a.prev = u_prev;
    a.cur = u_cur;
    a.kappa = kappa;
    a.gx = reinterpret_cast<const float *>(scr + kOffGx);
    a.gy = reinterpret_cast<const float *>(scr + kOffGy);
    a.gz = reinterpret_cast<const float *>(scr + kOffGz);
    a.pitch = lay.pitch;
    a.plane = (long long)lay.pitch * d->ny;
    a.nx = d->nx;
    a.ny = d->ny;
    a.nz = d->nz;
    a.zchunk = L.zchunk;
    const double h2 = d->h * d->h, dz2 = d->dz * d->dz;
    a.w0 = (float)(c[0] * (2.0 / h2 + 1.0 / dz2));
    for (int l = 1; l <= R; ++l) {
        a.wxy[l] = (float)(c[l] / h2);
        a.wz[l] = (float)(c[l] / dz2);
        a.wxy2[l] = make_float2(a.wxy[l], a.wxy[l]);
        a.wz2[l] = make_float2(a.wz[l], a.wz[l]);
    }
    // the kernel reads sample tab[time index]; the status block's index is 0
    a.src = Source{reinterpret_cast<const float *>(scr + kOffSrc), has_src ? 1 : 0, has_src ? src_ix : -1,
                   src_iy, src_iz, 0};
    a.rec = RecLattice{};
    a.st = reinterpret_cast<DevState *>(scr + kOffState);
    a.skip_plane1 = (skip >= 0 && skip < d->nz) ? skip + 1 : 0;
    e = launch_iso(R, L, tm, a, s);
    if (e != cudaSuccess) return cuda_err(e, "sweep launch");
    if (status) {
        static_status_kernel<<<1, 1, 0, s>>>(status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(e, "status launch");
    }
    return FD_OK;
}
