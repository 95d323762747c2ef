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
// output (u^n, the stored older level that becomes u^{n+1}, kappa).
//
// Limits and behaviour:
//   * nx, ny, nz <= FD_STATIC_MAX_AXIS (8192); larger grids are rejected with
//     FD_ERR_OUT_OF_RANGE before anything is enqueued.
//   * g_scratch (about 97 KiB) exists on every GPU that loads the library and
//     stays allocated until the process exits.
//   * Every call shares g_scratch and overwrites it (status block cleared, tables
//     rewritten) on the caller's stream before its kernel.  Calls whose work can
//     overlap on the GPU -- on different streams without ordering between them,
//     or on different host threads -- race on it; order them on one stream.
//   * The first call on a device looks up g_scratch's device address with
//     cudaGetSymbolAddress (host code cannot use the symbol itself: on the host
//     it names a stand-in, not device memory).  Make that first call before any
//     stream capture on that device.
//   * Device-side wait timeouts set a flag inside g_scratch that this entry
//     point does not report; the grid API's fd_sync() reports them for grids.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include <cudaTypedefs.h>

#include "coeffs.h"
#include "fd.h"
#include "fd_internal.h"

namespace fdk {
int set_last_error(int code, const char *msg);
}

namespace {

using namespace fdk;

constexpr int kMaxAxis = FD_STATIC_MAX_AXIS;
constexpr size_t kOffState = 0;                                   // DevState (64 B)
constexpr size_t kOffGx = 256;                                    // kMaxAxis floats
constexpr size_t kOffGy = kOffGx + sizeof(float) * kMaxAxis;
constexpr size_t kOffGz = kOffGy + sizeof(float) * kMaxAxis;
constexpr size_t kOffSrc = kOffGz + sizeof(float) * kMaxAxis;     // one source sample
constexpr size_t kScratchBytes = kOffSrc + 256;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_dev[kMaxDevices] = {};   // device address of g_scratch, per device

// Host staging of one call's tables (no heap allocation on the call path).
struct HostTables {
    DevState st;
    float gx[kMaxAxis], gy[kMaxAxis], gz[kMaxAxis];
    float src;
};
thread_local HostTables t_tables;

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
                                  double amp, void *stream)
{
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
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return cuda_err(e, "cudaGetSymbolAddress(g_scratch)");
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    unsigned char *scr = g_scratch_dev[dev];
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // tables of this call (weights as in fd_create_grid, Eq. 4 on every axis)
    const int R = d->r_xy;
    double c[kMaxR + 1];
    central_d2(R, c);
    HostTables &T = t_tables;
    memset(&T.st, 0, sizeof T.st);                 // time index 0, CTA counter 0, no error
    for (int i = 0; i < lay.pitch; ++i) T.gx[i] = i < d->nx ? (float)cerjan(i, d->nx, d->sponge_width, d->sponge_a) : 1.f;
    for (int j = 0; j < d->ny; ++j) T.gy[j] = (float)cerjan(j, d->ny, d->sponge_width, d->sponge_a);
    for (int k = 0; k < d->nz; ++k) T.gz[k] = (float)cerjan(k, d->nz, d->sponge_width, d->sponge_a);
    const double scale = d->dt * d->dt / (d->h * d->h * d->dz);     // dt^2 / V, as the grid API
    T.src = has_src ? (float)(amp * ricker(n * d->dt - t0, freq_hz) * scale) : 0.f;

    struct Piece { size_t off; const void *src; size_t bytes; } pieces[] = {
        {kOffState, &T.st, sizeof(DevState)},
        {kOffGx, T.gx, sizeof(float) * lay.pitch},
        {kOffGy, T.gy, sizeof(float) * d->ny},
        {kOffGz, T.gz, sizeof(float) * d->nz},
        {kOffSrc, &T.src, sizeof(float)},
    };
    for (const Piece &pc : pieces) {
        e = cudaMemcpyAsync(scr + pc.off, pc.src, pc.bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_err(e, "scratch upload");
    }

    const Launch L = iso_default_launch(R, d->nx, d->ny, d->nz);
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
    e = launch_iso(R, L, tm, a, s);
    if (e != cudaSuccess) return cuda_err(e, "sweep launch");
    return FD_OK;
}
