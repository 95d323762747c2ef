// C ABI of libfd.so (include/fd.h): validation, layout, tables, launches,
// graphs, state and receiver copies.  Every step of the time loop runs in the
// CUDA kernels of iso_sweep.cu / vti_sweep.cu; this file only orders them.
#include "fd.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "coeffs.h"
#include "fd_internal.h"
#include "launch_policy.h"

using namespace fdk;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();   // clear a non-sticky error
    return fail(FD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_desc(const fd_desc *d)
{
    if (!d) return fail(FD_ERR_INVALID_ARG, "desc is NULL");
    if (d->mode != FD_MODE_ISO && d->mode != FD_MODE_VTI) return fail(FD_ERR_INVALID_ARG, "bad mode %d", d->mode);
    if (d->nx < 1 || d->ny < 1 || d->nz < 1)
        return fail(FD_ERR_INVALID_ARG, "grid %d x %d x %d: every axis needs >= 1 point", d->nx, d->ny, d->nz);
    if (d->nx > (1 << 20) || d->ny > (1 << 20) || d->nz > (1 << 20))
        return fail(FD_ERR_INVALID_ARG, "grid axis above 2^20 points");
    if (!finite_pos(d->h) || !finite_pos(d->dt)) return fail(FD_ERR_INVALID_ARG, "h and dt must be finite and > 0");
    if (!d->dz_k && !finite_pos(d->dz)) return fail(FD_ERR_INVALID_ARG, "dz must be finite and > 0");
    if (d->sponge_width < 0 || !(d->sponge_a >= 0.0) || !std::isfinite(d->sponge_a))
        return fail(FD_ERR_INVALID_ARG, "bad damping layer (width %d, a %g)", d->sponge_width, d->sponge_a);
    if (d->mode == FD_MODE_ISO) {
        if (d->r_xy != d->r_z) return fail(FD_ERR_INVALID_ARG, "isotropic mode needs r_xy == r_z");
        if (d->dz_k) return fail(FD_ERR_INVALID_ARG, "dz_k is a VTI option");
        if (!iso_supported(d->r_xy)) return fail(FD_ERR_UNSUPPORTED, "isotropic radius %d not built (4, 8)", d->r_xy);
    } else {
        if (!vti_supported(d->r_xy, d->r_z))
            return fail(FD_ERR_UNSUPPORTED, "VTI radii (%d, %d) not built ((12, 8), (4, 4))", d->r_xy, d->r_z);
        if (d->dz_k) {
            if (d->nz < 2) return fail(FD_ERR_INVALID_ARG, "dz_k needs nz >= 2");
            for (int k = 0; k < d->nz - 1; ++k)
                if (!finite_pos(d->dz_k[k])) return fail(FD_ERR_INVALID_ARG, "dz_k[%d] must be finite and > 0", k);
        }
    }
    return FD_OK;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void compute_layout(const fd_desc *d, fd_layout_t *L)
{
    L->pitch = (int)round_up((size_t)d->nx, 32);
    L->nfields = d->mode == FD_MODE_ISO ? 2 : 4;
    L->nmodel = d->mode == FD_MODE_ISO ? 1 : 3;
    L->field_bytes = round_up((size_t)L->pitch * d->ny * d->nz * sizeof(float), 256);
    L->arena_bytes = (size_t)(L->nfields + L->nmodel) * L->field_bytes;
}

Launch default_launch(const fd_desc *d)
{
    return d->mode == FD_MODE_ISO ? iso_grid_launch(d->r_xy, d->nx, d->ny, d->nz)
                                  : vti_default_launch(d->r_xy, d->r_z, d->nx, d->ny, d->nz);
}

}  // namespace

struct fd_grid {
    fd_desc d{};
    std::vector<double> dzk;
    int dev = 0;
    cudaStream_t stream = nullptr;
    fd_layout_t lay{};
    char *arena = nullptr;
    float *field[4] = {};        // ISO: u[0], u[1]; VTI: p[0], p[1], q[0], q[1]
    float *model[3] = {};        // ISO: kappa; VTI: kx, kn, kz
    int cur = 0;                 // buffer index holding u^n (p^n, q^n)
    int n = 0;                   // host time index
    bool model_set = false;
    DevState *st = nullptr;      // device status block
    DevState *st_host = nullptr; // pinned copy
    float *gx = nullptr, *gy = nullptr, *gz = nullptr;
    float *ztab = nullptr;
    std::vector<float> zrows;    // host copy of ztab (VTI)
    double cxy[kMaxR + 1] = {};  // unit-grid second-derivative weights along x and y (Eq. 4)
    double cz[kMaxR + 1] = {};   // along z when dz is uniform (Eq. 4; VTI: replaces Eq. 5's rows)
    bool custom_z = false;       // VTI: z rows from cz rather than from the plane spacings
    double sig_z = 0.0;          // Gershgorin bound of the 1D z operator (isotropic, unit grid)
    int kg0 = 0, nzg = 0;        // local plane k is plane kg0 + k of a column of nzg planes
    double zrow_max = 0.0;       // Gershgorin bound of the z operator (VTI)
    double sig_xy = 0.0;         // Gershgorin bound of the 1D x-y operator (unit grid)
    float w0 = 0.f, wxy[kMaxR + 1] = {}, wz[kMaxR + 1] = {};
    // source
    float *src_tab = nullptr;
    int src_len = 0, sx = -1, sy = -1, sz = -1, into_q = 0;
    // receivers
    int nrec = 0, rec_t0 = 0, rec_cap = 0;
    float *trace = nullptr;
    bool lattice = false;
    RecLattice lat{};
    int *rec_idx = nullptr;
    int debug_skip = -1;         // fd_debug_skip_copy: plane withheld in the next launch
    // injection lattice (additive per-step sources, e.g. adjoint residuals)
    RecLattice inj{};
    double *d_misfit = nullptr;
    // launch
    Launch L{};
    CUtensorMap tm_halo[2];      // u (p) buffers, box (tx + 2 r_xy) x (ty + 2 r_xy)
    CUtensorMap tm_tile[4];      // every wavefield buffer, box tx x ty
    CUtensorMap tm_model[3];     // every model buffer, box tx x ty
    // tensor maps of caller fields for the gradient sweep, by address and box
    struct CachedMap {
        const float *p;
        int bx, by;
        CUtensorMap m;
    };
    std::vector<CachedMap> map_cache;
    // graphs
    int graph_steps = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    // fd_run_to_host: trace rows go to the host on their own stream, one event per chunk of steps
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_ev;
};

namespace {

void drop_graphs(fd_grid *g)
{
    for (auto &e : g->gexec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
}

int make_tensor_maps(fd_grid *g)
{
    const fd_desc &d = g->d;
    const int R = d.r_xy, tx = g->L.tx, ty = g->L.ty;
    const long long pitch = g->lay.pitch;
    int r = 0;
    for (int b = 0; b < 2 && !r; ++b)
        r = encode_field_map(&g->tm_halo[b], g->field[b], d.nx, d.ny, d.nz, pitch, tx + 2 * R, ty + 2 * R);
    for (int b = 0; b < g->lay.nfields && !r; ++b)
        r = encode_field_map(&g->tm_tile[b], g->field[b], d.nx, d.ny, d.nz, pitch, tx, ty);
    for (int m = 0; m < g->lay.nmodel && !r; ++m)
        r = encode_field_map(&g->tm_model[m], g->model[m], d.nx, d.ny, d.nz, pitch, tx, ty);
    if (r) return fail(FD_ERR_CUDA, "tensor map encoding failed (%d)", r);
    return FD_OK;
}

int set_launch(fd_grid *g, const Launch &L)
{
    if (L.tx <= 0 || L.ty <= 0 || L.zchunk <= 0 || L.lookahead <= 0 || L.zchunk > kMaxChunk)
        return fail(FD_ERR_INVALID_ARG, "bad launch configuration (z chunk 1..%d)", kMaxChunk);
    if ((g->d.ny + L.ty - 1) / L.ty > 65535 || (g->d.nz + L.zchunk - 1) / L.zchunk > 65535)
        return fail(FD_ERR_INVALID_ARG, "launch grid too large");
    const bool built = g->d.mode == FD_MODE_ISO ? iso_config_built(g->d.r_xy, L)
                                                : vti_config_built(g->d.r_xy, g->d.r_z, L);
    if (!built)
        return fail(FD_ERR_UNSUPPORTED, "tile %d x %d, lookahead %d is not built for this radius", L.tx, L.ty,
                    L.lookahead);
    g->L = L;
    drop_graphs(g);
    return make_tensor_maps(g);
}

// Enqueue one time step on stream s (no host-side bookkeeping).
// Everything of an isotropic launch except the two buffer pointers.
IsoArgs iso_args(const fd_grid *g)
{
    const fd_desc &d = g->d;
    IsoArgs a{};
    a.kappa = g->model[0];
    a.gx = g->gx; a.gy = g->gy; a.gz = g->gz;
    a.pitch = g->lay.pitch;
    a.plane = (long long)g->lay.pitch * d.ny;
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz;
    a.zchunk = g->L.zchunk;
    a.w0 = g->w0;
    std::memcpy(a.wxy, g->wxy, sizeof a.wxy);
    std::memcpy(a.wz, g->wz, sizeof a.wz);
    for (int l = 0; l <= kMaxR; ++l) {
        a.wxy2[l] = make_float2(g->wxy[l], g->wxy[l]);
        a.wz2[l] = make_float2(g->wz[l], g->wz[l]);
    }
    a.src = Source{g->src_tab, g->src_len, g->sx, g->sy, g->sz, g->into_q};
    a.rec = g->lat;
    a.rec.on = (g->nrec > 0 && g->lattice) ? 1 : 0;
    a.inj = g->inj;
    a.st = g->st;
    return a;
}

// Planes [zb, nz - ztop) of the step from level `cur`; hold = 1: a later part
// completes the step (advances the time index and samples gathered receivers).
cudaError_t enqueue_part(fd_grid *g, int cur, int zb, int ztop, int hold, cudaStream_t s)
{
    const fd_desc &d = g->d;
    Source src{g->src_tab, g->src_len, g->sx, g->sy, g->sz, g->into_q};
    RecLattice rec = g->lat;
    rec.on = (g->nrec > 0 && g->lattice) ? 1 : 0;
    const long long pitch = g->lay.pitch, plane = (long long)g->lay.pitch * d.ny;
    cudaError_t e;
    float *newbuf;
    if (d.mode == FD_MODE_ISO) {
        IsoArgs a = iso_args(g);
        a.prev = g->field[1 - cur];
        a.cur = g->field[cur];
        a.skip_plane1 = g->debug_skip + 1;
        g->debug_skip = -1;
        a.zb = zb;
        a.ztop = ztop;
        a.hold = hold;
        const IsoMaps maps{g->tm_halo[cur], g->tm_tile[1 - cur], g->tm_model[0], g->tm_tile[cur]};
        e = launch_iso(d.r_xy, g->L, maps, a, s);
        newbuf = a.prev;
    } else {
        VtiArgs a{};
        a.pprev = g->field[1 - cur];
        a.qprev = g->field[2 + (1 - cur)];
        a.p = g->field[cur];
        a.q = g->field[2 + cur];
        a.kx = g->model[0]; a.kn = g->model[1]; a.kz = g->model[2];
        a.gx = g->gx; a.gy = g->gy; a.gz = g->gz;
        a.ztab = g->ztab;
        a.pitch = pitch; a.plane = plane;
        a.nx = d.nx; a.ny = d.ny; a.nz = d.nz;
        a.zchunk = g->L.zchunk;
        a.w0 = g->w0;
        std::memcpy(a.wxy, g->wxy, sizeof a.wxy);
        for (int l = 0; l <= kMaxR; ++l) a.wxy2[l] = make_float2(g->wxy[l], g->wxy[l]);
        a.src = src; a.rec = rec; a.st = g->st;
        a.zb = zb; a.ztop = ztop; a.hold = hold;
        a.skip_plane1 = g->debug_skip + 1;
        g->debug_skip = -1;
        const VtiMaps maps{g->tm_halo[cur],    g->tm_tile[2 + cur], g->tm_tile[1 - cur], g->tm_tile[3 - cur],
                           g->tm_model[0],     g->tm_model[1],      g->tm_model[2]};
        e = launch_vti(d.r_xy, d.r_z, g->L, maps, a, s);
        newbuf = a.pprev;
    }
    if (e != cudaSuccess) return e;
    if (!hold && g->nrec > 0 && !g->lattice)
        e = launch_gather(newbuf, pitch, plane, g->rec_idx, g->nrec, g->trace, g->rec_t0, g->rec_cap,
                          g->st, s);
    return e;
}

cudaError_t enqueue_step(fd_grid *g, int cur, cudaStream_t s) { return enqueue_part(g, cur, 0, 0, 0, s); }

int check_ready(fd_grid *g, int nsteps)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (!g->model_set) return fail(FD_ERR_BAD_STATE, "no model: call fd_set_model first");
    if (nsteps < 0) return fail(FD_ERR_INVALID_ARG, "negative step count");
    if ((long long)g->n + nsteps > 0x7fffffffLL) return fail(FD_ERR_OUT_OF_RANGE, "time index overflow");
    if (g->nrec > 0 && (long long)g->n + nsteps - g->rec_t0 > g->rec_cap)
        return fail(FD_ERR_OUT_OF_RANGE, "receiver buffer holds %d rows; step %d would need row %lld",
                    g->rec_cap, g->n + nsteps - 1, (long long)g->n + nsteps - 1 - g->rec_t0);
    if (g->inj.on && (long long)g->n + nsteps - g->inj.t0 > g->inj.cap)
        return fail(FD_ERR_OUT_OF_RANGE, "injection buffer holds %d rows", g->inj.cap);
    return FD_OK;
}

int check_dev_status(fd_grid *g)
{
    CU(cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream), "status copy");
    CU(cudaStreamSynchronize(g->stream), "stream synchronize");
    if (g->st_host->err & kErrTmaTimeout)
        return fail(FD_ERR_TIMEOUT, "a stencil CTA (%d) timed out waiting for a TMA copy", g->st_host->err_info - 1);
    return FD_OK;
}

// Replace a small device table, stream-ordered on s: the old table is freed
// after the work already enqueued on s, and no call synchronises the device
// (a server creates and destroys grids while other shots run).
int upload(void **dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (*dst) {
        cudaFreeAsync(*dst, s);
        *dst = nullptr;
    }
    if (bytes == 0) return FD_OK;
    cudaError_t e = cudaMallocAsync(dst, bytes, s);
    if (e != cudaSuccess) {
        *dst = nullptr;
        cudaGetLastError();
        return fail(FD_ERR_NO_MEMORY, "table allocation of %zu bytes failed", bytes);
    }
    // pageable source: staged before the call returns, so `src` may go away
    CU(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s), "table upload");
    return FD_OK;
}

// Tensor map of a caller's field in the grid's pitched layout (box bx x by x 1),
// encoded once per address and box: the gradient sweep is called every step
// with the same few buffers.
int cached_map(fd_grid *g, const float *p, int bx, int by, CUtensorMap *out)
{
    for (const auto &e : g->map_cache)
        if (e.p == p && e.bx == bx && e.by == by) {
            *out = e.m;
            return 0;
        }
    fd_grid::CachedMap e{p, bx, by, {}};
    const int r = encode_field_map(&e.m, p, g->d.nx, g->d.ny, g->d.nz, g->lay.pitch, bx, by);
    if (r) return r;
    if (g->map_cache.size() >= 256) g->map_cache.erase(g->map_cache.begin());
    g->map_cache.push_back(e);
    *out = e.m;
    return 0;
}

// Single-precision weights of the sweeps, their Gershgorin bounds and (VTI)
// the z rows, from the unit-grid weights cxy and cz.
int apply_weights(fd_grid *g)
{
    const fd_desc &d = g->d;
    const double h2 = d.h * d.h;
    g->sig_xy = row_abs_sum(g->cxy, d.r_xy);
    for (int l = 0; l <= kMaxR; ++l) {
        g->wxy[l] = (l >= 1 && l <= d.r_xy) ? (float)(g->cxy[l] / h2) : 0.0f;
        g->wz[l] = 0.0f;
    }
    if (d.mode == FD_MODE_ISO) {
        const double dz2 = d.dz * d.dz;
        bool same = true;
        for (int l = 0; l <= d.r_xy; ++l) same = same && g->cxy[l] == g->cz[l];
        g->w0 = same ? (float)(g->cxy[0] * (2.0 / h2 + 1.0 / dz2)) : (float)(2.0 * g->cxy[0] / h2 + g->cz[0] / dz2);
        for (int l = 1; l <= d.r_z; ++l) g->wz[l] = (float)(g->cz[l] / dz2);
        g->sig_z = row_abs_sum(g->cz, d.r_z);
        return FD_OK;
    }
    g->w0 = (float)(2.0 * g->cxy[0] / h2);
    const int nw = 2 * d.r_z + 1;
    std::vector<double> tab((size_t)d.nz * nw);
    if (g->custom_z) {
        const double dz2 = d.dz * d.dz;
        for (int k = 0; k < d.nz; ++k)
            for (int l = -d.r_z; l <= d.r_z; ++l) tab[(size_t)k * nw + l + d.r_z] = g->cz[l < 0 ? -l : l] / dz2;
    } else {
        z_weights(d.nz, d.r_z, g->dzk.empty() ? nullptr : g->dzk.data(), d.dz, tab.data());
    }
    g->zrow_max = z_row_abs_max(tab.data(), d.nz, d.r_z);
    // one row per plane, copied whole into the sweep's shared memory: each
    // weight twice (an f32x2 operand), then the plane's damping factor
    // (filled in by upload_z_tables)
    const int zr = vti_zrow(d.r_z);
    g->zrows.assign((size_t)d.nz * zr, 0.0f);
    for (int k = 0; k < d.nz; ++k) {
        float *row = g->zrows.data() + (size_t)k * zr;
        for (int m = 0; m < nw; ++m) row[2 * m] = row[2 * m + 1] = (float)tab[(size_t)k * nw + m];
    }
    return FD_OK;
}

// Damping factors along z of the local planes (the planes kg0.. of a column
// of nzg planes), and for VTI the z rows that end with the same factor.
int upload_z_tables(fd_grid *g)
{
    const fd_desc &d = g->d;
    std::vector<float> pz(d.nz);
    for (int k = 0; k < d.nz; ++k) pz[k] = (float)cerjan(g->kg0 + k, g->nzg, d.sponge_width, d.sponge_a);
    int rc = upload(reinterpret_cast<void **>(&g->gz), pz.data(), pz.size() * 4, g->stream);
    if (rc || d.mode != FD_MODE_VTI) return rc;
    const int zr = vti_zrow(d.r_z), nw = 2 * d.r_z + 1;
    for (int k = 0; k < d.nz; ++k) g->zrows[(size_t)k * zr + 2 * nw] = pz[k];
    return upload(reinterpret_cast<void **>(&g->ztab), g->zrows.data(), g->zrows.size() * 4, g->stream);
}

// A receiver set that is a row-major lattice on one z plane with constant
// strides: fills the geometry of L (not its buffer, origin step or capacity).
bool detect_lattice(const int *idx, int nrec, RecLattice *L)
{
    int rnx = 1;
    while (rnx < nrec && idx[3 * rnx + 1] == idx[1]) ++rnx;
    const int rny = nrec / rnx;
    const int rsx = rnx > 1 ? idx[3] - idx[0] : 1;
    const int rsy = rny > 1 ? idx[3 * rnx + 1] - idx[1] : 1;
    if (rny * rnx != nrec || rsx <= 0 || rsy <= 0) return false;
    for (int r = 0; r < nrec; ++r) {
        const int ry = r / rnx, rx = r % rnx;
        if (idx[3 * r] != idx[0] + rx * rsx || idx[3 * r + 1] != idx[1] + ry * rsy || idx[3 * r + 2] != idx[2])
            return false;
    }
    *L = RecLattice{};
    L->nrec = nrec;
    L->rk = idx[2];
    L->rx0 = idx[0];
    L->ry0 = idx[1];
    L->rsx = rsx;
    L->rsy = rsy;
    L->rnx = rnx;
    L->rny = rny;
    return true;
}

double source_volume(const fd_grid *g, int iz)
{
    const fd_desc &d = g->d;
    if (d.mode == FD_MODE_VTI && !g->dzk.empty()) {
        const double lo = iz >= 1 ? g->dzk[iz - 1] : g->dzk[0];
        const double hi = iz <= d.nz - 2 ? g->dzk[iz] : g->dzk[d.nz - 2];
        return d.h * d.h * 0.5 * (lo + hi);
    }
    return d.h * d.h * d.dz;
}

int set_source_table(fd_grid *g, int ix, int iy, int iz, const std::vector<double> &s, int inject_q)
{
    const fd_desc &d = g->d;
    if (ix < 0 || ix >= d.nx || iy < 0 || iy >= d.ny || iz < 0 || iz >= d.nz)
        return fail(FD_ERR_INVALID_ARG, "source cell (%d, %d, %d) outside the grid", ix, iy, iz);
    if (inject_q && d.mode != FD_MODE_VTI) return fail(FD_ERR_INVALID_ARG, "inject_q is a VTI option");
    const double scale = d.dt * d.dt / source_volume(g, iz);
    std::vector<float> tab(s.size());
    for (size_t i = 0; i < s.size(); ++i) tab[i] = (float)(s[i] * scale);
    int rc = upload(reinterpret_cast<void **>(&g->src_tab), tab.data(), tab.size() * sizeof(float), g->stream);
    if (rc) return rc;
    g->src_len = (int)tab.size();
    g->sx = ix; g->sy = iy; g->sz = iz;
    g->into_q = inject_q ? 1 : 0;
    drop_graphs(g);
    return FD_OK;
}

}  // namespace

namespace fdk {
// Lets other translation units of the library report through fd_last_error().
int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace fdk

extern "C" {

int fd_last_error(char *buf, size_t n)
{
    if (!buf || n == 0) return FD_ERR_INVALID_ARG;
    std::snprintf(buf, n, "%s", g_err.c_str());
    return FD_OK;
}

int fd_layout(const fd_desc *d, fd_layout_t *out)
{
    int rc = check_desc(d);
    if (rc) return rc;
    if (!out) return fail(FD_ERR_INVALID_ARG, "out is NULL");
    compute_layout(d, out);
    return FD_OK;
}

int fd_required_bytes(const fd_desc *d, size_t *bytes)
{
    fd_layout_t L;
    int rc = fd_layout(d, &L);
    if (rc) return rc;
    if (!bytes) return fail(FD_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = L.arena_bytes;
    return FD_OK;
}

int fd_stability_limit(const fd_desc *d, double vmax, double eps_max, double *dt_max)
{
    int rc = check_desc(d);
    if (rc) return rc;
    if (!dt_max || !finite_pos(vmax) || !std::isfinite(eps_max) || 1.0 + 2.0 * eps_max <= 0.0)
        return fail(FD_ERR_INVALID_ARG, "bad stability-limit arguments");
    double c[kMaxR + 1];
    central_d2(d->r_xy, c);
    const double sxy = row_abs_sum(c, d->r_xy);
    double rho;
    if (d->mode == FD_MODE_ISO) {
        rho = 2.0 * sxy / (d->h * d->h) + sxy / (d->dz * d->dz);
    } else {
        std::vector<double> tab((size_t)d->nz * (2 * d->r_z + 1));
        z_weights(d->nz, d->r_z, d->dz_k, d->dz, tab.data());
        rho = (1.0 + 2.0 * std::max(0.0, eps_max)) * 2.0 * sxy / (d->h * d->h) +
              z_row_abs_max(tab.data(), d->nz, d->r_z);
    }
    *dt_max = 2.0 / (vmax * std::sqrt(rho));
    return FD_OK;
}

int fd_create_grid(const fd_desc *d, void *arena, size_t arena_bytes, void *stream, fd_grid_t **out)
{
    int rc = check_desc(d);
    if (rc) return rc;
    if (!out) return fail(FD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    fd_layout_t lay;
    compute_layout(d, &lay);
    if (!arena) return fail(FD_ERR_INVALID_ARG, "arena is NULL");
    if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) return fail(FD_ERR_INVALID_ARG, "arena not 256-byte aligned");
    if (arena_bytes < lay.arena_bytes)
        return fail(FD_ERR_NO_MEMORY, "arena has %zu bytes, needs %zu", arena_bytes, lay.arena_bytes);
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, arena) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(FD_ERR_INVALID_ARG, "arena is not device memory");
    }

    fd_grid *g = new (std::nothrow) fd_grid;
    if (!g) return fail(FD_ERR_NO_MEMORY, "host allocation failed");
    g->d = *d;
    if (d->dz_k) g->dzk.assign(d->dz_k, d->dz_k + d->nz - 1);
    g->d.dz_k = nullptr;
    if (g->d.dz_k == nullptr && !g->dzk.empty() && !finite_pos(g->d.dz)) g->d.dz = g->dzk[0];
    g->stream = static_cast<cudaStream_t>(stream);
    g->lay = lay;
    g->arena = static_cast<char *>(arena);
    cudaGetDevice(&g->dev);
    for (int b = 0; b < lay.nfields; ++b) g->field[b] = reinterpret_cast<float *>(g->arena + b * lay.field_bytes);
    for (int m = 0; m < lay.nmodel; ++m)
        g->model[m] = reinterpret_cast<float *>(g->arena + (lay.nfields + m) * lay.field_bytes);

    auto bail = [&](int code) {
        fd_destroy_grid(g);
        return code;
    };
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&g->st), sizeof(DevState), g->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "status block allocation"));
    g->st_host = new (std::nothrow) DevState;
    if (!g->st_host) return bail(fail(FD_ERR_NO_MEMORY, "host allocation failed"));
    e = cudaMemsetAsync(g->st, 0, sizeof(DevState), g->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "status clear"));
    e = cudaMemsetAsync(g->arena, 0, (size_t)lay.nfields * lay.field_bytes, g->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "wavefield clear"));

    // weights (Eq. 4 on x-y; Eq. 4 on z for the isotropic case, Eq. 5 for VTI)
    central_d2(d->r_xy, g->cxy);
    central_d2(d->r_z, g->cz);
    if ((rc = apply_weights(g))) return bail(rc);
    // damping profiles (Cerjan), padded to the pitch for 128-bit loads
    std::vector<float> px(lay.pitch, 1.0f), py(d->ny);
    for (int i = 0; i < d->nx; ++i) px[i] = (float)cerjan(i, d->nx, d->sponge_width, d->sponge_a);
    for (int j = 0; j < d->ny; ++j) py[j] = (float)cerjan(j, d->ny, d->sponge_width, d->sponge_a);
    if ((rc = upload(reinterpret_cast<void **>(&g->gx), px.data(), px.size() * 4, g->stream)) ||
        (rc = upload(reinterpret_cast<void **>(&g->gy), py.data(), py.size() * 4, g->stream)))
        return bail(rc);
    g->kg0 = 0;
    g->nzg = d->nz;
    if ((rc = upload_z_tables(g))) return bail(rc);

    rc = set_launch(g, default_launch(d));
    if (rc) return bail(rc);
    *out = g;
    return FD_OK;
}

int fd_set_launch(fd_grid_t *g, int tx, int ty, int zchunk, int lookahead)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    Launch L{tx, ty, zchunk, lookahead};
    Launch old = g->L;
    int rc = set_launch(g, L);
    if (rc) {
        set_launch(g, old);
        return rc;
    }
    return FD_OK;
}

int fd_set_model(fd_grid_t *g, const float *vz, const float *eps, const float *delta, int ptr_kind)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    const fd_desc &d = g->d;
    const bool vti = d.mode == FD_MODE_VTI;
    if (!vz || (vti && (!eps || !delta)) || (!vti && (eps || delta)))
        return fail(FD_ERR_INVALID_ARG, vti ? "VTI needs vz, eps and delta" : "isotropic mode takes v only");
    if (ptr_kind != FD_PTR_HOST && ptr_kind != FD_PTR_DEVICE) return fail(FD_ERR_INVALID_ARG, "bad ptr_kind");
    g->model_set = false;
    drop_graphs(g);
    const long long pitch = g->lay.pitch;
    const size_t row = (size_t)d.nx * 4, rows = (size_t)d.ny * d.nz;
    CU(cudaMemsetAsync(reinterpret_cast<char *>(g->st) + offsetof(DevState, vmax), 0, 16, g->stream),
       "status clear");
    const float *in[3] = {vz, eps, delta};
    long long src_pitch = d.nx;
    if (ptr_kind == FD_PTR_HOST) {
        // stage the dense inputs in the model buffers, then convert in place
        float *stage[3] = {vti ? g->model[2] : g->model[0], g->model[0], g->model[1]};
        for (int m = 0; m < (vti ? 3 : 1); ++m) {
            CU(cudaMemcpy2DAsync(stage[m], pitch * 4, in[m], row, row, rows, cudaMemcpyHostToDevice, g->stream),
               "model upload");
            in[m] = stage[m];
        }
        src_pitch = pitch;
    }
    cudaError_t e;
    if (!vti)
        e = launch_model_iso(in[0], src_pitch, g->model[0], d.nx, d.ny, d.nz, pitch, d.dt, g->st, g->stream);
    else
        e = launch_model_vti(in[0], in[1], in[2], src_pitch, g->model[0], g->model[1], g->model[2], d.nx, d.ny,
                             d.nz, pitch, d.dt, g->st, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "model kernel");
    CU(cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream), "status copy");
    CU(cudaStreamSynchronize(g->stream), "stream synchronize");
    const DevState &s = *g->st_host;
    if (s.bad) return fail(FD_ERR_INVALID_ARG, "%u model values are not finite / not positive", s.bad);
    if (vti && s.eps_lt_delta)
        return fail(FD_ERR_INVALID_ARG, "%u cells have eps < delta (the VTI system is unstable there)", s.eps_lt_delta);
    const double dt = d.dt;
    const double kmax = (double)s.vmax * dt * (double)s.vmax * dt;
    double lam;
    if (!vti) {
        const double dz2 = d.dz * d.dz;
        lam = kmax * (2.0 * g->sig_xy / (d.h * d.h) + g->sig_z / dz2);
    } else {
        lam = (double)s.kxmax * 2.0 * g->sig_xy / (d.h * d.h) + kmax * g->zrow_max;
    }
    if (lam > 4.0 * (1.0 + 1e-9))
        return fail(FD_ERR_UNSTABLE_DT, "dt = %g exceeds the stability bound (%.6g of it) for v_max = %g", dt,
                    std::sqrt(lam / 4.0), (double)s.vmax);
    g->model_set = true;
    return FD_OK;
}

int fd_add_source(fd_grid_t *g, int ix, int iy, int iz, double freq_hz, double t0, double amp, int inject_q)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (!finite_pos(freq_hz) || !std::isfinite(t0) || !std::isfinite(amp))
        return fail(FD_ERR_INVALID_ARG, "bad Ricker parameters");
    // beyond t0 + 4/f the wavelet is below 1e-60 relative: the table stops there
    const double tend = t0 + 4.0 / freq_hz;
    const double nmax = std::ceil(tend / g->d.dt) + 1.0;
    if (nmax > (double)(1 << 26)) return fail(FD_ERR_INVALID_ARG, "source table too long (t0 + 4/f >> dt)");
    const int len = std::max(0, (int)nmax);
    std::vector<double> s(len);
    for (int n = 0; n < len; ++n) s[n] = amp * ricker(n * g->d.dt - t0, freq_hz);
    return set_source_table(g, ix, iy, iz, s, inject_q);
}

int fd_add_source_series(fd_grid_t *g, int ix, int iy, int iz, const float *s, int nt, int inject_q)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (nt < 0 || (nt > 0 && !s)) return fail(FD_ERR_INVALID_ARG, "bad source series");
    std::vector<double> v(s, s + nt);
    return set_source_table(g, ix, iy, iz, v, inject_q);
}

int fd_set_receivers(fd_grid_t *g, const int *idx, int nrec, float *trace_dev, int nt_cap)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    drop_graphs(g);
    if (nrec == 0) {
        g->nrec = 0;
        g->lattice = false;
        return FD_OK;
    }
    if (nrec < 0 || !idx || !trace_dev || nt_cap < 0) return fail(FD_ERR_INVALID_ARG, "bad receiver arguments");
    const fd_desc &d = g->d;
    for (int r = 0; r < nrec; ++r) {
        const int i = idx[3 * r], j = idx[3 * r + 1], k = idx[3 * r + 2];
        if (i < 0 || i >= d.nx || j < 0 || j >= d.ny || k < 0 || k >= d.nz)
            return fail(FD_ERR_INVALID_ARG, "receiver %d at (%d, %d, %d) outside the grid", r, i, j, k);
    }
    RecLattice L{};
    const bool lat = detect_lattice(idx, nrec, &L);
    g->lattice = lat;
    g->nrec = nrec;
    g->trace = trace_dev;
    g->rec_cap = nt_cap;
    g->rec_t0 = g->n;
    g->lat = RecLattice{};
    if (lat) {
        g->lat = L;
        g->lat.trace = trace_dev;
        g->lat.t0 = g->n;
        g->lat.cap = nt_cap;
    } else {
        int rc = upload(reinterpret_cast<void **>(&g->rec_idx), idx, (size_t)nrec * 3 * sizeof(int), g->stream);
        if (rc) {
            g->nrec = 0;
            return rc;
        }
    }
    return FD_OK;
}

int fd_step(fd_grid_t *g) { return fd_run(g, 1); }

int fd_set_injection(fd_grid_t *g, const int *idx, int nrec, const float *values_dev, int nt_cap)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    drop_graphs(g);
    if (nrec == 0) {
        g->inj = RecLattice{};
        return FD_OK;
    }
    if (g->d.mode != FD_MODE_ISO) return fail(FD_ERR_UNSUPPORTED, "injection lattices are isotropic-only");
    if (nrec < 0 || !idx || !values_dev || nt_cap < 0) return fail(FD_ERR_INVALID_ARG, "bad injection arguments");
    const fd_desc &d = g->d;
    for (int r = 0; r < nrec; ++r) {
        const int i = idx[3 * r], j = idx[3 * r + 1], k = idx[3 * r + 2];
        if (i < 0 || i >= d.nx || j < 0 || j >= d.ny || k < 0 || k >= d.nz)
            return fail(FD_ERR_INVALID_ARG, "injection point %d at (%d, %d, %d) outside the grid", r, i, j, k);
    }
    RecLattice L{};
    if (!detect_lattice(idx, nrec, &L))
        return fail(FD_ERR_UNSUPPORTED, "injection points must form a row-major lattice on one plane");
    L.trace = const_cast<float *>(values_dev);
    L.t0 = g->n;
    L.cap = nt_cap;
    L.on = 1;
    g->inj = L;
    return FD_OK;
}

int fd_adjoint_source(fd_grid_t *g, const float *traces, const float *dobs, int nt, float *inj, double *misfit)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (g->d.mode != FD_MODE_ISO) return fail(FD_ERR_UNSUPPORTED, "the adjoint is isotropic-only");
    if (!g->model_set) return fail(FD_ERR_BAD_STATE, "no model");
    if (g->nrec <= 0 || !g->lattice)
        return fail(FD_ERR_BAD_STATE, "the grid needs receivers on a lattice (they define the adjoint sources)");
    if (nt < 0 || (nt > 0 && (!traces || !dobs || !inj)) || !misfit) return fail(FD_ERR_INVALID_ARG, "bad arguments");
    if (!g->d_misfit) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&g->d_misfit), sizeof(double), g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "misfit allocation");
    }
    CU(cudaMemsetAsync(g->d_misfit, 0, sizeof(double), g->stream), "misfit clear");
    if (nt > 0) {
        cudaError_t e = launch_adjoint_source(g->lat, g->model[0], g->lay.pitch, (long long)g->lay.pitch * g->d.ny,
                                              traces, dobs, nt, inj, g->d_misfit, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint source kernel");
    }
    CU(cudaMemcpyAsync(misfit, g->d_misfit, sizeof(double), cudaMemcpyDeviceToHost, g->stream), "misfit copy");
    CU(cudaStreamSynchronize(g->stream), "stream synchronize");
    return FD_OK;
}

int fd_grad_accumulate(fd_grid_t *g, const float *z, const float *a, float *grad)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (g->d.mode != FD_MODE_ISO) return fail(FD_ERR_UNSUPPORTED, "the adjoint is isotropic-only");
    if (!g->model_set) return fail(FD_ERR_BAD_STATE, "no model");
    if (!z || !a || !grad) return fail(FD_ERR_INVALID_ARG, "NULL field");
    if ((reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(grad)) % 16)
        return fail(FD_ERR_INVALID_ARG, "fields must be 16-byte aligned");
    if (g->d.ny > 65535 || g->d.nz > 65535) return fail(FD_ERR_UNSUPPORTED, "grid too large for the gradient kernel");
    const fd_desc &d = g->d;
    const int R = d.r_xy;
    const Launch L = iso_grad_launch(R, d.nx, d.ny, d.nz);
    IsoMaps maps;
    CUtensorMap mg;
    if (cached_map(g, a, L.tx + 2 * R, L.ty + 2 * R, &maps.cur) || cached_map(g, a, L.tx, L.ty, &maps.cur_tile) ||
        cached_map(g, z, L.tx, L.ty, &maps.prev) ||
        cached_map(g, g->model[0], L.tx, L.ty, &maps.kappa) || cached_map(g, grad, L.tx, L.ty, &mg))
        return fail(FD_ERR_CUDA, "tensor map encoding failed");
    IsoArgs w = iso_args(g);
    w.prev = grad;
    w.cur = a;
    w.zchunk = L.zchunk;
    w.c2dt = (float)(2.0 * d.dt);
    cudaError_t e = launch_iso_grad(R, L, maps, mg, w, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gradient kernel");
    return FD_OK;
}

int fd_step_from(fd_grid_t *g, const float *cur, const float *prev, float *out)
{
    int rc = check_ready(g, 1);
    if (rc) return rc;
    if (g->d.mode != FD_MODE_ISO) return fail(FD_ERR_UNSUPPORTED, "fd_step_from takes isotropic grids");
    if (!cur || !prev || !out) return fail(FD_ERR_INVALID_ARG, "NULL field");
    if ((reinterpret_cast<uintptr_t>(cur) | reinterpret_cast<uintptr_t>(prev) | reinterpret_cast<uintptr_t>(out)) % 16)
        return fail(FD_ERR_INVALID_ARG, "fields must be 16-byte aligned");
    if (out == cur) return fail(FD_ERR_INVALID_ARG, "out must not be cur (its neighbours' halos read it)");
    const fd_desc &d = g->d;
    const int R = d.r_xy;
    const Launch &L = g->L;
    IsoMaps maps;
    if (cached_map(g, cur, L.tx + 2 * R, L.ty + 2 * R, &maps.cur) || cached_map(g, cur, L.tx, L.ty, &maps.cur_tile) ||
        cached_map(g, prev, L.tx, L.ty, &maps.prev))
        return fail(FD_ERR_CUDA, "tensor map encoding failed");
    maps.kappa = g->tm_model[0];
    IsoArgs a = iso_args(g);
    a.prev = out;               // written: u^{n+1} (read through the map of prev)
    a.cur = cur;
    cudaError_t e = launch_iso(R, L, maps, a, g->stream);
    if (e == cudaSuccess && g->nrec > 0 && !g->lattice)
        e = launch_gather(out, g->lay.pitch, (long long)g->lay.pitch * d.ny, g->rec_idx, g->nrec, g->trace, g->rec_t0,
                          g->rec_cap, g->st, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    g->n += 1;
    return FD_OK;
}

int fd_set_graph(fd_grid_t *g, int steps)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (steps != 0 && (steps < 2 || steps > 1024 || steps % 2))
        return fail(FD_ERR_INVALID_ARG, "graph steps must be 0 or even in 2..1024");
    drop_graphs(g);
    g->graph_steps = steps;
    return FD_OK;
}

int fd_step_planes(fd_grid_t *g, int k_begin, int k_end, int complete)
{
    if (g && (k_begin < 0 || k_end > g->d.nz || k_begin >= k_end))
        return fail(FD_ERR_INVALID_ARG, "planes [%d, %d) are not a non-empty range of 0..%d", k_begin, k_end, g->d.nz);
    int rc = check_ready(g, 1);
    if (rc) return rc;
    cudaError_t e = enqueue_part(g, g->cur, k_begin, g->d.nz - k_end, complete ? 0 : 1, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    if (complete) {
        g->cur ^= 1;
        g->n += 1;
    }
    return FD_OK;
}

int fd_run(fd_grid_t *g, int nsteps)
{
    int rc = check_ready(g, nsteps);
    if (rc) return rc;
    int left = nsteps;
    if (left > 0 && g->debug_skip >= 0) {
        // the test hook's launch runs outside any graph
        cudaError_t e = enqueue_step(g, g->cur, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step launch");
        g->cur ^= 1;
        g->n += 1;
        left -= 1;
    }
    const int K = g->graph_steps;
    while (K > 0 && left >= K) {
        cudaGraphExec_t &ge = g->gexec[g->cur];
        if (!ge) {
            if (!g->cap_stream) CU(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking), "stream create");
            CU(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = cudaSuccess;
            for (int j = 0; j < K && e == cudaSuccess; ++j) e = enqueue_step(g, (g->cur + j) & 1, g->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
            if (e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(e, "step capture");
            }
            if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
            e = cudaGraphInstantiate(&ge, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                ge = nullptr;
                return cuda_fail(e, "graph instantiate");
            }
        }
        CU(cudaGraphLaunch(ge, g->stream), "graph launch");
        g->n += K;   // K is even: the buffer parity is unchanged
        left -= K;
    }
    for (; left > 0; --left) {
        cudaError_t e = enqueue_step(g, g->cur, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step launch");
        g->cur ^= 1;
        g->n += 1;
    }
    return FD_OK;
}

int fd_run_to_host(fd_grid_t *g, int nsteps, float *host_dst, int chunk_steps)
{
    int rc = check_ready(g, nsteps);
    if (rc) return rc;
    if (g->nrec == 0) return fail(FD_ERR_BAD_STATE, "no receivers");
    if (chunk_steps < 0 || (nsteps > 0 && !host_dst)) return fail(FD_ERR_INVALID_ARG, "bad arguments");
    if (nsteps == 0) return FD_OK;
    // chunks: 64 steps unless asked otherwise, whole graphs when graphs are on,
    // at most 256 of them (one event each)
    int c = chunk_steps > 0 ? chunk_steps : 64;
    c = std::max(c, (nsteps + 255) / 256);
    if (g->graph_steps > 0) c = (c + g->graph_steps - 1) / g->graph_steps * g->graph_steps;
    const int nchunks = (nsteps + c - 1) / c;
    if (!g->copy_stream) CU(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking), "stream create");
    while ((int)g->copy_ev.size() < nchunks) {
        cudaEvent_t e = nullptr;
        CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
        g->copy_ev.push_back(e);
    }
    // every chunk's steps first (a pageable destination then still overlaps:
    // its staged copies run on the host while later chunks compute) ...
    const long long row0 = (long long)g->n - g->rec_t0;
    for (int i = 0; i < nchunks; ++i) {
        rc = fd_run(g, std::min(c, nsteps - i * c));
        if (rc) {
            cudaStreamSynchronize(g->stream);
            return rc;
        }
        CU(cudaEventRecord(g->copy_ev[i], g->stream), "event record");
    }
    // ... then each chunk's rows once its steps are done; copies already enqueued
    // are waited for on every path, so none writes host_dst after the return
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nchunks && e == cudaSuccess; ++i) {
        const int ci = std::min(c, nsteps - i * c);
        e = cudaStreamWaitEvent(g->copy_stream, g->copy_ev[i], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_dst + (size_t)i * c * g->nrec,
                                g->trace + (size_t)(row0 + (long long)i * c) * g->nrec,
                                (size_t)ci * g->nrec * sizeof(float), cudaMemcpyDeviceToHost, g->copy_stream);
    }
    const cudaError_t es = cudaStreamSynchronize(g->copy_stream);
    if (e != cudaSuccess) return cuda_fail(e, "trace copy");
    if (es != cudaSuccess) return cuda_fail(es, "copy stream synchronize");
    return check_dev_status(g);
}

int fd_read_receivers(fd_grid_t *g, int t_begin, int t_count, float *dst, int dst_kind)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (g->nrec == 0) return fail(FD_ERR_BAD_STATE, "no receivers");
    if (t_begin < 0 || t_count < 0 || (t_count > 0 && !dst)) return fail(FD_ERR_INVALID_ARG, "bad read arguments");
    if (dst_kind != FD_PTR_HOST && dst_kind != FD_PTR_DEVICE) return fail(FD_ERR_INVALID_ARG, "bad dst_kind");
    const long long written = (long long)g->n - g->rec_t0;
    if ((long long)t_begin + t_count > std::min<long long>(written, g->rec_cap))
        return fail(FD_ERR_OUT_OF_RANGE, "rows [%d, %d) requested, %lld written", t_begin, t_begin + t_count, written);
    const size_t bytes = (size_t)t_count * g->nrec * sizeof(float);
    if (bytes)
        CU(cudaMemcpyAsync(dst, g->trace + (size_t)t_begin * g->nrec, bytes,
                           dst_kind == FD_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream),
           "trace copy");
    if (dst_kind == FD_PTR_HOST) return check_dev_status(g);
    return FD_OK;
}

int fd_get_state(fd_grid_t *g, float *cur, float *prev, float *q_cur, float *q_prev, int ptr_kind, int *time_index)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (ptr_kind != FD_PTR_HOST && ptr_kind != FD_PTR_DEVICE) return fail(FD_ERR_INVALID_ARG, "bad ptr_kind");
    const fd_desc &d = g->d;
    if ((q_cur || q_prev) && d.mode != FD_MODE_VTI) return fail(FD_ERR_INVALID_ARG, "q is a VTI field");
    float *dst[4] = {cur, prev, q_cur, q_prev};
    const float *src[4] = {g->field[g->cur], g->field[1 - g->cur], g->field[2 + g->cur], g->field[3 - g->cur]};
    const size_t row = (size_t)d.nx * 4;
    for (int m = 0; m < 4; ++m)
        if (dst[m])
            CU(cudaMemcpy2DAsync(dst[m], row, src[m], (size_t)g->lay.pitch * 4, row, (size_t)d.ny * d.nz,
                                 ptr_kind == FD_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                 g->stream),
               "state copy");
    if (time_index) *time_index = g->n;
    if (ptr_kind == FD_PTR_HOST) return check_dev_status(g);
    return FD_OK;
}

int fd_set_state(fd_grid_t *g, const float *cur, const float *prev, const float *q_cur, const float *q_prev,
                 int ptr_kind, int time_index)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (ptr_kind != FD_PTR_HOST && ptr_kind != FD_PTR_DEVICE) return fail(FD_ERR_INVALID_ARG, "bad ptr_kind");
    if (time_index < 0) return fail(FD_ERR_INVALID_ARG, "negative time index");
    const fd_desc &d = g->d;
    if ((q_cur || q_prev) && d.mode != FD_MODE_VTI) return fail(FD_ERR_INVALID_ARG, "q is a VTI field");
    const float *src[4] = {cur, prev, q_cur, q_prev};
    float *dst[4] = {g->field[g->cur], g->field[1 - g->cur], g->field[2 + g->cur], g->field[3 - g->cur]};
    const size_t row = (size_t)d.nx * 4;
    for (int m = 0; m < 4; ++m)
        if (src[m])
            CU(cudaMemcpy2DAsync(dst[m], (size_t)g->lay.pitch * 4, src[m], row, row, (size_t)d.ny * d.nz,
                                 ptr_kind == FD_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                 g->stream),
               "state copy");
    g->st_host->step = time_index;
    CU(cudaMemcpyAsync(&g->st->step, &g->st_host->step, sizeof(int), cudaMemcpyHostToDevice, g->stream),
       "time index copy");
    CU(cudaStreamSynchronize(g->stream), "stream synchronize");
    g->n = time_index;
    return FD_OK;
}

int fd_field(fd_grid_t *g, int which, float **dev_ptr, int *pitch)
{
    if (!g || !dev_ptr) return fail(FD_ERR_INVALID_ARG, "NULL argument");
    if (which < 0 || which > 3 || (which > 1 && g->d.mode != FD_MODE_VTI)) return fail(FD_ERR_INVALID_ARG, "bad field");
    const int b[4] = {g->cur, 1 - g->cur, 2 + g->cur, 3 - g->cur};
    *dev_ptr = g->field[b[which]];
    if (pitch) *pitch = g->lay.pitch;
    return FD_OK;
}

int fd_optimized_weights(int radius, double kmax, double *weights)
{
    if (!weights) return fail(FD_ERR_INVALID_ARG, "weights is NULL");
    if (radius < 1 || radius > kMaxR) return fail(FD_ERR_INVALID_ARG, "radius %d outside 1..%d", radius, kMaxR);
    if (!(kmax > 0.0) || kmax > M_PI) return fail(FD_ERR_INVALID_ARG, "kmax %g outside (0, pi]", kmax);
    if (band_optimized_d2(radius, kmax, weights)) return fail(FD_ERR_INVALID_ARG, "weight fit failed");
    return FD_OK;
}

int fd_set_weights(fd_grid_t *g, const double *w_xy, const double *w_z)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (g->model_set) return fail(FD_ERR_BAD_STATE, "set the weights before the model (the stability check uses them)");
    const fd_desc &d = g->d;
    // a second-derivative stencil: exact on constants and on x^2 / 2
    auto consistent = [](const double *w, int R) {
        double s = w[0], a = std::fabs(w[0]), q = 0.0;
        for (int l = 1; l <= R; ++l) {
            if (!std::isfinite(w[l])) return false;
            s += 2.0 * w[l];
            a += 2.0 * std::fabs(w[l]);
            q += (double)l * l * w[l];
        }
        return std::isfinite(w[0]) && std::fabs(s) <= 1e-9 * a && std::fabs(q - 1.0) <= 1e-6;
    };
    if (w_xy && !consistent(w_xy, d.r_xy))
        return fail(FD_ERR_INVALID_ARG, "x-y weights are not a consistent second derivative");
    if (w_z) {
        if (!g->dzk.empty()) return fail(FD_ERR_UNSUPPORTED, "z weights need a uniform dz");
        if (!consistent(w_z, d.r_z)) return fail(FD_ERR_INVALID_ARG, "z weights are not a consistent second derivative");
    }
    if (w_xy) std::memcpy(g->cxy, w_xy, sizeof(double) * (d.r_xy + 1));
    if (w_z) {
        std::memcpy(g->cz, w_z, sizeof(double) * (d.r_z + 1));
        if (d.mode == FD_MODE_VTI) g->custom_z = true;
    }
    drop_graphs(g);
    int rc = apply_weights(g);
    if (rc) return rc;
    return (d.mode == FD_MODE_VTI && w_z) ? upload_z_tables(g) : FD_OK;
}

int fd_set_z_window(fd_grid_t *g, int kg0, int nz_global)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    if (kg0 < 0 || nz_global < 1 || (long long)kg0 + g->d.nz > nz_global)
        return fail(FD_ERR_INVALID_ARG, "planes [%d, %d) do not lie in a column of %d planes", kg0, kg0 + g->d.nz,
                    nz_global);
    if (!g->dzk.empty()) return fail(FD_ERR_UNSUPPORTED, "z windows need a uniform dz");
    g->kg0 = kg0;
    g->nzg = nz_global;
    drop_graphs(g);   // the tables move
    return upload_z_tables(g);
}

int fd_halo_exchange(fd_grid_t *lo, fd_grid_t *up, int planes)
{
    if (!lo || !up || lo == up) return fail(FD_ERR_INVALID_ARG, "need two distinct grids");
    const fd_desc &a = lo->d, &b = up->d;
    if (a.mode != b.mode || a.nx != b.nx || a.ny != b.ny || a.r_xy != b.r_xy || a.r_z != b.r_z)
        return fail(FD_ERR_INVALID_ARG, "slabs differ in mode, radius or x-y size");
    if (lo->dev != up->dev || lo->stream != up->stream)
        return fail(FD_ERR_INVALID_ARG, "slabs must share a device and a stream");
    const int rz = a.mode == FD_MODE_ISO ? a.r_xy : a.r_z;
    if (planes < rz) return fail(FD_ERR_INVALID_ARG, "%d ghost planes, the z stencil needs %d", planes, rz);
    if (a.nz < 2 * planes || b.nz < 2 * planes)
        return fail(FD_ERR_INVALID_ARG, "slabs of %d and %d planes cannot hold %d ghost planes", a.nz, b.nz, planes);
    if (lo->nzg != up->nzg || up->kg0 != lo->kg0 + a.nz - 2 * planes)
        return fail(FD_ERR_INVALID_ARG, "z windows [%d, %d) and [%d, %d) do not overlap by %d planes", lo->kg0,
                    lo->kg0 + a.nz, up->kg0, up->kg0 + b.nz, 2 * planes);
    if (lo->n != up->n) return fail(FD_ERR_BAD_STATE, "slabs at time indices %d and %d", lo->n, up->n);
    const size_t plane = (size_t)lo->lay.pitch * a.ny;
    const size_t bytes = plane * planes * sizeof(float);
    // current level: u (ISO), p and q (VTI)
    const int nf = a.mode == FD_MODE_ISO ? 1 : 2;
    for (int f = 0; f < nf; ++f) {
        float *fl = lo->field[2 * f + lo->cur], *fu = up->field[2 * f + up->cur];
        CU(cudaMemcpyAsync(fu, fl + (a.nz - 2 * planes) * plane, bytes, cudaMemcpyDeviceToDevice, lo->stream),
           "ghost planes up");
        CU(cudaMemcpyAsync(fl + (a.nz - planes) * plane, fu + planes * plane, bytes, cudaMemcpyDeviceToDevice,
                           lo->stream),
           "ghost planes down");
    }
    return FD_OK;
}

int fd_debug_skip_copy(fd_grid_t *g, int plane)
{
    if (!g) {
        // the next fd_iso_step_static() on this host thread
        if (plane < 0) return fail(FD_ERR_INVALID_ARG, "plane %d is negative", plane);
        t_static_skip = plane;
        return FD_OK;
    }
    if (plane < 0 || plane >= g->d.nz) return fail(FD_ERR_INVALID_ARG, "plane %d outside 0..%d", plane, g->d.nz - 1);
    g->debug_skip = plane;
    return FD_OK;
}

int fd_time_index(fd_grid_t *g, int *n)
{
    if (!g || !n) return fail(FD_ERR_INVALID_ARG, "NULL argument");
    *n = g->n;
    return FD_OK;
}

int fd_sync(fd_grid_t *g)
{
    if (!g) return fail(FD_ERR_INVALID_ARG, "grid is NULL");
    return check_dev_status(g);
}

int fd_destroy_grid(fd_grid_t *g)
{
    if (!g) return FD_OK;
    drop_graphs(g);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->copy_stream) {
        cudaStreamSynchronize(g->copy_stream);
        cudaStreamDestroy(g->copy_stream);
    }
    for (cudaEvent_t e : g->copy_ev) cudaEventDestroy(e);
    // stream-ordered frees: after this grid's enqueued work, without a device-wide sync
    void *bufs[] = {g->st, g->gx, g->gy, g->gz, g->ztab, g->src_tab, g->rec_idx, g->d_misfit};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, g->stream);
    cudaStreamSynchronize(g->stream);
    delete g->st_host;
    delete g;
    cudaGetLastError();
    return FD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched isotropic shots: one launch per time step over every member's tiles.

struct fd_batch {
    struct Member {
        fd_grid *g;
        int n_end;
    };
    cudaStream_t stream = nullptr;
    std::vector<Member> members;
    Launch L[2];                        // radius 4, radius 8 (zchunk 0 = each member's own)
    BatchShot *d_shots = nullptr;
    size_t cap_shots = 0;
    int4 *d_items = nullptr;
    size_t cap_items = 0;
    int nitems[2] = {0, 0}, off[2] = {0, 0}, max_zc[2] = {1, 1};
    bool dirty = true;
    int graph_steps = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // radius-8 members run on a stream of their own, forked from and joined
    // back into the batch stream around every run, so the two kernels of a
    // step overlap (each fills the other's last partial wave)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // pinned host staging of the table uploads (two, used in turn)
    struct Staging {
        void *host = nullptr;
        size_t cap = 0;
        cudaEvent_t done = nullptr;
    };
    Staging stage[2];
    int next_stage = 0;
};

namespace {

int radius_slot(int R) { return R == 4 ? 0 : (R == 8 ? 1 : -1); }

void batch_drop_graph(fd_batch *b)
{
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

int batch_rebuild(fd_batch *b)
{
    const size_t ns = b->members.size();
    std::vector<BatchShot> shots(ns);
    std::vector<int4> items[2];
    for (int r = 0; r < 2; ++r) b->max_zc[r] = 1;
    for (size_t i = 0; i < ns; ++i) {
        fd_grid *g = b->members[i].g;
        const fd_desc &d = g->d;
        const int ri = radius_slot(d.r_xy), R = d.r_xy;
        const Launch &L = b->L[ri];
        BatchShot &s = shots[i];
        std::memset(static_cast<void *>(&s), 0, sizeof s);
        const long long pitch = g->lay.pitch;
        int r = 0;
        for (int k = 0; k < 2 && !r; ++k)
            r = encode_field_map(&s.halo[k], g->field[k], d.nx, d.ny, d.nz, pitch, L.tx + 2 * R, L.ty + 2 * R);
        for (int k = 0; k < 2 && !r; ++k)
            r = encode_field_map(&s.tile[k], g->field[k], d.nx, d.ny, d.nz, pitch, L.tx, L.ty);
        if (!r) r = encode_field_map(&s.kappa, g->model[0], d.nx, d.ny, d.nz, pitch, L.tx, L.ty);
        if (r) return fail(FD_ERR_CUDA, "tensor map encoding failed (%d)", r);
        s.a = iso_args(g);
        const int zc = L.zchunk > 0 ? std::min(L.zchunk, d.nz) : g->L.zchunk;
        s.a.zchunk = zc;
        s.buf[0] = g->field[0];
        s.buf[1] = g->field[1];
        s.n0 = g->n;
        s.cur0 = g->cur;
        s.n_end = b->members[i].n_end;
        const int gx = (d.nx + L.tx - 1) / L.tx, gy = (d.ny + L.ty - 1) / L.ty, gz = (d.nz + zc - 1) / zc;
        s.ncta = (unsigned)gx * gy * gz;
        s.a.ncta = s.ncta;
        b->max_zc[ri] = std::max(b->max_zc[ri], zc);
        for (int bz = 0; bz < gz; ++bz)
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) items[ri].push_back(make_int4((int)i, bx, by, bz));
    }
    const size_t nit = items[0].size() + items[1].size();
    if (nit > 0x7fffffff) return fail(FD_ERR_OUT_OF_RANGE, "batch has too many work items");
    // device tables: stream-ordered (re)allocation, so that growing them neither
    // synchronises the device nor frees a table a queued launch still reads
    if (ns > b->cap_shots) {
        if (b->d_shots) cudaFreeAsync(b->d_shots, b->stream);
        b->d_shots = nullptr;
        b->cap_shots = 0;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&b->d_shots), ns * sizeof(BatchShot), b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch descriptor allocation");
        b->cap_shots = ns;
    }
    if (nit > b->cap_items) {
        if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
        b->d_items = nullptr;
        b->cap_items = 0;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&b->d_items), std::max<size_t>(nit, 1) * sizeof(int4),
                                        b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch work-list allocation");
        b->cap_items = std::max<size_t>(nit, 1);
    }
    // Uploads from pinned staging (a pageable source would make the host wait for
    // the launches already queued), alternating between two buffers; a buffer is
    // reused once its previous upload has run.
    fd_batch::Staging &st = b->stage[b->next_stage];
    b->next_stage ^= 1;
    if (st.done) CU(cudaEventSynchronize(st.done), "staging reuse");
    else CU(cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming), "event create");
    const size_t need = ns * sizeof(BatchShot) + nit * sizeof(int4);
    if (need > st.cap) {
        if (st.host) cudaFreeHost(st.host);
        st.host = nullptr;
        st.cap = 0;
        CU(cudaMallocHost(&st.host, need), "staging allocation");
        st.cap = need;
    }
    char *hp = static_cast<char *>(st.host);
    if (ns) std::memcpy(hp, shots.data(), ns * sizeof(BatchShot));
    int4 *hi = reinterpret_cast<int4 *>(hp + ns * sizeof(BatchShot));
    if (!items[0].empty()) std::memcpy(hi, items[0].data(), items[0].size() * sizeof(int4));
    if (!items[1].empty()) std::memcpy(hi + items[0].size(), items[1].data(), items[1].size() * sizeof(int4));
    if (ns) CU(cudaMemcpyAsync(b->d_shots, hp, ns * sizeof(BatchShot), cudaMemcpyHostToDevice, b->stream),
               "batch descriptor upload");
    if (nit) CU(cudaMemcpyAsync(b->d_items, hi, nit * sizeof(int4), cudaMemcpyHostToDevice, b->stream),
                "batch work-list upload");
    CU(cudaEventRecord(st.done, b->stream), "event record");
    b->off[0] = 0;
    b->nitems[0] = (int)items[0].size();
    b->off[1] = b->nitems[0];
    b->nitems[1] = (int)items[1].size();
    // No synchronisation: the uploads are ordered on the batch stream after the
    // launches that read the previous lists (the radius-8 stream joins the batch
    // stream at the end of every run).
    b->dirty = false;
    batch_drop_graph(b);
    return FD_OK;
}

// `steps` batch steps on stream s; radius-8 members on b->side when both radii
// are present (forked from s after everything already on s, joined back).
cudaError_t batch_enqueue_steps(fd_batch *b, int steps, cudaStream_t s)
{
    const int radii[2] = {4, 8};
    const bool split = b->nitems[0] && b->nitems[1];
    cudaError_t e = cudaSuccess;
    if (split) {
        if (!b->side) {
            if ((e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        if ((e = cudaEventRecord(b->ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(b->side, b->ev_fork, 0)) != cudaSuccess) return e;
    }
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        if (!b->nitems[r]) continue;
        cudaStream_t sr = (split && r == 1) ? b->side : s;
        for (int j = 0; j < steps && e == cudaSuccess; ++j)
            e = launch_iso_batch(radii[r], b->L[r], b->d_items + b->off[r], b->nitems[r], b->d_shots,
                                 b->max_zc[r], sr);
    }
    if (split) {
        // join even after a failed launch, so that no capture is left forked
        cudaError_t e1 = cudaEventRecord(b->ev_join, b->side);
        cudaError_t e2 = cudaStreamWaitEvent(s, b->ev_join, 0);
        if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
    return e;
}

}  // namespace

extern "C" {

int fd_batch_create(void *stream, fd_batch_t **out)
{
    if (!out) return fail(FD_ERR_INVALID_ARG, "out is NULL");
    fd_batch *b = new (std::nothrow) fd_batch;
    if (!b) return fail(FD_ERR_NO_MEMORY, "host allocation failed");
    b->stream = static_cast<cudaStream_t>(stream);
    b->L[0] = Launch{64, 16, 64, 3};
    b->L[1] = Launch{32, 32, 64, 2};
    *out = b;
    return FD_OK;
}

int fd_batch_set_launch(fd_batch_t *b, int radius, int tx, int ty, int zchunk, int lookahead)
{
    if (!b) return fail(FD_ERR_INVALID_ARG, "batch is NULL");
    const int ri = radius_slot(radius);
    if (ri < 0) return fail(FD_ERR_UNSUPPORTED, "batches hold isotropic radius 4 or 8 shots");
    if (zchunk < 0 || zchunk > kMaxChunk) return fail(FD_ERR_INVALID_ARG, "z chunk 0..%d", kMaxChunk);
    Launch L{tx, ty, zchunk, lookahead};
    if (!iso_config_built(radius, L))
        return fail(FD_ERR_UNSUPPORTED, "tile %d x %d, lookahead %d is not built for radius %d", tx, ty, lookahead,
                    radius);
    b->L[ri] = L;
    b->dirty = true;
    return FD_OK;
}

int fd_batch_set_graph(fd_batch_t *b, int steps)
{
    if (!b) return fail(FD_ERR_INVALID_ARG, "batch is NULL");
    if (steps < 0 || steps > 1024) return fail(FD_ERR_INVALID_ARG, "graph steps must be 0..1024");
    batch_drop_graph(b);
    b->graph_steps = steps;
    return FD_OK;
}

int fd_batch_add(fd_batch_t *b, fd_grid_t *g, int nsteps)
{
    if (!b || !g) return fail(FD_ERR_INVALID_ARG, "NULL argument");
    if (g->d.mode != FD_MODE_ISO || radius_slot(g->d.r_xy) < 0)
        return fail(FD_ERR_UNSUPPORTED, "batches hold isotropic radius 4 or 8 shots");
    if (!g->model_set) return fail(FD_ERR_BAD_STATE, "no model: call fd_set_model first");
    if (nsteps < 0 || (long long)g->n + nsteps > 0x7fffffffLL) return fail(FD_ERR_INVALID_ARG, "bad step count");
    if (g->nrec > 0 && !g->lattice)
        return fail(FD_ERR_UNSUPPORTED, "batched shots need receivers on a lattice of one plane");
    if (g->nrec > 0 && (long long)g->n + nsteps - g->rec_t0 > g->rec_cap)
        return fail(FD_ERR_OUT_OF_RANGE, "receiver buffer too small for %d more steps", nsteps);
    if (g->inj.on) return fail(FD_ERR_UNSUPPORTED, "batched shots take no injection lattice");
    for (const auto &m : b->members)
        if (m.g == g) return fail(FD_ERR_INVALID_ARG, "grid is already in the batch");
    // the grid's own setup (tables, source, state) may sit on another stream
    if (g->stream != b->stream) CU(cudaStreamSynchronize(g->stream), "member setup");
    b->members.push_back({g, g->n + nsteps});
    b->dirty = true;
    return FD_OK;
}

int fd_batch_remove(fd_batch_t *b, fd_grid_t *g)
{
    if (!b || !g) return fail(FD_ERR_INVALID_ARG, "NULL argument");
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->members[i].g == g) {
            b->members.erase(b->members.begin() + i);
            b->dirty = true;
            return FD_OK;
        }
    return fail(FD_ERR_INVALID_ARG, "grid is not in the batch");
}

int fd_batch_steps_left(fd_batch_t *b, fd_grid_t *g, int *left)
{
    if (!b || !g || !left) return fail(FD_ERR_INVALID_ARG, "NULL argument");
    for (const auto &m : b->members)
        if (m.g == g) {
            *left = std::max(0, m.n_end - g->n);
            return FD_OK;
        }
    return fail(FD_ERR_INVALID_ARG, "grid is not in the batch");
}

int fd_batch_run(fd_batch_t *b, int max_steps, int *steps_run)
{
    if (!b) return fail(FD_ERR_INVALID_ARG, "batch is NULL");
    if (max_steps < 0) return fail(FD_ERR_INVALID_ARG, "negative step count");
    if (steps_run) *steps_run = 0;
    int need = 0;
    for (const auto &m : b->members) need = std::max(need, m.n_end - m.g->n);
    const int steps = std::min(max_steps, need);
    if (steps == 0) return FD_OK;
    if (b->dirty) {
        int rc = batch_rebuild(b);
        if (rc) return rc;
    }
    int left = steps;
    const int K = b->graph_steps;
    while (K > 0 && left >= K) {
        if (!b->gexec) {
            if (!b->cap_stream) CU(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream create");
            CU(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = batch_enqueue_steps(b, K, b->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
            if (e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(e, "batch capture");
            }
            if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
            e = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->gexec = nullptr;
                return cuda_fail(e, "graph instantiate");
            }
        }
        CU(cudaGraphLaunch(b->gexec, b->stream), "graph launch");
        left -= K;
    }
    if (left > 0) {
        cudaError_t e = batch_enqueue_steps(b, left, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    }
    for (auto &m : b->members) {
        const int adv = std::max(0, std::min(steps, m.n_end - m.g->n));
        m.g->n += adv;
        m.g->cur ^= (adv & 1);
    }
    if (steps_run) *steps_run = steps;
    return FD_OK;
}

int fd_batch_destroy(fd_batch_t *b)
{
    if (!b) return FD_OK;
    cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->side) {
        cudaStreamSynchronize(b->side);
        cudaStreamDestroy(b->side);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->d_shots) cudaFreeAsync(b->d_shots, b->stream);
    if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
    cudaStreamSynchronize(b->stream);
    for (auto &st : b->stage) {
        if (st.done) cudaEventDestroy(st.done);
        if (st.host) cudaFreeHost(st.host);
    }
    delete b;
    cudaGetLastError();
    return FD_OK;
}

}  // extern "C"
