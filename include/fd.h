/*
 * fd.h -- C ABI of the GB300 finite-difference wave-propagation library (libfd.so).
 *
 * One explicit time step of the high-order central finite-difference wave
 * equation of Medina, St-Cyr & Warburton, "High-Order Finite-differences on
 * multi-threaded architectures using OCCA" (arXiv 1410.1387):
 *   - the centred leapfrog of Sec. 1, Eq. 3:  u^{n+1} = 2u^n - u^{n-1} + dt^2 F(u^n);
 *   - F for the isotropic acoustic case: v^2 (d_xx + d_yy + d_zz) u + s(t) delta;
 *   - F for the VTI pseudo-acoustic system of Eqs. 1-2 (p, q fields, velocities
 *     nu_x = nu_z sqrt(1+2 eps), nu_n = nu_z sqrt(1+2 delta));
 *   - the symmetric x-y stencil of radius R_xy (Eq. 4) and the per-plane z
 *     stencil of radius R_z (Eq. 5, variable dz_k absorbed into the weights);
 *   - the Ricker source of Sec. 1 (f = 15 Hz in the paper), the Cerjan damping
 *     layer and the zero halo beyond the grid (Sec. 1, last paragraph);
 *   - receivers sampling the new level every step (an addition: the paper has
 *     no receivers; seismic imaging needs them).
 *
 * Conventions
 *   Every call returns an int status: FD_OK (0) or a negative FD_ERR_* code.
 *   fd_last_error() gives a message for the calling thread's last failure.
 *   No call throws, exits or aborts.  All calls are thread-compatible, not
 *   thread-safe: one grid must not be used from two threads at once.
 *
 * Layout
 *   Fields are single precision, x fastest: element (i, j, k) sits at
 *   i + pitch*(j + ny*k), pitch = fd_layout().pitch (a multiple of 32 floats,
 *   so every row starts on a 128-byte boundary).  Dense arrays passed in or
 *   out of the library (models, states) have pitch nx instead.
 *   Points outside 0..n-1 on any axis hold the value zero (the zero halo).
 *
 * Ownership
 *   The caller owns all large device memory: it allocates one device arena of
 *   fd_required_bytes() bytes (256-byte aligned) and the receiver trace buffer,
 *   and keeps both alive until fd_destroy_grid().  The library allocates only
 *   small tables (weights, damping profiles, source samples, receiver indices,
 *   a 64-byte device status block) and frees them in fd_destroy_grid().
 *   All device work is ordered on the stream given to fd_create_grid()
 *   (a cudaStream_t; NULL = the legacy default stream).  Calls that return
 *   data to the host (fd_read_receivers to host memory, fd_get_state to host
 *   memory, fd_sync, fd_set_model) synchronise that stream.
 */
#ifndef FD_H
#define FD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FD_OK                0
#define FD_ERR_INVALID_ARG  (-1)   /* bad size, radius, pointer, index, model value */
#define FD_ERR_UNSTABLE_DT  (-2)   /* dt above the leapfrog stability bound */
#define FD_ERR_OUT_OF_RANGE (-3)   /* receiver rows / steps beyond the buffers */
#define FD_ERR_BAD_STATE    (-4)   /* call out of order (e.g. step before model) */
#define FD_ERR_CUDA         (-5)   /* a CUDA runtime call failed */
#define FD_ERR_TIMEOUT      (-6)   /* a device-side bounded wait gave up */
#define FD_ERR_NO_MEMORY    (-7)   /* arena too small, or a small table allocation failed */
#define FD_ERR_UNSUPPORTED  (-8)   /* radius / mode combination not compiled in */

/* ---- enums ------------------------------------------------------------- */
#define FD_MODE_ISO    0           /* isotropic acoustic, one field u */
#define FD_MODE_VTI    1           /* VTI pseudo-acoustic, fields p and q (Eqs. 1-2) */
#define FD_PTR_HOST    0
#define FD_PTR_DEVICE  1

typedef struct fd_grid fd_grid_t;  /* opaque handle */

/* Problem description (Sec. 1: grid, spacings, radii, time step, damping). */
typedef struct fd_desc {
    int mode;             /* FD_MODE_ISO or FD_MODE_VTI */
    int nx, ny, nz;       /* points per axis, >= 1 each; the damping layer is inside */
    int r_xy;             /* x-y radius R_xy of Eq. 4: ISO 4 or 8, VTI 12 */
    int r_z;              /* z radius R_z of Eq. 5: ISO == r_xy, VTI 8 */
    double h;             /* dx = dy (> 0) */
    double dz;            /* uniform dz (> 0), used when dz_k == NULL */
    const double *dz_k;   /* VTI only, optional: nz-1 plane spacings (host; copied).
                             Ghost planes beyond the grid continue the end spacing. */
    double dt;            /* time step (> 0) */
    int sponge_width;     /* Cerjan layer width in cells on every face; 0 = none */
    double sponge_a;      /* Cerjan constant a: factor exp(-(a d)^2) per axis, d = 1..width */
} fd_desc;

/* Memory layout chosen for a description. */
typedef struct fd_layout_t {
    int pitch;            /* floats per row of every field */
    int nfields;          /* wavefield buffers: ISO 2, VTI 4 */
    int nmodel;           /* model buffers: ISO 1 (kappa), VTI 3 (kappa_x, kappa_n, kappa_z) */
    size_t field_bytes;   /* bytes of one field buffer (pitch*ny*nz*4, rounded to 256) */
    size_t arena_bytes;   /* (nfields + nmodel) * field_bytes */
} fd_layout_t;

/* Bytes of device arena that fd_create_grid() needs for d.  Pure host call. */
int fd_required_bytes(const fd_desc *d, size_t *bytes);

/* Pitch and buffer split for d.  Pure host call. */
int fd_layout(const fd_desc *d, fd_layout_t *out);

/*
 * Largest stable dt for d with maximum velocity vmax (ISO: v; VTI: nu_z) and,
 * for VTI, the maximum eps.  The bound is (v dt)^2 * rho <= 4 with rho the
 * Gershgorin bound of the discrete operator's spectrum (exact for uniform
 * spacing: rho = 2 sigma_xy / h^2 + sigma_z / dz^2, sigma = the stencil's
 * symbol at the Nyquist frequency).  d->dt is ignored.  Pure host call.
 */
int fd_stability_limit(const fd_desc *d, double vmax, double eps_max, double *dt_max);

/*
 * Create a grid on `arena` (device memory of at least fd_required_bytes(d),
 * 256-byte aligned, owned by the caller) ordered on `stream` (cudaStream_t).
 * Zero-fills the wavefields (u^0 = u^{-1} = 0, the paper's quiescent start)
 * and uploads the weight and damping tables.  The current CUDA device must be
 * the one that owns the arena.  Time index starts at 0.
 */
int fd_create_grid(const fd_desc *d, void *arena, size_t arena_bytes, void *stream,
                   fd_grid_t **out);

/*
 * Set the model from dense nz x ny x nx float arrays (pitch nx), host or
 * device per ptr_kind.  ISO: vz = velocity, eps = delta = NULL.  VTI: vz =
 * nu_z, eps, delta = Thomsen parameters (Sec. 1).  Stores kappa = (v dt)^2
 * (VTI: kappa_z = (nu_z dt)^2, kappa_x = kappa_z (1+2 eps), kappa_n =
 * kappa_z (1+2 delta)), computed in double and rounded to float.
 * Errors: FD_ERR_INVALID_ARG for a non-finite or non-positive velocity, or
 * (VTI) eps < delta somewhere (the operator is unstable there: the paper's
 * "eps - delta <= 0" is read as eps >= delta) or 1 + 2 delta <= 0;
 * FD_ERR_UNSTABLE_DT when dt exceeds fd_stability_limit() for the model's
 * maxima.  On error the grid has no model.  Synchronises the stream.
 */
int fd_set_model(fd_grid_t *g, const float *vz, const float *eps, const float *delta,
                 int ptr_kind);

/*
 * Stencil weights.  By default a grid uses the maximal-order (Taylor) weights
 * of Eq. 4, c_l = 2 (-1)^{l+1} (R!)^2 / (l^2 (R-l)! (R+l)!), c_0 = -2 sum c_l,
 * and the per-plane Eq. 5 weights in z.  Sec. 1 notes that the weights can be
 * optimised instead (after Holberg 1987; the paper gives no method or values).
 *
 * fd_optimized_weights writes radius + 1 band-optimised weights c_0..c_R of
 * the unit-grid second derivative (the stencil c_0 u_0 + sum c_l (u_l + u_-l)):
 * exact on quadratics (sum l^2 c_l = 1, c_0 = -2 sum c_l) and, among those,
 * the least-squares minimum of the relative symbol error
 *   int_0^kmax (4 sum_l c_l sin^2(l k / 2) / k^2 - 1)^2 dk,
 * so the numerical phase velocity stays closest to the true one for
 * wavenumbers k h <= kmax.  1 <= radius <= 12, 0 < kmax <= pi.  Pure host call.
 *
 * fd_set_weights installs unit-grid weights (radius + 1 doubles, in units of
 * 1/h^2 and 1/dz^2) for the x-y stencil and, with a uniform dz, the z stencil;
 * NULL keeps the current ones.  They must be exact on constants and quadratics
 * (FD_ERR_INVALID_ARG otherwise); z weights on a grid with dz_k return
 * FD_ERR_UNSUPPORTED.  Call it before fd_set_model (FD_ERR_BAD_STATE after),
 * whose stability check uses the installed weights; fd_stability_limit()
 * assumes the default ones.
 */
int fd_optimized_weights(int radius, double kmax, double *weights);
int fd_set_weights(fd_grid_t *g, const double *w_xy, const double *w_z);

/*
 * Ricker point source (Sec. 1) at cell (ix, iy, iz): step n adds
 *   dt^2 * amp * s(n dt - t0) / V,  s(t) = (1 - 2 pi^2 f^2 t^2) exp(-pi^2 f^2 t^2),
 * to the new level of p (ISO: u), and of q too when inject_q != 0 (VTI only).
 * V = h*h*dz (VTI with dz_k: h*h times the mean of the two spacings beside iz).
 * A grid has one source; a second call replaces it.
 */
int fd_add_source(fd_grid_t *g, int ix, int iy, int iz, double freq_hz, double t0, double amp,
                  int inject_q);

/* As fd_add_source() with an arbitrary wavelet: step n adds dt^2 * s[n] / V
   for n < nt (host array, copied), nothing after. */
int fd_add_source_series(fd_grid_t *g, int ix, int iy, int iz, const float *s, int nt,
                         int inject_q);

/*
 * Receivers at cells idx_xyz[3r..3r+2] (host ints, copied), r < nrec.  After
 * the step that makes level n+1, trace_dev[(n - n_set) * nrec + r] = p^{n+1}
 * (ISO: u^{n+1}) at receiver r, where n_set is the time index at this call.
 * trace_dev is device memory of nt_cap * nrec floats owned by the caller.
 * A set that is a row-major lattice on one z plane is sampled inside the
 * stencil kernel; any other set by a small gather kernel after each step.
 * nrec = 0 removes the receivers.
 */
int fd_set_receivers(fd_grid_t *g, const int *idx_xyz, int nrec, float *trace_dev, int nt_cap);

/* One time step (Eq. 3): enqueue one stencil launch.  FD_ERR_BAD_STATE without
   a model; FD_ERR_OUT_OF_RANGE if the receiver buffer is full. */
int fd_step(fd_grid_t *g);

/* nsteps time steps (one launch each, or replays of a captured CUDA graph, see
   fd_set_graph).  Checks all of them against the receiver buffer first. */
int fd_run(fd_grid_t *g, int nsteps);

/* One time step of g's operator (Eq. 3) between caller-owned levels: reads u^n
   from cur and the stored older level from prev, writes u^{n+1} to out (device
   arrays in g's pitched layout, 16-byte aligned; out may be prev -- the
   in-place step -- but not cur).  g's model, damping layer, source and
   receivers apply at g's time index, which advances; g's own levels are left
   as they are.  Isotropic grids.  Lets a caller keep a run of consecutive
   levels without copying them (the adjoint's recomputed segments).  Tensor
   maps of these buffers are cached on g (by address). */
int fd_step_from(fd_grid_t *g, const float *cur, const float *prev, float *out);

/* Use replays of a CUDA graph of `steps` launches (even, 2..1024) in fd_run;
   0 = plain launches (the default). */
int fd_set_graph(fd_grid_t *g, int steps);

/*
 * Copy receiver rows [t_begin, t_begin + t_count) (row m = step n_set + m) to
 * dst (t_count * nrec floats, host or device per dst_kind).  Host copies
 * synchronise the stream and report device-side errors.  FD_ERR_OUT_OF_RANGE
 * for rows not written yet.
 */
int fd_read_receivers(fd_grid_t *g, int t_begin, int t_count, float *dst, int dst_kind);

/*
 * nsteps time steps, as fd_run, with their receiver rows streamed to the host
 * while later steps compute: host_dst receives nsteps * nrec floats, row m
 * holding step n_call + m (n_call = the time index at this call; receiver
 * order as in fd_set_receivers).  The steps run in chunks of chunk_steps
 * (0 = 64; at least nsteps / 256; rounded up to whole graphs when fd_set_graph
 * is on); each chunk's rows are copied on a stream of the grid's own once the
 * chunk's steps are done.  host_dst belongs to the caller and should be pinned
 * (cudaHostAlloc or registered) for the copies to run asynchronously; pageable
 * memory works, its copies staged by the host.  Returns after the last row has
 * arrived and the device status has been read (FD_ERR_TIMEOUT as fd_sync);
 * it synchronises, so it is not to be called while the grid's stream is being
 * captured into a graph.
 * FD_ERR_BAD_STATE without receivers or a model; FD_ERR_OUT_OF_RANGE if the
 * receiver buffer cannot hold the steps (nothing is enqueued then).  The paper
 * records no receivers; this is the host side of the fused receiver lattice.
 */
int fd_run_to_host(fd_grid_t *g, int nsteps, float *host_dst, int chunk_steps);

/*
 * Copy the stored state out as dense nz x ny x nx arrays (any pointer may be
 * NULL).  cur = u^n (VTI: p^n), prev = the stored older level, q_cur / q_prev
 * the same for q (VTI).  The older level is stored before its second damping
 * factor: with the Cerjan layer, the physical u^{n-1} is G * prev (G = 1
 * outside the layer), which is how the sweep applies both factors in one pass.
 * *time_index (may be NULL) receives n.  Synchronises for host destinations.
 */
int fd_get_state(fd_grid_t *g, float *cur, float *prev, float *q_cur, float *q_prev,
                 int ptr_kind, int *time_index);

/* Overwrite the stored state from dense arrays (same convention as
   fd_get_state; NULL = leave that level unchanged) and set the time index. */
int fd_set_state(fd_grid_t *g, const float *cur, const float *prev, const float *q_cur,
                 const float *q_prev, int ptr_kind, int time_index);

/* Device pointer and pitch of a stored level: which = 0 cur, 1 prev,
   2 q_cur, 3 q_prev (VTI).  Valid until the next step. */
int fd_field(fd_grid_t *g, int which, float **dev_ptr, int *pitch);

/*
 * Tile and pipeline of the stencil kernel (a tuning knob; results do not
 * depend on it).  tx x ty points per CTA (tx a multiple of 4), zchunk planes
 * per CTA, `lookahead` staged planes in flight.  A (tx, ty, lookahead)
 * combination that is not built into the library returns FD_ERR_UNSUPPORTED
 * and leaves the previous configuration in place.  Built: isotropic radius 4:
 * 64 x 16 (lookahead 2, 3, 4), 64 x 8, 128 x 8, 32 x 16 (lookahead 3),
 * 32 x 32 (lookahead 2, 3); radius 8: 64 x 8 (lookahead 2, 3), 32 x 16,
 * 32 x 32 (lookahead 2); VTI (12, 8): 64 x 8 (lookahead 2, 3), 32 x 16,
 * 32 x 32 (lookahead 2).  32 x 32 tiles keep the z queues in tensor memory.
 * A new grid starts with 32 x 32, lookahead 3 (isotropic radius 4; 64 x 16,
 * lookahead 3 on a grid too small to fill the GPU with 32 x 32 CTAs), 32 x 32,
 * lookahead 2 (radius 8; VTI at R_z = 8) or 64 x 8, lookahead 2 (other VTI
 * radii), and a z chunk fitted to whole waves of the CTAs the GPU holds at
 * once: 32-96 planes (isotropic), 32-64 (VTI).
 */
int fd_set_launch(fd_grid_t *g, int tx, int ty, int zchunk, int lookahead);

/*
 * Failure-detection test hook: in the next step (run outside any graph), the
 * sweep's CTA (0,0,0) withholds the copy of plane `plane` of u^n (VTI: p^n), a
 * plane inside its z chunk.  Its consumers' bounded wait (about
 * one second) runs out; the CTA records the timeout in the grid's status
 * block, waits (bounded) for its copies in flight and exits, and the next
 * fd_sync / host read-back returns FD_ERR_TIMEOUT.  The context stays usable;
 * the grid's results are then undefined and its status stays failed.  With
 * g == NULL the hook applies to the next fd_iso_step_static() call made on the
 * calling host thread (plane checked against that call's grid).  Not for
 * production use.
 */
int fd_debug_skip_copy(fd_grid_t *g, int plane);

/* Current time index n (host-side count of enqueued steps). */
int fd_time_index(fd_grid_t *g, int *n);

/* Wait for the grid's stream; FD_ERR_TIMEOUT if a kernel's bounded wait gave up. */
int fd_sync(fd_grid_t *g);

/* Release the grid and its small tables (not the caller's arena or traces). */
int fd_destroy_grid(fd_grid_t *g);

/* Copy the calling thread's last error message into buf (always terminated). */
int fd_last_error(char *buf, size_t n);

/* ---- z slabs of one shot ------------------------------------------------------
 * One grid (Sec. 1) cut along z into slabs, each a grid of its own (all on one
 * GPU, or one per GPU), stored with P >= R ghost planes (VTI: R_z) on every
 * side that has a neighbour: slab s owns planes [a_s, b_s) and stores
 * [a_s - P, b_s + P) clipped to the column.  A step only reads points within R
 * of the point it updates, so after every step it suffices to replace the
 * ghost planes of the new level by the neighbours' planes there; the interior
 * of every slab then holds, bit for bit, the values of the unsplit grid.  The
 * source and the receivers go to the slab that owns their plane (local
 * indices).  An extension for shots larger than one GPU: the paper runs one
 * grid per device.
 */

/* Declare that local plane k of g is plane kg0 + k of a column of nz_global
   planes, so that the damping layer along z follows the column rather than
   the slab.  Uniform dz only (FD_ERR_UNSUPPORTED when the grid has dz_k).
   Invalidates g's step graphs; call it before g joins a batch. */
int fd_set_z_window(fd_grid_t *g, int kg0, int nz_global);

/* Ghost-plane exchange between the z-neighbours `lower` and `upper` on one
   device: copies the current level (ISO: u; VTI: p and q) of lower's planes
   [nz_l - 2P, nz_l - P) to upper's [0, P) and upper's [P, 2P) to lower's
   [nz_l - P, nz_l), P = planes.  Requires P >= the z radius, z windows that
   overlap by 2P planes (upper's kg0 = lower's kg0 + nz_l - 2P), equal mode,
   radii, nx, ny and time index, and one stream for both grids (the copies are
   asynchronous on it).  Across GPUs the same planes travel point to point
   between ranks instead. */
int fd_halo_exchange(fd_grid_t *lower, fd_grid_t *upper, int planes);

/* Part of one time step (Eq. 3 at planes [k_begin, k_end) only; every point
   still reads u^n within R of it, ghost planes included).  A step may be
   enqueued as several parts on g's stream, each plane in at most one part;
   the part with complete != 0 comes last: it advances the time index, samples
   gathered receivers and makes the new level current.  Planes no part covers
   keep their older stored value -- a slab's ghost planes, which the exchange
   then overwrites.  This lets a slab update the planes its neighbours need
   first, start their exchange, and update its interior while the planes are
   in flight.  Parts run outside any CUDA graph.  FD_ERR_INVALID_ARG for an
   empty or out-of-range range; otherwise as fd_step. */
int fd_step_planes(fd_grid_t *g, int k_begin, int k_end, int complete);

/* ---- adjoint and velocity gradient -----------------------------------------
 * For J = 1/2 sum_n sum_r (u^{n+1}(x_r) - dobs[n][r])^2 of an isotropic run
 * (an extension: the paper computes no gradients; its use is imaging).  The
 * step of fd_step is x_{n+1} = A x_n + f_n on the stored pair (u^n, u_prev)
 * with A = [[G (2 + K L), -G^2], [1, 0]], K = (v dt)^2.  Its transpose,
 * written for z = K G alpha (alpha the adjoint of u), is the same step run
 * backward in time:
 *   z_n = G (2 z_{n+1} - G z_{n+2} + K L z_{n+1} + K R^T r_{n-1}),
 * i.e. fd_step on a second grid with the residuals injected at the receivers,
 * and dJ/dv = sum_n 2 dt z_{n+1} (L u^n) / sqrt(K).
 */

/* Additive sources on a lattice (one z plane, row-major, constant strides):
   at step n, point r gets values_dev[(n - n_set) * nrec + r] added inside the
   damping bracket (like the Ricker source).  values_dev: device, nt_cap rows,
   owned by the caller.  nrec = 0 removes them.  Isotropic grids only. */
int fd_set_injection(fd_grid_t *g, const int *idx_xyz, int nrec, const float *values_dev, int nt_cap);

/* From device traces and data (nt x nrec, row n = step n, g's receiver lattice):
   inj[m][r] = K(x_r) (traces - dobs)[nt-1-m][r] (device, nt x nrec; the
   adjoint run's injection rows) and *misfit = J (host; synchronises). */
int fd_adjoint_source(fd_grid_t *g, const float *traces, const float *dobs, int nt, float *inj,
                      double *misfit);

/* grad += 2 dt z (L a) / sqrt(K) over g's grid; z, a, grad are device arrays
   in g's pitched layout (fd_layout), 16-byte aligned (FD_ERR_INVALID_ARG
   otherwise).  Asynchronous on g's stream. */
int fd_grad_accumulate(fd_grid_t *g, const float *z, const float *a, float *grad);

/* ---- batched shots --------------------------------------------------------
 * Many independent isotropic shots (radius 4 or 8, any sizes and step counts)
 * advanced together: each launch performs one time step (Eq. 3, exactly the
 * arithmetic of fd_step) of every member shot, its CTAs drawn from one work
 * list of (shot, tile, z chunk) items, so that small grids share the GPU
 * instead of each leaving most SMs idle.  Each member keeps its own buffers,
 * model, source and receivers (a receiver set must be a lattice on one plane).
 * A shot's own time index picks its current buffer on the device, so a CUDA
 * graph of several batch launches replays without per-step arguments; members
 * that have run their steps skip their items.  An extension of the paper's
 * single-shot step for seismic surveys (many shots per model).
 */
typedef struct fd_batch fd_batch_t;

/* New empty batch ordered on `stream` (the member grids' work must be ordered
   before it by the caller, e.g. by using the same stream). */
int fd_batch_create(void *stream, fd_batch_t **out);

/* Tile (tx x ty, lookahead) and z chunk used for members of the given radius;
   zchunk 0 = each member grid's own (fd_set_launch).  Defaults: radius 4:
   64 x 16, 64 planes, lookahead 3; radius 8: 32 x 32, 64 planes, lookahead 2. */
int fd_batch_set_launch(fd_batch_t *b, int radius, int tx, int ty, int zchunk, int lookahead);

/* Replay CUDA graphs of `steps` batch launches in fd_batch_run (0 = plain launches). */
int fd_batch_set_graph(fd_batch_t *b, int steps);

/* Add grid g (isotropic, model set) to run `nsteps` more steps in the batch.
   If g uses another stream, that stream is synchronised first so that its
   setup precedes the batch launches.  The grid stays owned by the caller and
   must outlive every batch launch enqueued while it was a member. */
int fd_batch_add(fd_batch_t *b, fd_grid_t *g, int nsteps);

/* Detach g (finished, or cancelled between runs). */
int fd_batch_remove(fd_batch_t *b, fd_grid_t *g);

/* Steps g still has to run in the batch. */
int fd_batch_steps_left(fd_batch_t *b, fd_grid_t *g, int *left);

/* Up to max_steps batch launches, fewer when every member is done;
   *steps_run (may be NULL) receives the number of launches. */
int fd_batch_run(fd_batch_t *b, int max_steps, int *steps_run);

/* Release the batch (not its member grids). */
int fd_batch_destroy(fd_batch_t *b);

/*
 * One isotropic step that allocates no device memory.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc -- a serving
 * process whose own pool allocator owns all device memory, or a
 * latency-critical loop that cannot take the device-wide synchronisation that
 * cudaMalloc / cudaFree may cause -- and so cannot use fd_create_grid().
 *
 * Same arithmetic and kernel as fd_step() on an isotropic grid, and the same
 * results bit for bit: u_prev holds the stored older level on entry and
 * u^{n+1} on return (in place), u_cur is u^n, kappa = (v dt)^2; all three are
 * device arrays in the pitched layout of fd_layout(d) (16-byte aligned), owned
 * by the caller.  n is the time index of u_cur and selects the Ricker sample
 * s(n dt - t0) of the source at (src_ix, src_iy, src_iz); src_ix < 0 means no
 * source.  No receivers.  status (optional, device memory owned by the caller,
 * NULL to skip) receives FD_OK, or FD_ERR_TIMEOUT when a bounded device wait
 * of the sweep ran out (the step's output is then undefined); it is written
 * on `stream` after the sweep.  Asynchronous on `stream`: the call enqueues
 * kernels only and makes the host wait for nothing.
 *
 * Its scratch (status block, damping profiles, source sample) lives in a
 * fixed __device__ array of about 97 KiB that every GPU loading the library
 * holds until exit.  Grids with an axis above FD_STATIC_MAX_AXIS points, or a
 * damping layer wider than FD_STATIC_MAX_SPONGE cells, are rejected with
 * FD_ERR_OUT_OF_RANGE.  Every call rewrites that array on its stream, so
 * calls that may overlap on the GPU (different streams or host threads
 * without ordering) race; the first call on a device looks up the array's
 * address and should come before any stream capture on that device.
 * fd_debug_skip_copy(NULL, plane) arms the failure-detection hook for the next
 * call made on the same host thread.
 */
#define FD_STATIC_MAX_AXIS 8192
#define FD_STATIC_MAX_SPONGE 512
int fd_iso_step_static(const fd_desc *d, const float *u_cur, float *u_prev, const float *kappa,
                       int n, int src_ix, int src_iy, int src_iz, double freq_hz, double t0,
                       double amp, int *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FD_H */
