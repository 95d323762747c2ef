/*
 * FP64 CPU oracle for the high-order finite-difference wave propagator of
 * Medina, St-Cyr & Warburton, "High-Order Finite-differences on multi-threaded
 * architectures using OCCA" (arXiv 1410.1387).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * legs of the benchmark are the only callers.  The CUDA library neither links
 * nor calls this file and shares no code with it (its weights, sponge, source
 * and stepping are written separately there).
 *
 * Everything is written the slow, obvious way: double precision, plain loops,
 * a bounds test for every neighbour (values outside the grid are zero: the zero
 * halo of Sec. 1), OpenMP over z planes only.  Fields are dense nx*ny*nz
 * arrays, x fastest, index i + nx*(j + ny*k).
 *
 * Pins (tests/test_oracle_*.py): weight moments and textbook values, polynomial
 * exactness, the plane-wave dispersion relation, discrete energy conservation,
 * a dense-matrix brute force, the VTI -> isotropic reduction, the leapfrog
 * stability boundary, and closed forms for the source and the sponge.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Stencil weights                                                           */
/* ------------------------------------------------------------------------ */

/*
 * Central second-derivative weights of order 2R on a uniform unit grid
 * (the symmetric x-y stencil of Eq. 4, read as the maximal-order Taylor
 * stencil because the paper prints no weights):
 *   c_l = 2 (-1)^(l+1) (R!)^2 / (l^2 (R-l)! (R+l)!),  l = 1..R
 *   c_0 = -2 sum_l c_l.
 * The factorial ratio is formed as prod_{m=1..l} (R-l+m)/(R+m).
 * Returns 0, or -1 for R outside 1..32.
 */
int or_taylor_weights(int R, double *c)
{
    if (R < 1 || R > 32) return -1;
    double sum = 0.0;
    for (int l = 1; l <= R; ++l) {
        double ratio = 1.0;
        for (int m = 1; m <= l; ++m) ratio *= (double)(R - l + m) / (double)(R + m);
        double sign = (l % 2 == 1) ? 1.0 : -1.0;
        c[l] = 2.0 * sign * ratio / ((double)l * (double)l);
        sum += c[l];
    }
    c[0] = -2.0 * sum;
    return 0;
}

/*
 * Second-derivative weights at node z[k] from the n nodes z[0..n-1]: the
 * second derivative of the Lagrange interpolant, w_j = L_j''(z[k]) with
 *   L_j(x) = prod_{m != j} (x - z[m]) / (z[j] - z[m]).
 * The second derivative of a product of n-1 linear factors is the sum over
 * ordered pairs (a, b), a != b, of the product of the other factors.
 * This is the variable-spacing z stencil of Eq. 5, with dz absorbed.
 */
int or_lagrange_d2(const double *z, int n, int k, double *w)
{
    if (n < 3 || k < 0 || k >= n) return -1;
    double x = z[k];
    for (int j = 0; j < n; ++j) {
        double denom = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != j) denom *= (z[j] - z[m]);
        double num = 0.0;
        for (int a = 0; a < n; ++a) {
            if (a == j) continue;
            for (int b = 0; b < n; ++b) {
                if (b == j || b == a) continue;
                double prod = 1.0;
                for (int m = 0; m < n; ++m)
                    if (m != j && m != a && m != b) prod *= (x - z[m]);
                num += prod;
            }
        }
        w[j] = num / denom;
    }
    return 0;
}

/*
 * Node coordinates of plane k (any integer, ghosts included).  Planes are
 * z_0 = 0, z_{k+1} = z_k + dzk[k] for k = 0..nz-2; ghost planes continue with
 * the spacing of the nearest interior interval.  dzk == NULL means uniform dz.
 */
static double or_zcoord(int nz, const double *dzk, double dz, int k)
{
    if (dzk == NULL || nz < 2) return dz * (double)k;
    if (k <= 0) return dzk[0] * (double)k;
    double z = 0.0;
    int kin = k < nz - 1 ? k : nz - 1;
    for (int m = 0; m < kin; ++m) z += dzk[m];
    if (k > nz - 1) z += dzk[nz - 2] * (double)(k - (nz - 1));
    return z;
}

/*
 * Per-plane z weights of Eq. 5: tab[k*(2Rz+1) + (l+Rz)] is the weight of
 * plane k+l in the second z derivative at plane k, l = -Rz..Rz.
 */
int or_z_table(int nz, int Rz, const double *dzk, double dz, double *tab)
{
    if (nz < 1 || Rz < 1 || Rz > 32) return -1;
    int n = 2 * Rz + 1;
    double *zn = (double *)malloc(sizeof(double) * (size_t)n);
    if (!zn) return -2;
    for (int k = 0; k < nz; ++k) {
        for (int l = -Rz; l <= Rz; ++l) zn[l + Rz] = or_zcoord(nz, dzk, dz, k + l);
        or_lagrange_d2(zn, n, Rz, tab + (size_t)k * (size_t)n);
    }
    free(zn);
    return 0;
}

/*
 * Symbol of the 1D second-difference stencil at the grid Nyquist frequency,
 * sigma_R = -(c_0 + 2 sum_l (-1)^l c_l), on a unit grid.  It is the largest
 * eigenvalue magnitude of the 1D operator on an infinite grid.
 */
double or_nyquist_symbol(int R)
{
    double c[33];
    if (or_taylor_weights(R, c) != 0) return -1.0;
    double s = c[0];
    for (int l = 1; l <= R; ++l) s += 2.0 * ((l % 2 == 0) ? 1.0 : -1.0) * c[l];
    return -s;
}

/*
 * Largest stable Courant number v*dt/h of the isotropic 3D leapfrog scheme
 * (Eq. 3) with h = dx = dy = dz: the leapfrog recurrence is stable while
 * (v dt)^2 * lambda_max(-L) <= 4, and lambda_max(-L) = 3 sigma_R / h^2.
 */
double or_iso_courant_limit(int R)
{
    double s = or_nyquist_symbol(R);
    if (s <= 0.0) return -1.0;
    return 2.0 / sqrt(3.0 * s);
}

/* ------------------------------------------------------------------------ */
/* Source and sponge                                                         */
/* ------------------------------------------------------------------------ */

/* Ricker wavelet of Sec. 1: s(t) = (1 - 2 pi^2 f^2 t^2) exp(-pi^2 f^2 t^2). */
double or_ricker(double t, double f)
{
    double a = OR_PI * OR_PI * f * f * t * t;
    return (1.0 - 2.0 * a) * exp(-a);
}

/*
 * Cerjan damping factor along one axis (reading of Sec. 1's damping layer):
 * d = number of cells into the layer counted from its inner edge (1..nb at
 * the nb outermost cells of each end, 0 elsewhere), factor exp(-(a d)^2).
 */
double or_sponge_axis(int i, int n, int nb, double a)
{
    int d = 0;
    if (nb <= 0) return 1.0;
    if (i < nb) d = nb - i;
    else if (i >= n - nb) d = i - (n - nb - 1);
    double ad = a * (double)d;
    return exp(-ad * ad);
}

/* ------------------------------------------------------------------------ */
/* Operators                                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;       /* grid points per axis; the damping layer is inside */
    int r_xy, r_z;        /* stencil radii; the isotropic case uses r_xy == r_z */
    double h;             /* dx = dy */
    double dz;            /* uniform dz, used when ztab == NULL */
    const double *ztab;   /* optional nz*(2 r_z + 1) z weights (or_z_table) */
    double dt;            /* time step */
    int nb;               /* damping-layer width in cells, 0 = none */
    double sponge_a;      /* damping constant a */
    int src_on;           /* 1: inject the Ricker source */
    int sx, sy, sz;       /* source cell */
    double src_f, src_t0, src_amp;
    int src_into_q;       /* VTI: inject into q as well as p */
    double src_volume;    /* cell volume dividing the point source */
    int nrec;             /* receivers */
    const int *rec;       /* 3*nrec cell indices (ix, iy, iz) */
    const double *cxy;    /* optional r_xy+1 unit-grid weights c_0..c_R along x and y (NULL: Taylor) */
    const double *cz;     /* optional r_z+1 unit-grid weights along z for a uniform dz (NULL: Taylor) */
} or_cfg;

/* The weights a run uses: the caller's (cxy, cz) where given, else Taylor's. */
static int stencil_weights(const or_cfg *c, double *cw, double *cz)
{
    if (c->cxy) {
        for (int l = 0; l <= c->r_xy; ++l) cw[l] = c->cxy[l];
    } else if (or_taylor_weights(c->r_xy, cw)) {
        return -1;
    }
    if (c->cz) {
        for (int l = 0; l <= c->r_z; ++l) cz[l] = c->cz[l];
    } else if (or_taylor_weights(c->r_z, cz)) {
        return -1;
    }
    return 0;
}

static inline double at(const double *u, const or_cfg *c, int i, int j, int k)
{
    if (i < 0 || i >= c->nx || j < 0 || j >= c->ny || k < 0 || k >= c->nz) return 0.0;
    return u[(size_t)i + (size_t)c->nx * ((size_t)j + (size_t)c->ny * (size_t)k)];
}

static inline size_t idx(const or_cfg *c, int i, int j, int k)
{
    return (size_t)i + (size_t)c->nx * ((size_t)j + (size_t)c->ny * (size_t)k);
}

/* Horizontal part of Eq. 4 divided by h^2, radius r_xy: (d_xx + d_yy) u. */
static double op_h(const or_cfg *c, const double *cw, const double *u, int i, int j, int k)
{
    double s = 2.0 * cw[0] * at(u, c, i, j, k);
    for (int l = 1; l <= c->r_xy; ++l)
        s += cw[l] * (at(u, c, i + l, j, k) + at(u, c, i - l, j, k) +
                      at(u, c, i, j + l, k) + at(u, c, i, j - l, k));
    return s / (c->h * c->h);
}

/* Vertical second derivative of Eq. 5, radius r_z. */
static double op_z(const or_cfg *c, const double *cz, const double *u, int i, int j, int k)
{
    double s = 0.0;
    if (c->ztab) {
        const double *w = c->ztab + (size_t)k * (size_t)(2 * c->r_z + 1);
        for (int l = -c->r_z; l <= c->r_z; ++l) s += w[l + c->r_z] * at(u, c, i, j, k + l);
        return s;
    }
    s = cz[0] * at(u, c, i, j, k);
    for (int l = 1; l <= c->r_z; ++l) s += cz[l] * (at(u, c, i, j, k + l) + at(u, c, i, j, k - l));
    return s / (c->dz * c->dz);
}

/* Isotropic Laplacian L u = (d_xx + d_yy + d_zz) u, zero outside the grid. */
int or_iso_laplacian(const or_cfg *c, const double *u, double *Lu)
{
    double cw[33], cz[33];
    if (stencil_weights(c, cw, cz)) return -1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i)
                Lu[idx(c, i, j, k)] = op_h(c, cw, u, i, j, k) + op_z(c, cz, u, i, j, k);
    return 0;
}

/* The two VTI operators: Hp = (d_xx + d_yy) p (Eq. 4), Dq = d_zz q (Eq. 5). */
int or_vti_operators(const or_cfg *c, const double *p, const double *q, double *Hp, double *Dq)
{
    double cw[33], cz[33];
    if (stencil_weights(c, cw, cz)) return -1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                Hp[idx(c, i, j, k)] = op_h(c, cw, p, i, j, k);
                Dq[idx(c, i, j, k)] = op_z(c, cz, q, i, j, k);
            }
    return 0;
}

static double sponge_at(const or_cfg *c, int i, int j, int k)
{
    return or_sponge_axis(i, c->nx, c->nb, c->sponge_a) *
           or_sponge_axis(j, c->ny, c->nb, c->sponge_a) *
           or_sponge_axis(k, c->nz, c->nb, c->sponge_a);
}

/* Source term added to the new level of step n: dt^2 * amp * s(n dt - t0) / V. */
static double source_term(const or_cfg *c, int n)
{
    double s = c->src_amp * or_ricker((double)n * c->dt - c->src_t0, c->src_f);
    return c->dt * c->dt * s / c->src_volume;
}

/* ------------------------------------------------------------------------ */
/* Time stepping                                                             */
/* ------------------------------------------------------------------------ */

/*
 * Isotropic leapfrog (Eq. 3 with F = v^2 L u + s delta):
 *   u^{n+1} = 2 u^n - u^{n-1} + (v dt)^2 L u^n + dt^2 s(t^n) delta_h,
 * then the Cerjan layer multiplies both u^{n+1} and u^n by G.
 * u holds u^{n0}, uprev u^{n0-1} (true values); both are advanced by nsteps.
 * traces (nsteps x nrec, may be NULL) receives u^{n+1} at the receivers.
 */
int or_iso_run(const or_cfg *c, const double *v, double *u, double *uprev,
               int n0, int nsteps, double *traces)
{
    double cw[33], cz[33];
    if (stencil_weights(c, cw, cz)) return -1;
    size_t N = (size_t)c->nx * (size_t)c->ny * (size_t)c->nz;
    double *un = (double *)malloc(sizeof(double) * (N ? N : 1));
    double *cur = (double *)malloc(sizeof(double) * (N ? N : 1));
    double *prv = (double *)malloc(sizeof(double) * (N ? N : 1));
    if (!un || !cur || !prv) { free(un); free(cur); free(prv); return -2; }
    memcpy(cur, u, sizeof(double) * N);
    memcpy(prv, uprev, sizeof(double) * N);

    for (int s = 0; s < nsteps; ++s) {
        int n = n0 + s;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    size_t p = idx(c, i, j, k);
                    double kappa = v[p] * c->dt * v[p] * c->dt;
                    double Lu = op_h(c, cw, cur, i, j, k) + op_z(c, cz, cur, i, j, k);
                    un[p] = 2.0 * cur[p] - prv[p] + kappa * Lu;
                }
        if (c->src_on) un[idx(c, c->sx, c->sy, c->sz)] += source_term(c, n);
        if (c->nb > 0) {
#pragma omp parallel for schedule(static)
            for (int k = 0; k < c->nz; ++k)
                for (int j = 0; j < c->ny; ++j)
                    for (int i = 0; i < c->nx; ++i) {
                        double g = sponge_at(c, i, j, k);
                        un[idx(c, i, j, k)] *= g;
                        cur[idx(c, i, j, k)] *= g;
                    }
        }
        if (traces)
            for (int r = 0; r < c->nrec; ++r)
                traces[(size_t)s * (size_t)c->nrec + (size_t)r] =
                    un[idx(c, c->rec[3 * r], c->rec[3 * r + 1], c->rec[3 * r + 2])];
        double *t = prv; prv = cur; cur = un; un = t;
    }
    memcpy(u, cur, sizeof(double) * N);
    memcpy(uprev, prv, sizeof(double) * N);
    free(un); free(cur); free(prv);
    return 0;
}

/*
 * VTI leapfrog (Eqs. 1-3): with kx = vz^2 (1+2 eps) dt^2, kn = vz^2 (1+2 delta) dt^2,
 * kz = vz^2 dt^2 (Sec. 1's nu_x, nu_n, nu_z),
 *   p^{n+1} = 2p^n - p^{n-1} + kx Hp^n + kz Dq^n + dt^2 s delta_h
 *   q^{n+1} = 2q^n - q^{n-1} + kn Hp^n + kz Dq^n   (+ the source if src_into_q)
 * then the Cerjan layer multiplies both time levels of p and q by G.
 * traces receive p^{n+1}.
 */
int or_vti_run(const or_cfg *c, const double *vz, const double *eps, const double *delta,
               double *p, double *pprev, double *q, double *qprev,
               int n0, int nsteps, double *traces)
{
    double cw[33], cz[33];
    if (stencil_weights(c, cw, cz)) return -1;
    size_t N = (size_t)c->nx * (size_t)c->ny * (size_t)c->nz;
    size_t B = sizeof(double) * (N ? N : 1);
    double *pn = malloc(B), *pc = malloc(B), *pp = malloc(B);
    double *qn = malloc(B), *qc = malloc(B), *qp = malloc(B);
    if (!pn || !pc || !pp || !qn || !qc || !qp) {
        free(pn); free(pc); free(pp); free(qn); free(qc); free(qp);
        return -2;
    }
    memcpy(pc, p, sizeof(double) * N); memcpy(pp, pprev, sizeof(double) * N);
    memcpy(qc, q, sizeof(double) * N); memcpy(qp, qprev, sizeof(double) * N);

    for (int s = 0; s < nsteps; ++s) {
        int n = n0 + s;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    size_t m = idx(c, i, j, k);
                    double v2 = vz[m] * vz[m] * c->dt * c->dt;
                    double kx = v2 * (1.0 + 2.0 * eps[m]);
                    double kn = v2 * (1.0 + 2.0 * delta[m]);
                    double Hp = op_h(c, cw, pc, i, j, k);
                    double Dq = op_z(c, cz, qc, i, j, k);
                    pn[m] = 2.0 * pc[m] - pp[m] + kx * Hp + v2 * Dq;
                    qn[m] = 2.0 * qc[m] - qp[m] + kn * Hp + v2 * Dq;
                }
        if (c->src_on) {
            double st = source_term(c, n);
            pn[idx(c, c->sx, c->sy, c->sz)] += st;
            if (c->src_into_q) qn[idx(c, c->sx, c->sy, c->sz)] += st;
        }
        if (c->nb > 0) {
#pragma omp parallel for schedule(static)
            for (int k = 0; k < c->nz; ++k)
                for (int j = 0; j < c->ny; ++j)
                    for (int i = 0; i < c->nx; ++i) {
                        size_t m = idx(c, i, j, k);
                        double g = sponge_at(c, i, j, k);
                        pn[m] *= g; pc[m] *= g; qn[m] *= g; qc[m] *= g;
                    }
        }
        if (traces)
            for (int r = 0; r < c->nrec; ++r)
                traces[(size_t)s * (size_t)c->nrec + (size_t)r] =
                    pn[idx(c, c->rec[3 * r], c->rec[3 * r + 1], c->rec[3 * r + 2])];
        double *t = pp; pp = pc; pc = pn; pn = t;
        t = qp; qp = qc; qc = qn; qn = t;
    }
    memcpy(p, pc, sizeof(double) * N); memcpy(pprev, pp, sizeof(double) * N);
    memcpy(q, qc, sizeof(double) * N); memcpy(qprev, qp, sizeof(double) * N);
    free(pn); free(pc); free(pp); free(qn); free(qc); free(qp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One step at sampled points, from single-precision state                   */
/* ------------------------------------------------------------------------ */

static inline double atf(const float *u, const or_cfg *c, int i, int j, int k)
{
    if (i < 0 || i >= c->nx || j < 0 || j >= c->ny || k < 0 || k >= c->nz) return 0.0;
    return (double)u[(size_t)i + (size_t)c->nx * ((size_t)j + (size_t)c->ny * (size_t)k)];
}

/*
 * One isotropic step evaluated only at npts points (pts = 3*npts cell
 * indices), from a single-precision state u^n (dense, full grid) and the true
 * previous level at those points (uprev_pts).  out[m] = G (2u - u^{n-1} +
 * (v dt)^2 L u + source) at point m, i.e. u^{n+1} after the Cerjan factor.
 * Lets a test check a full-size GPU step point by point.
 */
int or_iso_step_points(const or_cfg *c, const float *v, const float *u,
                       int npts, const int *pts, const double *uprev_pts, int n, double *out)
{
    double cw[33], cz[33];
    if (stencil_weights(c, cw, cz)) return -1;
#pragma omp parallel for schedule(static)
    for (int m = 0; m < npts; ++m) {
        int i = pts[3 * m], j = pts[3 * m + 1], k = pts[3 * m + 2];
        double s = 2.0 * cw[0] * atf(u, c, i, j, k);
        for (int l = 1; l <= c->r_xy; ++l)
            s += cw[l] * (atf(u, c, i + l, j, k) + atf(u, c, i - l, j, k) +
                          atf(u, c, i, j + l, k) + atf(u, c, i, j - l, k));
        double Lu = s / (c->h * c->h);
        double sz = cz[0] * atf(u, c, i, j, k);
        for (int l = 1; l <= c->r_z; ++l) sz += cz[l] * (atf(u, c, i, j, k + l) + atf(u, c, i, j, k - l));
        Lu += sz / (c->dz * c->dz);
        size_t p = idx(c, i, j, k);
        double vv = (double)v[p] * c->dt;
        double val = 2.0 * atf(u, c, i, j, k) - uprev_pts[m] + vv * vv * Lu;
        if (c->src_on && i == c->sx && j == c->sy && k == c->sz) val += source_term(c, n);
        out[m] = val * (c->nb > 0 ? sponge_at(c, i, j, k) : 1.0);
    }
    return 0;
}

/*
 * One VTI step at npts points from single-precision p^n, q^n (full grid) and
 * the true previous levels at those points.  outp/outq receive p^{n+1}, q^{n+1}.
 */
int or_vti_step_points(const or_cfg *c, const float *vz, const float *eps, const float *delta,
                       const float *p, const float *q, int npts, const int *pts,
                       const double *pprev_pts, const double *qprev_pts, int n,
                       double *outp, double *outq)
{
    double cw[33], cz[33];
    if (stencil_weights(c, cw, cz)) return -1;
    int nw = 2 * c->r_z + 1;
#pragma omp parallel for schedule(static)
    for (int m = 0; m < npts; ++m) {
        int i = pts[3 * m], j = pts[3 * m + 1], k = pts[3 * m + 2];
        double s = 2.0 * cw[0] * atf(p, c, i, j, k);
        for (int l = 1; l <= c->r_xy; ++l)
            s += cw[l] * (atf(p, c, i + l, j, k) + atf(p, c, i - l, j, k) +
                          atf(p, c, i, j + l, k) + atf(p, c, i, j - l, k));
        double Hp = s / (c->h * c->h);
        double Dq = 0.0;
        if (c->ztab) {
            const double *w = c->ztab + (size_t)k * (size_t)nw;
            for (int l = -c->r_z; l <= c->r_z; ++l) Dq += w[l + c->r_z] * atf(q, c, i, j, k + l);
        } else {
            Dq = cz[0] * atf(q, c, i, j, k);
            for (int l = 1; l <= c->r_z; ++l) Dq += cz[l] * (atf(q, c, i, j, k + l) + atf(q, c, i, j, k - l));
            Dq /= c->dz * c->dz;
        }
        size_t ix = idx(c, i, j, k);
        double v2 = (double)vz[ix] * (double)vz[ix] * c->dt * c->dt;
        double kx = v2 * (1.0 + 2.0 * (double)eps[ix]);
        double kn = v2 * (1.0 + 2.0 * (double)delta[ix]);
        double pv = 2.0 * atf(p, c, i, j, k) - pprev_pts[m] + kx * Hp + v2 * Dq;
        double qv = 2.0 * atf(q, c, i, j, k) - qprev_pts[m] + kn * Hp + v2 * Dq;
        if (c->src_on && i == c->sx && j == c->sy && k == c->sz) {
            double st = source_term(c, n);
            pv += st;
            if (c->src_into_q) qv += st;
        }
        double g = c->nb > 0 ? sponge_at(c, i, j, k) : 1.0;
        outp[m] = pv * g;
        outq[m] = qv * g;
    }
    return 0;
}

/*
 * Misfit and velocity gradient of the isotropic run (zero initial state,
 * source, damping and receivers as in or_iso_run):
 *   J = 1/2 sum_{n<N} sum_r (u^{n+1}(x_r) - dobs[n][r])^2.
 * Written in the physical variables of the literal Cerjan recurrence: with
 * p^n the damped older level, one step is
 *   u^{n+1} = G (2 u^n - p^n + K L u^n + S_n),   p^{n+1} = G u^n,   K = (v dt)^2,
 * i.e. x_{n+1} = A x_n + f_n with A = [[G (2 + K L), -G], [G, 0]].  The
 * adjoint state (alpha, beta) runs backward with the transpose of A (L is
 * symmetric, G and K diagonal):
 *   alpha_n = (2 + L K) G alpha_{n+1} + G beta_{n+1} + R^T r_{n-1},
 *   beta_n  = -G alpha_{n+1},
 * from alpha_N = R^T r_{N-1}, beta_N = 0 (r_n = data residual of step n), and
 *   dJ/dK(x) = sum_{n<N} alpha_{n+1}(x) G(x) (L u^n)(x),  dJ/dv = dJ/dK 2 v dt^2.
 * Stores every forward level: for small grids only.  grad_v may be NULL.
 */
int or_iso_misfit_grad(const or_cfg *c, const double *v, const double *dobs, int nsteps, double *J,
                       double *grad_v)
{
    double cw[33], cz[33];
    if (stencil_weights(c, cw, cz)) return -1;
    const size_t N = (size_t)c->nx * (size_t)c->ny * (size_t)c->nz;
    const size_t B = sizeof(double) * (N ? N : 1);
    double *U = (double *)calloc((size_t)(nsteps + 1) * (N ? N : 1), sizeof(double));   /* u^0..u^N */
    double *P = (double *)calloc(N ? N : 1, sizeof(double));
    double *G = (double *)malloc(B), *K = (double *)malloc(B), *Lu = (double *)malloc(B);
    double *al = (double *)calloc(N ? N : 1, sizeof(double)), *be = (double *)calloc(N ? N : 1, sizeof(double));
    double *aln = (double *)malloc(B), *w = (double *)malloc(B), *gk = (double *)calloc(N ? N : 1, sizeof(double));
    double *res = (double *)malloc(sizeof(double) * (size_t)(nsteps > 0 ? nsteps : 1) * (size_t)(c->nrec > 0 ? c->nrec : 1));
    if (!U || !P || !G || !K || !Lu || !al || !be || !aln || !w || !gk || !res) {
        free(U); free(P); free(G); free(K); free(Lu); free(al); free(be); free(aln); free(w); free(gk); free(res);
        return -2;
    }
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                size_t m = idx(c, i, j, k);
                G[m] = c->nb > 0 ? sponge_at(c, i, j, k) : 1.0;
                K[m] = v[m] * c->dt * v[m] * c->dt;
            }
    /* forward, keeping every level */
    double Jsum = 0.0;
    for (int n = 0; n < nsteps; ++n) {
        double *u = U + (size_t)n * N, *un = U + (size_t)(n + 1) * N;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    size_t m = idx(c, i, j, k);
                    double L = op_h(c, cw, u, i, j, k) + op_z(c, cz, u, i, j, k);
                    un[m] = G[m] * (2.0 * u[m] - P[m] + K[m] * L);
                }
        if (c->src_on) {
            size_t s = idx(c, c->sx, c->sy, c->sz);
            un[s] += G[s] * source_term(c, n);
        }
        for (size_t m = 0; m < N; ++m) P[m] = G[m] * u[m];
        for (int r = 0; r < c->nrec; ++r) {
            double d = un[idx(c, c->rec[3 * r], c->rec[3 * r + 1], c->rec[3 * r + 2])] -
                       dobs[(size_t)n * (size_t)c->nrec + (size_t)r];
            res[(size_t)n * (size_t)c->nrec + (size_t)r] = d;
            Jsum += 0.5 * d * d;
        }
    }
    *J = Jsum;
    if (grad_v) {
        /* backward: alpha_{n} from alpha_{n+1}, beta_{n+1}; gradient term with u^n */
        for (int n = nsteps; n >= 1; --n) {
            /* al, be hold (alpha_{n+1}, beta_{n+1}) (zero for n = N) */
#pragma omp parallel for schedule(static)
            for (size_t m = 0; m < N; ++m) w[m] = K[m] * G[m] * al[m];
#pragma omp parallel for schedule(static)
            for (int k = 0; k < c->nz; ++k)
                for (int j = 0; j < c->ny; ++j)
                    for (int i = 0; i < c->nx; ++i) {
                        size_t m = idx(c, i, j, k);
                        double Lw = op_h(c, cw, w, i, j, k) + op_z(c, cz, w, i, j, k);
                        aln[m] = 2.0 * G[m] * al[m] + Lw + G[m] * be[m];
                    }
            for (int r = 0; r < c->nrec; ++r)
                aln[idx(c, c->rec[3 * r], c->rec[3 * r + 1], c->rec[3 * r + 2])] +=
                    res[(size_t)(n - 1) * (size_t)c->nrec + (size_t)r];
            for (size_t m = 0; m < N; ++m) {
                be[m] = -G[m] * al[m];
                al[m] = aln[m];
            }
            /* al = alpha_n: gradient term of step n-1 uses alpha_n and u^{n-1} */
            const double *u = U + (size_t)(n - 1) * N;
#pragma omp parallel for schedule(static)
            for (int k = 0; k < c->nz; ++k)
                for (int j = 0; j < c->ny; ++j)
                    for (int i = 0; i < c->nx; ++i) {
                        size_t m = idx(c, i, j, k);
                        double L = op_h(c, cw, u, i, j, k) + op_z(c, cz, u, i, j, k);
                        gk[m] += al[m] * G[m] * L;
                    }
        }
        for (size_t m = 0; m < N; ++m) grad_v[m] = gk[m] * 2.0 * v[m] * c->dt * c->dt;
    }
    free(U); free(P); free(G); free(K); free(Lu); free(al); free(be); free(aln); free(w); free(gk); free(res);
    return 0;
}

/* Sponge factor G at a cell (product over the three axes). */
double or_sponge_at(const or_cfg *c, int i, int j, int k)
{
    return c->nb > 0 ? sponge_at(c, i, j, k) : 1.0;
}

/* Number of OpenMP threads a parallel region of the oracle will use. */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
