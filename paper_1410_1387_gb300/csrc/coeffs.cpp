// Stencil weights and stability bounds used by the library.
//
// All weights come from Fornberg's recursion (B. Fornberg, "Generation of
// finite difference formulas on arbitrarily spaced grids", Math. Comp. 51,
// 1988), which builds the weights of every derivative order up to M at x0 from
// the nodes one node at a time.  On the uniform nodes -R..R it gives the
// symmetric weights of Eq. 4; on the planes z_{k-Rz}..z_{k+Rz} it gives the
// per-plane weights of Eq. 5 with the spacings absorbed.
#include "coeffs.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace fdk {

void fornberg(double x0, const double *x, int n, int M, double *out)
{
    // d[m][j]: weight of node j for derivative m, over the nodes seen so far
    std::vector<double> d((size_t)(M + 1) * n, 0.0);
    auto D = [&](int m, int j) -> double & { return d[(size_t)m * n + j]; };
    D(0, 0) = 1.0;
    double c1 = 1.0;
    double c4 = x[0] - x0;
    for (int i = 1; i < n; ++i) {
        const int mn = std::min(i, M);
        double c2 = 1.0;
        const double c5 = c4;
        c4 = x[i] - x0;
        for (int j = 0; j < i; ++j) {
            const double c3 = x[i] - x[j];
            c2 *= c3;
            if (j == i - 1) {
                // the new node's weights, from the previous last node's
                for (int m = mn; m >= 1; --m) D(m, i) = c1 * (m * D(m - 1, i - 1) - c5 * D(m, i - 1)) / c2;
                D(0, i) = -c1 * c5 * D(0, i - 1) / c2;
            }
            for (int m = mn; m >= 1; --m) D(m, j) = (c4 * D(m, j) - m * D(m - 1, j)) / c3;
            D(0, j) = c4 * D(0, j) / c3;
        }
        c1 = c2;
    }
    for (int j = 0; j < n; ++j) out[j] = D(M, j);
}

void central_d2(int R, double *c)
{
    std::vector<double> x(2 * R + 1), w(2 * R + 1);
    for (int j = 0; j <= 2 * R; ++j) x[j] = (double)(j - R);
    fornberg(0.0, x.data(), 2 * R + 1, 2, w.data());
    // symmetric: average the two sides to remove rounding asymmetry
    c[0] = w[R];
    for (int l = 1; l <= R; ++l) c[l] = 0.5 * (w[R + l] + w[R - l]);
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's iteration on P_n from
// the first guess cos(pi (i + 3/4) / (n + 1/2)), P_n by the three-term recurrence.
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double step = p1 / dp;
            t -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

int band_optimized_d2(int R, double kmax, double *c)
{
    if (R < 1 || R > 32 || !(kmax > 0.0) || kmax > M_PI) return -1;
    if (R == 1) {
        c[0] = -2.0;
        c[1] = 1.0;
        return 0;
    }
    // relative symbol error e(k) = sum_l c_l phi_l(k) - 1, phi_l = 4 sin^2(l k / 2) / k^2
    // (phi_l(0) = l^2); with c_1 = 1 - sum_{l>=2} l^2 c_l the constraint e(0) = 0
    // holds and e = sum_{l>=2} c_l (phi_l - l^2 phi_1) - (1 - phi_1): a linear least-
    // squares problem in c_2..c_R, sampled at composite Gauss-Legendre points.
    constexpr int NQ = 16, NS = 32;
    double gx[NQ], gw[NQ];
    gauss_legendre(NQ, gx, gw);
    const int M = NQ * NS, P = R - 1;
    std::vector<double> A((size_t)M * P), b(M);
    auto phi = [](int l, double k) {
        const double s = std::sin(0.5 * l * k);
        return 4.0 * s * s / (k * k);
    };
    for (int si = 0; si < NS; ++si)
        for (int q = 0; q < NQ; ++q) {
            const int row = si * NQ + q;
            const double k = (si + 0.5 * (gx[q] + 1.0)) * kmax / NS;
            const double sw = std::sqrt(0.5 * gw[q] * kmax / NS);
            const double p1 = phi(1, k);
            for (int l = 2; l <= R; ++l) A[(size_t)row * P + (l - 2)] = sw * (phi(l, k) - l * l * p1);
            b[row] = sw * (1.0 - p1);
        }
    // Householder QR of A, applied to b as it goes; then back substitution
    for (int j = 0; j < P; ++j) {
        double nrm = 0.0;
        for (int i = j; i < M; ++i) nrm += A[(size_t)i * P + j] * A[(size_t)i * P + j];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return -1;
        const double a0 = A[(size_t)j * P + j];
        const double alpha = a0 > 0.0 ? -nrm : nrm;
        std::vector<double> v(M - j);
        v[0] = a0 - alpha;
        for (int i = j + 1; i < M; ++i) v[i - j] = A[(size_t)i * P + j];
        double vv = 0.0;
        for (double e : v) vv += e * e;
        if (vv == 0.0) continue;
        for (int col = j; col <= P; ++col) {   // col == P is b
            double dot = 0.0;
            for (int i = j; i < M; ++i) dot += v[i - j] * (col < P ? A[(size_t)i * P + col] : b[i]);
            const double f = 2.0 * dot / vv;
            for (int i = j; i < M; ++i) (col < P ? A[(size_t)i * P + col] : b[i]) -= f * v[i - j];
        }
    }
    std::vector<double> xs(P);
    for (int j = P - 1; j >= 0; --j) {
        double s = b[j];
        for (int m = j + 1; m < P; ++m) s -= A[(size_t)j * P + m] * xs[m];
        xs[j] = s / A[(size_t)j * P + j];
    }
    double c1 = 1.0, sum = 0.0;
    for (int l = 2; l <= R; ++l) {
        c[l] = xs[l - 2];
        c1 -= (double)l * l * c[l];
        sum += c[l];
    }
    c[1] = c1;
    c[0] = -2.0 * (sum + c1);
    for (int l = 0; l <= R; ++l)
        if (!std::isfinite(c[l])) return -1;
    return 0;
}

double row_abs_sum(const double *c, int R)
{
    double s = std::fabs(c[0]);
    for (int l = 1; l <= R; ++l) s += 2.0 * std::fabs(c[l]);
    return s;
}

static double plane_z(int nz, const double *dzk, double dz, long k)
{
    if (!dzk || nz < 2) return dz * (double)k;
    if (k <= 0) return dzk[0] * (double)k;
    double z = 0.0;
    const long kin = std::min<long>(k, nz - 1);
    for (long m = 0; m < kin; ++m) z += dzk[m];
    if (k > nz - 1) z += dzk[nz - 2] * (double)(k - (nz - 1));
    return z;
}

void z_weights(int nz, int Rz, const double *dzk, double dz, double *tab)
{
    const int nw = 2 * Rz + 1;
    std::vector<double> zn(nw);
    // prefix sums make plane coordinates O(1) after the first pass
    std::vector<double> zc(nz);
    for (int k = 0; k < nz; ++k) zc[k] = (k == 0) ? 0.0 : (dzk ? zc[k - 1] + dzk[k - 1] : dz * k);
    for (int k = 0; k < nz; ++k) {
        for (int l = -Rz; l <= Rz; ++l) {
            const long kk = (long)k + l;
            zn[l + Rz] = (kk >= 0 && kk < nz) ? zc[kk] : plane_z(nz, dzk, dz, kk);
        }
        fornberg(zn[Rz], zn.data(), nw, 2, tab + (size_t)k * nw);
    }
}

double z_row_abs_max(const double *tab, int nz, int Rz)
{
    const int nw = 2 * Rz + 1;
    double m = 0.0;
    for (int k = 0; k < nz; ++k) {
        double s = 0.0;
        for (int j = 0; j < nw; ++j) s += std::fabs(tab[(size_t)k * nw + j]);
        m = std::max(m, s);
    }
    return m;
}

double cerjan(int i, int n, int width, double a)
{
    if (width <= 0) return 1.0;
    int d = 0;
    if (i < width) d = width - i;
    else if (i >= n - width) d = i - (n - width - 1);
    const double ad = a * d;
    return std::exp(-ad * ad);
}

double ricker(double t, double f)
{
    const double pf = M_PI * f * t;
    const double a = pf * pf;
    return (1.0 - 2.0 * a) * std::exp(-a);
}

}  // namespace fdk
