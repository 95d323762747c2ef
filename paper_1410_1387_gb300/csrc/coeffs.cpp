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
