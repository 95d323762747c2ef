// Host-side weights, damping profile and wavelet of the library (coeffs.cpp).
#pragma once

namespace fdk {

// Fornberg's recursion: weights out[0..n-1] of the M-th derivative at x0 from nodes x.
void fornberg(double x0, const double *x, int n, int M, double *out);
// Symmetric order-2R second-derivative weights c[0..R] on a unit grid (Eq. 4).
void central_d2(int R, double *c);
// Band-optimised symmetric second-derivative weights c[0..R] on a unit grid:
// exact on quadratics (sum_l l^2 c_l = 1, c_0 = -2 sum c_l) and, within that,
// least-squares optimal for the relative error of the symbol,
// int_0^kmax (-S(k) / k^2 - 1)^2 dk with S(k) = c_0 + 2 sum_l c_l cos(l k)
// (the optimised weights of Sec. 1, after Holberg 1987).  0 < kmax <= pi.
// Returns 0, or -1 for bad arguments.
int band_optimized_d2(int R, double kmax, double *c);
// |c_0| + 2 sum |c_l|: the Gershgorin bound of the 1D operator's spectrum
// (equal to its symbol at the Nyquist frequency for the alternating Taylor weights).
double row_abs_sum(const double *c, int R);
// Per-plane z weights tab[k*(2Rz+1) + l+Rz] (Eq. 5); dzk = nz-1 spacings or NULL.
void z_weights(int nz, int Rz, const double *dzk, double dz, double *tab);
double z_row_abs_max(const double *tab, int nz, int Rz);
// Cerjan factor along one axis: exp(-(a d)^2), d = cells into the layer (1..width).
double cerjan(int i, int n, int width, double a);
// Ricker wavelet (1 - 2 pi^2 f^2 t^2) exp(-pi^2 f^2 t^2).
double ricker(double t, double f);

}  // namespace fdk
