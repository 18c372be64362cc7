// Look-up table for the erfc-Coulomb pair terms (Sec. 3.3: the expensive error
// function and exponential of Eq. 10 replaced by precomputed values and
// polynomial interpolation, with a separate treatment of short distances).
//
// Over s = r^2 in [0, s_max] (s_max = r_cut^2 plus a relative margin of 1e-6) the
// table holds n cubic pieces on a uniform grid.  Two factors are tabulated:
//   force  f(s) = [erfc(sqrt(alpha s)) / sqrt(s) + 2 sqrt(alpha/pi) e^{-alpha s}] / s
//          (the Coulomb pair force is coulomb_k q_i q_j f(s) (r_i - r_j));
//   energy e(s) = erfc(sqrt(alpha s)) / sqrt(s).
// Both are singular at s = 0, so the pieces below the knot s0 (the first knot at
// or above (r_cut/3)^2) hold the smooth remainders f(s) - s^{-3/2} and
// e(s) - s^{-1/2}; the kernel adds the bare Coulomb term there, exactly.  This is
// this library's form of the paper's short-distance series: the remainders are
// entire functions of s whose Taylor series (in powers of alpha s) is used to
// evaluate them where the closed forms would cancel.  Above s0 the factors are
// smooth and tabulated directly.
//
// Piece k covers [k h, (k+1) h] with h = s_max / n; in the local coordinate
// t = s/h - k in [0, 1] its value is c0 + c1 t + c2 t^2 + c3 t^3, the cubic through
// the exact values at t = 0, 1/3, 2/3, 1 (FP64 on the host).  Coefficients are
// stored as {c0, c1, c2, c3} for the force factor of piece k at [2k] and for the
// energy factor at [2k + 1].
#include <math.h>
#include <string.h>

#include <vector>

#include "rbmd_internal.cuh"

namespace rbmd {
namespace {

// Remainder f(s) - s^{-3/2} by its series:
//   (2 sqrt(alpha/pi)) sum_{k>=0} (-alpha)^{k+1} s^k 2 (k+1) / ((k+1)! (2k+3))
// (from the series of erf and exp; the s^{-1} terms cancel), used for alpha s < 2.
double force_rem_series(double alpha, double s)
{
    const double x = -alpha * s;
    double term = -alpha;  // (-alpha)^{k+1} s^k / (k+1)! at k = 0
    double acc = 0.0;
    for (int k = 0; k < 80; ++k) {
        acc += term * 2.0 * (k + 1) / (2.0 * k + 3.0);
        term *= x / (double)(k + 2);
        if (fabs(term) < 1e-30) break;
    }
    return 2.0 * sqrt(alpha / kPi) * acc;
}

// Remainder e(s) - s^{-1/2} = -erf(sqrt(alpha s)) / sqrt(s) by its series
//   -(2 sqrt(alpha/pi)) sum_{n>=0} (-alpha s)^n / (n! (2n+1)), used for alpha s < 2.
double energy_rem_series(double alpha, double s)
{
    const double x = -alpha * s;
    double term = 1.0;
    double acc = 0.0;
    for (int n = 0; n < 80; ++n) {
        acc += term / (2.0 * n + 1.0);
        term *= x / (double)(n + 1);
        if (fabs(term) < 1e-30) break;
    }
    return -2.0 * sqrt(alpha / kPi) * acc;
}

double force_factor(double alpha, double s)
{
    const double r = sqrt(s);
    return (erfc(sqrt(alpha) * r) / r + 2.0 * sqrt(alpha / kPi) * exp(-alpha * s)) / s;
}

double energy_factor(double alpha, double s)
{
    const double r = sqrt(s);
    return erfc(sqrt(alpha) * r) / r;
}

double force_rem(double alpha, double s)
{
    if (alpha * s < 2.0) return force_rem_series(alpha, s);
    return force_factor(alpha, s) - pow(s, -1.5);
}

double energy_rem(double alpha, double s)
{
    if (alpha * s < 2.0) return energy_rem_series(alpha, s);
    return energy_factor(alpha, s) - 1.0 / sqrt(s);
}

// Cubic through (0, y0), (1/3, y1), (2/3, y2), (1, y3): Newton form converted to
// monomial coefficients.
void cubic4(const double y[4], double c[4])
{
    const double h = 1.0 / 3.0;
    const double d1 = (y[1] - y[0]) / h, d2 = (y[2] - y[1]) / h, d3 = (y[3] - y[2]) / h;
    const double e1 = (d2 - d1) / (2 * h), e2 = (d3 - d2) / (2 * h);
    const double g1 = (e2 - e1) / (3 * h);
    // p(t) = y0 + d1 t + e1 t (t - h) + g1 t (t - h)(t - 2h)
    c[0] = y[0];
    c[1] = d1 - e1 * h + g1 * 2 * h * h;
    c[2] = e1 - g1 * 3 * h;
    c[3] = g1;
}

}  // namespace

rbmd_status pair_table_host(double alpha, double r_cut, int n, std::vector<double> &coef,
                            int32_t *i0, double *inv_h)
{
    if (!(alpha > 0.0) || !(r_cut > 0.0) || n < 16) return RBMD_ERR_INVALID;
    const double smax = r_cut * r_cut * (1.0 + 1e-6);
    const double h = smax / n;
    const double s0 = r_cut * r_cut / 9.0;
    int k0 = (int)ceil(s0 / h);  // pieces [0, k0) hold the remainders
    if (k0 < 1) k0 = 1;
    if (k0 > n) k0 = n;
    coef.assign((size_t)8 * n, 0.0);
    for (int k = 0; k < n; ++k) {
        double yf[4], ye[4];
        for (int j = 0; j < 4; ++j) {
            const double s = (k + j / 3.0) * h;
            if (k < k0) {
                yf[j] = force_rem(alpha, s);
                ye[j] = energy_rem(alpha, s);
            } else {
                yf[j] = force_factor(alpha, s);
                ye[j] = energy_factor(alpha, s);
            }
        }
        cubic4(yf, &coef[(size_t)8 * k]);
        cubic4(ye, &coef[(size_t)8 * k + 4]);
    }
    *i0 = k0;
    *inv_h = 1.0 / h;
    return RBMD_OK;
}

}  // namespace rbmd

extern "C" rbmd_status rbmd_pair_table(double alpha, double r_cut, int32_t n, int32_t *i0,
                                       double *inv_h, double *coef)
{
    if (!i0 || !inv_h) return RBMD_ERR_INVALID;
    std::vector<double> c;
    rbmd_status s = rbmd::pair_table_host(alpha, r_cut, n, c, i0, inv_h);
    if (s != RBMD_OK) return s;
    if (coef) memcpy(coef, c.data(), sizeof(double) * c.size());
    return RBMD_OK;
}
