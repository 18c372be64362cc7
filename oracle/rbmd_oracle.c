/*
 * rbmd_oracle.c -- plain, slow FP64 reference of the random-batch nonbonded step
 * (random batch Ewald + random batch list) of arXiv 2407.09315.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header, table or constant generator
 * with the CUDA path: every definition below is written out again from the paper
 * and from the readings listed at the top of each function.
 *
 * Conventions (reduced units, cubic periodic box of side L, volume V = L^3):
 *   - state: fractional fixed-point coordinates u in [0, 2^32), decoded here as
 *     x = u * (L / 2^32) in FP64;
 *   - k = 2*pi*m/L with m in Z^3 (Sec. 2.2, below Eq. 8);
 *   - all energies and forces carry the Coulomb prefactor coulomb_k (Eq. 3 with
 *     1/(4 pi eps0) -> coulomb_k);
 *   - every random choice is driven by Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), written here from
 *     that publication.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math), see build.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO32 4294967296.0
#define ORC_TWO64 18446744073709551616.0
#define ORC_PI 3.14159265358979323846

/* Counter word 3 tags which random stream a draw belongs to. */
#define ORC_STREAM_RBE 1u
#define ORC_STREAM_RBL 2u
#define ORC_STREAM_LANGEVIN 3u
#define ORC_STREAM_METROPOLIS 4u
#define ORC_MAX_ATTEMPTS 256

/* Host threads of the per-mode and per-atom loops (1 unless orc_set_threads
 * raises it; every element is computed by the same operations in the same
 * order whatever the count, only the order of the RBL sums over atoms changes). */
static int orc_threads = 1;

void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }

int orc_get_threads(void) { return orc_threads; }

static int orc_thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 3): 10 rounds of two 32x32->64 multiplies with  */
/* the published multipliers and Weyl key increments.                        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* golden ratio */
            k1 += 0xBB67AE85u; /* sqrt(3) - 1 */
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void orc_seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
}

/* ------------------------------------------------------------------------ */
/* RBE sampling distribution (Sec. 2.2 around Eq. 12, Algorithm 1 step 1).   */
/* P(m) ~ exp(-k^2/(4 alpha)) = prod_d exp(-a m_d^2), a = pi^2/(alpha L^2).  */
/* Reading: the modes are drawn i.i.d. (the unbiasedness statement below     */
/* Eq. 12 assumes it) by exact per-dimension inverse CDF over |m_d| <= M,    */
/* with M the smallest integer with a M^2 >= ln(1e16).                       */
/* ------------------------------------------------------------------------ */
double orc_sampler_a(double L, double alpha)
{
    return ORC_PI * ORC_PI / (alpha * L * L);
}

int orc_sampler_M(double L, double alpha)
{
    double a = orc_sampler_a(L, alpha);
    return (int)ceil(sqrt(16.0 * log(10.0) / a));
}

/* Thresholds T[j] = min(2^64-1, floor(CDF_j * 2^64)), j = 0..2M, where
 * CDF_j = sum_{i<=j} w_i / sum_i w_i and w_i = exp(-a (i-M)^2).
 * Returns H = sum_{m=-M}^{M} exp(-a m^2) (1-D theta sum). */
double orc_sampler_table(double L, double alpha, int M, uint64_t *T)
{
    double a = orc_sampler_a(L, alpha);
    int n = 2 * M + 1;
    double *cum = (double *)malloc(sizeof(double) * (size_t)n);
    double total = 0.0;
    for (int j = 0; j < n; ++j) {
        double m = (double)(j - M);
        total += exp(-a * m * m);
        cum[j] = total;
    }
    for (int j = 0; j < n; ++j) {
        double x = (cum[j] / total) * ORC_TWO64;
        T[j] = (x >= ORC_TWO64) ? UINT64_MAX : (uint64_t)x;
    }
    free(cum);
    return total;
}

/* Normaliser of the sampling density over k != 0:
 * S = sum_{m != 0} exp(-a |m|^2) = H^3 - 1 (the paper's Q, Eq. 12). */
double orc_rbe_S(double L, double alpha)
{
    int M = orc_sampler_M(L, alpha);
    uint64_t *T = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
    double H = orc_sampler_table(L, alpha, M, T);
    free(T);
    return H * H * H - 1.0;
}

/* m_d for one 64-bit uniform: the number of thresholds T[0..2M-1] that are
 * <= U (the smallest j with U < T[j], T[2M] taken as infinite), minus M. */
static int orc_draw_index(uint64_t U, const uint64_t *T, int M)
{
    int count = 0;
    for (int j = 0; j < 2 * M; ++j)
        if (T[j] <= U) ++count;
    return count - M;
}

/* Draw the P modes of one step.  Sample l, attempt t:
 *   words = Philox(ctr = (l, t, step, STREAM_RBE | replica<<8), key = seed)
 *   U_x = w0<<32 | w1, U_y = w2<<32 | w3;
 *   words' = Philox(ctr = (l, t | 0x80000000, step, ...)), U_z = w0'<<32 | w1'.
 * m = 0 is rejected and retried with t+1 (k != 0 in Eq. 12); after 256
 * rejections the mode stays 0 and carries zero weight.  m_out: [P][3]. */
void orc_rbe_sample(uint64_t seed, int64_t step, uint32_t replica, int P,
                    double L, double alpha, int32_t *m_out)
{
    int M = orc_sampler_M(L, alpha);
    uint64_t *T = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
    orc_sampler_table(L, alpha, M, T);
    uint32_t key[2];
    orc_seed_key(seed, key);
    for (int l = 0; l < P; ++l) {
        int mx = 0, my = 0, mz = 0;
        for (uint32_t t = 0; t < ORC_MAX_ATTEMPTS; ++t) {
            uint32_t ctr[4] = {(uint32_t)l, t, (uint32_t)step, ORC_STREAM_RBE | (replica << 8)};
            uint32_t w[4], w2[4];
            orc_philox4x32_10(ctr, key, w);
            ctr[1] = t | 0x80000000u;
            orc_philox4x32_10(ctr, key, w2);
            uint64_t ux = ((uint64_t)w[0] << 32) | w[1];
            uint64_t uy = ((uint64_t)w[2] << 32) | w[3];
            uint64_t uz = ((uint64_t)w2[0] << 32) | w2[1];
            mx = orc_draw_index(ux, T, M);
            my = orc_draw_index(uy, T, M);
            mz = orc_draw_index(uz, T, M);
            if (mx != 0 || my != 0 || mz != 0) break;
        }
        m_out[3 * l + 0] = mx;
        m_out[3 * l + 1] = my;
        m_out[3 * l + 2] = mz;
    }
    free(T);
}

/* All m != 0 with |m_d| <= M, in lexicographic (mx, my, mz) order, and their
 * Gaussian weights exp(-k^2/(4 alpha)) (the full Fourier series of Eq. 11).
 * Returns the count (2M+1)^3 - 1; m_out/w_out may be NULL to query it. */
int64_t orc_full_modes(double L, double alpha, int M, int32_t *m_out, double *w_out)
{
    double a = orc_sampler_a(L, alpha);
    int64_t c = 0;
    for (int mx = -M; mx <= M; ++mx)
        for (int my = -M; my <= M; ++my)
            for (int mz = -M; mz <= M; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                if (m_out) {
                    m_out[3 * c + 0] = mx;
                    m_out[3 * c + 1] = my;
                    m_out[3 * c + 2] = mz;
                }
                if (w_out) w_out[c] = exp(-a * (double)(mx * mx + my * my + mz * mz));
                ++c;
            }
    return c;
}

static void orc_decode(int64_t n, const uint32_t *u, double L, double *x)
{
    for (int64_t i = 0; i < 3 * n; ++i) x[i] = (double)u[i] * (L / ORC_TWO32);
}

/* ------------------------------------------------------------------------ */
/* Structure factors, Eq. 9: rho(k) = sum_j q_j exp(i k . r_j).              */
/* rho_out: [nm][2] (real, imaginary).                                       */
/* ------------------------------------------------------------------------ */
void orc_structure_factor(int64_t n, const uint32_t *u, const double *q, double L,
                          int64_t nm, const int32_t *m, double *rho_out)
{
    double *x = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    orc_decode(n, u, L, x);
#pragma omp parallel for num_threads(orc_threads) schedule(static)
    for (int64_t l = 0; l < nm; ++l) {
        double kx = 2.0 * ORC_PI * m[3 * l + 0] / L;
        double ky = 2.0 * ORC_PI * m[3 * l + 1] / L;
        double kz = 2.0 * ORC_PI * m[3 * l + 2] / L;
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double th = kx * x[3 * j] + ky * x[3 * j + 1] + kz * x[3 * j + 2];
            re += q[j] * cos(th);
            im += q[j] * sin(th);
        }
        rho_out[2 * l] = re;
        rho_out[2 * l + 1] = im;
    }
    free(x);
}

/* ------------------------------------------------------------------------ */
/* Weighted Fourier-mode force and energy.  With weights W_l it computes     */
/*   F_i = - coulomb_k sum_l W_l (4 pi q_i k_l / (V k_l^2)) Im(e^{-i k_l.r_i} rho_l)
 *   E   =   coulomb_k sum_l W_l (2 pi / V) |rho_l|^2 / k_l^2                */
/* W_l = exp(-k^2/4alpha) over all m != 0 gives the Ewald long-range force   */
/* (Eq. 11) and energy (second term of Eq. 8); W_l = S/P over P sampled      */
/* modes gives the RBE force (Eq. 12) and the matching energy estimate       */
/* (reading: the paper states no energy estimator; this one is unbiased for  */
/* Eq. 8's term and its exact gradient is Eq. 12).                           */
/* Forces are computed only for the n_sel atoms listed in sel (all if sel is */
/* NULL); F_out is [n_sel][3] (or [n][3]); rho is always summed over all n.  */
/* ------------------------------------------------------------------------ */
void orc_mode_forces(int64_t n, const uint32_t *u, const double *q, double L,
                     double coulomb_k, int64_t nm, const int32_t *m, const double *W,
                     int64_t n_sel, const int64_t *sel, double *F_out, double *E_out,
                     double *rho_out)
{
    double V = L * L * L;
    double *x = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    double *rho = (double *)malloc(sizeof(double) * (size_t)(2 * nm));
    orc_decode(n, u, L, x);
    orc_structure_factor(n, u, q, L, nm, m, rho);
    int64_t ns = sel ? n_sel : n;
    double E = 0.0;
    for (int64_t l = 0; l < nm; ++l) {
        double kx = 2.0 * ORC_PI * m[3 * l + 0] / L;
        double ky = 2.0 * ORC_PI * m[3 * l + 1] / L;
        double kz = 2.0 * ORC_PI * m[3 * l + 2] / L;
        double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 == 0.0) continue; /* exhausted sample: zero weight */
        double re = rho[2 * l], im = rho[2 * l + 1];
        E += coulomb_k * W[l] * (2.0 * ORC_PI / V) * (re * re + im * im) / k2;
    }
    /* every atom sums its modes in mode order */
#pragma omp parallel for num_threads(orc_threads) schedule(static)
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = sel ? sel[s] : s;
        double f[3] = {0.0, 0.0, 0.0};
        for (int64_t l = 0; l < nm; ++l) {
            double kx = 2.0 * ORC_PI * m[3 * l + 0] / L;
            double ky = 2.0 * ORC_PI * m[3 * l + 1] / L;
            double kz = 2.0 * ORC_PI * m[3 * l + 2] / L;
            double k2 = kx * kx + ky * ky + kz * kz;
            if (k2 == 0.0) continue;
            double re = rho[2 * l], im = rho[2 * l + 1];
            double th = kx * x[3 * i] + ky * x[3 * i + 1] + kz * x[3 * i + 2];
            /* Im(e^{-i th} (re + i im)) = im cos th - re sin th */
            double imag = im * cos(th) - re * sin(th);
            double c = -coulomb_k * W[l] * 4.0 * ORC_PI * q[i] / (V * k2) * imag;
            f[0] += c * kx;
            f[1] += c * ky;
            f[2] += c * kz;
        }
        F_out[3 * s + 0] = f[0];
        F_out[3 * s + 1] = f[1];
        F_out[3 * s + 2] = f[2];
    }
    if (E_out) *E_out = E;
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)(2 * nm));
    free(rho);
    free(x);
}

/* RBE force of one step (Eq. 12): P modes drawn by orc_rbe_sample, each with
 * weight S/P.  m_out ([P][3]) and rho_out ([P][2]) may be NULL. */
void orc_rbe_forces(int64_t n, const uint32_t *u, const double *q, double L, double alpha,
                    double coulomb_k, int P, uint64_t seed, int64_t step, uint32_t replica,
                    int64_t n_sel, const int64_t *sel, double *F_out, double *E_out,
                    int32_t *m_out, double *rho_out)
{
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * P));
    double *W = (double *)malloc(sizeof(double) * (size_t)P);
    orc_rbe_sample(seed, step, replica, P, L, alpha, m);
    double S = orc_rbe_S(L, alpha);
    for (int l = 0; l < P; ++l) W[l] = S / (double)P;
    orc_mode_forces(n, u, q, L, coulomb_k, P, m, W, n_sel, sel, F_out, E_out, rho_out);
    if (m_out) memcpy(m_out, m, sizeof(int32_t) * (size_t)(3 * P));
    free(W);
    free(m);
}

/* ------------------------------------------------------------------------ */
/* Virial tensor of the weighted Fourier-mode energy (pressure, Sec. 2.2).   */
/* The virial is W_ab = -dE/d e_ab, the derivative of the energy under the   */
/* affine strain x -> (1 + e) x of the box and of every position at fixed    */
/* fractional coordinates (reading: the paper names the virial among its     */
/* outputs but prints no formula).  Under that strain V -> V (1 + tr e),     */
/* k -> (1 - e^T) k and every phase k.r_j is unchanged, so rho(k) is too.    */
/* For the mode energy e_l = coulomb_k W_l (2 pi/V) |rho_l|^2 / k_l^2 with   */
/* W_l = exp(-k_l^2/4 alpha) (the Ewald term of Eq. 8) the derivative is     */
/*   W_ab = sum_l e_l [delta_ab - 2 k_a k_b (1/k_l^2 + 1/(4 alpha))],        */
/* the 1/(4 alpha) part coming from the Gaussian.  The RBE estimate (Eq. 12 */
/* sampling) reuses it with W_l = S/P: it is then an unbiased estimate of    */
/* the Ewald virial, not the derivative of the RBE energy estimate (whose   */
/* modes and S depend on L).  W_out[6] = xx, yy, zz, xy, xz, yz.            */
/* ------------------------------------------------------------------------ */
void orc_mode_virial(int64_t n, const uint32_t *u, const double *q, double L, double alpha,
                     double coulomb_k, int64_t nm, const int32_t *m, const double *W,
                     double *W_out)
{
    double V = L * L * L;
    double *rho = (double *)malloc(sizeof(double) * (size_t)(2 * (nm > 0 ? nm : 1)));
    orc_structure_factor(n, u, q, L, nm, m, rho);
    for (int c = 0; c < 6; ++c) W_out[c] = 0.0;
    for (int64_t l = 0; l < nm; ++l) {
        double k[3];
        for (int d = 0; d < 3; ++d) k[d] = 2.0 * ORC_PI * m[3 * l + d] / L;
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        if (k2 == 0.0) continue;
        double re = rho[2 * l], im = rho[2 * l + 1];
        double e = coulomb_k * W[l] * (2.0 * ORC_PI / V) * (re * re + im * im) / k2;
        double b = 2.0 * (1.0 / k2 + 1.0 / (4.0 * alpha));
        W_out[0] += e * (1.0 - b * k[0] * k[0]);
        W_out[1] += e * (1.0 - b * k[1] * k[1]);
        W_out[2] += e * (1.0 - b * k[2] * k[2]);
        W_out[3] += e * (-b * k[0] * k[1]);
        W_out[4] += e * (-b * k[0] * k[2]);
        W_out[5] += e * (-b * k[1] * k[2]);
    }
    free(rho);
}

/* RBE virial estimate of one step: the modes of orc_rbe_sample, W_l = S/P. */
void orc_rbe_virial(int64_t n, const uint32_t *u, const double *q, double L, double alpha,
                    double coulomb_k, int P, uint64_t seed, int64_t step, uint32_t replica,
                    double *W_out)
{
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * P));
    double *W = (double *)malloc(sizeof(double) * (size_t)P);
    orc_rbe_sample(seed, step, replica, P, L, alpha, m);
    double S = orc_rbe_S(L, alpha);
    for (int l = 0; l < P; ++l) W[l] = S / (double)P;
    orc_mode_virial(n, u, q, L, alpha, coulomb_k, P, m, W, W_out);
    free(W);
    free(m);
}

/* ------------------------------------------------------------------------ */
/* Full Ewald sum (Eqs. 8, 10, 11) as the physics reference.                 */
/*  real space: explicit images n with |r_ij + nL| < r_cut (i != j or n != 0)*/
/*  reciprocal: all m != 0 with |m_d| <= M                                   */
/*  self: -sqrt(alpha/pi) sum q^2                                            */
/* Tin-foil boundary (no surface term).  Real-space force sign: like charges */
/* repel, F_i along +(r_i - r_j) (reading of Eq. 10's r_ij).                  */
/* ------------------------------------------------------------------------ */
void orc_ewald(int64_t n, const uint32_t *u, const double *q, double L, double alpha,
               double coulomb_k, double r_cut, int M, double *F_real, double *F_recip,
               double *E_real, double *E_recip, double *E_self)
{
    double *x = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    orc_decode(n, u, L, x);
    double sa = sqrt(alpha);
    int nimg = (int)ceil(r_cut / L) + 1;
    double Er = 0.0;
    for (int64_t s = 0; s < 3 * n; ++s) F_real[s] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            for (int a = -nimg; a <= nimg; ++a)
                for (int b = -nimg; b <= nimg; ++b)
                    for (int c = -nimg; c <= nimg; ++c) {
                        if (i == j && a == 0 && b == 0 && c == 0) continue;
                        double rx = x[3 * i] - x[3 * j] + a * L;
                        double ry = x[3 * i + 1] - x[3 * j + 1] + b * L;
                        double rz = x[3 * i + 2] - x[3 * j + 2] + c * L;
                        double r = sqrt(rx * rx + ry * ry + rz * rz);
                        if (r >= r_cut) continue;
                        double qq = coulomb_k * q[i] * q[j];
                        Er += 0.5 * qq * erfc(sa * r) / r;
                        double g = qq * (erfc(sa * r) / (r * r) +
                                         2.0 * sa / sqrt(ORC_PI) * exp(-alpha * r * r) / r);
                        F_real[3 * i] += g * rx / r;
                        F_real[3 * i + 1] += g * ry / r;
                        F_real[3 * i + 2] += g * rz / r;
                    }
    *E_real = Er;
    int64_t nm = orc_full_modes(L, alpha, M, NULL, NULL);
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * nm));
    double *W = (double *)malloc(sizeof(double) * (size_t)nm);
    orc_full_modes(L, alpha, M, m, W);
    orc_mode_forces(n, u, q, L, coulomb_k, nm, m, W, 0, NULL, F_recip, E_recip, NULL);
    double q2 = 0.0;
    for (int64_t i = 0; i < n; ++i) q2 += q[i] * q[i];
    *E_self = -coulomb_k * sqrt(alpha / ORC_PI) * q2;
    free(W);
    free(m);
    free(x);
}

/* Virial tensor of the full Ewald sum (same readings as orc_ewald): the     */
/* real-space part over explicit images, 1/2 sum over ordered pairs of       */
/* r_ij (x) F_ij with F_ij the erfc-Coulomb force on i from j (Eq. 10) and   */
/* r_ij = r_i - r_j + nL; the Fourier part from orc_mode_virial over every   */
/* m != 0 with |m_d| <= M.  The self term does not depend on the strain.     */
void orc_ewald_virial(int64_t n, const uint32_t *u, const double *q, double L, double alpha,
                      double coulomb_k, double r_cut, int M, double *W_real, double *W_recip)
{
    double *x = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    orc_decode(n, u, L, x);
    double sa = sqrt(alpha);
    int nimg = (int)ceil(r_cut / L) + 1;
    for (int c = 0; c < 6; ++c) W_real[c] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            for (int a = -nimg; a <= nimg; ++a)
                for (int b = -nimg; b <= nimg; ++b)
                    for (int c = -nimg; c <= nimg; ++c) {
                        if (i == j && a == 0 && b == 0 && c == 0) continue;
                        double r3[3] = {x[3 * i] - x[3 * j] + a * L,
                                        x[3 * i + 1] - x[3 * j + 1] + b * L,
                                        x[3 * i + 2] - x[3 * j + 2] + c * L};
                        double r = sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
                        if (r >= r_cut) continue;
                        double qq = coulomb_k * q[i] * q[j];
                        double g = qq * (erfc(sa * r) / (r * r) +
                                         2.0 * sa / sqrt(ORC_PI) * exp(-alpha * r * r) / r);
                        double f[3] = {g * r3[0] / r, g * r3[1] / r, g * r3[2] / r};
                        W_real[0] += 0.5 * r3[0] * f[0];
                        W_real[1] += 0.5 * r3[1] * f[1];
                        W_real[2] += 0.5 * r3[2] * f[2];
                        W_real[3] += 0.5 * r3[0] * f[1];
                        W_real[4] += 0.5 * r3[0] * f[2];
                        W_real[5] += 0.5 * r3[1] * f[2];
                    }
    int64_t nm = orc_full_modes(L, alpha, M, NULL, NULL);
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * nm));
    double *W = (double *)malloc(sizeof(double) * (size_t)nm);
    orc_full_modes(L, alpha, M, m, W);
    orc_mode_virial(n, u, q, L, alpha, coulomb_k, nm, m, W, W_recip);
    free(W);
    free(m);
    free(x);
}

/* ------------------------------------------------------------------------ */
/* Random batch list, Sec. 2.3 (Eqs. 13-16) and Algorithm 2.                 */
/*                                                                          */
/* Readings:                                                                */
/*  - names: r_core is the paper's inner radius r_c, r_cut its outer r_s;   */
/*  - membership is decided on integers: d = (int32)(u_j - u_i) per          */
/*    dimension (the minimum image), D = sum d^2 in uint64, core if          */
/*    D < Rc2, shell if Rc2 <= D <= Rs2 (Eq. 13 read literally), with        */
/*    R2 = floor((r * 2^32 / L)^2);                                          */
/*  - the batch B(i) is a uniform p-subset of S(i) without replacement: the  */
/*    p shell members with the smallest 64-bit priority                      */
/*    Philox(ctr = (i, j, step, STREAM_RBL | replica<<8), key = seed),       */
/*    words w0<<32 | w1, ties to the smaller j; if N_s <= p, B = S;          */
/*  - shell weight N_s/p (Eq. 15), 1 when N_s <= p;                         */
/*  - pair force = erfc-Coulomb (Eq. 10) + LJ (Eq. 2) with Lorentz-Berthelot */
/*    mixing (Eq. 4), both truncated at r_cut without a shift;              */
/*  - F_corr = -(1/N) sum_i (F_core + F_shell*) over all atoms (Eq. 16);     */
/*  - energy: E = 1/2 sum_i [sum_{C(i)} u_ij + w_i sum_{B(i)} u_ij] (the     */
/*    paper gives no energy for the batched list).                          */
/* Atom ids are the array indices.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    const uint32_t *u;
    const double *q;
    const int32_t *type;
    int32_t n_types;
    const double *eps;
    const double *sig;
    double L, alpha, coulomb_k, r_core, r_cut;
    int32_t p;
    uint64_t seed;
    int64_t step;
    uint32_t replica;
    int32_t exact; /* 1: every shell member kept with weight 1 */
    uint64_t Rc2, Rs2;
    /* cell list (only when use_cells) */
    int32_t nc;
    int64_t *cell_start;
    int64_t *cell_atoms;
} orc_rbl_sys;

uint64_t orc_rbl_R2(double r, double L)
{
    double s = r * (ORC_TWO32 / L);
    return (uint64_t)floor(s * s);
}

/* Classify pair (i, j): 0 none, 1 core, 2 shell. */
static int orc_classify(const orc_rbl_sys *S, int64_t i, int64_t j)
{
    if (i == j) return 0;
    uint64_t D = 0;
    for (int d = 0; d < 3; ++d) {
        int32_t dd = (int32_t)(S->u[3 * j + d] - S->u[3 * i + d]);
        int64_t e = (int64_t)dd;
        D += (uint64_t)(e * e);
    }
    if (D < S->Rc2) return 1;
    if (D <= S->Rs2) return 2;
    return 0;
}

static uint64_t orc_priority(const orc_rbl_sys *S, int64_t i, int64_t j)
{
    uint32_t key[2], w[4];
    orc_seed_key(S->seed, key);
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)j, (uint32_t)S->step,
                       ORC_STREAM_RBL | (S->replica << 8)};
    orc_philox4x32_10(ctr, key, w);
    return ((uint64_t)w[0] << 32) | w[1];
}

/* Pair energy and the force on i from j (vector along r_i - r_j, min image).
 * rij (may be NULL) receives r_i - r_j, gparts (may be NULL) the Coulomb and LJ
 * parts of -dU/dr. */
static void orc_pair(const orc_rbl_sys *S, const double *x, int64_t i, int64_t j,
                     double *e_coul, double *e_lj, double f[3], double rij[3], double gparts[2])
{
    double r3[3];
    for (int d = 0; d < 3; ++d) {
        double dd = x[3 * i + d] - x[3 * j + d];
        dd -= S->L * nearbyint(dd / S->L);
        r3[d] = dd;
    }
    double r = sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
    double sa = sqrt(S->alpha);
    double qq = S->coulomb_k * S->q[i] * S->q[j];
    int ti = S->type[i], tj = S->type[j];
    double eps = sqrt(S->eps[ti] * S->eps[tj]);
    double sig = 0.5 * (S->sig[ti] + S->sig[tj]);
    double sr6 = pow(sig / r, 6.0);
    double sr12 = sr6 * sr6;
    *e_coul = qq * erfc(sa * r) / r;
    *e_lj = 4.0 * eps * (sr12 - sr6);
    /* -dU/dr */
    double gc = qq * (erfc(sa * r) / (r * r) + 2.0 * sa / sqrt(ORC_PI) * exp(-S->alpha * r * r) / r);
    double gl = 24.0 * eps * (2.0 * sr12 - sr6) / r;
    double g = gc + gl;
    for (int d = 0; d < 3; ++d) f[d] = g * r3[d] / r;
    if (rij) for (int d = 0; d < 3; ++d) rij[d] = r3[d];
    if (gparts) { gparts[0] = gc; gparts[1] = gl; }
}

/* Adds s * r (x) (g r / |r|) to the 6-component tensor acc (xx yy zz xy xz yz). */
static void orc_add_virial(double *acc, double s, const double r3[3], double g)
{
    double r = sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
    double h = s * g / r;
    acc[0] += h * r3[0] * r3[0];
    acc[1] += h * r3[1] * r3[1];
    acc[2] += h * r3[2] * r3[2];
    acc[3] += h * r3[0] * r3[1];
    acc[4] += h * r3[0] * r3[2];
    acc[5] += h * r3[1] * r3[2];
}

/* Candidate enumeration: brute force over all j, or the 27 (deduplicated)
 * neighbour cells of a plain cell list with cells of side >= r_cut. */
typedef struct {
    int64_t *ids;
    int64_t count, cap;
} orc_list;

static void orc_list_push(orc_list *l, int64_t v)
{
    if (l->count == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 64;
        l->ids = (int64_t *)realloc(l->ids, sizeof(int64_t) * (size_t)l->cap);
    }
    l->ids[l->count++] = v;
}

static int orc_cell_of(uint32_t uc, int32_t nc)
{
    return (int)(((uint64_t)uc * (uint64_t)nc) >> 32);
}

static void orc_candidates(const orc_rbl_sys *S, int64_t i, orc_list *out)
{
    out->count = 0;
    if (!S->cell_start) {
        for (int64_t j = 0; j < S->n; ++j) orc_list_push(out, j);
        return;
    }
    int nc = S->nc;
    int ci[3];
    for (int d = 0; d < 3; ++d) ci[d] = orc_cell_of(S->u[3 * i + d], nc);
    /* distinct neighbour offsets per dimension */
    int offs[3], noff;
    if (nc >= 3) { offs[0] = -1; offs[1] = 0; offs[2] = 1; noff = 3; }
    else if (nc == 2) { offs[0] = 0; offs[1] = 1; noff = 2; }
    else { offs[0] = 0; noff = 1; }
    for (int a = 0; a < noff; ++a)
        for (int b = 0; b < noff; ++b)
            for (int c = 0; c < noff; ++c) {
                int cx = (ci[0] + offs[a] + nc) % nc;
                int cy = (ci[1] + offs[b] + nc) % nc;
                int cz = (ci[2] + offs[c] + nc) % nc;
                int64_t cell = ((int64_t)cx * nc + cy) * nc + cz;
                for (int64_t k = S->cell_start[cell]; k < S->cell_start[cell + 1]; ++k)
                    orc_list_push(out, S->cell_atoms[k]);
            }
}

/* Per-atom classification and batch.  batch_out: p entries, ids ascending,
 * -1 padded.  Returns weight w_i. */
static double orc_rbl_lists(const orc_rbl_sys *S, int64_t i, orc_list *cand, orc_list *core,
                            orc_list *shell, int64_t *batch, int32_t *nb_out)
{
    orc_candidates(S, i, cand);
    core->count = 0;
    shell->count = 0;
    for (int64_t k = 0; k < cand->count; ++k) {
        int64_t j = cand->ids[k];
        int c = orc_classify(S, i, j);
        if (c == 1) orc_list_push(core, j);
        else if (c == 2) orc_list_push(shell, j);
    }
    int64_t Ns = shell->count;
    int p = S->p;
    int32_t nb = 0;
    double w = 1.0;
    if (S->exact || Ns <= p) {
        for (int64_t k = 0; k < Ns; ++k) batch[nb++] = shell->ids[k];
    } else {
        /* p smallest (priority, id) by repeated selection over the shell */
        uint64_t *pr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)Ns);
        char *taken = (char *)calloc((size_t)Ns, 1);
        for (int64_t k = 0; k < Ns; ++k) pr[k] = orc_priority(S, i, shell->ids[k]);
        for (int t = 0; t < p; ++t) {
            int64_t best = -1;
            for (int64_t k = 0; k < Ns; ++k) {
                if (taken[k]) continue;
                if (best < 0 || pr[k] < pr[best] ||
                    (pr[k] == pr[best] && shell->ids[k] < shell->ids[best]))
                    best = k;
            }
            taken[best] = 1;
            batch[nb++] = shell->ids[best];
        }
        free(taken);
        free(pr);
        w = (double)Ns / (double)p;
    }
    /* ids ascending for comparison */
    for (int a = 1; a < nb; ++a) {
        int64_t v = batch[a];
        int b = a - 1;
        while (b >= 0 && batch[b] > v) { batch[b + 1] = batch[b]; --b; }
        batch[b + 1] = v;
    }
    *nb_out = nb;
    return w;
}

static void orc_build_cells(orc_rbl_sys *S)
{
    int nc = (int)floor(S->L / S->r_cut);
    if (nc < 1) nc = 1;
    S->nc = nc;
    int64_t ncell = (int64_t)nc * nc * nc;
    S->cell_start = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    S->cell_atoms = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->n > 0 ? S->n : 1));
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->n > 0 ? S->n : 1));
    for (int64_t i = 0; i < S->n; ++i) {
        int cx = orc_cell_of(S->u[3 * i], nc), cy = orc_cell_of(S->u[3 * i + 1], nc),
            cz = orc_cell_of(S->u[3 * i + 2], nc);
        cell_of[i] = ((int64_t)cx * nc + cy) * nc + cz;
        S->cell_start[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) S->cell_start[c + 1] += S->cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, S->cell_start, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < S->n; ++i) S->cell_atoms[fill[cell_of[i]]++] = i;
    free(fill);
    free(cell_of);
}

/*
 * orc_rbl: short-range forces of Algorithm 2.
 *   sel/n_sel : atoms whose outputs are wanted (all if sel == NULL)
 *   F_out     : [n_sel][3] F_core + F_shell* (before the correction)
 *   n_core/n_shell/n_batch/batch : per selected atom; batch [n_sel][p] ids
 *               ascending, -1 padded (batch only if p-width fits; any may be NULL)
 *   Fsum_out  : sum over ALL atoms of F_core + F_shell* (so F_corr = -Fsum/N)
 *   E_coul_out, E_lj_out : energy of Sec. 2.3 reading, over ALL atoms
 *   W_coul_out, W_lj_out : (may be NULL) virial tensors [6] (xx yy zz xy xz yz)
 *               of the erfc-Coulomb and LJ parts of that energy, over ALL
 *               atoms: W = -dE/d(strain) with the list weights held fixed,
 *               1/2 sum_i [sum_{C(i)} r_ij (x) F_ij + w_i sum_{B(i)} r_ij (x) F_ij],
 *               r_ij = r_i - r_j (minimum image), F_ij the pair force on i.
 *               The momentum correction (Eq. 16) is not a pair force and
 *               adds nothing (reading).
 *   want_all  : 1 to evaluate every atom (needed for Fsum and energies)
 */
void orc_rbl(int64_t n, const uint32_t *u, const double *q, const int32_t *type,
             int32_t n_types, const double *eps, const double *sig, double L, double alpha,
             double coulomb_k, double r_core, double r_cut, int32_t p, uint64_t seed,
             int64_t step, uint32_t replica, int32_t exact, int32_t use_cells, int64_t n_sel,
             const int64_t *sel, double *F_out, int32_t *n_core, int32_t *n_shell,
             int32_t *n_batch, int64_t *batch, int32_t want_all, double *Fsum_out,
             double *E_coul_out, double *E_lj_out, double *W_coul_out, double *W_lj_out)
{
    orc_rbl_sys S;
    memset(&S, 0, sizeof(S));
    S.n = n; S.u = u; S.q = q; S.type = type; S.n_types = n_types; S.eps = eps; S.sig = sig;
    S.L = L; S.alpha = alpha; S.coulomb_k = coulomb_k; S.r_core = r_core; S.r_cut = r_cut;
    S.p = p; S.seed = seed; S.step = step; S.replica = replica; S.exact = exact;
    S.Rc2 = orc_rbl_R2(r_core, L);
    S.Rs2 = orc_rbl_R2(r_cut, L);
    if (use_cells) orc_build_cells(&S);
    double *x = (double *)malloc(sizeof(double) * (size_t)(3 * (n > 0 ? n : 1)));
    orc_decode(n, u, L, x);

    /* per-atom evaluation; the sums over atoms are kept per thread (atoms in
     * contiguous static chunks) and added in thread order */
    enum { ACC_F = 0, ACC_EC = 3, ACC_EL = 4, ACC_WC = 5, ACC_WL = 11, ACC_N = 17 };
    const int nth = orc_threads;
    double *acc_all = (double *)calloc((size_t)nth * ACC_N, sizeof(double));
    int64_t ns = sel ? n_sel : n;
    int64_t nloop = want_all ? n : ns;
    /* map atom -> selected slot when both are needed */
    int64_t *slot = NULL;
    if (sel && want_all) {
        slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) slot[i] = -1;
        for (int64_t s = 0; s < n_sel; ++s) slot[sel[s]] = s;
    }
#pragma omp parallel num_threads(nth)
    {
        double *acc = acc_all + (size_t)orc_thread_id() * ACC_N;
        orc_list cand = {0}, core = {0}, shell = {0};
        int64_t cap_b = 16;
        int64_t *bt = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap_b);
#pragma omp for schedule(static)
        for (int64_t it = 0; it < nloop; ++it) {
            int64_t i, s;
            if (want_all) { i = it; s = sel ? slot[i] : i; }
            else { s = it; i = sel ? sel[it] : it; }
            orc_candidates(&S, i, &cand);
            if (cand.count > cap_b) {
                cap_b = cand.count;
                bt = (int64_t *)realloc(bt, sizeof(int64_t) * (size_t)cap_b);
            }
            int32_t nb = 0;
            double w = orc_rbl_lists(&S, i, &cand, &core, &shell, bt, &nb);
            double Fi[3] = {0, 0, 0}, ec, el, f[3], r3[3], gp[2];
            for (int64_t k = 0; k < core.count; ++k) {
                orc_pair(&S, x, i, core.ids[k], &ec, &el, f, r3, gp);
                acc[ACC_EC] += 0.5 * ec; acc[ACC_EL] += 0.5 * el;
                orc_add_virial(acc + ACC_WC, 0.5, r3, gp[0]);
                orc_add_virial(acc + ACC_WL, 0.5, r3, gp[1]);
                for (int d = 0; d < 3; ++d) Fi[d] += f[d];
            }
            double Fb[3] = {0, 0, 0};
            for (int k = 0; k < nb; ++k) {
                orc_pair(&S, x, i, bt[k], &ec, &el, f, r3, gp);
                acc[ACC_EC] += 0.5 * w * ec; acc[ACC_EL] += 0.5 * w * el;
                orc_add_virial(acc + ACC_WC, 0.5 * w, r3, gp[0]);
                orc_add_virial(acc + ACC_WL, 0.5 * w, r3, gp[1]);
                for (int d = 0; d < 3; ++d) Fb[d] += f[d];
            }
            for (int d = 0; d < 3; ++d) Fi[d] += w * Fb[d];
            for (int d = 0; d < 3; ++d) acc[ACC_F + d] += Fi[d];
            if (s >= 0) {
                if (F_out) for (int d = 0; d < 3; ++d) F_out[3 * s + d] = Fi[d];
                if (n_core) n_core[s] = (int32_t)core.count;
                if (n_shell) n_shell[s] = (int32_t)shell.count;
                if (n_batch) n_batch[s] = nb;
                if (batch) {
                    for (int k = 0; k < p; ++k) batch[(int64_t)p * s + k] = (k < nb) ? bt[k] : -1;
                }
            }
        }
        free(bt);
        free(cand.ids); free(core.ids); free(shell.ids);
    }
    double tot[ACC_N];
    for (int c = 0; c < ACC_N; ++c) tot[c] = 0.0;
    for (int t = 0; t < nth; ++t)
        for (int c = 0; c < ACC_N; ++c) tot[c] += acc_all[(size_t)t * ACC_N + c];
    free(acc_all);
    if (Fsum_out) for (int d = 0; d < 3; ++d) Fsum_out[d] = tot[ACC_F + d];
    if (E_coul_out) *E_coul_out = tot[ACC_EC];
    if (E_lj_out) *E_lj_out = tot[ACC_EL];
    if (W_coul_out) for (int c = 0; c < 6; ++c) W_coul_out[c] = tot[ACC_WC + c];
    if (W_lj_out) for (int c = 0; c < 6; ++c) W_lj_out[c] = tot[ACC_WL + c];
    free(slot);
    free(x);
    free(S.cell_start);
    free(S.cell_atoms);
}

/* ------------------------------------------------------------------------ */
/* Total nonbonded force of one step: RBE (Eq. 12) + RBL (Eqs. 14-15) with   */
/* the momentum correction of Eq. 16 added to every atom.  F_out: [n][3].    */
/* E_out (may be NULL): [4] = {E_coul_real, E_lj, E_rbe, E_self}.            */
/* ------------------------------------------------------------------------ */
void orc_forces(int64_t n, const uint32_t *u, const double *q, const int32_t *type,
                int32_t n_types, const double *eps, const double *sig, double L, double alpha,
                double coulomb_k, double r_core, double r_cut, int32_t p, int32_t P,
                uint64_t seed, int64_t step, uint32_t replica, int32_t exact, double *F_out,
                double *E_out)
{
    double *Fr = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    double *Fs = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    double Erbe = 0.0, Ec = 0.0, El = 0.0, Fsum[3];
    orc_rbe_forces(n, u, q, L, alpha, coulomb_k, P, seed, step, replica, 0, NULL, Fr, &Erbe,
                   NULL, NULL);
    orc_rbl(n, u, q, type, n_types, eps, sig, L, alpha, coulomb_k, r_core, r_cut, p, seed, step,
            replica, exact, 1, 0, NULL, Fs, NULL, NULL, NULL, NULL, 1, Fsum, &Ec, &El, NULL,
            NULL);
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            F_out[3 * i + d] = Fr[3 * i + d] + Fs[3 * i + d] - Fsum[d] / (double)n;
    if (E_out) {
        double q2 = 0.0;
        for (int64_t i = 0; i < n; ++i) q2 += q[i] * q[i];
        E_out[0] = Ec;
        E_out[1] = El;
        E_out[2] = Erbe;
        E_out[3] = -coulomb_k * sqrt(alpha / ORC_PI) * q2;
    }
    free(Fs);
    free(Fr);
}

/* ------------------------------------------------------------------------ */
/* Metropolis mode chains (Algorithm 1 step 1: the paper draws the modes by  */
/* the Metropolis procedure).  Reading: P independent chains, one per mode   */
/* slot, each a random walk on Z^3 \ {0} with the symmetric proposal         */
/* m' = m + delta e_d (axis d uniform, delta = +-1) accepted with            */
/* min(1, exp(-a (|m'|^2 - |m|^2))), a = pi^2/(alpha L^2); m' = 0 rejected.    */
/* |m'|^2 - |m|^2 = 2 delta m_d + 1: moves that lower |m| are always        */
/* accepted; the others, with k = |m_d|, when the 64-bit uniform U is below  */
/* A_k = min(2^64 - 1, floor(exp(-a (2k + 1)) 2^64)), k = 0..2M (beyond 2M   */
/* the move is rejected: exp(-a (4M + 1)) < 1e-32).                          */
/* Chain l starts at step 0 from the exact draw of step 0 (orc_rbe_sample),   */
/* so it is stationary from the start; every later step s makes `moves`       */
/* moves; move t uses Philox(ctr = (l, t, s, 4 | replica<<8), key = seed):    */
/* d = w0 mod 3, delta = +1 if w1 is odd else -1, U = w2<<32 | w3.           */
/* ------------------------------------------------------------------------ */
void orc_metropolis_table(double L, double alpha, int M, uint64_t *A)
{
    const double a = ORC_PI * ORC_PI / (alpha * L * L);
    for (int k = 0; k <= 2 * M; ++k) {
        double x = exp(-a * (2.0 * k + 1.0)) * ORC_TWO64;
        A[k] = (x >= ORC_TWO64) ? UINT64_MAX : (uint64_t)x;
    }
}

void orc_rbe_metropolis(uint64_t seed, int64_t step, uint32_t replica, int P, double L,
                        double alpha, int moves, int32_t *m_out)
{
    orc_rbe_sample(seed, 0, replica, P, L, alpha, m_out);
    const int M = orc_sampler_M(L, alpha);
    uint64_t *A = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
    orc_metropolis_table(L, alpha, M, A);
    uint32_t key[2];
    orc_seed_key(seed, key);
    for (int l = 0; l < P; ++l) {
        int32_t *m = m_out + 3 * l;
        for (int64_t st = 1; st <= step; ++st) {
            for (int t = 0; t < moves; ++t) {
                uint32_t ctr[4] = {(uint32_t)l, (uint32_t)t, (uint32_t)st,
                                   ORC_STREAM_METROPOLIS | (replica << 8)};
                uint32_t w[4];
                orc_philox4x32_10(ctr, key, w);
                const int d = (int)(w[0] % 3u);
                const int delta = (w[1] & 1u) ? 1 : -1;
                const uint64_t U = ((uint64_t)w[2] << 32) | w[3];
                int32_t mn[3] = {m[0], m[1], m[2]};
                mn[d] += delta;
                if (mn[0] == 0 && mn[1] == 0 && mn[2] == 0) continue;
                int accept;
                if (delta * m[d] < 0) {
                    accept = 1;
                } else {
                    const int k = m[d] < 0 ? -m[d] : m[d];
                    accept = k <= 2 * M && U < A[k];
                }
                if (accept) m[d] = mn[d];
            }
        }
    }
    free(A);
}

/* ------------------------------------------------------------------------ */
/* Standard normal deviates of the Langevin random force for atom `id` at    */
/* force evaluation `step`: one Philox4x32-10 call, key = seed, counter      */
/* (id, step, 0, 3 | replica << 8); uniforms u_k = (w_k + 1/2) / 2^32 in     */
/* (0, 1); Box-Muller: g_x, g_y = sqrt(-2 ln u_0) (cos, sin)(2 pi u_1),      */
/* g_z = sqrt(-2 ln u_2) cos(2 pi u_3).                                      */
/* ------------------------------------------------------------------------ */
void orc_langevin_normals(uint64_t seed, uint32_t id, int64_t step, uint32_t replica,
                          double g[3])
{
    uint32_t key[2], w[4];
    orc_seed_key(seed, key);
    const uint32_t ctr[4] = {id, (uint32_t)step, 0u, ORC_STREAM_LANGEVIN | (replica << 8)};
    orc_philox4x32_10(ctr, key, w);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)w[k] + 0.5) / ORC_TWO32;
    const double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    g[0] = r0 * cos(2.0 * ORC_PI * u[1]);
    g[1] = r0 * sin(2.0 * ORC_PI * u[1]);
    g[2] = r1 * cos(2.0 * ORC_PI * u[3]);
}

/* ------------------------------------------------------------------------ */
/* Velocity-Verlet (Sec. 2.1) with the thermostats of Sec. 2.1.             */
/* Readings: unit masses and k_B = 1 (reduced units, Sec. 4.1); positions    */
/* are the fixed-point u, drifted by rint(v_d * (dt * 2^32 / L)) and wrapped */
/* mod 2^32; T = 2 KE / g with g = 3N - 3 degrees of freedom.                */
/*  thermostat 0: none (NVE).                                                */
/*  thermostat 1: Berendsen, lambda = sqrt(1 + (dt/tau)(T0/T - 1)) clamped   */
/*     to [0.8, 1.25], applied to v after the second half-kick.              */
/*  thermostat 2: Langevin (Schneider-Stoll): after the forces of the new    */
/*     configuration, every atom gets F_L = -gamma v + sqrt(2 gamma T0 / dt) */
/*     G with gamma = 1/tau, v the half-step velocity and G standard normal  */
/*     (orc_langevin_normals, keyed by the step of that force evaluation);   */
/*     F + F_L drives the second half-kick and the next first half-kick.     */
/*  thermostat 3: Nose-Hoover, one thermostat variable xi, Q = g T0 tau^2,   */
/*     symmetric splitting: xi += dt/2 (2 KE - g T0)/Q; v *= e^{-xi dt/2};  */
/*     half-kick, drift, forces, half-kick; v *= e^{-xi dt/2};               */
/*     xi += dt/2 (2 KE - g T0)/Q (KE of the scaled velocities).             */
/*     *xi (in/out) carries the variable between calls.                      */
/*  thermostat 4: energy bath (NVE; Sec. 2.1 names the scheme without its    */
/*     steps).  Reading: a Berendsen-type relaxation of the total energy     */
/*     H = K + U toward the bath energy E0 (*xi, unchanged), with U the      */
/*     potential (all four terms of orc_forces, the random batches of that   */
/*     step) of the new configuration and K the kinetic energy after the     */
/*     second half-kick: K -> K + (dt/tau)(E0 - U - K), i.e.                 */
/*     lambda^2 = a = 1 + (dt/tau)((E0 - U)/K - 1), lambda = sqrt(a) with a  */
/*     clamped to [0.64, 1.5625] (lambda in [0.8, 1.25], as Berendsen); no  */
/*     rescale when K = 0.  tau = dt puts H at E0 after every step.          */
/* One call advances step0 -> step0 + n_steps.  F (in/out): the forces used  */
/* by the first half-kick (those of step0, plus its Langevin force if any);  */
/* on return those of step0 + n_steps.                                       */
/* ------------------------------------------------------------------------ */
static double orc_kinetic(int64_t n, const double *v)
{
    double ke = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) ke += 0.5 * v[i] * v[i];
    return ke;
}

void orc_vv(int64_t n, uint32_t *u, double *v, double *F, const double *q, const int32_t *type,
            int32_t n_types, const double *eps, const double *sig, double L, double alpha,
            double coulomb_k, double r_core, double r_cut, int32_t p, int32_t P, uint64_t seed,
            int64_t step0, uint32_t replica, int32_t exact, double dt, int32_t thermostat,
            double T0, double tau, int64_t n_steps, double *xi)
{
    double c = dt * (ORC_TWO32 / L);
    const double g = 3.0 * (double)n - 3.0;
    const double Q = g * T0 * tau * tau;
    for (int64_t s = 0; s < n_steps; ++s) {
        if (thermostat == 3 && n > 1) {
            *xi += 0.5 * dt * (2.0 * orc_kinetic(n, v) - g * T0) / Q;
            const double f = exp(-0.5 * dt * *xi);
            for (int64_t i = 0; i < 3 * n; ++i) v[i] *= f;
        }
        for (int64_t i = 0; i < 3 * n; ++i) {
            v[i] += 0.5 * dt * F[i];
            int64_t du = (int64_t)nearbyint(v[i] * c);
            u[i] = (uint32_t)((uint64_t)u[i] + (uint64_t)du);
        }
        double E[4] = {0.0, 0.0, 0.0, 0.0};
        orc_forces(n, u, q, type, n_types, eps, sig, L, alpha, coulomb_k, r_core, r_cut, p, P,
                   seed, step0 + s + 1, replica, exact, F, E);
        if (thermostat == 2) {
            const double gamma = 1.0 / tau, sd = sqrt(2.0 * gamma * T0 / dt);
            for (int64_t i = 0; i < n; ++i) {
                double gn[3];
                orc_langevin_normals(seed, (uint32_t)i, step0 + s + 1, replica, gn);
                for (int d = 0; d < 3; ++d) F[3 * i + d] += -gamma * v[3 * i + d] + sd * gn[d];
            }
        }
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * F[i];
        if (thermostat == 1 && n > 1) {
            double T = 2.0 * orc_kinetic(n, v) / g;
            double lam = sqrt(1.0 + (dt / tau) * (T0 / T - 1.0));
            if (lam < 0.8) lam = 0.8;
            if (lam > 1.25) lam = 1.25;
            for (int64_t i = 0; i < 3 * n; ++i) v[i] *= lam;
        }
        if (thermostat == 3 && n > 1) {
            const double f = exp(-0.5 * dt * *xi);
            for (int64_t i = 0; i < 3 * n; ++i) v[i] *= f;
            *xi += 0.5 * dt * (2.0 * orc_kinetic(n, v) - g * T0) / Q;
        }
        if (thermostat == 4) {
            const double K = orc_kinetic(n, v);
            const double U = E[0] + E[1] + E[2] + E[3];
            if (K > 0.0) {
                const double a = 1.0 + (dt / tau) * ((*xi - U) / K - 1.0);
                const double lam = a <= 0.64 ? 0.8 : (a >= 1.5625 ? 1.25 : sqrt(a));
                for (int64_t i = 0; i < 3 * n; ++i) v[i] *= lam;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Gradients of the total potential of one step,                            */
/*   E = E_coul_real + E_lj + E_rbe + E_self,                               */
/* with the list energy E_RBL = 1/2 sum_i sum_j W_ij u_ij (W_ij = 1 for j in */
/* C(i), N_s(i)/p for j in B(i), 0 otherwise; u_ij = coulomb_k q_i q_j       */
/* erfc(sqrt(alpha) r)/r + 4 eps_ij[(sigma_ij/r)^12 - (sigma_ij/r)^6],        */
/* Eqs. 2, 4, 10), the RBE estimate E_rbe = coulomb_k (2 pi S/(V P))         */
/* sum_l |rho_l|^2 / k_l^2 and E_self = -coulomb_k sqrt(alpha/pi) sum q^2.   */
/* The weights W are held fixed (they change only when a list membership    */
/* changes, where E is discontinuous).  Chain rule pair by pair: each       */
/* ordered pair (i, j) adds 1/2 W_ij du_ij to both atoms it touches.        */
/* Outputs: E_out[4] (as orc_forces), dr [n][3], dq [n], deps [T], dsig [T]. */
/* ------------------------------------------------------------------------ */
void orc_energy_grad(int64_t n, const uint32_t *u, const double *q, const int32_t *type,
                     int32_t n_types, const double *eps, const double *sig, double L,
                     double alpha, double coulomb_k, double r_core, double r_cut, int32_t p,
                     int32_t P, uint64_t seed, int64_t step, uint32_t replica, int32_t exact,
                     double *E_out, double *dr, double *dq, double *deps, double *dsig)
{
    double V = L * L * L;
    double sa = sqrt(alpha);
    double *x = (double *)malloc(sizeof(double) * (size_t)(3 * (n > 0 ? n : 1)));
    orc_decode(n, u, L, x);
    for (int64_t s = 0; s < 3 * n; ++s) dr[s] = 0.0;
    for (int64_t i = 0; i < n; ++i) dq[i] = 0.0;
    for (int t = 0; t < n_types; ++t) { deps[t] = 0.0; dsig[t] = 0.0; }
    double Ec = 0.0, El = 0.0;

    /* short range: lists of every atom */
    orc_rbl_sys S;
    memset(&S, 0, sizeof(S));
    S.n = n; S.u = u; S.q = q; S.type = type; S.n_types = n_types; S.eps = eps; S.sig = sig;
    S.L = L; S.alpha = alpha; S.coulomb_k = coulomb_k; S.r_core = r_core; S.r_cut = r_cut;
    S.p = p; S.seed = seed; S.step = step; S.replica = replica; S.exact = exact;
    S.Rc2 = orc_rbl_R2(r_core, L);
    S.Rs2 = orc_rbl_R2(r_cut, L);
    orc_build_cells(&S);
    orc_list cand = {0}, core = {0}, shell = {0};
    int64_t cap_b = 16;
    int64_t *bt = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap_b);
    for (int64_t i = 0; i < n; ++i) {
        orc_candidates(&S, i, &cand);
        if (cand.count > cap_b) {
            cap_b = cand.count;
            bt = (int64_t *)realloc(bt, sizeof(int64_t) * (size_t)cap_b);
        }
        int32_t nb = 0;
        double w = orc_rbl_lists(&S, i, &cand, &core, &shell, bt, &nb);
        int64_t ntot = core.count + nb;
        for (int64_t e = 0; e < ntot; ++e) {
            int64_t j = e < core.count ? core.ids[e] : bt[e - core.count];
            double W = e < core.count ? 1.0 : w;
            double r3[3];
            for (int d = 0; d < 3; ++d) {
                double dd = x[3 * i + d] - x[3 * j + d];
                dd -= L * nearbyint(dd / L);
                r3[d] = dd;
            }
            double r = sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
            int a = type[i], b = type[j];
            double eij = sqrt(eps[a] * eps[b]);
            double sij = 0.5 * (sig[a] + sig[b]);
            double sr6 = pow(sij / r, 6.0), sr12 = sr6 * sr6;
            double erfr = erfc(sa * r) / r;
            double uc = coulomb_k * q[i] * q[j] * erfr;
            double ul = 4.0 * eij * (sr12 - sr6);
            Ec += 0.5 * W * uc;
            El += 0.5 * W * ul;
            /* du/dr */
            double duc = -coulomb_k * q[i] * q[j] *
                         (erfc(sa * r) / (r * r) + 2.0 * sa / sqrt(ORC_PI) * exp(-alpha * r * r) / r);
            double dul = -24.0 * eij * (2.0 * sr12 - sr6) / r;
            double g = 0.5 * W * (duc + dul);
            for (int d = 0; d < 3; ++d) {
                dr[3 * i + d] += g * r3[d] / r;
                dr[3 * j + d] -= g * r3[d] / r;
            }
            /* charges */
            dq[i] += 0.5 * W * coulomb_k * q[j] * erfr;
            dq[j] += 0.5 * W * coulomb_k * q[i] * erfr;
            /* LJ parameters through Lorentz-Berthelot (Eq. 4) */
            double due = 4.0 * (sr12 - sr6);                   /* du/d eps_ij */
            double dus = 4.0 * eij * (12.0 * sr12 - 6.0 * sr6) / sij; /* du/d sigma_ij */
            deps[a] += 0.5 * W * due * 0.5 * sqrt(eps[b] / eps[a]);
            deps[b] += 0.5 * W * due * 0.5 * sqrt(eps[a] / eps[b]);
            dsig[a] += 0.5 * W * dus * 0.5;
            dsig[b] += 0.5 * W * dus * 0.5;
        }
    }
    free(bt);
    free(cand.ids); free(core.ids); free(shell.ids);
    free(S.cell_start);
    free(S.cell_atoms);

    /* RBE estimate: E = sum_l Wl (2 pi/V) |rho_l|^2/k^2 with Wl = coulomb_k S / P */
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * (P > 0 ? P : 1)));
    orc_rbe_sample(seed, step, replica, P, L, alpha, m);
    double Ssum = orc_rbe_S(L, alpha);
    double *rho = (double *)malloc(sizeof(double) * (size_t)(2 * (P > 0 ? P : 1)));
    orc_structure_factor(n, u, q, L, P, m, rho);
    double Erbe = 0.0;
    for (int l = 0; l < P; ++l) {
        double kx = 2.0 * ORC_PI * m[3 * l] / L, ky = 2.0 * ORC_PI * m[3 * l + 1] / L,
               kz = 2.0 * ORC_PI * m[3 * l + 2] / L;
        double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 == 0.0) continue;
        double c = coulomb_k * (Ssum / P) * (2.0 * ORC_PI / V) / k2;
        double re = rho[2 * l], im = rho[2 * l + 1];
        Erbe += c * (re * re + im * im);
        for (int64_t i = 0; i < n; ++i) {
            double th = kx * x[3 * i] + ky * x[3 * i + 1] + kz * x[3 * i + 2];
            double cs = cos(th), sn = sin(th);
            /* d|rho|^2/dq_i = 2 (re cos + im sin); d|rho|^2/dr_i = 2 q_i k (im cos - re sin) */
            dq[i] += c * 2.0 * (re * cs + im * sn);
            double gr = c * 2.0 * q[i] * (im * cs - re * sn);
            dr[3 * i] += gr * kx;
            dr[3 * i + 1] += gr * ky;
            dr[3 * i + 2] += gr * kz;
        }
    }
    free(rho);
    free(m);

    /* self energy */
    double q2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        q2 += q[i] * q[i];
        dq[i] += -2.0 * coulomb_k * sqrt(alpha / ORC_PI) * q[i];
    }
    if (E_out) {
        E_out[0] = Ec;
        E_out[1] = El;
        E_out[2] = Erbe;
        E_out[3] = -coulomb_k * sqrt(alpha / ORC_PI) * q2;
    }
    free(x);
}
