/*
 * orc_moments.c -- moments without a closed form (Sec. 2.3) and the Yukawa kernel (Sec. 3.2) for
 *                  the plain FP64 CPU oracle of arXiv 2107.03958.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.c).  Every routine writes out a definition of the paper:
 *   orc_bessel_k          K0, K1 by the integral K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt.
 *   orc_yukawa_moment     ghat(k) of g = K0(kappa|x|)/(2 pi) in closed form, from the indefinite
 *                         integral int rho K0(kappa rho) J0(s rho) d rho.
 *   orc_ghat_numeric_full ghat(k) = 2 pi p int_0^{a^{1/p}} g(tau^p) J0(s tau^p) tau^{2p-1} d tau
 *                         (Sec. 2.3, the substitution rho = tau^p) with the Clenshaw-Curtis points
 *                         and weights of eq. (cc_pts)/(cc_wts) as printed.
 *   orc_eta               the window eta_beta of Sec. 2.3 (localization).
 *   orc_ghat_localized_full  the multiplier of the localized scheme, eq. (io_split): the moments
 *                         of g eta_beta (trapezoidal rule in tau) plus the DFT of the trapezoidal-
 *                         rule weights h^2 g (1 - eta_beta) of the smooth part.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;
static const double PI = 3.14159265358979323846;

enum { ORC_LOG = 0, ORC_POW = 1, ORC_HELM = 2, ORC_YUKAWA = 3 };

void orc_fft2(int R, int C, double *data, int sign, double scale);
double orc_varkappa(double t);

/* K_nu(x), nu = 0 or 1, x > 0: int_0^inf exp(-x cosh t) cosh(nu t) dt by the trapezoidal rule
 * (the integrand is analytic and decays doubly exponentially, so the rule converges
 * exponentially in 1/h once h resolves the peak at t = 0, whose width is about 1/sqrt(x)):
 * step min(1/16, 1/(4 sqrt x)), summed until x cosh t > 745 (where exp underflows). */
double orc_bessel_k(int nu, double x)
{
    const double h = fmin(1.0 / 16.0, 0.25 / sqrt(x));
    double sum = 0.5 * exp(-x);
    for (int j = 1; j < 100000; ++j) {
        double t = j * h, c = cosh(t);
        if (x * c > 745.0) break;
        sum += exp(-x * c) * (nu ? cosh(t) : 1.0);
    }
    return h * sum;
}

/* 2 pi int_0^a (1/2pi) K0(kappa rho) J0(s rho) rho d rho.  With
 *   F(rho) = rho (s J1(s rho) K0(kappa rho) - kappa J0(s rho) K1(kappa rho)) / (s^2 + kappa^2),
 * F' = rho K0(kappa rho) J0(s rho) (from J0' = -J1, (rho J1)' = rho J0, K0' = -K1,
 * (rho K1)' = -rho K0), and F(0+) = -1/(s^2 + kappa^2) (rho K1(kappa rho) -> 1/kappa), so
 *   ghat = (1 + z J1(z) K0(kappa a) - kappa a J0(z) K1(kappa a)) / (s^2 + kappa^2),  z = s a. */
double orc_yukawa_moment(double kappa, double s, double a)
{
    double ka = kappa * a, z = s * a;
    return (1.0 + z * j1(z) * orc_bessel_k(0, ka) - ka * j0(z) * orc_bessel_k(1, ka)) / (s * s + kappa * kappa);
}

/* g(rho), unscaled: log rho, rho^gamma, (i/4) H0^(1)(kappa rho), K0(kappa rho)/(2 pi). */
static cplx kernel_g(int family, double gamma, double kappa, double rho)
{
    switch (family) {
    case ORC_LOG: return log(rho);
    case ORC_POW: return pow(rho, gamma);
    case ORC_HELM: return (I / 4.0) * (j0(kappa * rho) + I * y0(kappa * rho));
    default: return orc_bessel_k(0, kappa * rho) / (2.0 * PI);
    }
}

/* Eq. (cc_pts), (cc_wts) on [0, alpha], j = 1..npc:
 *   x_j = (alpha/2)(1 + cos((j - 1/2) pi/npc)),
 *   w_j = (alpha/npc) sum'_{k=0}^{npc} theta_k cos((j - 1/2) k pi / npc),
 * theta_k = -2/(k^2 - 1) for even k, 0 for odd k, the k = 0 term halved. */
void orc_cc_rule(int npc, double alpha, double *x, double *w)
{
    for (int j = 1; j <= npc; ++j) {
        double th = (j - 0.5) * PI / npc;
        x[j - 1] = 0.5 * alpha * (1.0 + cos(th));
        double acc = 0.0;
        for (int k = 0; k <= npc; k += 2) {
            double theta = -2.0 / ((double)k * k - 1.0);
            acc += (k == 0 ? 0.5 : 1.0) * theta * cos(k * th);
        }
        w[j - 1] = alpha / npc * acc;
    }
}

/* Writes the quadrant table quad[k1][k2] (h x h, h = M/2 + 1) into the full M x M table at FFT
 * index (k = q for q < M/2, else q - M), reading it by |k1|, |k2|. */
static void quadrant_to_full(const cplx *quad, int M, cplx *o)
{
    int h = M / 2 + 1;
#pragma omp parallel for schedule(static)
    for (int q1 = 0; q1 < M; ++q1) {
        int k1 = q1 < M / 2 ? q1 : M - q1;
        for (int q2 = 0; q2 < M; ++q2) {
            int k2 = q2 < M / 2 ? q2 : M - q2;
            o[(long)q1 * M + q2] = quad[(long)k1 * h + k2];
        }
    }
}

/* Moments by the quadrature of Sec. 2.3: after rho = tau^p,
 *   ghat(k) = 2 pi p int_0^{a^{1/p}} g(tau^p) J0(2 pi |k| tau^p / b) tau^{2p-1} d tau,
 * with the npc-point rule of eq. (cc_pts)/(cc_wts).  M x M table at FFT index, times scale. */
int orc_ghat_numeric_full(int family, double gamma, double kappa, double scale, double b, double a, int p,
                          int npc, int M, double *out)
{
    int h = M / 2 + 1;
    double *x = malloc(sizeof(double) * npc), *w = malloc(sizeof(double) * npc), *xp = malloc(sizeof(double) * npc);
    cplx *gw = malloc(sizeof(cplx) * npc);
    cplx *quad = malloc(sizeof(cplx) * (size_t)h * h);
    if (!x || !w || !xp || !gw || !quad) return 2;
    orc_cc_rule(npc, pow(a, 1.0 / p), x, w);
    for (int j = 0; j < npc; ++j) {
        xp[j] = pow(x[j], p);
        gw[j] = w[j] * kernel_g(family, gamma, kappa, xp[j]) * pow(x[j], 2 * p - 1);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int k1 = 0; k1 < h; ++k1)
        for (int k2 = 0; k2 < h; ++k2) {
            double s = 2.0 * PI * hypot((double)k1, (double)k2) / b;
            cplx acc = 0;
            for (int j = 0; j < npc; ++j) acc += gw[j] * j0(s * xp[j]);
            quad[(long)k1 * h + k2] = scale * 2.0 * PI * p * acc;
        }
    quadrant_to_full(quad, M, (cplx *)out);
    free(x);
    free(w);
    free(xp);
    free(gw);
    free(quad);
    return 0;
}

/* eta_beta(rho) of Sec. 2.3: C-infinity, 1 on [0, beta/2], 0 beyond beta; in between the
 * half-window varkappa of eq. (halfwindow1): eta = varkappa((rho - beta/2) / (beta/2)). */
double orc_eta(double rho, double beta)
{
    if (rho <= 0.5 * beta) return 1.0;
    if (rho >= beta) return 0.0;
    return orc_varkappa((rho - 0.5 * beta) / (0.5 * beta));
}

/* Multiplier of the localized scheme, eq. (io_split), on the M x M grid (M = n b, h = 1/n):
 *   (1) ghat_eta(k) = 2 pi int_0^beta g(rho) eta_beta(rho) J0(s rho) rho d rho, after rho = tau^p by
 *       the trapezoidal rule with npc intervals on [0, beta^{1/p}] (the integrand vanishes to high
 *       order at both ends);
 *   (2) the classical trapezoidal rule for the smooth kernel g (1 - eta_beta): weights
 *       W1(d) = h^2 g(|d| h) (1 - eta_beta(|d| h)) for 0 < |d| h < a, d in [-M/2, M/2)^2, whose
 *       discrete convolution with u is the FFT product with fft2(W1);
 * total: ghat_eta + fft2(W1), times scale, at FFT index. */
int orc_ghat_localized_full(int family, double gamma, double kappa, double scale, double b, double a, int n,
                            double beta, int p, int npc, double *out)
{
    int M = (int)llround(n * b), h = M / 2 + 1;
    double tb = pow(beta, 1.0 / p), ht = tb / npc;
    double *xp = malloc(sizeof(double) * (npc + 1));
    cplx *gw = malloc(sizeof(cplx) * (npc + 1));
    cplx *quad = malloc(sizeof(cplx) * (size_t)h * h);
    if (!xp || !gw || !quad) return 2;
    for (int j = 0; j <= npc; ++j) {
        double tau = j * ht, rho = pow(tau, p);
        xp[j] = rho;
        double wt = (j == 0 || j == npc) ? 0.5 * ht : ht;
        gw[j] = (j == 0) ? 0.0 : wt * kernel_g(family, gamma, kappa, rho) * orc_eta(rho, beta) * pow(tau, 2 * p - 1);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int k1 = 0; k1 < h; ++k1)
        for (int k2 = 0; k2 < h; ++k2) {
            double s = 2.0 * PI * hypot((double)k1, (double)k2) / b;
            cplx acc = 0;
            for (int j = 1; j <= npc; ++j) acc += gw[j] * j0(s * xp[j]);
            quad[(long)k1 * h + k2] = 2.0 * PI * p * acc;
        }
    cplx *o = (cplx *)out;
    quadrant_to_full(quad, M, o);
    cplx *W1 = calloc((size_t)M * M, sizeof(cplx));
    if (!W1) return 2;
    double hh = 1.0 / n;
    for (int q1 = 0; q1 < M; ++q1) {
        int d1 = q1 < M / 2 ? q1 : q1 - M;
        for (int q2 = 0; q2 < M; ++q2) {
            int d2 = q2 < M / 2 ? q2 : q2 - M;
            double r = hypot((double)d1, (double)d2) * hh;
            if (r == 0.0 || r >= a) continue;
            W1[(long)q1 * M + q2] = hh * hh * kernel_g(family, gamma, kappa, r) * (1.0 - orc_eta(r, beta));
        }
    }
    orc_fft2(M, M, (double *)W1, -1, 1.0);
    for (long i = 0; i < (long)M * M; ++i) o[i] = scale * (o[i] + W1[i]);
    free(W1);
    free(xp);
    free(gw);
    free(quad);
    return 0;
}

/* The non-radial kernel of Sec. 3.1: g(x) = -x1 / (2 pi |x|^2) = d/dx1 G with G = -(1/2pi) log|x|.
 * Its moments over B_a (eq. (bk)) in polar coordinates y = rho (cos t, sin t), xi = 2 pi k / b =
 * s (cos p, sin p):
 *   ghat(k) = int_0^a int_0^{2pi} -(cos t / 2pi) exp(-i s rho cos(t - p)) dt d rho
 *           = i cos p int_0^a J1(s rho) d rho = i (xi1 / s) (1 - J0(s a)) / s,      ghat(0) = 0,
 * using int_0^{2pi} cos t exp(-i z cos(t - p)) dt = -2 pi i J1(z) cos p.  It is odd in k1: at the
 * unpaired Nyquist index k1 = -M/2 of F_n the sum of eq. (An) would not return a real A_n u for
 * real u, so that mode's multiplier is taken as 0 (its real part).  M x M table at FFT index
 * (k = q for q < M/2, else q - M), times scale. */
void orc_ghat_full_dx1log(double scale, double b, double a, int M, double *out)
{
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (int q1 = 0; q1 < M; ++q1) {
        long k1 = q1 < M / 2 ? q1 : q1 - M;
        for (int q2 = 0; q2 < M; ++q2) {
            long k2 = q2 < M / 2 ? q2 : q2 - M;
            cplx v = 0;
            if ((k1 != 0 || k2 != 0) && q1 != M / 2) {
                double s = 2.0 * PI * hypot((double)k1, (double)k2) / b;
                double xi1 = 2.0 * PI * (double)k1 / b;
                v = I * scale * xi1 * (1.0 - j0(s * a)) / (s * s);
            }
            o[(long)q1 * M + q2] = v;
        }
    }
}
