/*
 * orc.c -- plain FP64 CPU oracle for the FFT convolution scheme of
 *          Tiwari, Pandey, Paul & Anand, "Fast accurate approximation of convolutions
 *          with weakly singular kernel and its applications" (arXiv 2107.03958).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  The product (CUDA) path shares no code with it and
 * never calls it.
 *
 * Every routine writes out the paper's definition directly, in FP64 / complex128, with no
 * pruning, fusion or blocking:
 *   orc_fft / orc_fft2   discrete Fourier transform (recursive mixed-radix Cooley-Tukey);
 *                        the "FFT" the scheme of eq. (An) in Sec. 2.1 relies on.
 *   orc_ghat_radial      moments ghat(k) of Sec. 2.2: eq. (ghat) and the closed forms that
 *                        follow it (log, Helmholtz with the k=0 sign corrected, |x|^gamma
 *                        via the Lommel-function form), plus plain quadrature where the
 *                        closed form loses digits.
 *   orc_conv             A_n u of eq. (An): crop_n( ifft2( ghat (.) fft2( zero-extend_M(u) ) ) ).
 *   orc_direct           the quadrature form eq. (quad)/(quad_wts): an O(n^4) double sum
 *                        with weights w(d) built by plain sums (no FFT).
 *   orc_fs_mask          Fourier smoothing of Sec. 2.4: chi^n_Omega of eq. (tfs) times psi.
 *   orc_gmres            restarted GMRES for the Nystrom system eq. (descretls) of Sec. 3.3.
 *
 * Complex arrays cross the ABI as interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;
#define PI_L 3.141592653589793238462643383279502884L
static const double PI = 3.14159265358979323846;

enum { ORC_LOG = 0, ORC_POW = 1, ORC_HELM = 2, ORC_YUKAWA = 3 };

double orc_yukawa_moment(double kappa, double s, double a); /* orc_moments.c */

/* ------------------------------------------------------------------------------------------
 * Discrete Fourier transform.
 *   X[k] = sum_{j<N} x[j] exp(sign * 2 pi i j k / N)
 * computed by recursive decimation in time over the smallest prime factor p of N:
 *   X[q + m r] = sum_{s<p} exp(sign 2 pi i s (q + m r)/N) * FFT_m(x[s], x[s+p], ...)[q],  N = p m.
 * ------------------------------------------------------------------------------------------ */
static int least_factor(int n)
{
    for (int p = 2; (long)p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* w[t] = exp(sign 2 pi i t / N) for t in [0, N), evaluated in long double. */
static cplx *twiddle_table(int N, int sign)
{
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    for (int t = 0; t < N; ++t) {
        long double ang = 2.0L * PI_L * (long double)t / (long double)N;
        w[t] = (double)cosl(ang) + I * ((double)sign * (double)sinl(ang));
    }
    return w;
}

static void fft_rec(int N, const cplx *in, long istride, cplx *out, const cplx *w, long wstride,
                    cplx *tmp)
{
    if (N == 1) {
        out[0] = in[0];
        return;
    }
    int p = least_factor(N), m = N / p;
    for (int s = 0; s < p; ++s)
        fft_rec(m, in + s * istride, istride * p, out + (long)s * m, w, wstride * p, tmp);
    for (int q = 0; q < m; ++q) {
        for (int s = 0; s < p; ++s) tmp[s] = out[(long)s * m + q];
        for (int r = 0; r < p; ++r) {
            cplx acc = 0;
            long k = q + (long)m * r;
            for (int s = 0; s < p; ++s) acc += w[((long)s * k % N) * wstride] * tmp[s];
            out[k] = acc;
        }
    }
}

static int max_factor(int N)
{
    int mx = 1;
    while (N > 1) {
        int p = least_factor(N);
        if (p > mx) mx = p;
        N /= p;
    }
    return mx;
}

/* In-place 1-D transform of N interleaved complex values (unnormalised). */
void orc_fft(int N, double *data, int sign)
{
    cplx *x = (cplx *)data;
    cplx *w = twiddle_table(N, sign);
    cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)max_factor(N));
    fft_rec(N, x, 1, out, w, 1, tmp);
    memcpy(x, out, sizeof(cplx) * (size_t)N);
    free(w);
    free(out);
    free(tmp);
}

/* In-place 2-D transform of an R x C row-major complex array (first index = rows),
 * rows then columns; scale multiplies the result. */
static void fft2(int R, int C, cplx *a, int sign, double scale)
{
    cplx *wc = twiddle_table(C, sign);
    cplx *wr = twiddle_table(R, sign);
    int pf = max_factor(R > C ? R : C);
#pragma omp parallel
    {
        cplx *in = (cplx *)malloc(sizeof(cplx) * (size_t)(R > C ? R : C));
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)(R > C ? R : C));
        cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)pf);
#pragma omp for schedule(static)
        for (int r = 0; r < R; ++r) {
            fft_rec(C, a + (long)r * C, 1, out, wc, 1, tmp);
            memcpy(a + (long)r * C, out, sizeof(cplx) * (size_t)C);
        }
#pragma omp for schedule(static)
        for (int c = 0; c < C; ++c) {
            for (int r = 0; r < R; ++r) in[r] = a[(long)r * C + c];
            fft_rec(R, in, 1, out, wr, 1, tmp);
            for (int r = 0; r < R; ++r) a[(long)r * C + c] = out[r] * scale;
        }
        free(in);
        free(out);
        free(tmp);
    }
    free(wc);
    free(wr);
}

void orc_fft2(int R, int C, double *data, int sign, double scale)
{
    fft2(R, C, (cplx *)data, sign, scale);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------------------------
 * Gauss-Legendre rule on [-1, 1] by Newton iteration on P_n (three-term recurrence).
 * ------------------------------------------------------------------------------------------ */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            pp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

#define GL_N 20
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;
static void gl_init(void)
{
    if (!gl_ready) {
        gauss_legendre(GL_N, gl_x, gl_w);
        gl_ready = 1;
    }
}

/* ------------------------------------------------------------------------------------------
 * Moments ghat(k), Sec. 2.2.  All kernels are radial; s = 2 pi |k| / b, z = s a.
 *   ORC_LOG : g(x) = scale * log|x|.  The closed form printed for -(1/2pi) log|x| is scaled by
 *             -2 pi scale.
 *   ORC_POW : g(x) = scale * |x|^gamma.  The closed form printed for (1/2pi)|x|^gamma is scaled
 *             by 2 pi scale.  It equals s^{-2-gamma} I(z) with I(z) = int_0^z t^{1+gamma} J0(t) dt.
 *   ORC_HELM: g(x) = scale * (i/4) H0^(1)(kappa |x|).
 *   ORC_YUKAWA: g(x) = scale * K0(kappa |x|) / (2 pi) (Sec. 3.2), closed form in orc_moments.c.
 * ------------------------------------------------------------------------------------------ */

/* I(z) = int_0^z t^{1+gamma} J0(t) dt by the power series of J0, term by term (z <= 8). */
static double pow_moment_series(double gamma, double z)
{
    double sum = 0.0, c = 1.0; /* c = (-1)^m / (4^m (m!)^2) */
    double zp = pow(z, 2.0 + gamma);
    for (int m = 0; m < 200; ++m) {
        double term = c * zp / (2.0 * m + 2.0 + gamma);
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum) && m > 2) break;
        c *= -1.0 / (4.0 * (m + 1.0) * (m + 1.0));
        zp *= z * z;
    }
    return sum;
}

/* int_{z0}^{z1} t^{1+gamma} J0(t) dt by 20-point Gauss-Legendre on pieces of length <= 1/2
 * (the integrand is analytic there; J0 varies on a unit scale). */
static double pow_moment_gl(double gamma, double z0, double z1)
{
    gl_init();
    int pieces = (int)ceil((z1 - z0) / 0.5);
    if (pieces < 1) pieces = 1;
    double h = (z1 - z0) / pieces, sum = 0.0;
    for (int p = 0; p < pieces; ++p) {
        double lo = z0 + p * h, mid = lo + 0.5 * h;
        for (int i = 0; i < GL_N; ++i) {
            double t = mid + 0.5 * h * gl_x[i];
            sum += 0.5 * h * gl_w[i] * pow(t, 1.0 + gamma) * j0(t);
        }
    }
    return sum;
}

/* Lommel's second function S_{mu,nu}(z) by its large-z asymptotic expansion
 *   S ~ z^{mu-1} sum_m (-1)^m prod_{j=1..m} ((mu-2j+1)^2 - nu^2) z^{-2m},
 * summed until the terms stop decreasing (or vanish: the series terminates when
 * mu +- nu is an odd positive integer). */
static double lommel_S_asym(double mu, double nu, double z)
{
    double sum = 1.0, term = 1.0, prev = INFINITY;
    for (int m = 1; m < 400; ++m) {
        double f = ((mu - 2.0 * m + 1.0) * (mu - 2.0 * m + 1.0) - nu * nu) / (z * z);
        term *= -f;
        if (term == 0.0) break;
        if (fabs(term) >= prev) break;
        sum += term;
        prev = fabs(term);
        if (fabs(term) < 1e-18 * fabs(sum)) break;
    }
    return pow(z, mu - 1.0) * sum;
}

#define ORC_POW_ZASYM 45.0

/* I(z) = int_0^z t^{1+gamma} J0(t) dt, gamma > -2. */
double orc_pow_moment(double gamma, double z)
{
    if (z <= 8.0) return pow_moment_series(gamma, z);
    if (z <= ORC_POW_ZASYM) return pow_moment_series(gamma, 8.0) + pow_moment_gl(gamma, 8.0, z);
    /* closed form of Sec. 2.2 for |x|^gamma:
     *   I(z) = 2^{1+gamma} Gamma(1+gamma/2)/Gamma(-gamma/2)
     *          + z (gamma J0(z) S_{gamma,-1}(z) + J1(z) S_{1+gamma,0}(z)) */
    double c = pow(2.0, 1.0 + gamma) * tgamma(1.0 + 0.5 * gamma) / tgamma(-0.5 * gamma);
    return c + z * (gamma * j0(z) * lommel_S_asym(gamma, -1.0, z) +
                    j1(z) * lommel_S_asym(1.0 + gamma, 0.0, z));
}

/* 2 pi (i/4) int_0^a H0^(1)(kappa rho) J0(s rho) rho d rho by Gauss-Legendre in tau, rho = tau^2
 * (removes the log singularity's effect on the rule), on pieces of tau-length <= 0.05. */
static cplx helm_moment_quad(double kappa, double s, double a)
{
    gl_init();
    double ta = sqrt(a);
    int pieces = (int)ceil(ta / 0.02);
    double h = ta / pieces;
    cplx sum = 0.0;
    for (int p = 0; p < pieces; ++p) {
        double mid = (p + 0.5) * h;
        for (int i = 0; i < GL_N; ++i) {
            double tau = mid + 0.5 * h * gl_x[i], rho = tau * tau;
            cplx H0 = j0(kappa * rho) + I * y0(kappa * rho);
            sum += 0.5 * h * gl_w[i] * H0 * j0(s * rho) * rho * 2.0 * tau;
        }
    }
    return 2.0 * PI * (I / 4.0) * sum;
}

/* Band around the resonance s = kappa where the k != 0 closed form is a near 0/0 quotient (its
 * numerator vanishes at s = kappa) and loses up to ~log10(1/|s/kappa - 1|) digits: quadrature there. */
#define ORC_HELM_RES_REL 5e-2

/* ghat for one |k| (kmag >= 0). */
cplx orc_ghat_radial_c(int family, double gamma, double kappa, double scale, double b, double a,
                       double kmag)
{
    double s = 2.0 * PI * kmag / b, z = s * a;
    if (family == ORC_LOG) {
        double G;
        if (kmag == 0.0)
            G = a * a / 4.0 * (1.0 - 2.0 * log(a));
        else
            G = -a * log(a) * j1(z) / s + (1.0 - j0(z)) / (s * s);
        return -2.0 * PI * scale * G;
    }
    if (family == ORC_POW) {
        if (kmag == 0.0) return 2.0 * PI * scale * pow(a, 2.0 + gamma) / (2.0 + gamma);
        return 2.0 * PI * scale * pow(s, -2.0 - gamma) * orc_pow_moment(gamma, z);
    }
    if (family == ORC_YUKAWA) return scale * orc_yukawa_moment(kappa, s, a);
    /* ORC_HELM */
    double ka = kappa * a;
    cplx H0 = j0(ka) + I * y0(ka), H1 = j1(ka) + I * y1(ka);
    if (kmag == 0.0) {
        /* k = 0 closed form with the sign of the 2/(kappa pi) term corrected: it is the
         * s -> 0 limit of the k != 0 form and what the defining integral gives. */
        return scale * (PI / (2.0 * kappa)) * (I * a * j1(ka) - a * y1(ka) - 2.0 / (kappa * PI));
    }
    if (fabs(s - kappa) < ORC_HELM_RES_REL * kappa) return scale * helm_moment_quad(kappa, s, a);
    return scale * (I * PI / 2.0) * (z * j1(z) * H0 - ka * j0(z) * H1 - 2.0 * I / PI) /
           (s * s - kappa * kappa);
}

void orc_ghat_radial(int family, double gamma, double kappa, double scale, double b, double a,
                     double kmag, double *out2)
{
    cplx v = orc_ghat_radial_c(family, gamma, kappa, scale, b, a, kmag);
    out2[0] = creal(v);
    out2[1] = cimag(v);
}

/* Helmholtz moment at exactly s = kappa (resonance line of Sec. 2.2). */
void orc_ghat_helm_resonant(double kappa, double scale, double a, double *out2)
{
    double ka = kappa * a;
    cplx H0 = j0(ka) + I * y0(ka), H1 = j1(ka) + I * y1(ka);
    cplx v = scale * (I / 4.0) * PI * a * a * (j0(ka) * H0 + j1(ka) * H1);
    out2[0] = creal(v);
    out2[1] = cimag(v);
}

void orc_ghat_helm_quad(double kappa, double scale, double s, double a, double *out2)
{
    cplx v = scale * helm_moment_quad(kappa, s, a);
    out2[0] = creal(v);
    out2[1] = cimag(v);
}

/* Full M x M table of ghat(k) for k in F_n, stored at FFT index q (k = q for q < M/2, else q - M).
 * ghat depends on |k| only, so the quadrant 0 <= k1, k2 <= M/2 is evaluated and read back by |k1|, |k2|. */
void orc_ghat_full(int family, double gamma, double kappa, double scale, double b, double a, int M,
                   double *out)
{
    int h = M / 2 + 1;
    cplx *quad = (cplx *)malloc(sizeof(cplx) * (size_t)h * h);
    gl_init(); /* before the threads start */
#pragma omp parallel for schedule(dynamic, 4)
    for (int k1 = 0; k1 < h; ++k1)
        for (int k2 = 0; k2 < h; ++k2)
            quad[(long)k1 * h + k2] =
                orc_ghat_radial_c(family, gamma, kappa, scale, b, a, hypot((double)k1, (double)k2));
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (int q1 = 0; q1 < M; ++q1) {
        int k1 = q1 < M / 2 ? q1 : M - q1;
        for (int q2 = 0; q2 < M; ++q2) {
            int k2 = q2 < M / 2 ? q2 : M - q2;
            o[(long)q1 * M + q2] = quad[(long)k1 * h + k2];
        }
    }
    free(quad);
}

/* ------------------------------------------------------------------------------------------
 * The scheme A_n of eq. (An), Sec. 2.1:
 *   u_e = zero-extension of the n x n grid data u_j = u(j/n) to the M x M grid of [0,b)^2 (M = n b),
 *   hat u_{e,n} = (1/M^2) fft2(u_e),  A_n u (x_j) = sum_{k in F_n} ghat(k) hat u_{e,n}(k) e^{2 pi i k.j/M},
 * i.e. A_n u = crop_n( ifft2( ghat (.) fft2(u_e) ) ) with ifft2 carrying the 1/M^2.
 * ghat_full is the M x M table of orc_ghat_full.  u and out are n x n complex, row-major
 * (first index <-> x1).  Batched over `batch` densities.
 * ------------------------------------------------------------------------------------------ */
int orc_conv(int n, int M, const double *ghat_full, const double *u, double *out, int batch)
{
    if (n <= 0 || M < n) return 1;
    const cplx *g = (const cplx *)ghat_full;
    cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)M * M);
    if (!a) return 2;
    for (int bi = 0; bi < batch; ++bi) {
        const cplx *ub = (const cplx *)u + (long)bi * n * n;
        cplx *ob = (cplx *)out + (long)bi * n * n;
        memset(a, 0, sizeof(cplx) * (size_t)M * M);
        for (int j1 = 0; j1 < n; ++j1)
            for (int j2 = 0; j2 < n; ++j2) a[(long)j1 * M + j2] = ub[(long)j1 * n + j2];
        fft2(M, M, a, -1, 1.0);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)M * M; ++i) a[i] *= g[i];
        fft2(M, M, a, +1, 1.0 / ((double)M * (double)M));
        for (int j1 = 0; j1 < n; ++j1)
            for (int j2 = 0; j2 < n; ++j2) ob[(long)j1 * n + j2] = a[(long)j1 * M + j2];
    }
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Quadrature form eq. (quad)/(quad_wts):  (A_n u)(x_i) = sum_j w(i - j) u_j,
 *   w(d) = (1/M^2) sum_{k in F_n} ghat(k) e^{2 pi i k.d / M},  d in [-(n-1), n-1]^2.
 * The weight sum is a plain double sum over k1 and k2 (separable exponential, no FFT);
 * the application is the O(n^4) sum.  Outputs only the rows i1 in [r0, r1) (all i2).
 * ------------------------------------------------------------------------------------------ */
int orc_direct(int n, int M, const double *ghat_full, const double *u, double *out, int r0, int r1)
{
    const cplx *g = (const cplx *)ghat_full;
    int D = 2 * n - 1;
    /* E[di][q] = exp(2 pi i k(q) d / M) with d = di - (n-1), k(q) the F_n index of FFT slot q. */
    cplx *E = (cplx *)malloc(sizeof(cplx) * (size_t)D * M);
    cplx *T = (cplx *)malloc(sizeof(cplx) * (size_t)D * M); /* T[d1][q2] = sum_q1 E[d1][q1] g[q1][q2] */
    cplx *W = (cplx *)malloc(sizeof(cplx) * (size_t)D * D);
    if (!E || !T || !W) return 2;
    for (int di = 0; di < D; ++di) {
        long d = di - (n - 1);
        for (int q = 0; q < M; ++q) {
            long k = q < M / 2 ? q : q - M;
            long r = ((k * d) % M + M) % M;
            long double ang = 2.0L * PI_L * (long double)r / (long double)M;
            E[(long)di * M + q] = (double)cosl(ang) + I * (double)sinl(ang);
        }
    }
#pragma omp parallel for schedule(static)
    for (int d1 = 0; d1 < D; ++d1)
        for (int q2 = 0; q2 < M; ++q2) {
            cplx acc = 0;
            for (int q1 = 0; q1 < M; ++q1) acc += E[(long)d1 * M + q1] * g[(long)q1 * M + q2];
            T[(long)d1 * M + q2] = acc;
        }
    double inv = 1.0 / ((double)M * (double)M);
#pragma omp parallel for schedule(static)
    for (int d1 = 0; d1 < D; ++d1)
        for (int d2 = 0; d2 < D; ++d2) {
            cplx acc = 0;
            for (int q2 = 0; q2 < M; ++q2) acc += T[(long)d1 * M + q2] * E[(long)d2 * M + q2];
            W[(long)d1 * D + d2] = acc * inv;
        }
    const cplx *uu = (const cplx *)u;
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (int i1 = r0; i1 < r1; ++i1)
        for (int i2 = 0; i2 < n; ++i2) {
            cplx acc = 0;
            for (int j1 = 0; j1 < n; ++j1)
                for (int j2 = 0; j2 < n; ++j2)
                    acc += W[(long)(i1 - j1 + n - 1) * D + (i2 - j2 + n - 1)] * uu[(long)j1 * n + j2];
            o[(long)(i1 - r0) * n + i2] = acc;
        }
    free(E);
    free(T);
    free(W);
    return 0;
}

/* Weight table w(d) alone (D x D, D = 2n-1, d = index - (n-1)), same definition as above. */
int orc_weights(int n, int M, const double *ghat_full, double *wout)
{
    /* Reuse orc_direct on unit impulses would cost O(n^4); build the table directly instead. */
    const cplx *g = (const cplx *)ghat_full;
    int D = 2 * n - 1;
    cplx *E = (cplx *)malloc(sizeof(cplx) * (size_t)D * M);
    cplx *T = (cplx *)malloc(sizeof(cplx) * (size_t)D * M);
    if (!E || !T) return 2;
    for (int di = 0; di < D; ++di) {
        long d = di - (n - 1);
        for (int q = 0; q < M; ++q) {
            long k = q < M / 2 ? q : q - M;
            long r = ((k * d) % M + M) % M;
            long double ang = 2.0L * PI_L * (long double)r / (long double)M;
            E[(long)di * M + q] = (double)cosl(ang) + I * (double)sinl(ang);
        }
    }
    for (int d1 = 0; d1 < D; ++d1)
        for (int q2 = 0; q2 < M; ++q2) {
            cplx acc = 0;
            for (int q1 = 0; q1 < M; ++q1) acc += E[(long)d1 * M + q1] * g[(long)q1 * M + q2];
            T[(long)d1 * M + q2] = acc;
        }
    cplx *W = (cplx *)wout;
    double inv = 1.0 / ((double)M * (double)M);
    for (int d1 = 0; d1 < D; ++d1)
        for (int d2 = 0; d2 < D; ++d2) {
            cplx acc = 0;
            for (int q2 = 0; q2 < M; ++q2) acc += T[(long)d1 * M + q2] * E[(long)d2 * M + q2];
            W[(long)d1 * D + d2] = acc * inv;
        }
    free(E);
    free(T);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Fourier smoothing, Sec. 2.4.  chi^n_Omega(x) = sum_{k in F_n} chihat_b(k) e^{2 pi i k.x/b},
 *   chihat_b(k) = (1/b^2) int_Omega e^{-2 pi i k.y/b} dy   (period-b reading of eq. (tfs)),
 * sampled at x_j = j/n:  chi^n(x_j) = M^2 ifft2(chihat_b)[j], real part kept.
 * shape 0: disk, geom = (c1, c2, r):
 *   chihat_b = e^{-2 pi i k.c/b} r J1(2 pi |k| r/b) / (b |k|),  k = 0: pi r^2 / b^2.
 * shape 1: rectangle [g0,g1] x [g2,g3]: product over the two axes of
 *   (e^{-2 pi i k s0/b} - e^{-2 pi i k s1/b}) / (2 pi i k),  k = 0: (s1 - s0)/b.
 * psi(x) = w(x1) w(x2), w = 1 on [delta, 1-delta], w(t) = varkappa((delta - t)/delta) for t < delta,
 * mirrored for t > 1 - delta, with varkappa(t) = exp(2 e^{-1/t} / (t - 1)) of eq. (halfwindow1).
 * Output: mask = chi^n psi on the n x n grid (real).  delta <= 0 omits psi.
 * ------------------------------------------------------------------------------------------ */
double orc_varkappa(double t)
{
    if (t <= 0.0) return 1.0;
    if (t >= 1.0) return 0.0;
    return exp(2.0 * exp(-1.0 / t) / (t - 1.0));
}

double orc_psi1(double t, double delta)
{
    if (delta <= 0.0) return 1.0;
    if (t < delta) return orc_varkappa((delta - t) / delta);
    if (t > 1.0 - delta) return orc_varkappa((t - (1.0 - delta)) / delta);
    return 1.0;
}

static cplx rect_factor(long k, double s0, double s1, double b)
{
    if (k == 0) return (s1 - s0) / b;
    long double a0 = -2.0L * PI_L * (long double)k * s0 / b, a1 = -2.0L * PI_L * (long double)k * s1 / b;
    cplx e0 = (double)cosl(a0) + I * (double)sinl(a0), e1 = (double)cosl(a1) + I * (double)sinl(a1);
    return (e0 - e1) / (2.0 * PI * I * (double)k);
}

int orc_fs_mask(int n, int M, double b, int shape, const double *geom, double delta, double *mask)
{
    cplx *c = (cplx *)malloc(sizeof(cplx) * (size_t)M * M);
    if (!c) return 2;
#pragma omp parallel for schedule(static)
    for (int q1 = 0; q1 < M; ++q1) {
        long k1 = q1 < M / 2 ? q1 : q1 - M;
        for (int q2 = 0; q2 < M; ++q2) {
            long k2 = q2 < M / 2 ? q2 : q2 - M;
            cplx v;
            if (shape == 0) {
                double c1 = geom[0], c2 = geom[1], r = geom[2];
                double km = hypot((double)k1, (double)k2);
                if (k1 == 0 && k2 == 0)
                    v = PI * r * r / (b * b);
                else {
                    long double ph = -2.0L * PI_L * ((long double)k1 * c1 + (long double)k2 * c2) / b;
                    v = ((double)cosl(ph) + I * (double)sinl(ph)) * r * j1(2.0 * PI * km * r / b) / (b * km);
                }
            } else {
                v = rect_factor(k1, geom[0], geom[1], b) * rect_factor(k2, geom[2], geom[3], b);
            }
            c[(long)q1 * M + q2] = v;
        }
    }
    fft2(M, M, c, +1, 1.0);
    for (int j1 = 0; j1 < n; ++j1)
        for (int j2 = 0; j2 < n; ++j2)
            mask[(long)j1 * n + j2] =
                creal(c[(long)j1 * M + j2]) * orc_psi1((double)j1 / n, delta) * orc_psi1((double)j2 / n, delta);
    free(c);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Lippmann-Schwinger Nystrom system eq. (descretls), Sec. 3.3:
 *   L x = x + kappa^2 A_n(m x) = f  on the n x n grid,
 * solved by restarted GMRES (Arnoldi with modified Gram-Schmidt, Givens rotations), x0 given.
 * Stops when ||f - L x||_2 / ||f||_2 <= tol (Arnoldi estimate, confirmed by the true residual at
 * each restart) or after maxit matvecs.  Returns 0 if converged, 3 otherwise.
 * ------------------------------------------------------------------------------------------ */
static void ls_apply(int n, int M, const cplx *g, double kappa2, const double *m, const cplx *x,
                     cplx *y, cplx *tmp)
{
    for (long i = 0; i < (long)n * n; ++i) tmp[i] = m[i] * x[i];
    orc_conv(n, M, (const double *)g, (const double *)tmp, (double *)y, 1);
    for (long i = 0; i < (long)n * n; ++i) y[i] = x[i] + kappa2 * y[i];
}

static double nrm2(long N, const cplx *v)
{
    double s = 0.0;
    for (long i = 0; i < N; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return sqrt(s);
}

void orc_ls_apply(int n, int M, const double *ghat_full, double kappa, const double *m,
                  const double *x, double *y)
{
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n * n);
    ls_apply(n, M, (const cplx *)ghat_full, kappa * kappa, m, (const cplx *)x, (cplx *)y, tmp);
    free(tmp);
}

int orc_gmres(int n, int M, const double *ghat_full, double kappa, const double *m, const double *f,
              double *x_io, int restart, int maxit, double tol, int *iters_out, double *relres_out)
{
    const cplx *g = (const cplx *)ghat_full;
    const cplx *fb = (const cplx *)f;
    cplx *x = (cplx *)x_io;
    long N = (long)n * n;
    double k2 = kappa * kappa;
    cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)N * (restart + 1));
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *H = (cplx *)calloc((size_t)(restart + 1) * restart, sizeof(cplx));
    cplx *cs = (cplx *)malloc(sizeof(cplx) * restart), *sn = (cplx *)malloc(sizeof(cplx) * restart);
    cplx *e = (cplx *)malloc(sizeof(cplx) * (restart + 1)), *y = (cplx *)malloc(sizeof(cplx) * restart);
    double fn = nrm2(N, fb);
    if (fn == 0.0) fn = 1.0;
    int it = 0, conv = 0;
    double rel = 1.0;
    while (it < maxit) {
        ls_apply(n, M, g, k2, m, x, w, tmp);
        for (long i = 0; i < N; ++i) V[i] = fb[i] - w[i];
        double beta = nrm2(N, V);
        rel = beta / fn;
        if (rel <= tol) {
            conv = 1;
            break;
        }
        for (long i = 0; i < N; ++i) V[i] /= beta;
        memset(e, 0, sizeof(cplx) * (restart + 1));
        e[0] = beta;
        int j;
        for (j = 0; j < restart && it < maxit; ++j, ++it) {
            ls_apply(n, M, g, k2, m, V + (long)j * N, w, tmp);
            for (int i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
                cplx h = 0;
                const cplx *vi = V + (long)i * N;
                for (long t = 0; t < N; ++t) h += conj(vi[t]) * w[t];
                for (long t = 0; t < N; ++t) w[t] -= h * vi[t];
                H[(long)i * restart + j] = h;
            }
            double hn = nrm2(N, w);
            H[(long)(j + 1) * restart + j] = hn;
            cplx *vn = V + (long)(j + 1) * N;
            for (long t = 0; t < N; ++t) vn[t] = hn > 0 ? w[t] / hn : 0;
            for (int i = 0; i < j; ++i) { /* apply the previous rotations to column j */
                cplx h0 = H[(long)i * restart + j], h1 = H[(long)(i + 1) * restart + j];
                H[(long)i * restart + j] = conj(cs[i]) * h0 + conj(sn[i]) * h1;
                H[(long)(i + 1) * restart + j] = -sn[i] * h0 + cs[i] * h1;
            }
            cplx h0 = H[(long)j * restart + j], h1 = H[(long)(j + 1) * restart + j];
            double r = sqrt(creal(h0 * conj(h0)) + creal(h1 * conj(h1)));
            cs[j] = r > 0 ? h0 / r : 1;
            sn[j] = r > 0 ? h1 / r : 0;
            H[(long)j * restart + j] = r;
            H[(long)(j + 1) * restart + j] = 0;
            e[j + 1] = -sn[j] * e[j];
            e[j] = conj(cs[j]) * e[j];
            rel = cabs(e[j + 1]) / fn;
            if (rel <= tol) {
                ++j;
                ++it;
                break;
            }
        }
        /* back substitution H(0:j,0:j) y = e(0:j), x += V y */
        for (int i = j - 1; i >= 0; --i) {
            cplx acc = e[i];
            for (int t = i + 1; t < j; ++t) acc -= H[(long)i * restart + t] * y[t];
            y[i] = acc / H[(long)i * restart + i];
        }
        for (int i = 0; i < j; ++i)
            for (long t = 0; t < N; ++t) x[t] += y[i] * V[(long)i * N + t];
    }
    if (!conv) { /* final true residual */
        ls_apply(n, M, g, k2, m, x, w, tmp);
        for (long i = 0; i < N; ++i) w[i] = fb[i] - w[i];
        rel = nrm2(N, w) / fn;
        conv = rel <= tol;
    }
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
    free(V);
    free(w);
    free(tmp);
    free(H);
    free(cs);
    free(sn);
    free(e);
    free(y);
    return conv ? 0 : 3;
}
