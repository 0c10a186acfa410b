// ghat.cu -- FP64 moment table ghat(|k|) of Sec. 2.2, built on the GPU once per plan.
//
//   ghat(k) = 2 pi int_0^a g(rho) J0(s rho) rho d rho,   s = 2 pi |k| / b,  z = s a   (eq. (ghat))
//
// Table layout: quadrant [k2][k1], 0 <= k1, k2 <= M/2; ghat depends on |k| only, so every k in
// F_n is read as ghat(|k1|, |k2|).
//
//   log      g = scale log|x|: the closed form printed for -(1/2pi) log|x|, times -2 pi scale.
//   |x|^gam  g = scale |x|^gamma: 2 pi scale s^{-2-gamma} I(z), I(z) = int_0^z t^{1+gamma} J0(t) dt.
//            z > 60: I(z) = C - T(z) with C = 2^{1+gamma} Gamma(1+gamma/2)/Gamma(-gamma/2) (the
//            constant of Sec. 2.2's closed form) and the tail T(z) = int_z^inf t^{1+gamma} J0 dt
//            expanded by repeated integration by parts (pow_tail below; the same function as the
//            Lommel-function form printed in Sec. 2.2, derived and summed independently);
//            z <= 60: the moment integral directly, rho = a t^2 (the p = 2 substitution of Sec. 2.2,
//            which makes t^{3 + 2 gamma} a polynomial for 2 gamma integer), panel Clenshaw-Curtis.
//   Helmholtz g = scale (i/4) H0^(1)(kappa |x|): the closed forms of Sec. 2.2, with the k = 0 value
//            taken with -2/(kappa pi) (the s -> 0 limit of the k != 0 line; the printed sign is
//            wrong), and direct quadrature when |s - kappa| < 0.08 kappa, where the k != 0 line is a
//            near 0/0 quotient (its numerator vanishes at s = kappa) and loses digits.  The band
//            quadrature uses rho = a u^4 (p = 4: the integrand u^7 H0 J0 is smooth at 0 despite H0's
//            logarithm) and panel Clenshaw-Curtis; H0 and H1 at the single argument kappa a, and H0
//            at the quadrature nodes, are tabulated once on the host (the C library's
//            j0/y0/j1/y1); the device evaluates J0, J1 at z = s a per k.
// The switch points (z = 60, 8% band) sit beyond where the closed forms lose digits; between
// them and the oracle's own switch points the two sides evaluate the moments by different methods.
#include <cmath>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

// Clenshaw-Curtis rule of CC_N + 1 points on [-1, 1] (cc_rule_host below), for the panel quadratures
__constant__ double c_ccx[CC_N + 1];
__constant__ double c_ccw[CC_N + 1];

#define POW_ZTAIL 60.0
#define HELM_BAND 8e-2  // quadrature band |s - kappa| < 8% kappa (the closed form cancels there)

// Tail of the |x|^gamma moment integral, nu = 1 + gamma:
//   T(z) = int_z^inf t^nu J0(t) dt   (Abel-summed where it does not converge absolutely).
// With t J0 = (t J1)' and J1 = -J0', two integrations by parts give
//   A_mu = int_z^inf t^mu J0 = -z^mu J1(z) - (mu - 1) z^{mu-1} J0(z) - (mu - 1)^2 A_{mu-2},
// so that T(z) = -J1(z) z^nu sum_k c_k - J0(z) z^{nu-1} sum_k c_k (nu - 1 - 2k), with
// c_0 = 1, c_{k+1} = -c_k (nu - 1 - 2k)^2 / z^2: an asymptotic series, summed up to its smallest
// term.  Returns I(z) = C - T(z).
__device__ double pow_tail(double gamma, double z, double C)
{
    const double nu = 1.0 + gamma, iz2 = 1.0 / (z * z);
    double P = 0.0, Q = 0.0, c = 1.0, last = 1e300;
    for (int k = 0; k < 200; ++k) {
        const double qk = c * (nu - 1.0 - 2.0 * k);
        const double mag = fabs(c) + fabs(qk);
        if (mag >= last) break;  // the series has started to diverge
        P += c;
        Q += qk;
        last = mag;
        if (mag < 1e-18 * (fabs(P) + fabs(Q))) break;
        const double f = nu - 1.0 - 2.0 * k;
        c *= -f * f * iz2;
    }
    return C + j1(z) * pow(z, nu) * P + j0(z) * pow(z, nu - 1.0) * Q;
}

// int_0^a rho^{1+gamma} J0(s rho) d rho = 2 a^{2+gamma} int_0^1 t^{3+2 gamma} J0(z t^2) dt, on
// 4 + ceil(z/2) panels of the Clenshaw-Curtis rule (z <= 60: at most 34 panels).
__device__ double pow_moment_cc(double gamma, double s, double a)
{
    const double z = s * a;
    const int P = 4 + (int)ceil(0.5 * z);
    const double hw = 0.5 / P;
    double sum = 0.0;
    for (int p = 0; p < P; ++p) {
        const double mid = (p + 0.5) / P;
        for (int i = 0; i <= CC_N; ++i) {
            const double t = mid + hw * c_ccx[i];
            sum += c_ccw[i] * pow(t, 3.0 + 2.0 * gamma) * j0(z * t * t);
        }
    }
    return 2.0 * pow(a, 2.0 + gamma) * hw * sum;
}

// 2 pi (i/4) int_0^a H0(kappa rho) J0(s rho) rho d rho = i 2 pi a^2 int_0^1 H0(kappa a u^4) J0(s a u^4) u^7 du
// by panel Clenshaw-Curtis.  The nodes' H0(kappa a u^4) do not depend on s; k_helm_band_table
// tabulates them once per plan (tab: per node u, weight, Re H0, Im H0), so only J0 is evaluated
// here.
// Entries in the resonance band |s - kappa| < HELM_BAND kappa, k1 >= k2 (k_ghat leaves them, and
// their mirrors, to this kernel): one warp per entry, the lanes taking every 32nd node of the
// table, the partial sums combined by shuffles.  Block k2 covers the band's k1 range of row k2.
__global__ void k_ghat_band(double kappa, double scale, double b, double a, int h, double *out,
                            const double *__restrict__ tab, int nodes)
{
    const int k2 = blockIdx.x;
    if (k2 >= h) return;
    const double kr = kappa * b / (2.0 * M_PI);  // |k| where s = kappa
    const double rlo = kr * (1.0 - HELM_BAND), rhi = kr * (1.0 + HELM_BAND), k2d = (double)k2;
    const int lo = max(k2, (int)floor(sqrt(fmax(0.0, rlo * rlo - k2d * k2d))) - 1);
    const int hi = min(h - 1, (int)ceil(sqrt(fmax(0.0, rhi * rhi - k2d * k2d))) + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k1 = lo + warp; k1 <= hi; k1 += nw) {
        // the same test as k_ghat's, on the same arithmetic
        const double km = hypot((double)k1, k2d);
        const double s = 2.0 * M_PI * km / b;
        if (km == 0.0 || !(fabs(s - kappa) < HELM_BAND * kappa)) continue;
        double sr = 0.0, si = 0.0;
        for (int i = lane; i < nodes; i += 32) {
            const double u = tab[4 * i], u4 = u * u * u * u;
            const double w = tab[4 * i + 1] * j0(s * a * u4) * u4 * u * u * u;
            sr += w * tab[4 * i + 2];
            si += w * tab[4 * i + 3];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) {
            const double c = 2.0 * M_PI * a * a;
            const long long idx = (long long)k2 * h + k1, mirror = (long long)k1 * h + k2;
            out[2 * idx] = out[2 * mirror] = scale * (-c * si);
            out[2 * idx + 1] = out[2 * mirror + 1] = scale * (c * sr);
        }
    }
}

// The band quadrature's node table (per node u, weight, Re H0, Im H0 of H0(kappa a u^4)): P
// panels of CC_N + 1 Clenshaw-Curtis nodes on [q/P, (q+1)/P], one thread per node.  The integrand's
// limit at u = 0 is 0 (u^7 log u); H0 itself is infinite there.
__global__ void k_helm_band_table(double *__restrict__ tab, int P, double ka)
{
    const int nodes = P * (CC_N + 1);
    const double hw = 0.5 / P;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nodes; t += gridDim.x * blockDim.x) {
        const int q = t / (CC_N + 1), i = t - q * (CC_N + 1);
        const double u = (q + 0.5) / P + hw * c_ccx[i], arg = ka * u * u * u * u;
        double *e = tab + 4 * (size_t)t;
        e[0] = u;
        e[1] = hw * c_ccw[i];
        e[2] = arg > 0.0 ? j0(arg) : 0.0;
        e[3] = arg > 0.0 ? y0(arg) : 0.0;
    }
}

// hka = (J0, Y0, J1, Y1)(kappa a), tabulated on the host.  Helmholtz entries in the resonance band
// are left to k_ghat_band.
__global__ void k_ghat(int family, double gamma, double kappa, double scale, double b, double a,
                       int h, double *out, double4 hka)
{
    const long long N = (long long)h * h;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k2 = (int)(idx / h), k1 = (int)(idx - (long long)k2 * h);
        const double km = hypot((double)k1, (double)k2);
        const double s = 2.0 * M_PI * km / b, z = s * a;
        if (family == CONV_K_DX1LOG) {
            // the non-radial kernel: T(|k1|, |k2|) = scale (2 pi |k1| / b)(1 - J0(s a)) / s^2, the
            // passes multiply by i sgn(k1) T; not symmetric in k1 <-> k2, so no mirror
            out[idx] = km == 0.0 ? 0.0 : scale * (2.0 * M_PI * k1 / b) * (1.0 - j0(z)) / (s * s);
            continue;
        }
        // ghat depends on |k| only: each entry with k1 >= k2 also fills its mirror [k1][k2]
        if (k1 < k2) continue;
        const long long mirror = (long long)k1 * h + k2;
        if (family == CONV_K_LOG) {
            double G;
            if (km == 0.0) G = 0.25 * a * a * (1.0 - 2.0 * log(a));
            else G = -a * log(a) * j1(z) / s + (1.0 - j0(z)) / (s * s);
            out[idx] = out[mirror] = -2.0 * M_PI * scale * G;
        } else if (family == CONV_K_POW) {
            double v;
            if (km == 0.0) v = pow(a, 2.0 + gamma) / (2.0 + gamma);
            else if (z <= POW_ZTAIL) v = pow_moment_cc(gamma, s, a);
            else {
                const double C = pow(2.0, 1.0 + gamma) * tgamma(1.0 + 0.5 * gamma) / tgamma(-0.5 * gamma);
                v = pow(s, -2.0 - gamma) * pow_tail(gamma, z, C);
            }
            out[idx] = out[mirror] = 2.0 * M_PI * scale * v;
        } else if (family == CONV_K_YUKAWA) {
            // closed form (Sec. 3.2 kernel K0(kappa|x|)/(2 pi)); hka.x, hka.y = K0, K1 at kappa a
            const double ka = kappa * a;
            const double v = (1.0 + z * j1(z) * hka.x - ka * j0(z) * hka.y) / (s * s + kappa * kappa);
            out[idx] = out[mirror] = scale * v;
        } else {
            const double ka = kappa * a;
            double2 r;
            if (km == 0.0) {
                // (pi/(2 kappa)) (i a J1(ka) - a Y1(ka) - 2/(kappa pi))
                double c = M_PI / (2.0 * kappa);
                r = make_double2(c * (-a * hka.w - 2.0 / (kappa * M_PI)), c * a * hka.z);
            } else if (fabs(s - kappa) < HELM_BAND * kappa) {
                continue;  // k_ghat_band
            } else {
                // (i pi/2) (z J1(z) H0(ka) - ka J0(z) H1(ka) - 2i/pi) / (s^2 - kappa^2)
                double J0z = j0(z), J1z = j1(z);
                double H0r = hka.x, H0i = hka.y, H1r = hka.z, H1i = hka.w;
                double nr = z * J1z * H0r - ka * J0z * H1r;
                double ni = z * J1z * H0i - ka * J0z * H1i - 2.0 / M_PI;
                double d = 0.5 * M_PI / (s * s - kappa * kappa);
                r = make_double2(-ni * d, nr * d);
            }
            out[2 * idx] = out[2 * mirror] = scale * r.x;
            out[2 * idx + 1] = out[2 * mirror + 1] = scale * r.y;
        }
    }
}

__global__ void k_to_f32(const double *__restrict__ in, float *__restrict__ out, long long N)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// Clenshaw-Curtis rule on [-1, 1]: nodes x_j = cos(j pi / N), j = 0..N (N even), and the weights
// that integrate the interpolating Chebyshev polynomial exactly: with int_{-1}^1 T_{2k} = -2/(4k^2-1),
//   w_j = (c_j / N) (1 - sum_{k=1}^{N/2} beta_k cos(2 k j pi / N) / (4k^2 - 1)),
// c_j = 1 at the two ends and 2 inside, beta_k = 1 for k = N/2 and 2 below.
void cc_rule_host(int N, double *x, double *w)
{
    for (int j = 0; j <= N; ++j) {
        x[j] = std::cos(j * M_PI / N);
        double acc = 0.0;
        for (int k = 1; k <= N / 2; ++k)
            acc += (k == N / 2 ? 1.0 : 2.0) * std::cos(2.0 * k * j * M_PI / N) / (4.0 * k * k - 1.0);
        w[j] = ((j == 0 || j == N) ? 1.0 : 2.0) / N * (1.0 - acc);
    }
}

conv_status build_compact_table(const double *ghat, bool cplx, int n, int M, double *g2_out, cudaStream_t st);

// The FP64 tables of plan src (same kernel, period, n, radius and embedding) copied into p, then
// p's FP32 multiplier from them if p is FP32.
conv_status copy_ghat(conv_plan_s *p, const conv_plan_s *src)
{
    cudaStream_t st = p->setup_stream;
    p->ghat_bytes = src->ghat_bytes;
    if (dev_alloc(&p->ghat_paper, p->ghat_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(CONV_ENOMEM, "cudaMalloc of the moment table failed");
    }
    WSC_CUDA(cudaMemcpyAsync(p->ghat_paper, src->ghat_paper, p->ghat_bytes, cudaMemcpyDeviceToDevice, st));
    if (p->compact) {
        p->table_bytes = src->table_bytes;
        if (dev_alloc(&p->ghat64, p->table_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "cudaMalloc of the compact multiplier failed");
        }
        WSC_CUDA(cudaMemcpyAsync(p->ghat64, src->ghat64, p->table_bytes, cudaMemcpyDeviceToDevice, st));
    } else {
        p->ghat64 = p->ghat_paper;
        p->table_bytes = p->ghat_bytes;
    }
    if (p->prec == CONV_P_FP32) {
        const long long NT = (long long)(p->table_bytes / sizeof(double));
        if (dev_alloc(&p->ghat32, (size_t)NT * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "cudaMalloc of the FP32 multiplier failed");
        }
        const int b2 = (int)std::min<long long>((NT + 255) / 256, 152LL * 16);
        k_to_f32<<<b2, 256, 0, st>>>(p->ghat64, reinterpret_cast<float *>(p->ghat32), NT);
        WSC_CUDA(cudaGetLastError());
    }
    WSC_CUDA(cudaStreamSynchronize(st));
    return CONV_OK;
}

conv_status build_ghat(conv_plan_s *p)
{
    double cx[CC_N + 1], cw[CC_N + 1];
    cc_rule_host(CC_N, cx, cw);
    cudaStream_t st = p->setup_stream;
    WSC_CUDA(cudaMemcpyToSymbolAsync(c_ccx, cx, sizeof(cx), 0, cudaMemcpyHostToDevice, st));
    WSC_CUDA(cudaMemcpyToSymbolAsync(c_ccw, cw, sizeof(cw), 0, cudaMemcpyHostToDevice, st));
    const int hb = p->Mb / 2 + 1;
    const long long N = (long long)hb * hb;
    const int comps = p->complex_ghat ? 2 : 1;
    p->ghat_bytes = (size_t)N * comps * sizeof(double);
    if (dev_alloc(&p->ghat_paper, p->ghat_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(CONV_ENOMEM, "cudaMalloc of the moment table failed");
    }
    const double scale = p->kern.scale == 0.0 ? 1.0 : p->kern.scale;
    // Helmholtz: H0, H1 at kappa a and the quadrature table for the resonance band
    double4 hka = make_double4(0, 0, 0, 0);
    double *htab = nullptr;
    int hnodes = 0;
    const bool closed = p->moments.method == CONV_MOMENTS_CLOSED;
    if (closed && p->kern.family == CONV_K_YUKAWA) {
        double k0 = 0.0, k1 = 0.0;
        bessel_k01_host(p->kern.kappa * p->a, &k0, &k1);
        hka = make_double4(k0, k1, 0.0, 0.0);
    }
    if (closed && p->kern.family == CONV_K_HELMHOLTZ) {
        const double kappa = p->kern.kappa, a = p->a, ka = kappa * a;
        hka = make_double4(::j0(ka), ::y0(ka), ::j1(ka), ::y1(ka));
        // panels in u = (rho/a)^{1/4}: 8 + ceil(1.5 (kappa + s) a) for s up to the band's top, each
        // holding about two thirds of an oscillation of H0(kappa a u^4) J0(s a u^4) at u = 1; the
        // nodes' H0 values are computed on the device (thousands of nodes at large kappa a)
        const int P = 8 + (int)std::ceil(1.5 * (2.0 + HELM_BAND) * kappa * a);
        hnodes = P * (CC_N + 1);
        if (cudaMallocAsync(&htab, 4 * (size_t)hnodes * sizeof(double), st) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "cudaMalloc of the Helmholtz quadrature table failed");
        }
        k_helm_band_table<<<(hnodes + 255) / 256, 256, 0, st>>>(htab, P, ka);
        WSC_CUDA(cudaGetLastError());
    }
    if (closed) {
        int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
        k_ghat<<<blocks, 256, 0, st>>>(p->kern.family, p->kern.gamma, p->kern.kappa, scale, p->b, p->a, hb,
                                       p->ghat_paper, hka);
        if (htab)  // the resonance band's entries
            k_ghat_band<<<hb, 256, 0, st>>>(p->kern.kappa, scale, p->b, p->a, hb, p->ghat_paper, htab, hnodes);
        if (htab) cudaFreeAsync(htab, st);  // in stream order, after the kernels that read it
        WSC_CUDA(cudaGetLastError());
    } else {
        conv_status rc = build_moments_numeric(p, scale, p->ghat_paper, st);
        if (rc != CONV_OK) return rc;
    }
    // the passes' multiplier: the moments themselves, or the compact-embedding table built from them
    if (p->compact) {
        const size_t nq = (size_t)(p->n + 1) * (p->n + 1) * comps;
        p->table_bytes = nq * sizeof(double);
        if (dev_alloc(&p->ghat64, p->table_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "cudaMalloc of the compact multiplier failed");
        }
        conv_status rc = build_compact_table(p->ghat_paper, p->complex_ghat, p->n, p->Mb, p->ghat64, st);
        if (rc != CONV_OK) return rc;
    } else {
        p->ghat64 = p->ghat_paper;
        p->table_bytes = p->ghat_bytes;
    }
    if (p->prec == CONV_P_FP32) {
        const long long NT = (long long)(p->table_bytes / sizeof(double));
        if (dev_alloc(&p->ghat32, (size_t)NT * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "cudaMalloc of the FP32 multiplier failed");
        }
        const int b2 = (int)std::min<long long>((NT + 255) / 256, 152LL * 16);
        k_to_f32<<<b2, 256, 0, st>>>(p->ghat64, reinterpret_cast<float *>(p->ghat32), NT);
        WSC_CUDA(cudaGetLastError());
    }
    WSC_CUDA(cudaStreamSynchronize(st));
    return CONV_OK;
}

}  // namespace wsc
