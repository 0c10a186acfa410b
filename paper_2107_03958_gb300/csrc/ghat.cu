// ghat.cu -- FP64 moment table ghat(|k|) of Sec. 2.2, built on the GPU once per plan.
//
//   ghat(k) = 2 pi int_0^a g(rho) J0(s rho) rho d rho,   s = 2 pi |k| / b,  z = s a   (eq. (ghat))
//
// Table layout: quadrant [k2][k1], 0 <= k1, k2 <= M/2; ghat depends on |k| only, so every k in
// F_n is read as ghat(|k1|, |k2|).
//
//   log      g = scale log|x|: the closed form printed for -(1/2pi) log|x|, times -2 pi scale.
//   |x|^gam  g = scale |x|^gamma: 2 pi scale s^{-2-gamma} I(z), I(z) = int_0^z t^{1+gamma} J0(t) dt.
//            z > 45: I(z) = 2^{1+gamma} Gamma(1+gamma/2)/Gamma(-gamma/2)
//                           + z (gamma J0(z) S_{gamma,-1}(z) + J1(z) S_{1+gamma,0}(z))
//            with Lommel's S by its large-z expansion (closed form of Sec. 2.2);
//            z <= 45: the moment integral directly, rho = a t^2 (the p = 2 substitution of Sec. 2.2,
//            which makes t^{3 + 2 gamma} a polynomial for 2 gamma integer), composite Gauss-Legendre.
//   Helmholtz g = scale (i/4) H0^(1)(kappa |x|): the closed forms of Sec. 2.2, with the k = 0 value
//            taken with -2/(kappa pi) (the s -> 0 limit of the k != 0 line; the printed sign is
//            wrong), and direct quadrature when |s - kappa| < 0.05 kappa, where the k != 0 line is a
//            near 0/0 quotient (its numerator vanishes at s = kappa) and loses digits.  H0 and H1
//            at the single argument kappa a, and H0 at the quadrature nodes, are tabulated once on
//            the host (the C library's j0/y0/j1/y1); the device evaluates J0, J1 at z = s a per k.
#include <cmath>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

#define GL_NODES 16
__constant__ double c_glx[GL_NODES];
__constant__ double c_glw[GL_NODES];

#define POW_ZQUAD 45.0
#define HELM_RES_REL 5e-2  // quadrature band |s - kappa| < 5% kappa (the closed form cancels there)

__device__ double lommel_S_large(double mu, double nu, double z)
{
    double sum = 1.0, term = 1.0, prev = 1e300;
    for (int m = 1; m < 200; ++m) {
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

// int_0^a rho^{1+gamma} J0(s rho) d rho = 2 a^{2+gamma} int_0^1 t^{3+2 gamma} J0(z t^2) dt
__device__ double pow_moment_quad(double gamma, double s, double a)
{
    const double z = s * a;
    const int P = 16;
    const double hw = 0.5 / P;
    double sum = 0.0;
    for (int p = 0; p < P; ++p) {
        double mid = (p + 0.5) / P;
        for (int i = 0; i < GL_NODES; ++i) {
            double t = mid + hw * c_glx[i];
            sum += c_glw[i] * pow(t, 3.0 + 2.0 * gamma) * j0(z * t * t);
        }
    }
    return 2.0 * pow(a, 2.0 + gamma) * hw * sum;
}

// 2 pi (i/4) int_0^a H0(kappa rho) J0(s rho) rho d rho = i pi a^2 int_0^1 H0(kappa a t^2) J0(s a t^2) t^3 dt
// by composite Gauss-Legendre.  The nodes' H0(kappa a t^2) do not depend on s; the host tabulates
// them once per plan (tab: per node t, weight, Re H0, Im H0), so only J0 is evaluated here.
__device__ double2 helm_moment_quad(const double *__restrict__ tab, int nodes, double s, double a)
{
    double sr = 0.0, si = 0.0;
    for (int i = 0; i < nodes; ++i) {
        const double t = tab[4 * i], t2 = t * t;
        const double w = tab[4 * i + 1] * j0(s * a * t2) * t2 * t;
        sr += w * tab[4 * i + 2];
        si += w * tab[4 * i + 3];
    }
    const double c = M_PI * a * a;
    return make_double2(-c * si, c * sr);
}

// hka = (J0, Y0, J1, Y1)(kappa a), tabulated on the host.
__global__ void k_ghat(int family, double gamma, double kappa, double scale, double b, double a,
                       int h, double *out, double4 hka, const double *__restrict__ htab, int hnodes)
{
    const long long N = (long long)h * h;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k2 = (int)(idx / h), k1 = (int)(idx - (long long)k2 * h);
        // ghat depends on |k| only: each entry with k1 >= k2 also fills its mirror [k1][k2]
        if (k1 < k2) continue;
        const long long mirror = (long long)k1 * h + k2;
        const double km = hypot((double)k1, (double)k2);
        const double s = 2.0 * M_PI * km / b, z = s * a;
        if (family == CONV_K_LOG) {
            double G;
            if (km == 0.0) G = 0.25 * a * a * (1.0 - 2.0 * log(a));
            else G = -a * log(a) * j1(z) / s + (1.0 - j0(z)) / (s * s);
            out[idx] = out[mirror] = -2.0 * M_PI * scale * G;
        } else if (family == CONV_K_POW) {
            double v;
            if (km == 0.0) v = pow(a, 2.0 + gamma) / (2.0 + gamma);
            else if (z <= POW_ZQUAD) v = pow_moment_quad(gamma, s, a);
            else {
                double c = pow(2.0, 1.0 + gamma) * tgamma(1.0 + 0.5 * gamma) / tgamma(-0.5 * gamma);
                double I = c + z * (gamma * j0(z) * lommel_S_large(gamma, -1.0, z) +
                                    j1(z) * lommel_S_large(1.0 + gamma, 0.0, z));
                v = pow(s, -2.0 - gamma) * I;
            }
            out[idx] = out[mirror] = 2.0 * M_PI * scale * v;
        } else {
            const double ka = kappa * a;
            double2 r;
            if (km == 0.0) {
                // (pi/(2 kappa)) (i a J1(ka) - a Y1(ka) - 2/(kappa pi))
                double c = M_PI / (2.0 * kappa);
                r = make_double2(c * (-a * hka.w - 2.0 / (kappa * M_PI)), c * a * hka.z);
            } else if (fabs(s - kappa) < HELM_RES_REL * kappa) {
                r = helm_moment_quad(htab, hnodes, s, a);
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

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n.
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
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
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

conv_status build_compact_table(const double *ghat, bool cplx, int n, int M, double *g2_out, cudaStream_t st);

// The FP64 tables of plan src (same kernel, period, n, radius and embedding) copied into p, then
// p's FP32 multiplier from them if p is FP32.
conv_status copy_ghat(conv_plan_s *p, const conv_plan_s *src)
{
    cudaStream_t st = p->setup_stream;
    p->ghat_bytes = src->ghat_bytes;
    if (cudaMalloc(&p->ghat_paper, p->ghat_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(CONV_ENOMEM, "cudaMalloc of the moment table failed");
    }
    WSC_CUDA(cudaMemcpyAsync(p->ghat_paper, src->ghat_paper, p->ghat_bytes, cudaMemcpyDeviceToDevice, st));
    if (p->compact) {
        p->table_bytes = src->table_bytes;
        if (cudaMalloc(&p->ghat64, p->table_bytes) != cudaSuccess) {
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
        if (cudaMalloc(&p->ghat32, (size_t)NT * sizeof(float)) != cudaSuccess) {
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
    double gx[GL_NODES], gw[GL_NODES];
    gauss_legendre(GL_NODES, gx, gw);
    cudaStream_t st = p->setup_stream;
    WSC_CUDA(cudaMemcpyToSymbolAsync(c_glx, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, st));
    WSC_CUDA(cudaMemcpyToSymbolAsync(c_glw, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, st));
    const int hb = p->Mb / 2 + 1;
    const long long N = (long long)hb * hb;
    const int comps = p->complex_ghat ? 2 : 1;
    p->ghat_bytes = (size_t)N * comps * sizeof(double);
    if (cudaMalloc(&p->ghat_paper, p->ghat_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(CONV_ENOMEM, "cudaMalloc of the moment table failed");
    }
    const double scale = p->kern.scale == 0.0 ? 1.0 : p->kern.scale;
    // Helmholtz: H0, H1 at kappa a and the quadrature table for the resonance band
    double4 hka = make_double4(0, 0, 0, 0);
    double *htab = nullptr;
    int hnodes = 0;
    if (p->kern.family == CONV_K_HELMHOLTZ) {
        const double kappa = p->kern.kappa, a = p->a, ka = kappa * a;
        hka = make_double4(::j0(ka), ::y0(ka), ::j1(ka), ::y1(ka));
        // panels of t-width 1/P with (kappa + s) a / P <= 3 for s up to the band's top
        const int P = std::max(32, (int)std::ceil((2.0 + HELM_RES_REL) * kappa * a / 3.0));
        std::vector<double> tab(4 * (size_t)P * GL_NODES);
        const double hw = 0.5 / P;
        for (int q = 0; q < P; ++q)
            for (int i = 0; i < GL_NODES; ++i) {
                const double t = (q + 0.5) / P + hw * gx[i], arg = ka * t * t;
                double *e = &tab[4 * ((size_t)q * GL_NODES + i)];
                e[0] = t;
                e[1] = hw * gw[i];
                e[2] = ::j0(arg);
                e[3] = ::y0(arg);
            }
        hnodes = P * GL_NODES;
        if (cudaMallocAsync(&htab, tab.size() * sizeof(double), st) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "cudaMalloc of the Helmholtz quadrature table failed");
        }
        WSC_CUDA(cudaMemcpyAsync(htab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
    k_ghat<<<blocks, 256, 0, st>>>(p->kern.family, p->kern.gamma, p->kern.kappa, scale, p->b, p->a, hb,
                                   p->ghat_paper, hka, htab, hnodes);
    if (htab) cudaFreeAsync(htab, st);  // in stream order, after the kernel that reads it
    WSC_CUDA(cudaGetLastError());
    // the passes' multiplier: the moments themselves, or the compact-embedding table built from them
    if (p->compact) {
        const size_t nq = (size_t)(p->n + 1) * (p->n + 1) * comps;
        p->table_bytes = nq * sizeof(double);
        if (cudaMalloc(&p->ghat64, p->table_bytes) != cudaSuccess) {
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
        if (cudaMalloc(&p->ghat32, (size_t)NT * sizeof(float)) != cudaSuccess) {
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
