// moments.cu -- moment tables of kernels without a usable closed form (Sec. 2.3), and the Yukawa
// kernel g = K0(kappa |x|)/(2 pi) of Sec. 3.2.
//
//   quadrature (CONV_MOMENTS_QUADRATURE), Sec. 2.3: after rho = tau^p,
//       ghat(k) = 2 pi p int_0^{a^{1/p}} g(tau^p) J0(s tau^p) tau^{2p-1} d tau,   s = 2 pi |k| / b,
//     on a fixed set of nodes tau_j (panel Clenshaw-Curtis, the first panel graded geometrically
//     toward tau = 0 so that any algebraic or logarithmic singularity of g is integrated to full
//     accuracy), with c_j = w_j g(tau_j^p) tau_j^{2p-1} tabulated once on the host: every entry of
//     the table is the Bessel sum 2 pi p sum_j c_j J0(s tau_j^p), one thread per entry.
//   localized (CONV_MOMENTS_LOCALIZED), eq. (io_split): A u = int g (1 - eta_beta) u + int g eta_beta u.
//     The singular part's moments ghat_eta(k) = 2 pi int_0^beta g eta_beta J0(s rho) rho d rho are
//     the same Bessel sum with the trapezoidal rule in tau on [0, beta^{1/p}] (the integrand vanishes
//     to high order at both ends); the smooth part is the classical trapezoidal rule, i.e. the
//     discrete convolution with W1(d) = h^2 g(|d| h)(1 - eta_beta(|d| h)), 0 < |d| h < a, whose
//     multiplier is the M x M DFT of W1 (even in both indices: two passes of the plan-time FP64
//     line transforms).  The table is ghat_eta + DFT(W1).
//   eta_beta(rho) = 1 for rho <= beta/2, varkappa((rho - beta/2)/(beta/2)) for beta/2 < rho < beta,
//     0 beyond, with varkappa(t) = exp(2 e^{-1/t}/(t - 1)) of eq. (halfwindow1).
//   Yukawa closed form: ghat = (1 + z J1(z) K0(kappa a) - kappa a J0(z) K1(kappa a)) / (s^2 + kappa^2),
//     z = s a, from d/d rho [rho (s J1(s rho) K0(kappa rho) - kappa J0(s rho) K1(kappa rho))] =
//     (s^2 + kappa^2) rho K0(kappa rho) J0(s rho) and rho K1(kappa rho) -> 1/kappa at rho = 0.
#include <cmath>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

// K0(x), K1(x) for x > 0.  x <= 2: the ascending series (Abramowitz & Stegun 9.6.13, 9.6.11)
//   K0 = -(log(x/2) + gamma_E) I0(x) + sum_{k>=1} H_k y^k/(k!)^2,  y = x^2/4,
//   K1 = 1/x + log(x/2) I1(x) - (x/4) sum_{k>=0} (psi(k+1) + psi(k+2)) y^k/(k!(k+1)!);
// x > 2: K_nu(x) = e^{-x} int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt by the trapezoidal rule with
// step min(1/4, 1/(2 sqrt x)), which resolves the peak of width ~1/sqrt(x) at t = 0 (the
// integrand is analytic and decays doubly exponentially).
__host__ __device__ void bessel_k01(double x, double &k0, double &k1)
{
    const double euler_gamma = 0.57721566490153286061;
    if (x <= 2.0) {
        const double y = 0.25 * x * x, lx = log(0.5 * x);
        double t = 1.0, i0 = 0.0, s0 = 0.0, hk = 0.0;
        for (int k = 1; k < 60; ++k) {
            i0 += t;
            s0 += hk * t;
            t *= y / ((double)k * k);
            hk += 1.0 / k;
            if (t < 1e-18 * i0) break;
        }
        k0 = -(lx + euler_gamma) * i0 + s0;
        double u = 1.0, i1 = 0.0, s1 = 0.0, p1 = -euler_gamma, p2 = 1.0 - euler_gamma;
        for (int k = 1; k < 60; ++k) {
            i1 += u;
            s1 += (p1 + p2) * u;
            u *= y / ((double)k * (k + 1));
            p1 += 1.0 / k;
            p2 += 1.0 / (k + 1);
            if (u < 1e-18 * i1) break;
        }
        k1 = 1.0 / x + lx * 0.5 * x * i1 - 0.25 * x * s1;
        return;
    }
    const double h = fmin(0.25, 0.5 / sqrt(x));
    double a0 = 0.5, a1 = 0.5;
    for (int j = 1; j < 4096; ++j) {
        const double t = j * h, e = exp(-x * (cosh(t) - 1.0));
        if (e < 1e-18) break;
        a0 += e;
        a1 += e * cosh(t);
    }
    const double f = h * exp(-x);
    k0 = f * a0;
    k1 = f * a1;
}

void bessel_k01_host(double x, double *k0, double *k1) { bessel_k01(x, *k0, *k1); }

__host__ __device__ double eta_window(double rho, double beta)
{
    if (rho <= 0.5 * beta) return 1.0;
    if (rho >= beta) return 0.0;
    const double t = (rho - 0.5 * beta) / (0.5 * beta);
    return exp(2.0 * exp(-1.0 / t) / (t - 1.0));
}

// g(rho) of the kernel family, unscaled (re, im): log rho, rho^gamma, (i/4) H0^(1)(kappa rho),
// K0(kappa rho)/(2 pi).
__host__ __device__ double2 kernel_at(int family, double gamma, double kappa, double rho)
{
    if (family == CONV_K_LOG) return make_double2(log(rho), 0.0);
    if (family == CONV_K_POW) return make_double2(pow(rho, gamma), 0.0);
    if (family == CONV_K_HELMHOLTZ) return make_double2(-0.25 * y0(kappa * rho), 0.25 * j0(kappa * rho));
    double k0, k1;
    bessel_k01(kappa * rho, k0, k1);
    return make_double2(k0 / (2.0 * M_PI), 0.0);
}

// out[k2][k1] (+)= scale sum_j c_j J0(s r_j) over the quadrant k1, k2 < h (entries k1 >= k2, the
// mirror written too).  Nodes staged through shared memory in chunks shared by the block.
#define MOM_CHUNK 512
__global__ void __launch_bounds__(256) k_bessel_sum(const double *__restrict__ r, const double2 *__restrict__ c,
                                                    int nodes, double b, int h, double scale, int cplx,
                                                    int accumulate, double *__restrict__ out)
{
    __shared__ double sr[MOM_CHUNK];
    __shared__ double2 sc[MOM_CHUNK];
    const long long N = (long long)h * (h + 1) / 2;  // k1 >= k2
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += stride) {
        const long long idx = base + threadIdx.x;
        // idx -> (k1, k2) with k1 >= k2: row k1 holds k1 + 1 entries
        int k1 = 0, k2 = 0;
        if (idx < N) {
            k1 = (int)floor((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
            while ((long long)k1 * (k1 + 1) / 2 > idx) --k1;
            while ((long long)(k1 + 1) * (k1 + 2) / 2 <= idx) ++k1;
            k2 = (int)(idx - (long long)k1 * (k1 + 1) / 2);
        }
        const double s = 2.0 * M_PI * hypot((double)k1, (double)k2) / b;
        double ar = 0.0, ai = 0.0;
        for (int j0b = 0; j0b < nodes; j0b += MOM_CHUNK) {
            const int m = min(MOM_CHUNK, nodes - j0b);
            __syncthreads();
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                sr[t] = r[j0b + t];
                sc[t] = c[j0b + t];
            }
            __syncthreads();
            if (idx < N)
                for (int t = 0; t < m; ++t) {
                    const double v = j0(s * sr[t]);
                    ar += sc[t].x * v;
                    ai += sc[t].y * v;
                }
        }
        if (idx < N) {
            const long long i1 = (long long)k2 * h + k1, i2 = (long long)k1 * h + k2;
            ar *= scale;
            ai *= scale;
            if (cplx) {
                if (accumulate) {
                    ar += out[2 * i1];
                    ai += out[2 * i1 + 1];
                }
                out[2 * i1] = out[2 * i2] = ar;
                out[2 * i1 + 1] = out[2 * i2 + 1] = ai;
            } else {
                if (accumulate) ar += out[i1];
                out[i1] = out[i2] = ar;
            }
        }
    }
}

// Quadrant [k2][k1] (k < hq) of the smooth part's weights W1(d), d = (k1, k2), of the localized scheme.
__global__ void k_w1(int family, double gamma, double kappa, double hh, double a, double beta, int hq, int cplx,
                     double *__restrict__ out)
{
    const long long N = (long long)hq * hq;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k2 = (int)(idx / hq), k1 = (int)(idx - (long long)k2 * hq);
        const double r = hypot((double)k1, (double)k2) * hh;
        double2 v = make_double2(0.0, 0.0);
        if (r > 0.0 && r < a) {
            const double w = hh * hh * (1.0 - eta_window(r, beta));
            if (w != 0.0) {
                const double2 g = kernel_at(family, gamma, kappa, r);
                v = make_double2(w * g.x, w * g.y);
            }
        }
        if (cplx) {
            out[2 * idx] = v.x;
            out[2 * idx + 1] = v.y;
        } else {
            out[idx] = v.x;
        }
    }
}

// fsmask.cu: acc (+)= scale * DFT_{M x M}(table), for a table even in both indices given by its
// quadrant [k2][k1], k < M/2 + 1 (real or complex); acc the same quadrant layout.
conv_status add_even_dft2(const double *quad, bool cplx, int M, double scale, double *acc, cudaStream_t st);

// Nodes of the Sec. 2.3 quadrature on [0, alpha] in tau: P panels of the (CC_N + 1)-point
// Clenshaw-Curtis rule, the first panel split geometrically into 16 pieces toward 0.
static void panel_nodes(double alpha, int P, const double *x, const double *w, int npt, std::vector<double> &t,
                        std::vector<double> &wt)
{
    auto add_panel = [&](double lo, double hi) {
        const double mid = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
        for (int i = 0; i < npt; ++i) {
            t.push_back(mid + hw * x[i]);
            wt.push_back(hw * w[i]);
        }
    };
    const double H = alpha / P;
    double hi = H;
    for (int l = 0; l < 16; ++l) {
        add_panel(0.5 * hi, hi);
        hi *= 0.5;
    }
    add_panel(0.0, hi);
    for (int q = 1; q < P; ++q) add_panel(q * H, (q + 1) * H);
}

void cc_rule_host(int N, double *x, double *w);  // ghat.cu

conv_status build_moments_numeric(conv_plan_s *p, double scale, double *table, cudaStream_t st)
{
    const conv_moments &mo = p->moments;
    const int family = p->kern.family, hb = p->Mb / 2 + 1;
    const double gamma = p->kern.gamma, kappa = p->kern.kappa, a = p->a, b = p->b;
    const int pp = mo.p > 0 ? mo.p : 4;
    const bool localized = mo.method == CONV_MOMENTS_LOCALIZED;
    const double beta = mo.beta > 0.0 ? mo.beta : 1.0;
    const double R = localized ? beta : a;  // the integral runs over [0, R] in rho
    const double alpha = std::pow(R, 1.0 / pp);
    // largest phase s R over the table: the quadrant's corner
    const double zmax = 2.0 * M_PI * std::sqrt(2.0) * (hb - 1) / b * R;
    std::vector<double> t, wt;
    if (localized) {
        // trapezoidal rule in tau with Nt intervals: the phase s tau^p rises at most p zmax per unit of
        // tau / alpha; 2 + 3/pi nodes per radian of it, plus a floor
        const int Nt = mo.nodes > 0 ? mo.nodes : 64 + (int)std::ceil(pp * zmax);
        const double h = alpha / Nt;
        for (int j = 1; j < Nt; ++j) {  // both ends contribute 0 (tau^{2p-1} at 0, eta at beta)
            t.push_back(j * h);
            wt.push_back(h);
        }
    } else {
        double x[CC_N + 1], w[CC_N + 1];
        cc_rule_host(CC_N, x, w);
        // each panel spans at most 4 radians of the phase s tau^p at the table's largest s
        const int P = mo.nodes > 0 ? std::max(1, mo.nodes / (CC_N + 1)) : 4 + (int)std::ceil(0.25 * pp * zmax);
        panel_nodes(alpha, P, x, w, CC_N + 1, t, wt);
    }
    const int nodes = (int)t.size();
    std::vector<double> rr(nodes);
    std::vector<double2> cc(nodes);
    for (int j = 0; j < nodes; ++j) {
        const double rho = std::pow(t[j], pp);
        rr[j] = rho;
        double2 g = rho > 0.0 ? kernel_at(family, gamma, kappa, rho) : make_double2(0.0, 0.0);
        double f = wt[j] * std::pow(t[j], 2 * pp - 1) * (localized ? eta_window(rho, beta) : 1.0);
        if (rho == 0.0) f = 0.0;
        cc[j] = make_double2(f * g.x, f * g.y);
    }
    double *dr = nullptr;
    double2 *dc = nullptr;
    if (cudaMallocAsync(&dr, nodes * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync(&dc, nodes * sizeof(double2), st) != cudaSuccess) {
        cudaGetLastError();
        if (dr) cudaFreeAsync(dr, st);
        return fail(CONV_ENOMEM, "moment quadrature nodes");
    }
    WSC_CUDA(cudaMemcpyAsync(dr, rr.data(), nodes * sizeof(double), cudaMemcpyHostToDevice, st));
    WSC_CUDA(cudaMemcpyAsync(dc, cc.data(), nodes * sizeof(double2), cudaMemcpyHostToDevice, st));
    const bool cplx = p->complex_ghat;
    const long long NE = (long long)hb * (hb + 1) / 2;
    const int blocks = (int)std::min<long long>((NE + 255) / 256, 152LL * 8);
    k_bessel_sum<<<blocks, 256, 0, st>>>(dr, dc, nodes, b, hb, scale * 2.0 * M_PI * pp, cplx ? 1 : 0, 0, table);
    cudaFreeAsync(dr, st);
    cudaFreeAsync(dc, st);
    WSC_CUDA(cudaGetLastError());
    if (localized) {
        // the smooth part: W1 on the quadrant of the period-Mb lattice, then its DFT added in
        double *w1 = nullptr;
        const size_t bytes = (size_t)hb * hb * (cplx ? 2 : 1) * sizeof(double);
        if (cudaMallocAsync(&w1, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "localized weights");
        }
        const long long NQ = (long long)hb * hb;
        k_w1<<<(int)std::min<long long>((NQ + 255) / 256, 152LL * 16), 256, 0, st>>>(
            family, gamma, kappa, 1.0 / p->n, a, beta, hb, cplx ? 1 : 0, w1);
        conv_status rc = cudaGetLastError() == cudaSuccess ? add_even_dft2(w1, cplx, p->Mb, scale, table, st)
                                                           : fail(CONV_ECUDA, "localized weights kernel");
        cudaFreeAsync(w1, st);
        if (rc != CONV_OK) return rc;
    }
    return CONV_OK;
}

}  // namespace wsc
