// fsmask.cu -- Fourier-smoothed indicator of Sec. 2.4 (eq. (tfs)), built on the GPU in FP64.
//
//   mask_j = Re chi^n_Omega(x_j) * psi(x_j),  x_j = j/n,
//   chi^n_Omega(x) = sum_{k in F_n} chihat_b(k) e^{2 pi i k.x/b},  chihat_b(k) = (1/b^2) int_Omega e^{-2 pi i k.y/b} dy,
//
// read with period b and the index set F_n of eq. (An) (the printed e^{2 pi i k.x} with k in F_n
// mixes period 1 and nb modes; the period-b reading makes chi^n the trigonometric interpolant the
// scheme itself uses).  Its samples are one M x M inverse DFT of chihat_b cropped to n x n:
// a column kernel generates chihat_b(., k2) analytically, inverse-transforms it along k1 and keeps
// rows j1 < n; the complex row pass then transforms along k2 and keeps j2 < n.
//   disk  (c1, c2, r):   chihat_b = e^{-2 pi i k.c/b} r J1(2 pi |k| r/b) / (b |k|),  k = 0: pi r^2/b^2
//   rect  (x0, x1, y0, y1): product over the axes of (e^{-2 pi i k s0/b} - e^{-2 pi i k s1/b})/(2 pi i k),
//                         k = 0: (s1 - s0)/b
// psi(x) = w(x1) w(x2), w = 1 on [delta, 1 - delta], w(t) = varkappa((delta - t)/delta) below delta and
// mirrored above 1 - delta, with the half-window varkappa(t) = exp(2 e^{-1/t}/(t - 1)) of eq. (halfwindow1).
#include <cmath>
#include <vector>

#include "passes.cuh"

namespace wsc {

__device__ double2 chihat(int shape, const double *g, double b, int M, int q1, int q2)
{
    const long long k1 = q1 < M / 2 ? q1 : q1 - M, k2 = q2 < M / 2 ? q2 : q2 - M;
    if (shape == 0) {
        if (k1 == 0 && k2 == 0) return make_double2(M_PI * g[2] * g[2] / (b * b), 0.0);
        const double km = hypot((double)k1, (double)k2);
        double sn, cs;
        sincospi(-2.0 * ((double)k1 * g[0] + (double)k2 * g[1]) / b, &sn, &cs);
        const double amp = g[2] * j1(2.0 * M_PI * km * g[2] / b) / (b * km);
        return make_double2(amp * cs, amp * sn);
    }
    double2 f[2];
    const long long kk[2] = {k1, k2};
    for (int d = 0; d < 2; ++d) {
        const double s0 = g[2 * d], s1 = g[2 * d + 1];
        if (kk[d] == 0) {
            f[d] = make_double2((s1 - s0) / b, 0.0);
        } else {
            double sa, ca, sb, cb;
            sincospi(2.0 * (double)kk[d] * s0 / b, &sa, &ca);
            sincospi(2.0 * (double)kk[d] * s1 / b, &sb, &cb);
            // (e^{-i a} - e^{-i b}) / (2 pi i k) = (d_im - i d_re) / (2 pi k), d = e^{-ia} - e^{-ib}
            const double dr = ca - cb, di = -sa + sb, den = 2.0 * M_PI * (double)kk[d];
            f[d] = make_double2(di / den, -dr / den);
        }
    }
    return make_double2(f[0].x * f[1].x - f[0].y * f[1].y, f[0].x * f[1].y + f[0].y * f[1].x);
}

// Column k2 of chihat_b, inverse DFT along k1 (unnormalised, e^{+}), rows j1 < n into W[k2][j1].
__global__ void __launch_bounds__(512, 1) k_fs_cols(double2 *__restrict__ W, const FFTDesc *__restrict__ P,
                                                    const double2 *__restrict__ tw, int n, int M, int tpt,
                                                    int shape, double g0, double g1, double g2, double g3, double b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *buf = reinterpret_cast<double2 *>(smem_raw);
    const double geom[4] = {g0, g1, g2, g3};
    const int lt = threadIdx.x;
    for (int k2 = blockIdx.x; k2 < M; k2 += gridDim.x) {
        for (int e = lt; e < M; e += tpt) buf[pidx<double>(e)] = chihat(shape, geom, b, M, e, k2);
        __syncthreads();
        fft_smem<double, 0, true, false>(buf, P, tw, lt, tpt);
        for (int e = lt; e < n; e += tpt) W[(size_t)k2 * n + e] = buf[pidx<double>(e)];
        __syncthreads();
    }
}

__device__ double varkappa(double t)
{
    if (t <= 0.0) return 1.0;
    if (t >= 1.0) return 0.0;
    return exp(2.0 * exp(-1.0 / t) / (t - 1.0));
}

__device__ double psi1(double t, double delta)
{
    if (delta <= 0.0) return 1.0;
    if (t < delta) return varkappa((delta - t) / delta);
    if (t > 1.0 - delta) return varkappa((t - (1.0 - delta)) / delta);
    return 1.0;
}

template <typename T>
__global__ void k_fs_finish(const double2 *__restrict__ chi, T *__restrict__ mask, int n, double delta)
{
    const long long N = (long long)n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int j1 = (int)(i / n), j2 = (int)(i - (long long)j1 * n);
        mask[i] = (T)(chi[i].x * psi1((double)j1 / n, delta) * psi1((double)j2 / n, delta));
    }
}

int generic_threads(const FFTDesc &P);
bool factorize_any(int L, FFTDesc &d);
void stage_twiddles(const FFTDesc &d, std::vector<double> &re_im);

}  // namespace wsc

using namespace wsc;

extern "C" conv_status conv_fs_mask(conv_plan_t p, int shape, const double *geom, double delta, void *mask,
                                    void *stream)
{
    if (!p || !geom || !mask) return fail(CONV_EINVAL, "bad argument");
    if (shape != 0 && shape != 1) return fail(CONV_EINVAL, "shape must be 0 (disk) or 1 (rectangle)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n = p->n, M = p->M;
    FFTDesc d;
    if (!factorize_any(M, d)) return fail(CONV_EUNSUPPORTED, "transform length not 2^a 3^b 5^c");
    const int tpt = generic_threads(d);
    const size_t smem = (size_t)padded_len<double>(M) * sizeof(double2);
    int smem_optin = 0, sms = 0;
    WSC_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    WSC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    if (smem > (size_t)smem_optin || tpt > 512)
        return fail(CONV_EUNSUPPORTED, "FP64 transform of length M does not fit one CTA");
    std::vector<double> twh;
    stage_twiddles(d, twh);
    double2 *tw = nullptr, *W = nullptr, *chi = nullptr;
    FFTDesc *dd = nullptr;
    bool ok = cudaMalloc(&tw, twh.size() * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&W, (size_t)M * n * sizeof(double2)) == cudaSuccess &&
              cudaMalloc(&chi, (size_t)n * n * sizeof(double2)) == cudaSuccess &&
              cudaMalloc(&dd, sizeof(FFTDesc)) == cudaSuccess;
    conv_status rc = CONV_OK;
    if (!ok) {
        cudaGetLastError();
        rc = fail(CONV_ENOMEM, "FS mask buffers");
    }
    if (rc == CONV_OK) {
        cudaMemcpyAsync(tw, twh.data(), twh.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dd, &d, sizeof(FFTDesc), cudaMemcpyHostToDevice, st);
        cudaFuncSetAttribute(k_fs_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_c2c_rows_inv<double, 0, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_fs_cols<<<std::min(M, sms), tpt, smem, st>>>(W, dd, tw, n, M, tpt, shape, geom[0], geom[1], geom[2],
                                                     shape == 1 ? geom[3] : 0.0, p->b);
        PassArgs<double> a;
        a.in = W;
        a.mask = nullptr;
        a.out = chi;
        a.ghat = nullptr;
        a.u = nullptr;
        a.tw = tw;
        a.tw_len = d.tw_len;
        a.P = dd;
        a.n = n;
        a.h = p->h;
        a.M = M;
        a.tpt = tpt;
        a.units = n;
        a.batch = 1;
        a.alpha = make_double2(1.0, 0.0);
        a.beta = 0.0;
        k_c2c_rows_inv<double, 0, false, false><<<std::min(n, sms), tpt, smem, st>>>(a);
        int blocks = (int)std::min<long long>(((long long)n * n + 255) / 256, (long long)sms * 8);
        if (p->prec == CONV_P_FP64)
            k_fs_finish<double><<<blocks, 256, 0, st>>>(chi, reinterpret_cast<double *>(mask), n, delta);
        else
            k_fs_finish<float><<<blocks, 256, 0, st>>>(chi, reinterpret_cast<float *>(mask), n, delta);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "conv_fs_mask");
    }
    cudaFree(tw);
    cudaFree(W);
    cudaFree(chi);
    cudaFree(dd);
    return rc;
}
