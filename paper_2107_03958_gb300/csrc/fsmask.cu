// fsmask.cu -- plan-time FP64 line transforms: the Fourier-smoothed indicator of Sec. 2.4 and the
// compact-embedding multiplier.
//
// k_lines transforms `nlines` lines of length L in FP64, each generated on the fly (an analytic
// coefficient table, a moment-table lookup, a mirrored weight table, or a strided read), and
// stores the first `keep` outputs of each line with arbitrary strides.  Chained, two such launches
// give a pruned 2-D transform.
//
// (1) Fourier smoothing (Sec. 2.4, eq. (tfs) read with period b and the index set F_n of eq. (An)):
//   mask_j = Re chi^n_Omega(x_j) * psi(x_j),  chi^n_Omega(x) = sum_{k in F_n} chihat_b(k) e^{2 pi i k.x/b},
//   chihat_b(k) = (1/b^2) int_Omega e^{-2 pi i k.y/b} dy,
//   disk  (c1, c2, r):   chihat_b = e^{-2 pi i k.c/b} r J1(2 pi |k| r/b) / (b |k|),  k = 0: pi r^2/b^2
//   rect  (x0, x1, y0, y1): product over the axes of (e^{-2 pi i k s0/b} - e^{-2 pi i k s1/b})/(2 pi i k),
//                           k = 0: (s1 - s0)/b
//   psi(x) = w(x1) w(x2), w = 1 on [delta, 1 - delta], w(t) = varkappa((delta - t)/delta) below delta
//   and mirrored above 1 - delta, with varkappa(t) = exp(2 e^{-1/t}/(t - 1)) of eq. (halfwindow1).
//   Its samples are one M x M inverse DFT of chihat_b cropped to n x n.
//
// (2) Compact embedding.  A_n u is the quadrature of eq. (quad): (A_n u)_i = sum_j w(i - j) u_j with
//   w(d) = (1/M^2) sum_{k in F_n} ghat(k) e^{2 pi i k.d/M}, |d1|, |d2| <= n - 1 (eq. (quad_wts)).  Placing
//   w on the 2n-periodic lattice (w(d) at d mod 2n, zero at the unused index n) turns the same sum into
//   a cyclic convolution of period L = 2n, so A_n u = crop_n(ifft2_L(G2 . fft2_L(pad_L u))) with
//   G2 = fft2_L(w), exactly (up to rounding).  G2 is built here from the moment table: an M x M inverse
//   DFT cropped to the n x n quadrant of w (w is even in each index), then an L x L forward DFT whose
//   (n+1) x (n+1) quadrant is kept (G2 is even as well).
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "passes.cuh"

namespace wsc {

struct LineGen {
    int mode;             // 0 disk chihat, 1 rect chihat, 2 real quadrant, 3 complex quadrant,
                          // 4 mirrored n x n table on the L-periodic lattice, 5 strided read,
                          // 6 strided read of an even line stored for e <= L/2 only
    int L;                // line length
    double b, g[4];       // modes 0, 1
    const double *quad;   // modes 2, 3: quadrant [k2][k1] of a table of period L, h = L/2 + 1 per row
    int h;
    const double2 *src;   // modes 4, 5
    int n;                // mode 4: table side
    long long sl, se;     // modes 5, 6: src[line * sl + e * se] (6: e folded to L - e above L/2)
    int nvalid;           // mode 5: elements e >= nvalid read as zero (0: all valid)
    const void *dens;     // mode 7: density rows (line j1, element e < n), zero beyond n
    int dens_kind;        // mode 7: 0 FP32 real, 1 FP64 real, 2 FP32 complex, 3 FP64 complex
    const void *dmask;    // mode 7: optional n x n multiplier (FP32 for kinds 0, 2; FP64 otherwise)
};

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

__device__ __forceinline__ double2 line_value(const LineGen &G, int line, int e)
{
    switch (G.mode) {
    case 0:
    case 1: return chihat(G.mode, G.g, G.b, G.L, e, line);
    case 2:
    case 3: {
        const int k1 = e <= G.L / 2 ? e : G.L - e, k2 = line <= G.L / 2 ? line : G.L - line;
        const size_t i = (size_t)k2 * G.h + k1;
        return G.mode == 2 ? make_double2(G.quad[i], 0.0) : make_double2(G.quad[2 * i], G.quad[2 * i + 1]);
    }
    case 4: {
        // w(d1, d2) with d = e for e < n, L - e for e > n, nothing at e = n
        const int d1 = line < G.n ? line : (line > G.L - G.n ? G.L - line : -1);
        const int d2 = e < G.n ? e : (e > G.L - G.n ? G.L - e : -1);
        if (d1 < 0 || d2 < 0) return make_double2(0.0, 0.0);
        return G.src[(size_t)d1 * G.n + d2];
    }
    case 6: {
        const int f = e <= G.L / 2 ? e : G.L - e;
        return G.src[line * G.sl + f * G.se];
    }
    case 7: {
        if (e >= G.n) return make_double2(0.0, 0.0);
        const size_t i = (size_t)line * G.n + e;
        const bool f32 = (G.dens_kind & 1) == 0;
        double m = 1.0;
        if (G.dmask) m = f32 ? (double)reinterpret_cast<const float *>(G.dmask)[i] : reinterpret_cast<const double *>(G.dmask)[i];
        switch (G.dens_kind) {
        case 0: return make_double2(m * reinterpret_cast<const float *>(G.dens)[i], 0.0);
        case 1: return make_double2(m * reinterpret_cast<const double *>(G.dens)[i], 0.0);
        case 2: {
            const float2 v = reinterpret_cast<const float2 *>(G.dens)[i];
            return make_double2(m * v.x, m * v.y);
        }
        default: {
            const double2 v = reinterpret_cast<const double2 *>(G.dens)[i];
            return make_double2(m * v.x, m * v.y);
        }
        }
    }
    default:
        if (G.nvalid > 0 && e >= G.nvalid) return make_double2(0.0, 0.0);
        return G.src[line * G.sl + e * G.se];
    }
}

// out[line * ol + e * oe] = scale * DFT_L(line)[e] for e < keep (INV: e^{+}, unnormalised).
template <bool INV>
__global__ void __launch_bounds__(512, 1) k_lines(LineGen G, double2 *__restrict__ out, int nlines, int keep,
                                                  long long ol, long long oe, double scale,
                                                  const FFTDesc *__restrict__ P, const double2 *__restrict__ tw,
                                                  int tpt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *buf = reinterpret_cast<double2 *>(smem_raw);
    const int lt = threadIdx.x;
    for (int line = blockIdx.x; line < nlines; line += gridDim.x) {
        for (int e = lt; e < G.L; e += tpt) buf[pidx<double>(e)] = line_value(G, line, e);
        __syncthreads();
        fft_smem<double, 0, INV, false>(buf, P, tw, lt, tpt);
        for (int e = lt; e < keep; e += tpt) {
            const double2 v = buf[pidx<double>(e)];
            out[line * ol + e * oe] = make_double2(scale * v.x, scale * v.y);
        }
        __syncthreads();
    }
}

// Lines longer than one CTA holds: DFT_L = DFT_L2 after twiddles after DFT_L1 (L = L1 L2, the
// four-step split).  X[k1 + L1 k2] = sum_{n2} W_L2^{n2 k2} W_L^{n2 k1} sum_{n1} W_L1^{n1 k1} x[L2 n1 + n2]
// (W_N = e^{-+2 pi i/N}).  Step 1: per (line, n2), the length-L1 transform over n1, times the
// twiddle, into T[line][k1][n2]; step 2: per (line, k1), the length-L2 transform over n2, outputs
// k = k1 + L1 k2 < keep.  T lives in global memory (plan time only).
template <bool INV>
__global__ void __launch_bounds__(512, 1) k_lines_split1(LineGen G, double2 *__restrict__ T, int nlines, int L1, int L2,
                                                         const FFTDesc *__restrict__ P, const double2 *__restrict__ tw,
                                                         int tpt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *buf = reinterpret_cast<double2 *>(smem_raw);
    const int lt = threadIdx.x;
    const long long L = (long long)L1 * L2, subs = (long long)nlines * L2;
    for (long long sidx = blockIdx.x; sidx < subs; sidx += gridDim.x) {
        const int line = (int)(sidx / L2), n2 = (int)(sidx - (long long)line * L2);
        for (int e = lt; e < L1; e += tpt) buf[pidx<double>(e)] = line_value(G, line, e * L2 + n2);
        __syncthreads();
        fft_smem<double, 0, INV, false>(buf, P, tw, lt, tpt);
        for (int k1 = lt; k1 < L1; k1 += tpt) {
            const double2 v = buf[pidx<double>(k1)];
            double sn, cs;
            // W_L^{n2 k1} = e^{-+2 pi i n2 k1 / L}: sincospi of 2 (n2 k1 mod L) / L
            sincospi(2.0 * (double)(((long long)n2 * k1) % L) / (double)L, &sn, &cs);
            if (!INV) sn = -sn;
            T[((size_t)line * L1 + k1) * L2 + n2] = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
        }
        __syncthreads();
    }
}

template <bool INV>
__global__ void __launch_bounds__(512, 1) k_lines_split2(const double2 *__restrict__ T, double2 *__restrict__ out,
                                                         int nlines, int L1, int L2, int keep, long long ol,
                                                         long long oe, double scale, const FFTDesc *__restrict__ P,
                                                         const double2 *__restrict__ tw, int tpt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *buf = reinterpret_cast<double2 *>(smem_raw);
    const int lt = threadIdx.x;
    const long long subs = (long long)nlines * L1;
    for (long long sidx = blockIdx.x; sidx < subs; sidx += gridDim.x) {
        const int line = (int)(sidx / L1), k1 = (int)(sidx - (long long)line * L1);
        const double2 *src = T + ((size_t)line * L1 + k1) * L2;
        for (int e = lt; e < L2; e += tpt) buf[pidx<double>(e)] = src[e];
        __syncthreads();
        fft_smem<double, 0, INV, false>(buf, P, tw, lt, tpt);
        for (int k2 = lt; k2 < L2; k2 += tpt) {
            const long long k = k1 + (long long)L1 * k2;
            if (k < keep) {
                const double2 v = buf[pidx<double>(k2)];
                out[line * ol + k * oe] = make_double2(scale * v.x, scale * v.y);
            }
        }
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

// quadrant [k2][k1] of G2 (real or complex) from the complex transform output
__global__ void k_take_quadrant(const double2 *__restrict__ in, double *__restrict__ out, long long N, int cplx)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (cplx) {
            out[2 * i] = in[i].x;
            out[2 * i + 1] = in[i].y;
        } else {
            out[i] = in[i].x;
        }
    }
}

int generic_threads(const FFTDesc &P);
bool factorize_any(int L, FFTDesc &d);
void stage_twiddles(const FFTDesc &d, std::vector<double> &re_im);

// Device-side FFT set-up of one line length (descriptor, twiddles, launch shape).  A line that one
// CTA cannot hold (or any line with WSCONV_LINE_SPLIT=1, for tests) runs as the four-step split
// L = L1 L2 into two shorter line transforms with a global-memory buffer between them.
struct LineFFT {
    FFTDesc d;
    FFTDesc *dd = nullptr;
    double2 *tw = nullptr;
    int tpt = 0;
    size_t smem = 0;
    std::vector<double> twh;
    int L = 0, L1 = 0, L2 = 0;                 // L1 > 0: the split path
    LineFFT *f1 = nullptr, *f2 = nullptr;      // its two line lengths
    cudaStream_t st_ = nullptr;                // the tables are allocated and freed in its order
    ~LineFFT()
    {
        if (dd) cudaFreeAsync(dd, st_);
        if (tw) cudaFreeAsync(tw, st_);
        delete f1;
        delete f2;
    }
    static bool fits(int L, int &tpt_out)
    {
        FFTDesc d;
        if (!factorize_any(L, d)) return false;
        const int tpt = generic_threads(d);
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        tpt_out = tpt;
        return (size_t)padded_len<double>(L) * sizeof(double2) <= (size_t)optin && tpt <= 512;
    }
    conv_status init(int Lin, cudaStream_t st)
    {
        L = Lin;
        int t = 0;
        const char *force = getenv("WSCONV_LINE_SPLIT");
        const bool split = !fits(L, t) || (force && atoi(force) == 1 && L >= 16);
        if (split) {
            // the most balanced factor pair whose parts both fit (L1 <= L2)
            for (int a = (int)std::sqrt((double)L); a >= 2 && !L1; --a) {
                if (L % a) continue;
                int t1 = 0, t2 = 0;
                if (fits(a, t1) && fits(L / a, t2)) {
                    L1 = a;
                    L2 = L / a;
                }
            }
            if (!L1) return fail(CONV_EUNSUPPORTED, "FP64 line length " + std::to_string(L) + " has no four-step split");
            f1 = new LineFFT();
            f2 = new LineFFT();
            conv_status rc = f1->init_direct(L1, st);
            if (rc == CONV_OK) rc = f2->init_direct(L2, st);
            return rc;
        }
        return init_direct(L, st);
    }
    conv_status init_direct(int Lin, cudaStream_t st)
    {
        L = Lin;
        st_ = st;
        if (!factorize_any(L, d)) return fail(CONV_EUNSUPPORTED, "line length not 2^a 3^b 5^c");
        tpt = generic_threads(d);
        smem = (size_t)padded_len<double>(L) * sizeof(double2);
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (smem > (size_t)optin || tpt > 512) return fail(CONV_EUNSUPPORTED, "FP64 line transform does not fit one CTA");
        stage_twiddles(d, twh);
        if (cudaMallocAsync(&dd, sizeof(FFTDesc), st) != cudaSuccess ||
            cudaMallocAsync(&tw, twh.size() * sizeof(double), st) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "line transform tables");
        }
        WSC_CUDA(cudaMemcpyAsync(dd, &d, sizeof(FFTDesc), cudaMemcpyHostToDevice, st));
        WSC_CUDA(cudaMemcpyAsync(tw, twh.data(), twh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        // the opt-in maximum, so line transforms of any length can follow each other
        WSC_CUDA(cudaFuncSetAttribute(k_lines<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        WSC_CUDA(cudaFuncSetAttribute(k_lines<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        WSC_CUDA(cudaFuncSetAttribute(k_lines_split1<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        WSC_CUDA(cudaFuncSetAttribute(k_lines_split1<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        WSC_CUDA(cudaFuncSetAttribute(k_lines_split2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        WSC_CUDA(cudaFuncSetAttribute(k_lines_split2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        return CONV_OK;
    }
    // T: NULL (the four-step buffer of nlines x L values is allocated in stream order) or a buffer
    // of that size the caller owns
    template <bool INV>
    conv_status run(const LineGen &G, double2 *out, int nlines, int keep, long long ol, long long oe, double scale,
                    int sms, cudaStream_t st, double2 *Tbuf = nullptr) const
    {
        if (!L1) {
            k_lines<INV><<<std::min(nlines, sms * 2), tpt, smem, st>>>(G, out, nlines, keep, ol, oe, scale, dd, tw, tpt);
            return CONV_OK;
        }
        double2 *T = Tbuf;
        if (!T && cudaMallocAsync(&T, (size_t)nlines * L * sizeof(double2), st) != cudaSuccess) {
            cudaGetLastError();
            return fail(CONV_ENOMEM, "four-step line buffer");
        }
        const long long s1 = (long long)nlines * L2, s2 = (long long)nlines * L1;
        k_lines_split1<INV><<<(int)std::min<long long>(s1, sms * 2LL), f1->tpt, f1->smem, st>>>(G, T, nlines, L1, L2,
                                                                                             f1->dd, f1->tw, f1->tpt);
        k_lines_split2<INV><<<(int)std::min<long long>(s2, sms * 2LL), f2->tpt, f2->smem, st>>>(
            T, out, nlines, L1, L2, keep, ol, oe, scale, f2->dd, f2->tw, f2->tpt);
        if (!Tbuf) WSC_CUDA(cudaFreeAsync(T, st));
        return CONV_OK;
    }
};

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Compact-embedding multiplier G2 (quadrant [k2][k1], k1, k2 <= n, FP64, real or complex) from the
// period-M moment quadrant ghat (h = M/2 + 1 per row).  Synchronises `st`.
conv_status build_compact_table(const double *ghat, bool cplx, int n, int M, double *g2_out, cudaStream_t st)
{
    const int L = 2 * n, h = M / 2 + 1, sms = sm_count();
    LineFFT fm, fl;
    conv_status rc = fm.init(M, st);
    if (rc == CONV_OK) rc = fl.init(L, st);
    if (rc != CONV_OK) return rc;
    double2 *t1 = nullptr, *w = nullptr, *t2 = nullptr, *g2 = nullptr;
    const size_t n1 = (size_t)n + 1;
    // scratch in stream order: freeing it does not wait for other work on the device (a serving
    // process builds plans while other requests run)
    auto release = [&] {
        for (double2 *q : {t1, w, t2, g2})
            if (q) cudaFreeAsync(q, st);
    };
    // ghat is even in k2 and w in d1: the lines k2 and M - k2 of the first transform, and e1 and
    // L - e1 of the third, are the same, so only the first half of each is formed and the next
    // transform reads the other half folded back (mode 6)
    const int hM = M / 2 + 1, hL = L / 2 + 1;
    bool ok = cudaMallocAsync(&t1, (size_t)hM * n * sizeof(double2), st) == cudaSuccess &&
              cudaMallocAsync(&w, (size_t)n * n * sizeof(double2), st) == cudaSuccess &&
              cudaMallocAsync(&t2, n1 * L * sizeof(double2), st) == cudaSuccess &&
              cudaMallocAsync(&g2, n1 * n1 * sizeof(double2), st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release();
        return fail(CONV_ENOMEM, "compact-embedding buffers");
    }
    LineGen G{};
    // w = (1/M^2) IDFT_M x M (ghat) on [0, n)^2: columns k2 (lines) along k1, keep d1 < n -> t1[k2][d1]
    G.mode = cplx ? 3 : 2;
    G.L = M;
    G.quad = ghat;
    G.h = h;
    if (rc == CONV_OK) rc = fm.run<true>(G, t1, hM, n, n, 1, 1.0, sms, st);
    // rows d1: along k2 (lines k2 > M/2 folded back), keep d2 < n -> w[d1][d2]
    G.mode = 6;
    G.src = t1;
    G.sl = 1;
    G.se = n;
    if (rc == CONV_OK) rc = fm.run<true>(G, w, n, n, n, 1, 1.0 / ((double)M * (double)M), sms, st);
    // G2 = DFT_L x L (w on the L-periodic lattice): rows e1 along e2, keep k2 <= n -> t2[k2][e1]
    G.mode = 4;
    G.L = L;
    G.src = w;
    G.n = n;
    if (rc == CONV_OK) rc = fl.run<false>(G, t2, hL, n + 1, 1, L, 1.0, sms, st);
    // columns k2 along e1 (lines e1 > L/2 folded back), keep k1 <= n -> g2[k2][k1]
    G.mode = 6;
    G.src = t2;
    G.sl = L;
    G.se = 1;
    if (rc == CONV_OK) rc = fl.run<false>(G, g2, n + 1, n + 1, n + 1, 1, 1.0, sms, st);
    const long long NQ = (long long)n1 * n1;
    if (rc == CONV_OK)
        k_take_quadrant<<<(int)std::min<long long>((NQ + 255) / 256, sms * 8LL), 256, 0, st>>>(g2, g2_out, NQ, cplx ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (rc != CONV_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "compact-embedding table");
    return CONV_OK;
}

__global__ void k_add_quadrant(const double2 *__restrict__ t, double *__restrict__ acc, long long N, int cplx,
                               double scale)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (cplx) {
            acc[2 * i] += scale * t[i].x;
            acc[2 * i + 1] += scale * t[i].y;
        } else {
            acc[i] += scale * t[i].x;
        }
    }
}

// acc += scale * DFT_{M x M}(table) for a table even in both indices (the localized scheme's
// smooth-part weights), given by its quadrant [k2][k1], k < h = M/2 + 1, real or complex; the
// result is even too and is added to the quadrant acc (same layout).  Lines k2 <= M/2 along k1
// first (the rest are their mirrors), then lines q1 along k2 read folded back.
conv_status add_even_dft2(const double *quad, bool cplx, int M, double scale, double *acc, cudaStream_t st)
{
    const int h = M / 2 + 1, sms = sm_count();
    LineFFT f;
    conv_status rc = f.init(M, st);
    if (rc != CONV_OK) return rc;
    double2 *t1 = nullptr, *t2 = nullptr;
    if (cudaMallocAsync(&t1, (size_t)h * h * sizeof(double2), st) != cudaSuccess ||
        cudaMallocAsync(&t2, (size_t)h * h * sizeof(double2), st) != cudaSuccess) {
        cudaGetLastError();
        if (t1) cudaFreeAsync(t1, st);
        return fail(CONV_ENOMEM, "even 2-D DFT buffers");
    }
    LineGen G{};
    G.mode = cplx ? 3 : 2;
    G.L = M;
    G.quad = quad;
    G.h = h;
    rc = f.run<false>(G, t1, h, h, h, 1, 1.0, sms, st);  // t1[k2][q1]
    G.mode = 6;
    G.src = t1;
    G.sl = 1;
    G.se = h;
    if (rc == CONV_OK) rc = f.run<false>(G, t2, h, h, 1, h, 1.0, sms, st);  // t2[q2][q1]
    const long long N = (long long)h * h;
    if (rc == CONV_OK)
        k_add_quadrant<<<(int)std::min<long long>((N + 255) / 256, sms * 8LL), 256, 0, st>>>(t2, acc, N, cplx ? 1 : 0,
                                                                                              scale);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(t1, st);
    cudaFreeAsync(t2, st);
    if (rc != CONV_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "even 2-D DFT");
    return CONV_OK;
}

// ---------------------------------------------------------------- lines beyond one CTA
// When one line of the transform (length L) does not fit one CTA's shared memory -- FP64 at
// n = 8192 (L = 16384 compact, 24576 on the period-3 grid), FP32 at L = 24576 -- the three passes
// run as FP64 line transforms of the full complex spectrum, each line that one CTA cannot hold
// split four-step (L = L1 L2, a global-memory buffer between the two halves):
//   pass 1: rows j1 < n of u (times the mask), zero-extended to L: X[k2][j1];
//   pass 2: per chunk of columns k2, the length-L transform of X[k2][j1 < n] (zero beyond n),
//           times the multiplier ghat(|k1|, |k2|), the inverse transform, the first n outputs back
//           into X[k2][j1];
//   pass 3: rows j1 of X along k2, inverse, the first n outputs: Y[j1][j2];
//   out = beta u + alpha Y / L^2 (real part for R2R), in the plan's type.
// Densities run one after another, so the workspace does not grow with the batch.  The arithmetic
// is FP64 in every plan precision.
#define LONG_CHUNK 2048
struct LongLines {
    LineFFT f;
    int chunk = 0;
};

static size_t long_ws_elems(const conv_plan_s *p)
{
    const size_t n = p->n, L = p->M, ch = std::min<size_t>(L, LONG_CHUNK);
    return n * L + ch * L + std::max(n, ch) * L + n * n;  // X, F, T, Y (complex FP64)
}

size_t long_lines_ws_bytes(const conv_plan_s *p) { return long_ws_elems(p) * sizeof(double2); }

conv_status long_lines_init(conv_plan_s *p)
{
    LongLines *ll = new LongLines();
    conv_status rc = ll->f.init(p->M, p->setup_stream);
    if (rc != CONV_OK) {
        delete ll;
        return rc;
    }
    ll->chunk = std::min(p->M, LONG_CHUNK);
    p->longl = ll;
    WSC_CUDA(cudaStreamSynchronize(p->setup_stream));
    return CONV_OK;
}

void long_lines_destroy(conv_plan_s *p)
{
    delete p->longl;
    p->longl = nullptr;
}

// F[c][k1] *= ghat(|k1|, |k2|), k2 = c0 + c: the multiplier quadrant [k2][k1], h = L/2 + 1
__global__ void k_long_multiply(double2 *__restrict__ F, int cols, int c0, int L, const double *__restrict__ g, int cplx,
                                int odd)
{
    const int h = L / 2 + 1;
    const long long N = (long long)cols * L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / L), k1 = (int)(i - (long long)c * L), k2 = c0 + c;
        const int a1 = k1 <= L / 2 ? k1 : L - k1, a2 = k2 <= L / 2 ? k2 : L - k2;
        const size_t q = (size_t)a2 * h + a1;
        const double2 v = F[i];
        if (odd) {  // i sgn(k1) g, 0 at the unpaired Nyquist index
            const double t = 2 * k1 == L ? 0.0 : (2 * k1 < L ? g[q] : -g[q]);
            F[i] = make_double2(-t * v.y, t * v.x);
        } else if (cplx) {
            const double gr = g[2 * q], gi = g[2 * q + 1];
            F[i] = make_double2(v.x * gr - v.y * gi, v.x * gi + v.y * gr);
        } else {
            F[i] = make_double2(v.x * g[q], v.y * g[q]);
        }
    }
}

// out = beta u + alpha Y (alpha complex; real part for R2R), in the plan's types
template <typename T>
__global__ void k_long_finish(const double2 *__restrict__ Y, const void *__restrict__ u, void *__restrict__ out,
                              long long N, int io, double are, double aim, double beta)
{
    typedef typename cvec<T>::t V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double2 y = Y[i];
        double zr = are * y.x - aim * y.y, zi = are * y.y + aim * y.x;
        if (beta != 0.0) {
            if (io == CONV_IO_C2C) {
                const V uv = reinterpret_cast<const V *>(u)[i];
                zr += beta * (double)uv.x;
                zi += beta * (double)uv.y;
            } else {
                zr += beta * (double)reinterpret_cast<const T *>(u)[i];
            }
        }
        if (io == CONV_IO_R2R) reinterpret_cast<T *>(out)[i] = (T)zr;
        else reinterpret_cast<V *>(out)[i] = cmk<V>((T)zr, (T)zi);
    }
}

conv_status long_lines_apply(conv_plan_s *p, const void *u, const void *mask, void *out, int batch, double are,
                             double aim, double beta, void *ws, cudaStream_t st)
{
    const LongLines *ll = p->longl;
    if (!ll) return fail(CONV_EUNSUPPORTED, "long-line transforms not set up");
    const int n = p->n, L = p->M, CH = ll->chunk, sms = sm_count();
    const bool f32 = p->prec == CONV_P_FP32;
    const size_t nL = (size_t)n * L;
    double2 *X = reinterpret_cast<double2 *>(ws), *F = X + nL, *Tb = F + (size_t)CH * L,
            *Y = Tb + std::max<size_t>(n, CH) * L;
    const double sc = 1.0 / ((double)L * (double)L);
    const size_t rsz = f32 ? 4 : 8;
    const size_t in_elem = (p->io == CONV_IO_C2C ? 2 : 1) * rsz, out_elem = (p->io == CONV_IO_R2R ? 1 : 2) * rsz;
    cudaEvent_t *ev = timing_slot(p);
    if (ev) cudaEventRecord(ev[0], st);
    conv_status rc = CONV_OK;
    for (int b = 0; b < batch && rc == CONV_OK; ++b) {
        const char *ub = reinterpret_cast<const char *>(u) + (size_t)b * n * n * in_elem;
        char *ob = reinterpret_cast<char *>(out) + (size_t)b * n * n * out_elem;
        LineGen G{};
        G.L = L;
        G.mode = 7;
        G.n = n;
        G.dens = ub;
        G.dens_kind = (f32 ? 0 : 1) + (p->io == CONV_IO_C2C ? 2 : 0);
        G.dmask = mask;
        rc = ll->f.run<false>(G, X, n, L, 1, n, 1.0, sms, st, Tb);  // X[k2][j1]
        if (ev && b == 0) cudaEventRecord(ev[1], st);
        for (int c0 = 0; c0 < L && rc == CONV_OK; c0 += CH) {
            const int cols = std::min(CH, L - c0);
            LineGen C{};
            C.L = L;
            C.mode = 5;
            C.src = X + (size_t)c0 * n;
            C.sl = n;
            C.se = 1;
            C.nvalid = n;
            rc = ll->f.run<false>(C, F, cols, L, L, 1, 1.0, sms, st, Tb);  // F[c][k1]
            if (rc != CONV_OK) break;
            const long long NF = (long long)cols * L;
            k_long_multiply<<<(int)std::min<long long>((NF + 255) / 256, sms * 8LL), 256, 0, st>>>(
                F, cols, c0, L, p->ghat64, p->complex_ghat ? 1 : 0, p->kern.family == CONV_K_DX1LOG ? 1 : 0);
            LineGen I{};
            I.L = L;
            I.mode = 5;
            I.src = F;
            I.sl = L;
            I.se = 1;
            rc = ll->f.run<true>(I, X + (size_t)c0 * n, cols, n, n, 1, 1.0, sms, st, Tb);  // X[k2][j1 < n]
        }
        if (ev && b == 0) cudaEventRecord(ev[2], st);
        if (rc != CONV_OK) break;
        LineGen R{};
        R.L = L;
        R.mode = 5;
        R.src = X;
        R.sl = 1;
        R.se = n;
        rc = ll->f.run<true>(R, Y, n, n, n, 1, sc, sms, st, Tb);  // Y[j1][j2]
        if (rc != CONV_OK) break;
        const long long NN = (long long)n * n;
        const int g2 = (int)std::min<long long>((NN + 255) / 256, sms * 8LL);
        if (f32) k_long_finish<float><<<g2, 256, 0, st>>>(Y, ub, ob, NN, p->io, are, aim, beta);
        else k_long_finish<double><<<g2, 256, 0, st>>>(Y, ub, ob, NN, p->io, are, aim, beta);
    }
    if (ev) cudaEventRecord(ev[3], st);
    WSC_CUDA(cudaGetLastError());
    return rc;
}

}  // namespace wsc

using namespace wsc;

extern "C" conv_status conv_fs_mask(conv_plan_t p, int shape, const double *geom, double delta, void *mask,
                                    void *stream)
{
    if (!p || !geom || !mask) return fail(CONV_EINVAL, "bad argument");
    if (shape != 0 && shape != 1) return fail(CONV_EINVAL, "shape must be 0 (disk) or 1 (rectangle)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n = p->n, M = p->Mb, sms = sm_count();
    LineFFT f;
    conv_status rc = f.init(M, st);
    if (rc != CONV_OK) return rc;
    double2 *W = nullptr, *chi = nullptr;
    if (cudaMallocAsync(&W, (size_t)M * n * sizeof(double2), st) != cudaSuccess ||
        cudaMallocAsync(&chi, (size_t)n * n * sizeof(double2), st) != cudaSuccess) {
        cudaGetLastError();
        if (W) cudaFreeAsync(W, st);
        return fail(CONV_ENOMEM, "FS mask buffers");
    }
    LineGen G{};
    G.mode = shape;
    G.L = M;
    G.b = p->b;
    for (int i = 0; i < (shape == 0 ? 3 : 4); ++i) G.g[i] = geom[i];
    // columns k2 (lines) of chihat along k1, keep j1 < n -> W[k2][j1]
    if (rc == CONV_OK) rc = f.run<true>(G, W, M, n, n, 1, 1.0, sms, st);
    // rows j1: along k2, keep j2 < n -> chi[j1][j2]
    G.mode = 5;
    G.src = W;
    G.sl = 1;
    G.se = n;
    if (rc == CONV_OK) rc = f.run<true>(G, chi, n, n, n, 1, 1.0, sms, st);
    const int blocks = (int)std::min<long long>(((long long)n * n + 255) / 256, (long long)sms * 8);
    if (rc != CONV_OK) {
        cudaFreeAsync(W, st);
        cudaFreeAsync(chi, st);
        cudaStreamSynchronize(st);
        return rc;
    }
    if (p->prec == CONV_P_FP64)
        k_fs_finish<double><<<blocks, 256, 0, st>>>(chi, reinterpret_cast<double *>(mask), n, delta);
    else
        k_fs_finish<float><<<blocks, 256, 0, st>>>(chi, reinterpret_cast<float *>(mask), n, delta);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(W, st);
    cudaFreeAsync(chi, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "conv_fs_mask");
    return CONV_OK;
}
