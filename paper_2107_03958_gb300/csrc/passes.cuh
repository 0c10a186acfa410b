// passes.cuh -- kernel templates of the three fused convolution passes (instantiated per
// precision in passes_f64*.cu / passes_f32*.cu; host dispatch in passes.cu).
//
// Every pass kernel is persistent: the grid holds as many CTAs as fit on the GPU at once, and
// each CTA loops over work items (a row pair, a row or a column of one density), G items at a
// time, one per thread group of `tpt` threads.  With TWS the CTA first copies the length-M
// twiddle table into shared memory once, so the butterflies' twiddle reads never leave the SM.
#pragma once
#include "wsconv_internal.h"

namespace wsc {

#define WSC_LB(T, E) __launch_bounds__(maxt<T, E>::v, 1)

template <typename T> struct PassArgs {
    typedef typename cvec<T>::t V;
    const void *in;        // pass 1: u; passes 2, 3: the spectrum workspace
    const T *mask;         // pass 1: optional n x n multiplier
    void *out;             // passes 1, 2: the workspace; pass 3: the result
    const void *ghat;      // pass 2: moment quadrant [k2][k1] (T or complex V)
    const void *u;         // pass 3: u for the beta term
    const V *tw;           // per-stage twiddle blocks (FFTDesc), global
    int tw_len;            // entries of the twiddle table (TWS: of its shared-memory copy)
    const FFTDesc *P;
    int n, h, M, tpt;
    int units;             // work items over the whole batch
    int batch;
    V alpha;               // pass 3 scale (already times 1/M^2)
    T beta;                // pass 3: out = beta u + alpha (.)
    int *err;              // the plan's device status word (CONV_ETIMEOUT: a bounded wait gave up)
    int give_up;           // injected fault (CONV_FAULT_WAIT): treat the first bounded wait as given up
    int stage_len;         // fused passes: elements V of each group's staging area (0: none)
    int pf;                // fused passes: this launch prefetches work items into the staging areas
    int vec;               // R2C pass 2: the output pairs may be stored as 16-byte vectors
    int tma;               // pass 1: spectra leave by TMA stores; pass 3: spectra arrive by TMA loads
    CUtensorMap tmap;      // the spectrum array's map for those copies (kernel parameter space)
    int odd;               // pass 2: the multiplier is i sgn(k1) T(|k1|, |k2|) (the non-radial kernel)
    int nsel;              // pass 2: 0, or the batch's own multiplier per density (conv_apply_kernels)
    const void *gsel[WSC_MAX_SEL];
    void *scratch;         // split pass 2 with one buffer per group: one global line per group
};

// x times the odd multiplier i sgn(k1) t at transform index o of a length-L column (k1 = o below
// L/2, o - L above it; the unpaired Nyquist index L/2 gets 0).
template <typename V, typename T>
__device__ __forceinline__ V odd_mul(V x, T t, int o, int L)
{
    if (2 * o == L) return cmk<V>((T)0, (T)0);
    const T st = 2 * o < L ? t : -t;
    return cmk<V>(-st * x.y, st * x.x);
}

// The multiplier table of density b in pass 2: the plan's, or the batch's own per density.
template <typename T>
__device__ __forceinline__ const void *mult_of(const PassArgs<T> &a, int b)
{
    return a.nsel ? a.gsel[b] : a.ghat;
}

// Staging of a fused pass 1 with TMA stores: [input rows (prefetch), rounded to 128 bytes]
// [output pairs: nbox x TMA_ROWS x 2 elements]; pass 3 with TMA loads: [nbox x TMA_ROWS x 2].
template <typename T> __host__ __device__ inline int tma_boxes(int h) { return (h + TMA_ROWS - 1) / TMA_ROWS; }
template <typename T> __host__ __device__ inline int stage_in_len(int n, bool pf)
{
    const int per128 = 128 / (int)(2 * sizeof(T));
    return pf ? (n + per128 - 1) / per128 * per128 : 0;
}

// Shared-memory carve-up: [twiddles (M) if TWS][group 0 buffer][group 1 buffer]...
template <typename T, bool TWS>
__device__ __forceinline__ typename cvec<T>::t *setup_smem(const PassArgs<T> &a, const typename cvec<T>::t *&twp,
                                                           int g)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *base = reinterpret_cast<V *>(smem_raw);
    if (TWS) {
        for (int t = threadIdx.x; t < a.tw_len; t += blockDim.x) base[t] = __ldg(&a.tw[t]);
        __syncthreads();
        twp = base;
        base += a.tw_len;
    } else {
        twp = a.tw;
    }
    return base + (size_t)g * padded_len<T>(a.M);
}

// Fused passes continue the carve-up with [staging 0]...[staging G-1][mbarrier 0]...[mbarrier G-1],
// the staging block starting on a 128-byte shared-memory address and every area a multiple of
// 128 bytes long
// (pass_smem on the host computes the same sizes).  A pass with NBUF transform buffers per group
// takes buffers NBUF g ... NBUF g + NBUF - 1 of the carve-up.
template <typename T, bool TWS, int NBUF = 1>
__device__ __forceinline__ typename cvec<T>::t *stage_area(const PassArgs<T> &a, int g, int G,
                                                           unsigned long long *&bar)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t off = (TWS ? (size_t)a.tw_len * sizeof(V) : 0) + (size_t)NBUF * G * padded_len<T>(a.M) * sizeof(V);
    // 128-byte aligned shared address (TMA boxes); the host reserves 128 bytes of slack for it
    const size_t base = (size_t)__cvta_generic_to_shared(smem_raw);
    off = ((base + off + 127) & ~(size_t)127) - base;
    const size_t st = ((size_t)a.stage_len * sizeof(V) + 127) & ~(size_t)127;
    bar = reinterpret_cast<unsigned long long *>(smem_raw + off + (size_t)G * st) + g;
    return reinterpret_cast<V *>(smem_raw + off + (size_t)g * st);
}

// ============================================================================ R2R pipeline
// pass 1: two real rows j1, j1+1 packed as z = u_a + i u_b, zero-extended to M, forward FFT,
// Hermitian split A_k = (Z_k + conj Z_{M-k})/2, B_k = (Z_k - conj Z_{M-k})/(2i), k <= M/2.
template <typename T, int E, bool TWS>
__global__ void WSC_LB(T, E) k_r2r_rows_fwd(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M, h = a.h, pairs = (n + 1) / 2;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int b = valid ? unit / pairs : 0, j1 = valid ? 2 * (unit - b * pairs) : 0;
        const bool has2 = valid && j1 + 1 < n;
        const T *ua = reinterpret_cast<const T *>(a.in) + (size_t)b * n * n + (size_t)j1 * n;
        const T *ma = a.mask ? a.mask + (size_t)j1 * n : nullptr;
        for (int e = lt; e < M; e += a.tpt) {
            V z = cmk<V>(0, 0);
            if (valid && e < n) {
                T x = ua[e], y = has2 ? ua[n + e] : (T)0;
                if (ma) {
                    x *= ma[e];
                    if (has2) y *= ma[n + e];
                }
                z = cmk<V>(x, y);
            }
            buf[pidx<T>(e)] = z;
        }
        __syncthreads();
        fft_smem<T, E, false, TWS>(buf, a.P, twp, lt, a.tpt);
        if (valid) {
            V *Wb = reinterpret_cast<V *>(a.out) + (size_t)b * h * n;
            for (int k = lt; k < h; k += a.tpt) {
                V Zk = buf[pidx<T>(k)], Zm = buf[pidx<T>(k == 0 ? 0 : M - k)];
                Wb[(size_t)k * n + j1] = cmk<V>((T)0.5 * (Zk.x + Zm.x), (T)0.5 * (Zk.y - Zm.y));
                if (has2) Wb[(size_t)k * n + j1 + 1] = cmk<V>((T)0.5 * (Zk.y + Zm.y), (T)-0.5 * (Zk.x - Zm.x));
            }
        }
        __syncthreads();
    }
}

// pass 2: per column k2 <= M/2 of one density: forward FFT over the n stored rows, times the real
// ghat(|k1|, k2), inverse FFT, keep rows j1 < n.  Work items run batch-fastest, so the CTAs
// handling one column for all densities run side by side and share its ghat column in L2.
template <typename T, int E, bool TWS>
__global__ void WSC_LB(T, E) k_r2r_cols(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M, h = a.h;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int k2 = valid ? unit / a.batch : 0, b = valid ? unit - k2 * a.batch : 0;
        const T *ghat = reinterpret_cast<const T *>(mult_of(a, b));
        V *col = reinterpret_cast<V *>(a.out) + (size_t)b * h * n + (size_t)k2 * n;
        for (int e = lt; e < M; e += a.tpt) buf[pidx<T>(e)] = (valid && e < n) ? col[e] : cmk<V>(0, 0);
        __syncthreads();
        fft_smem<T, E, false, TWS>(buf, a.P, twp, lt, a.tpt);
        const T *gc = ghat + (size_t)k2 * h;
        for (int e = lt; e < M; e += a.tpt) {
            const int k1 = e <= M / 2 ? e : M - e;
            buf[pidx<T>(e)] = a.odd ? odd_mul(buf[pidx<T>(e)], __ldg(&gc[k1]), e, M)
                                    : cscale(buf[pidx<T>(e)], __ldg(&gc[k1]));
        }
        __syncthreads();
        fft_smem<T, E, true, TWS>(buf, a.P, twp, lt, a.tpt);
        if (valid)
            for (int e = lt; e < n; e += a.tpt) col[e] = buf[pidx<T>(e)];
        __syncthreads();
    }
}

// pass 3: rows j1, j1+1: Z_k = A_k + i B_k (k <= M/2), Z_{M-k} = conj A_k + i conj B_k, inverse FFT,
// out_a = Re Z, out_b = Im Z on j2 < n, times alpha (1/M^2), plus beta u.
template <typename T, int E, bool TWS>
__global__ void WSC_LB(T, E) k_r2r_rows_inv(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M, h = a.h, pairs = (n + 1) / 2;
    const T alpha = a.alpha.x, beta = a.beta;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int b = valid ? unit / pairs : 0, j1 = valid ? 2 * (unit - b * pairs) : 0;
        const bool has2 = valid && j1 + 1 < n;
        const V *Wb = reinterpret_cast<const V *>(a.in) + (size_t)b * h * n;
        for (int k = lt; k < h; k += a.tpt) {
            V A = cmk<V>(0, 0), B = cmk<V>(0, 0);
            if (valid) {
                A = Wb[(size_t)k * n + j1];
                if (has2) B = Wb[(size_t)k * n + j1 + 1];
            }
            buf[pidx<T>(k)] = cmk<V>(A.x - B.y, A.y + B.x);
            if (k > 0 && k < M - k) buf[pidx<T>(M - k)] = cmk<V>(A.x + B.y, B.x - A.y);
        }
        __syncthreads();
        fft_smem<T, E, true, TWS>(buf, a.P, twp, lt, a.tpt);
        if (valid) {
            const size_t ro = (size_t)b * n * n + (size_t)j1 * n;
            T *oa = reinterpret_cast<T *>(a.out) + ro;
            const T *ua = reinterpret_cast<const T *>(a.u) + ro;
            for (int e = lt; e < n; e += a.tpt) {
                V z = buf[pidx<T>(e)];
                T ra = alpha * z.x, rb = alpha * z.y;
                if (beta != (T)0) {
                    ra += beta * ua[e];
                    if (has2) rb += beta * ua[n + e];
                }
                oa[e] = ra;
                if (has2) oa[n + e] = rb;
            }
        }
        __syncthreads();
    }
}

// ============================================================================ C2C pipeline
template <typename T, int E, bool TWS, bool IN_REAL>
__global__ void WSC_LB(T, E) k_c2c_rows_fwd(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int b = valid ? unit / n : 0, j1 = valid ? unit - b * n : 0;
        const size_t ro = (size_t)b * n * n + (size_t)j1 * n;
        const T *mr = a.mask ? a.mask + (size_t)j1 * n : nullptr;
        for (int e = lt; e < M; e += a.tpt) {
            V z = cmk<V>(0, 0);
            if (valid && e < n) {
                if (IN_REAL) z.x = reinterpret_cast<const T *>(a.in)[ro + e];
                else z = reinterpret_cast<const V *>(a.in)[ro + e];
                if (mr) z = cscale(z, mr[e]);
            }
            buf[pidx<T>(e)] = z;
        }
        __syncthreads();
        fft_smem<T, E, false, TWS>(buf, a.P, twp, lt, a.tpt);
        if (valid) {
            V *Wb = reinterpret_cast<V *>(a.out) + (size_t)b * M * n;
            for (int k = lt; k < M; k += a.tpt) Wb[(size_t)k * n + j1] = buf[pidx<T>(k)];
        }
        __syncthreads();
    }
}

// pass 2, complex pipeline: all M columns; ghat real (CG = false) or complex (CG = true).
template <typename T, int E, bool TWS, bool CG>
__global__ void WSC_LB(T, E) k_c2c_cols(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M, h = a.h;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int k2 = valid ? unit / a.batch : 0, b = valid ? unit - k2 * a.batch : 0;
        V *col = reinterpret_cast<V *>(a.out) + (size_t)b * M * n + (size_t)k2 * n;
        for (int e = lt; e < M; e += a.tpt) buf[pidx<T>(e)] = (valid && e < n) ? col[e] : cmk<V>(0, 0);
        __syncthreads();
        fft_smem<T, E, false, TWS>(buf, a.P, twp, lt, a.tpt);
        const int k2q = k2 <= M / 2 ? k2 : M - k2;
        for (int e = lt; e < M; e += a.tpt) {
            const int k1 = e <= M / 2 ? e : M - e;
            V z = buf[pidx<T>(e)];
            if (CG) z = cmul(z, __ldg(reinterpret_cast<const V *>(mult_of(a, b)) + (size_t)k2q * h + k1));
            else z = cscale(z, __ldg(reinterpret_cast<const T *>(mult_of(a, b)) + (size_t)k2q * h + k1));
            buf[pidx<T>(e)] = z;
        }
        __syncthreads();
        fft_smem<T, E, true, TWS>(buf, a.P, twp, lt, a.tpt);
        if (valid)
            for (int e = lt; e < n; e += a.tpt) col[e] = buf[pidx<T>(e)];
        __syncthreads();
    }
}

template <typename T, int E, bool TWS, bool IN_REAL>
__global__ void WSC_LB(T, E) k_c2c_rows_inv(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int b = valid ? unit / n : 0, j1 = valid ? unit - b * n : 0;
        const V *Wb = reinterpret_cast<const V *>(a.in) + (size_t)b * M * n;
        for (int k = lt; k < M; k += a.tpt) buf[pidx<T>(k)] = valid ? Wb[(size_t)k * n + j1] : cmk<V>(0, 0);
        __syncthreads();
        fft_smem<T, E, true, TWS>(buf, a.P, twp, lt, a.tpt);
        if (valid) {
            const size_t ro = (size_t)b * n * n + (size_t)j1 * n;
            V *o = reinterpret_cast<V *>(a.out) + ro;
            for (int e = lt; e < n; e += a.tpt) {
                V z = cmul(buf[pidx<T>(e)], a.alpha);
                if (a.beta != (T)0) {
                    if (IN_REAL) z.x += a.beta * reinterpret_cast<const T *>(a.u)[ro + e];
                    else {
                        V x = reinterpret_cast<const V *>(a.u)[ro + e];
                        z.x += a.beta * x.x;
                        z.y += a.beta * x.y;
                    }
                }
                o[e] = z;
            }
        }
        __syncthreads();
    }
}

// ============================================================================ host glue
template <typename T, int E, bool TWS> conv_status set_attrs(int smem)
{
#define WSC_ATTR(k) WSC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))
    WSC_ATTR((k_r2r_rows_fwd<T, E, TWS>));
    WSC_ATTR((k_r2r_cols<T, E, TWS>));
    WSC_ATTR((k_r2r_rows_inv<T, E, TWS>));
    WSC_ATTR((k_c2c_rows_fwd<T, E, TWS, true>));
    WSC_ATTR((k_c2c_rows_fwd<T, E, TWS, false>));
    WSC_ATTR((k_c2c_cols<T, E, TWS, true>));
    WSC_ATTR((k_c2c_cols<T, E, TWS, false>));
    WSC_ATTR((k_c2c_rows_inv<T, E, TWS, true>));
    WSC_ATTR((k_c2c_rows_inv<T, E, TWS, false>));
#undef WSC_ATTR
    return CONV_OK;
}

// CTAs of one pass kernel that fit on an SM at this launch shape.
template <typename T, int E, bool TWS> int blocks_per_sm(int threads, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_r2r_cols<T, E, TWS>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

template <typename T, int E, bool TWS>
conv_status run_pipeline(conv_plan_s *p, const void *u, const void *mask, void *out, int batch,
                         double are, double aim, double beta, void *ws, cudaStream_t st)
{
    typedef typename cvec<T>::t V;
    const int n = p->n, M = p->M, h = p->h;
    const double sc = 1.0 / ((double)M * (double)M);
    PassArgs<T> a{};
    a.mask = reinterpret_cast<const T *>(mask);
    a.ghat = p->prec == CONV_P_FP64 ? (const void *)p->ghat64 : p->ghat32;
    a.nsel = p->nsel;
    for (int i = 0; i < p->nsel; ++i) a.gsel[i] = p->sel[i];
    a.odd = p->kern.family == CONV_K_DX1LOG ? 1 : 0;
    a.u = u;
    a.tw = reinterpret_cast<const V *>(p->tw);
    a.tw_len = p->fft.tw_len;
    a.P = p->fft_dev;
    a.n = n;
    a.h = h;
    a.M = M;
    a.batch = batch;
    a.alpha = cmk<V>((T)(are * sc), (T)(aim * sc));
    a.beta = (T)beta;
    const LaunchShape &R = p->rows, &C = p->cols;
    auto grid = [&](const LaunchShape &S, int units) {
        long long need = (units + S.groups - 1) / S.groups;
        return (unsigned)std::min<long long>(need, (long long)S.max_ctas);
    };
    cudaEvent_t *ev = timing_slot(p);
    if (ev) cudaEventRecord(ev[0], st);
    if (p->io == CONV_IO_R2R) {
        a.tpt = R.tpt;
        a.in = u;
        a.out = ws;
        a.units = batch * ((n + 1) / 2);
        k_r2r_rows_fwd<T, E, TWS><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[1], st);
        a.tpt = C.tpt;
        a.in = ws;
        a.units = batch * h;
        k_r2r_cols<T, E, TWS><<<grid(C, a.units), C.tpt * C.groups, C.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[2], st);
        a.tpt = R.tpt;
        a.out = out;
        a.units = batch * ((n + 1) / 2);
        k_r2r_rows_inv<T, E, TWS><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
    } else {
        const bool in_real = p->io == CONV_IO_R2C;
        a.tpt = R.tpt;
        a.in = u;
        a.out = ws;
        a.units = batch * n;
        if (in_real)
            k_c2c_rows_fwd<T, E, TWS, true><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
        else
            k_c2c_rows_fwd<T, E, TWS, false><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[1], st);
        a.tpt = C.tpt;
        a.in = ws;
        a.units = batch * M;
        if (p->complex_ghat)
            k_c2c_cols<T, E, TWS, true><<<grid(C, a.units), C.tpt * C.groups, C.smem, st>>>(a);
        else
            k_c2c_cols<T, E, TWS, false><<<grid(C, a.units), C.tpt * C.groups, C.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[2], st);
        a.tpt = R.tpt;
        a.out = out;
        a.units = batch * n;
        if (in_real)
            k_c2c_rows_inv<T, E, TWS, true><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
        else
            k_c2c_rows_inv<T, E, TWS, false><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
    }
    if (ev) cudaEventRecord(ev[3], st);
    WSC_CUDA(cudaGetLastError());
    return CONV_OK;
}

}  // namespace wsc
