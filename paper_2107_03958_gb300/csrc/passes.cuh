// passes.cuh -- kernel templates of the three fused convolution passes (instantiated per
// precision in passes_f64.cu / passes_f32.cu; host dispatch in passes.cu).
#pragma once
#include "wsconv_internal.h"

namespace wsc {

#define WSC_LB(T, E) __launch_bounds__(maxt<T, E>::v, 1)

// ============================================================================ R2R pipeline
template <typename T, int E>
__global__ void WSC_LB(T, E)
k_r2r_rows_fwd(const T *__restrict__ u, const T *__restrict__ mask, typename cvec<T>::t *__restrict__ W,
               int n, int h, const FFTDesc *__restrict__ P, const typename cvec<T>::t *__restrict__ tw, int tpt)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = __ldg(&P->L);
    const int g = threadIdx.x / tpt, lt = threadIdx.x - g * tpt;
    const int G = blockDim.x / tpt;
    V *buf = reinterpret_cast<V *>(smem_raw) + (size_t)g * padded_len<T>(M);
    const int pair = blockIdx.x * G + g;
    const int j1 = 2 * pair;
    const bool valid = j1 < n, has2 = j1 + 1 < n;
    const size_t bo = (size_t)blockIdx.y * n * n;
    const T *ua = u + bo + (size_t)j1 * n, *ub = ua + n;
    const T *ma = mask ? mask + (size_t)j1 * n : nullptr, *mb = mask ? ma + n : nullptr;
    for (int e = lt; e < M; e += tpt) {
        V z = cmk<V>(0, 0);
        if (valid && e < n) {
            T a = ua[e], b = has2 ? ub[e] : (T)0;
            if (mask) {
                a *= ma[e];
                if (has2) b *= mb[e];
            }
            z = cmk<V>(a, b);
        }
        buf[pidx<T>(e)] = z;
    }
    __syncthreads();
    fft_smem<T, E, false>(buf, P, tw, lt, tpt);
    if (!valid) return;
    V *Wb = W + (size_t)blockIdx.y * h * n;
    for (int k = lt; k < h; k += tpt) {
        V Zk = buf[pidx<T>(k)], Zm = buf[pidx<T>(k == 0 ? 0 : M - k)];
        // A = (Z_k + conj Z_{M-k}) / 2,  B = (Z_k - conj Z_{M-k}) / (2i)
        V A = cmk<V>((T)0.5 * (Zk.x + Zm.x), (T)0.5 * (Zk.y - Zm.y));
        Wb[(size_t)k * n + j1] = A;
        if (has2) {
            V B = cmk<V>((T)0.5 * (Zk.y + Zm.y), (T)-0.5 * (Zk.x - Zm.x));
            Wb[(size_t)k * n + j1 + 1] = B;
        }
    }
}

// Column pass, real ghat.  grid = (batch, column blocks): the batch's CTAs for one column block
// run side by side, so each ghat column is fetched from HBM once per batch.
template <typename T, int E>
__global__ void WSC_LB(T, E)
k_r2r_cols(typename cvec<T>::t *__restrict__ W, const T *__restrict__ ghat, int n, int h,
           const FFTDesc *__restrict__ P, const typename cvec<T>::t *__restrict__ tw, int tpt)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = __ldg(&P->L);
    const int g = threadIdx.x / tpt, lt = threadIdx.x - g * tpt;
    const int G = blockDim.x / tpt;
    V *buf = reinterpret_cast<V *>(smem_raw) + (size_t)g * padded_len<T>(M);
    const int k2 = blockIdx.y * G + g;
    const bool valid = k2 < h;
    V *col = W + (size_t)blockIdx.x * h * n + (size_t)k2 * n;
    for (int e = lt; e < M; e += tpt) buf[pidx<T>(e)] = (valid && e < n) ? col[e] : cmk<V>(0, 0);
    __syncthreads();
    fft_smem<T, E, false>(buf, P, tw, lt, tpt);
    if (valid) {
        const T *gc = ghat + (size_t)k2 * h;
        for (int e = lt; e < M; e += tpt) {
            int k1 = e <= M / 2 ? e : M - e;
            buf[pidx<T>(e)] = cscale(buf[pidx<T>(e)], __ldg(&gc[k1]));
        }
    }
    __syncthreads();
    fft_smem<T, E, true>(buf, P, tw, lt, tpt);
    if (valid)
        for (int e = lt; e < n; e += tpt) col[e] = buf[pidx<T>(e)];
}

template <typename T, int E>
__global__ void WSC_LB(T, E)
k_r2r_rows_inv(const typename cvec<T>::t *__restrict__ W, const T *__restrict__ u, T *__restrict__ out,
               int n, int h, const FFTDesc *__restrict__ P, const typename cvec<T>::t *__restrict__ tw, int tpt,
               T alpha, T beta)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = __ldg(&P->L);
    const int g = threadIdx.x / tpt, lt = threadIdx.x - g * tpt;
    const int G = blockDim.x / tpt;
    V *buf = reinterpret_cast<V *>(smem_raw) + (size_t)g * padded_len<T>(M);
    const int pair = blockIdx.x * G + g;
    const int j1 = 2 * pair;
    const bool valid = j1 < n, has2 = j1 + 1 < n;
    const V *Wb = W + (size_t)blockIdx.y * h * n;
    // Z_k = A_k + i B_k for k <= M/2 and Z_{M-k} = conj(A_k) + i conj(B_k)
    for (int k = lt; k < h; k += tpt) {
        V A = cmk<V>(0, 0), B = cmk<V>(0, 0);
        if (valid) {
            A = Wb[(size_t)k * n + j1];
            if (has2) B = Wb[(size_t)k * n + j1 + 1];
        }
        buf[pidx<T>(k)] = cmk<V>(A.x - B.y, A.y + B.x);
        if (k > 0 && k < M - k) buf[pidx<T>(M - k)] = cmk<V>(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    fft_smem<T, E, true>(buf, P, tw, lt, tpt);
    if (!valid) return;
    const size_t bo = (size_t)blockIdx.y * n * n;
    T *oa = out + bo + (size_t)j1 * n, *ob = oa + n;
    const T *ua = u + bo + (size_t)j1 * n, *ub = ua + n;
    for (int e = lt; e < n; e += tpt) {
        V z = buf[pidx<T>(e)];
        T ra = alpha * z.x, rb = alpha * z.y;
        if (beta != (T)0) {
            ra += beta * ua[e];
            if (has2) rb += beta * ub[e];
        }
        oa[e] = ra;
        if (has2) ob[e] = rb;
    }
}

// ============================================================================ C2C pipeline
template <typename T, int E, bool IN_REAL>
__global__ void WSC_LB(T, E)
k_c2c_rows_fwd(const void *__restrict__ uin, const T *__restrict__ mask, typename cvec<T>::t *__restrict__ W,
               int n, const FFTDesc *__restrict__ P, const typename cvec<T>::t *__restrict__ tw, int tpt)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = __ldg(&P->L);
    const int g = threadIdx.x / tpt, lt = threadIdx.x - g * tpt;
    const int G = blockDim.x / tpt;
    V *buf = reinterpret_cast<V *>(smem_raw) + (size_t)g * padded_len<T>(M);
    const int j1 = blockIdx.x * G + g;
    const bool valid = j1 < n;
    const size_t ro = (size_t)blockIdx.y * n * n + (size_t)j1 * n;
    const T *mr = mask ? mask + (size_t)j1 * n : nullptr;
    for (int e = lt; e < M; e += tpt) {
        V z = cmk<V>(0, 0);
        if (valid && e < n) {
            if (IN_REAL) z.x = reinterpret_cast<const T *>(uin)[ro + e];
            else z = reinterpret_cast<const V *>(uin)[ro + e];
            if (mask) z = cscale(z, mr[e]);
        }
        buf[pidx<T>(e)] = z;
    }
    __syncthreads();
    fft_smem<T, E, false>(buf, P, tw, lt, tpt);
    if (!valid) return;
    V *Wb = W + (size_t)blockIdx.y * M * n;
    for (int k = lt; k < M; k += tpt) Wb[(size_t)k * n + j1] = buf[pidx<T>(k)];
}

// Column pass; ghat real (CG = false) or complex (CG = true), quadrant [k2'][k1'].
template <typename T, int E, bool CG>
__global__ void WSC_LB(T, E)
k_c2c_cols(typename cvec<T>::t *__restrict__ W, const void *__restrict__ ghat, int n, int h,
           const FFTDesc *__restrict__ P, const typename cvec<T>::t *__restrict__ tw, int tpt)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = __ldg(&P->L);
    const int g = threadIdx.x / tpt, lt = threadIdx.x - g * tpt;
    const int G = blockDim.x / tpt;
    V *buf = reinterpret_cast<V *>(smem_raw) + (size_t)g * padded_len<T>(M);
    const int k2 = blockIdx.y * G + g;
    const bool valid = k2 < M;
    V *col = W + (size_t)blockIdx.x * M * n + (size_t)k2 * n;
    for (int e = lt; e < M; e += tpt) buf[pidx<T>(e)] = (valid && e < n) ? col[e] : cmk<V>(0, 0);
    __syncthreads();
    fft_smem<T, E, false>(buf, P, tw, lt, tpt);
    if (valid) {
        const int k2q = k2 <= M / 2 ? k2 : M - k2;
        for (int e = lt; e < M; e += tpt) {
            int k1 = e <= M / 2 ? e : M - e;
            V z = buf[pidx<T>(e)];
            if (CG) z = cmul(z, __ldg(reinterpret_cast<const V *>(ghat) + (size_t)k2q * h + k1));
            else z = cscale(z, __ldg(reinterpret_cast<const T *>(ghat) + (size_t)k2q * h + k1));
            buf[pidx<T>(e)] = z;
        }
    }
    __syncthreads();
    fft_smem<T, E, true>(buf, P, tw, lt, tpt);
    if (valid)
        for (int e = lt; e < n; e += tpt) col[e] = buf[pidx<T>(e)];
}

template <typename T, int E, bool IN_REAL>
__global__ void WSC_LB(T, E)
k_c2c_rows_inv(const typename cvec<T>::t *__restrict__ W, const void *__restrict__ uin,
               typename cvec<T>::t *__restrict__ out, int n, const FFTDesc *__restrict__ P,
               const typename cvec<T>::t *__restrict__ tw, int tpt, typename cvec<T>::t alpha, T beta)
{
    typedef typename cvec<T>::t V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = __ldg(&P->L);
    const int g = threadIdx.x / tpt, lt = threadIdx.x - g * tpt;
    const int G = blockDim.x / tpt;
    V *buf = reinterpret_cast<V *>(smem_raw) + (size_t)g * padded_len<T>(M);
    const int j1 = blockIdx.x * G + g;
    const bool valid = j1 < n;
    const V *Wb = W + (size_t)blockIdx.y * M * n;
    for (int k = lt; k < M; k += tpt) buf[pidx<T>(k)] = valid ? Wb[(size_t)k * n + j1] : cmk<V>(0, 0);
    __syncthreads();
    fft_smem<T, E, true>(buf, P, tw, lt, tpt);
    if (!valid) return;
    const size_t ro = (size_t)blockIdx.y * n * n + (size_t)j1 * n;
    for (int e = lt; e < n; e += tpt) {
        V z = cmul(buf[pidx<T>(e)], alpha);
        if (beta != (T)0) {
            if (IN_REAL) z.x += beta * reinterpret_cast<const T *>(uin)[ro + e];
            else {
                V x = reinterpret_cast<const V *>(uin)[ro + e];
                z.x += beta * x.x;
                z.y += beta * x.y;
            }
        }
        out[ro + e] = z;
    }
}


template <typename T, int E> conv_status set_attrs(int smem)
{
#define WSC_ATTR(k) WSC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))
    WSC_ATTR((k_r2r_rows_fwd<T, E>));
    WSC_ATTR((k_r2r_cols<T, E>));
    WSC_ATTR((k_r2r_rows_inv<T, E>));
    WSC_ATTR((k_c2c_rows_fwd<T, E, true>));
    WSC_ATTR((k_c2c_rows_fwd<T, E, false>));
    WSC_ATTR((k_c2c_cols<T, E, true>));
    WSC_ATTR((k_c2c_cols<T, E, false>));
    WSC_ATTR((k_c2c_rows_inv<T, E, true>));
    WSC_ATTR((k_c2c_rows_inv<T, E, false>));
#undef WSC_ATTR
    return CONV_OK;
}

template <typename T, int E>
conv_status run_pipeline(conv_plan_s *p, const void *u, const void *mask, void *out, int batch,
                       double are, double aim, double beta, void *ws, cudaStream_t st)
{
    typedef typename cvec<T>::t V;
    const int n = p->n, M = p->M, h = p->h;
    const double sc = 1.0 / ((double)M * (double)M);
    const V *tw = reinterpret_cast<const V *>(p->tw);
    V *W = reinterpret_cast<V *>(ws);
    const T *mk = reinterpret_cast<const T *>(mask);
    const void *gh = p->prec == CONV_P_FP64 ? (const void *)p->ghat64 : p->ghat32;
    const LaunchShape &R = p->rows, &C = p->cols;
    const FFTDesc *fd = p->fft_dev;
    cudaEvent_t *ev = timing_slot(p);
    if (ev) cudaEventRecord(ev[0], st);
    if (p->io == CONV_IO_R2R) {
        int units = (n + 1) / 2;
        dim3 g1((units + R.groups - 1) / R.groups, batch);
        k_r2r_rows_fwd<T, E><<<g1, R.tpt * R.groups, R.smem, st>>>(reinterpret_cast<const T *>(u), mk, W, n, h, fd, tw, R.tpt);
        if (ev) cudaEventRecord(ev[1], st);
        dim3 g2(batch, (h + C.groups - 1) / C.groups);
        k_r2r_cols<T, E><<<g2, C.tpt * C.groups, C.smem, st>>>(W, reinterpret_cast<const T *>(gh), n, h, fd, tw, C.tpt);
        if (ev) cudaEventRecord(ev[2], st);
        k_r2r_rows_inv<T, E><<<g1, R.tpt * R.groups, R.smem, st>>>(W, reinterpret_cast<const T *>(u), reinterpret_cast<T *>(out), n, h, fd, tw, R.tpt, (T)(are * sc), (T)beta);
    } else {
        const bool in_real = p->io == CONV_IO_R2C;
        dim3 g1((n + R.groups - 1) / R.groups, batch);
        if (in_real)
            k_c2c_rows_fwd<T, E, true><<<g1, R.tpt * R.groups, R.smem, st>>>(u, mk, W, n, fd, tw, R.tpt);
        else
            k_c2c_rows_fwd<T, E, false><<<g1, R.tpt * R.groups, R.smem, st>>>(u, mk, W, n, fd, tw, R.tpt);
        if (ev) cudaEventRecord(ev[1], st);
        dim3 g2(batch, (M + C.groups - 1) / C.groups);
        if (p->complex_ghat)
            k_c2c_cols<T, E, true><<<g2, C.tpt * C.groups, C.smem, st>>>(W, gh, n, h, fd, tw, C.tpt);
        else
            k_c2c_cols<T, E, false><<<g2, C.tpt * C.groups, C.smem, st>>>(W, gh, n, h, fd, tw, C.tpt);
        if (ev) cudaEventRecord(ev[2], st);
        V al = cmk<V>((T)(are * sc), (T)(aim * sc));
        if (in_real)
            k_c2c_rows_inv<T, E, true><<<g1, R.tpt * R.groups, R.smem, st>>>(W, u, reinterpret_cast<V *>(out), n, fd, tw, R.tpt, al, (T)beta);
        else
            k_c2c_rows_inv<T, E, false><<<g1, R.tpt * R.groups, R.smem, st>>>(W, u, reinterpret_cast<V *>(out), n, fd, tw, R.tpt, al, (T)beta);
    }
    if (ev) cudaEventRecord(ev[3], st);
    WSC_CUDA(cudaGetLastError());
    return CONV_OK;
}


}  // namespace wsc
