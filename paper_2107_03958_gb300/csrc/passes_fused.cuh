// passes_fused.cuh -- the three convolution passes on the fused transform of fft_fused.cuh:
//   pass 1: stage 0 reads the (masked, zero-extended) rows from global memory;
//   pass 2: stage 0 reads the column from global memory, the forward transform's last stage
//           multiplies by ghat before its shared-memory store, and the inverse transform's last
//           stage writes the n surviving rows to global memory;
//   pass 3: stage 0 reads the (Hermitian-completed) spectrum from global memory and the last stage
//           writes the cropped, scaled result (plus beta u) to global memory.
// Same work decomposition, layouts and results as passes.cuh; fewer shared-memory sweeps.
#pragma once
#include "fft_fused.cuh"
#include "passes.cuh"

namespace wsc {

// ============================================================================ R2R
// The two spectra of a row pair sit side by side (W[k][j1], W[k][j1+1]); with n even the pair
// starts on an even element, so FP32 moves it as one 16-byte access.
template <typename T>
__device__ __forceinline__ void load_pair(const typename cvec<T>::t *p, typename cvec<T>::t &A,
                                          typename cvec<T>::t &B, bool has2, bool vec)
{
    if constexpr (sizeof(T) == 4) {
        if (vec && has2) {
            const float4 q = *reinterpret_cast<const float4 *>(p);
            A = make_float2(q.x, q.y);
            B = make_float2(q.z, q.w);
            return;
        }
    }
    A = p[0];
    B = has2 ? p[1] : cmk<typename cvec<T>::t>(0, 0);
}

template <typename T>
__device__ __forceinline__ void store_pair(typename cvec<T>::t *p, typename cvec<T>::t A, typename cvec<T>::t B,
                                           bool has2, bool vec)
{
    if constexpr (sizeof(T) == 4) {
        if (vec && has2) {
            *reinterpret_cast<float4 *>(p) = make_float4(A.x, A.y, B.x, B.y);
            return;
        }
    }
    p[0] = A;
    if (has2) p[1] = B;
}

template <typename T, int E, int ED, bool TWS>
__global__ void WSC_LB(T, E) kf_r2r_rows_fwd(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M, h = a.h, pairs = (n + 1) / 2;
    const bool pair_vec = (n & 1) == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15) == 0;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int b = valid ? unit / pairs : 0, j1 = valid ? 2 * (unit - b * pairs) : 0;
        const bool has2 = valid && j1 + 1 < n;
        const T *ua = reinterpret_cast<const T *>(a.in) + (size_t)b * n * n + (size_t)j1 * n;
        const T *ma = a.mask ? a.mask + (size_t)j1 * n : nullptr;
        auto src = [&](int i) -> V {
            if (!valid || i >= n) return cmk<V>(0, 0);
            T x = ua[i], y = has2 ? ua[n + i] : (T)0;
            if (ma) {
                x *= ma[i];
                if (has2) y *= ma[n + i];
            }
            return cmk<V>(x, y);
        };
        fft_fused<T, E, ED, false, TWS>(buf, a.P, twp, lt, a.tpt, src, ToSmem{});
        if (valid) {
            V *Wb = reinterpret_cast<V *>(a.out) + (size_t)b * h * n;
            for (int k = lt; k < h; k += a.tpt) {
                V Zk = buf[pidx<T>(k)], Zm = buf[pidx<T>(k == 0 ? 0 : M - k)];
                const V A = cmk<V>((T)0.5 * (Zk.x + Zm.x), (T)0.5 * (Zk.y - Zm.y));
                const V B = cmk<V>((T)0.5 * (Zk.y + Zm.y), (T)-0.5 * (Zk.x - Zm.x));
                store_pair<T>(Wb + (size_t)k * n + j1, A, B, has2, pair_vec);
            }
        }
        __syncthreads();
    }
}

template <typename T, int E, int ED, bool TWS>
__global__ void WSC_LB(T, E) kf_r2r_cols(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M, h = a.h;
    const T *ghat = reinterpret_cast<const T *>(a.ghat);
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int k2 = valid ? unit / a.batch : 0, b = valid ? unit - k2 * a.batch : 0;
        V *col = reinterpret_cast<V *>(a.out) + (size_t)b * h * n + (size_t)k2 * n;
        const T *gc = ghat + (size_t)k2 * h;
        auto src = [&](int i) -> V { return (valid && i < n) ? col[i] : cmk<V>(0, 0); };
        auto mul = smem_hook([&](int o, V &x) {
            const int k1 = o <= M / 2 ? o : M - o;
            x = cscale(x, __ldg(&gc[k1]));
        });
        fft_fused<T, E, ED, false, TWS>(buf, a.P, twp, lt, a.tpt, src, mul);
        auto dst = [&](int o, V x) {
            if (valid && o < n) col[o] = x;
        };
        fft_fused<T, E, ED, true, TWS>(buf, a.P, twp, lt, a.tpt, FromSmem{}, dst);
        __syncthreads();
    }
}

template <typename T, int E, int ED, bool TWS>
__global__ void WSC_LB(T, E) kf_r2r_rows_inv(const PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    const int n = a.n, M = a.M, h = a.h, pairs = (n + 1) / 2;
    const bool pair_vec = (n & 1) == 0 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0;
    const T alpha = a.alpha.x, beta = a.beta;
    for (int base = blockIdx.x * G; base < a.units; base += gridDim.x * G) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        const int b = valid ? unit / pairs : 0, j1 = valid ? 2 * (unit - b * pairs) : 0;
        const bool has2 = valid && j1 + 1 < n;
        const V *Wb = reinterpret_cast<const V *>(a.in) + (size_t)b * h * n;
        // Z_k = A_k + i B_k (k <= M/2), Z_k = conj A_{M-k} + i conj B_{M-k} (k > M/2)
        auto src = [&](int i) -> V {
            if (!valid) return cmk<V>(0, 0);
            const bool lo = i <= M / 2;
            const size_t k = (size_t)(lo ? i : M - i);
            V A, B;
            load_pair<T>(Wb + k * n + j1, A, B, has2, pair_vec);
            return lo ? cmk<V>(A.x - B.y, A.y + B.x) : cmk<V>(A.x + B.y, B.x - A.y);
        };
        const size_t ro = (size_t)b * n * n + (size_t)j1 * n;
        T *oa = reinterpret_cast<T *>(a.out) + ro;
        const T *ua = reinterpret_cast<const T *>(a.u) + ro;
        auto dst = [&](int o, V z) {
            if (!valid || o >= n) return;
            T ra = alpha * z.x, rb = alpha * z.y;
            if (beta != (T)0) {
                ra += beta * ua[o];
                if (has2) rb += beta * ua[n + o];
            }
            oa[o] = ra;
            if (has2) oa[n + o] = rb;
        };
        fft_fused<T, E, ED, true, TWS>(buf, a.P, twp, lt, a.tpt, src, dst);
        __syncthreads();
    }
}

// ============================================================================ C2C
template <typename T, int E, int ED, bool TWS, bool IN_REAL>
__global__ void WSC_LB(T, E) kf_c2c_rows_fwd(const PassArgs<T> a)
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
        auto src = [&](int i) -> V {
            if (!valid || i >= n) return cmk<V>(0, 0);
            V z;
            if (IN_REAL) z = cmk<V>(reinterpret_cast<const T *>(a.in)[ro + i], (T)0);
            else z = reinterpret_cast<const V *>(a.in)[ro + i];
            return mr ? cscale(z, mr[i]) : z;
        };
        V *Wb = reinterpret_cast<V *>(a.out) + (size_t)b * M * n;
        auto dst = [&](int o, V z) {
            if (valid) Wb[(size_t)o * n + j1] = z;
        };
        fft_fused<T, E, ED, false, TWS>(buf, a.P, twp, lt, a.tpt, src, dst);
        __syncthreads();
    }
}

template <typename T, int E, int ED, bool TWS, bool CG>
__global__ void WSC_LB(T, E) kf_c2c_cols(const PassArgs<T> a)
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
        const int k2q = k2 <= M / 2 ? k2 : M - k2;
        auto src = [&](int i) -> V { return (valid && i < n) ? col[i] : cmk<V>(0, 0); };
        auto mul = smem_hook([&](int o, V &x) {
            const int k1 = o <= M / 2 ? o : M - o;
            if (CG) x = cmul(x, __ldg(reinterpret_cast<const V *>(a.ghat) + (size_t)k2q * h + k1));
            else x = cscale(x, __ldg(reinterpret_cast<const T *>(a.ghat) + (size_t)k2q * h + k1));
        });
        fft_fused<T, E, ED, false, TWS>(buf, a.P, twp, lt, a.tpt, src, mul);
        auto dst = [&](int o, V x) {
            if (valid && o < n) col[o] = x;
        };
        fft_fused<T, E, ED, true, TWS>(buf, a.P, twp, lt, a.tpt, FromSmem{}, dst);
        __syncthreads();
    }
}

template <typename T, int E, int ED, bool TWS, bool IN_REAL>
__global__ void WSC_LB(T, E) kf_c2c_rows_inv(const PassArgs<T> a)
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
        auto src = [&](int i) -> V { return valid ? Wb[(size_t)i * n + j1] : cmk<V>(0, 0); };
        const size_t ro = (size_t)b * n * n + (size_t)j1 * n;
        V *o_ = reinterpret_cast<V *>(a.out) + ro;
        auto dst = [&](int o, V z) {
            if (!valid || o >= n) return;
            z = cmul(z, a.alpha);
            if (a.beta != (T)0) {
                if (IN_REAL) z.x += a.beta * reinterpret_cast<const T *>(a.u)[ro + o];
                else {
                    const V x = reinterpret_cast<const V *>(a.u)[ro + o];
                    z.x += a.beta * x.x;
                    z.y += a.beta * x.y;
                }
            }
            o_[o] = z;
        };
        fft_fused<T, E, ED, true, TWS>(buf, a.P, twp, lt, a.tpt, src, dst);
        __syncthreads();
    }
}

// ============================================================================ host glue
template <typename T, int E, int ED, bool TWS> conv_status set_attrs_fused(int smem)
{
#define WSC_ATTR(k) WSC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))
    WSC_ATTR((kf_r2r_rows_fwd<T, E, ED, TWS>));
    WSC_ATTR((kf_r2r_cols<T, E, ED, TWS>));
    WSC_ATTR((kf_r2r_rows_inv<T, E, ED, TWS>));
    WSC_ATTR((kf_c2c_rows_fwd<T, E, ED, TWS, true>));
    WSC_ATTR((kf_c2c_rows_fwd<T, E, ED, TWS, false>));
    WSC_ATTR((kf_c2c_cols<T, E, ED, TWS, true>));
    WSC_ATTR((kf_c2c_cols<T, E, ED, TWS, false>));
    WSC_ATTR((kf_c2c_rows_inv<T, E, ED, TWS, true>));
    WSC_ATTR((kf_c2c_rows_inv<T, E, ED, TWS, false>));
#undef WSC_ATTR
    return CONV_OK;
}

template <typename T, int E, int ED, bool TWS> int blocks_per_sm_fused(int threads, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kf_r2r_cols<T, E, ED, TWS>, threads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

template <typename T, int E, int ED, bool TWS>
conv_status run_fused(conv_plan_s *p, const void *u, const void *mask, void *out, int batch, double are,
                      double aim, double beta, void *ws, cudaStream_t st)
{
    typedef typename cvec<T>::t V;
    const int n = p->n, M = p->M, h = p->h;
    const double sc = 1.0 / ((double)M * (double)M);
    PassArgs<T> a;
    a.mask = reinterpret_cast<const T *>(mask);
    a.ghat = p->prec == CONV_P_FP64 ? (const void *)p->ghat64 : p->ghat32;
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
    const LaunchShape &R = p->rows, &C = p->cols, &I = p->inv;
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
        kf_r2r_rows_fwd<T, E, ED, TWS><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[1], st);
        a.tpt = C.tpt;
        a.in = ws;
        a.units = batch * h;
        kf_r2r_cols<T, E, ED, TWS><<<grid(C, a.units), C.tpt * C.groups, C.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[2], st);
        a.tpt = I.tpt;
        a.out = out;
        a.units = batch * ((n + 1) / 2);
        kf_r2r_rows_inv<T, E, ED, false><<<grid(I, a.units), I.tpt * I.groups, I.smem, st>>>(a);
    } else {
        const bool in_real = p->io == CONV_IO_R2C;
        a.tpt = R.tpt;
        a.in = u;
        a.out = ws;
        a.units = batch * n;
        if (in_real)
            kf_c2c_rows_fwd<T, E, ED, TWS, true><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
        else
            kf_c2c_rows_fwd<T, E, ED, TWS, false><<<grid(R, a.units), R.tpt * R.groups, R.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[1], st);
        a.tpt = C.tpt;
        a.in = ws;
        a.units = batch * M;
        if (p->complex_ghat)
            kf_c2c_cols<T, E, ED, TWS, true><<<grid(C, a.units), C.tpt * C.groups, C.smem, st>>>(a);
        else
            kf_c2c_cols<T, E, ED, TWS, false><<<grid(C, a.units), C.tpt * C.groups, C.smem, st>>>(a);
        if (ev) cudaEventRecord(ev[2], st);
        a.tpt = I.tpt;
        a.out = out;
        a.units = batch * n;
        if (in_real)
            kf_c2c_rows_inv<T, E, ED, false, true><<<grid(I, a.units), I.tpt * I.groups, I.smem, st>>>(a);
        else
            kf_c2c_rows_inv<T, E, ED, false, false><<<grid(I, a.units), I.tpt * I.groups, I.smem, st>>>(a);
    }
    if (ev) cudaEventRecord(ev[3], st);
    WSC_CUDA(cudaGetLastError());
    return CONV_OK;
}

}  // namespace wsc
