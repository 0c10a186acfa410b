// passes_fused.cuh -- the three convolution passes on the fused transform of fft_fused.cuh:
//   pass 1: stage 0 reads the (masked, zero-extended) rows from global memory;
//   pass 2: stage 0 reads the column from global memory, the forward transform's last stage
//           multiplies by ghat before its shared-memory store, and the inverse transform's last
//           stage writes the n surviving rows to global memory;
//   pass 3: stage 0 reads the (Hermitian-completed) spectrum from global memory and the last stage
//           writes the cropped, scaled result (plus beta u) to global memory.
// Same work decomposition, layouts and results as passes.cuh; fewer shared-memory sweeps.
#pragma once
#include <type_traits>

#include "async_copy.cuh"
#include "fft_static.cuh"
#include "passes.cuh"

namespace wsc {

#define WSC_LBF(T, E, ED) __launch_bounds__(maxt_fused<T, E, ED>::v, 1)

// The compile-time-length kernels run only for n = L/2 (ED = 1000 + log2 L) or n = L/3
// (ED = 2000 + log2(L/3)), as the host selects them: their forward transforms see the zero
// extension beyond n and their inverse transforms' outputs are cropped to the first n.
template <int ED> __device__ constexpr bool pruned() { return ED >= 1000; }

// ---------------------------------------------------------------------------- prefetch
// With a.pf set, each thread group fetches the input of its next work item (unit + stride) into
// its staging area as soon as stage 0 of the current item has read the staged input, so the
// load latency hides behind the rest of the item's transforms.  Contiguous inputs (a row pair of
// u, a row of a complex input, a column of W) move as one bulk copy on the group's mbarrier;
// strided ones (the spectrum of a row pair or row, one element per k) as cp.async pieces.

// A bounded wait gave up: record CONV_ETIMEOUT, wait (bounded again) for the copy still in flight
// into this group's staging area, and let the caller leave the kernel.
static __device__ __noinline__ void abandon(int *err, unsigned long long *bar, unsigned par, bool pending)
{
    if (threadIdx.x == 0 && err) atomicExch(err, (int)CONV_ETIMEOUT);
    if (pending) mbar_wait(bar, par);
}

// Top of a work item in a bulk-copy pass: wait for its staged input.  False (for every thread of
// the CTA) when some wait gave up.
template <typename T>
__device__ __forceinline__ bool await_bulk(const PassArgs<T> &a, unsigned long long *bar, unsigned &par,
                                           bool valid)
{
    // with a.give_up (an injected fault) the wait is not even polled: the CTA abandons its first
    // item, draining the copy it issued with the ordinary bounded wait
    const bool ok = !valid || (!a.give_up && mbar_wait(bar, par));
    if (__syncthreads_or(!ok)) {
        abandon(a.err, bar, par, !ok);
        return false;
    }
    if (valid) par ^= 1u;
    return true;
}

// One thread of the group starts the bulk copy of `bytes` from `src` into the staging area.
__device__ __forceinline__ void issue_bulk(void *stg, const void *src, unsigned bytes, unsigned long long *bar)
{
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bytes);
    bulk_g2s(stg, src, bytes, bar);
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(typename cvec<T>::t *dst, const typename cvec<T>::t *src)
{
    if constexpr (sizeof(T) == 4) cp_async8(dst, src);
    else cp_async16(dst, src);
}

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

// Pass 1.  Staging: rows j1, j1 + 1 of u (adjacent in memory), n T each; one bulk copy
// (a.pf requires n sizeof(T) to be a multiple of 16 and u 16-byte aligned).
template <typename T, int E, int ED, bool TWS, bool PP = false>
__global__ void WSC_LBF(T, E, ED) kf_r2r_rows_fwd(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    // PP: two buffers per group, the transform ping-pongs between them (fft_static.cuh)
    V *buf = setup_smem<T, TWS>(a, twp, PP ? 2 * g : g);
    V *buf2 = PP ? buf + padded_len<T>(a.M) : buf;
    unsigned long long *bar;
    T *stg = reinterpret_cast<T *>(stage_area<T, TWS, PP ? 2 : 1>(a, g, G, bar));
    const int n = a.n, M = a.M, h = a.h, pairs = (n + 1) / 2, stride = gridDim.x * G;
    const bool pair_vec = (n & 1) == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15) == 0;
    // TMA stores: the spectrum pairs (A_k, B_k) of the item, k < h, side by side in shared memory
    V *ost = reinterpret_cast<V *>(stg) + stage_in_len<T>(n, a.pf);
    constexpr int WPE = (int)(sizeof(V) / 8);  // 8-byte words per element
    auto fetch = [&](int unit) {
        if (!a.pf || lt != 0 || unit >= a.units) return;
        const int b = unit / pairs, j1 = 2 * (unit - b * pairs);
        const unsigned bytes = (unsigned)((j1 + 1 < n ? 2 : 1) * (size_t)n * sizeof(T));
        issue_bulk(stg, reinterpret_cast<const T *>(a.in) + (size_t)b * n * n + (size_t)j1 * n, bytes, bar);
    };
    unsigned par = 0;
    if (a.pf) {
        if (lt == 0) mbar_init(bar);
        __syncthreads();
        fetch(blockIdx.x * G + g);
    }
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf && !await_bulk(a, bar, par, valid)) return;
        const int b = valid ? unit / pairs : 0, j1 = valid ? 2 * (unit - b * pairs) : 0;
        const bool has2 = valid && j1 + 1 < n;
        const T *ua = reinterpret_cast<const T *>(a.in) + (size_t)b * n * n + (size_t)j1 * n;
        const T *ma = a.mask ? a.mask + (size_t)j1 * n : nullptr;
        auto src = [&](int i) -> V {
            if (!valid || i >= n) return cmk<V>(0, 0);
            T x, y;
            if (a.pf) {
                x = stg[i];
                y = has2 ? stg[n + i] : (T)0;
            } else {
                x = ua[i];
                y = has2 ? ua[n + i] : (T)0;
            }
            if (ma) {
                x *= ma[i];
                if (has2) y *= ma[n + i];
            }
            return cmk<V>(x, y);
        };
        fft_any2<T, E, ED, false, TWS, pruned<ED>(), false, PP>(buf, buf2, a.P, twp, a.tw, lt, a.tpt, src, ToSmem{},
                                                                [&]() { fetch(unit + stride); });
        const V *spec = (PP && final_in_b1<ED>()) ? buf2 : buf;  // the spectrum Z
        if (a.tma) {
            // the previous item's stores have to have read the pairs before they are rewritten
            if (lt == 0) bulk_wait_read();
            __syncthreads();
        }
        if (valid) {
            V *Wb = reinterpret_cast<V *>(a.out) + (size_t)b * h * n;
            for (int k = lt; k < h; k += a.tpt) {
                V Zk = spec[pidx<T>(k)], Zm = spec[pidx<T>(k == 0 ? 0 : M - k)];
                const V A = cmk<V>((T)0.5 * (Zk.x + Zm.x), (T)0.5 * (Zk.y - Zm.y));
                const V B = cmk<V>((T)0.5 * (Zk.y + Zm.y), (T)-0.5 * (Zk.x - Zm.x));
                if (a.tma) {
                    ost[2 * k] = A;
                    ost[2 * k + 1] = B;
                } else {
                    store_pair<T>(Wb + (size_t)k * n + j1, A, B, has2, pair_vec);
                }
            }
        }
        if (a.tma) {
            fence_proxy_async_smem();
            __syncthreads();
            if (lt == 0 && valid) {
                for (int i = 0; i < tma_boxes<T>(h); ++i)
                    tma_store_3d(&a.tmap, j1 * WPE, i * TMA_ROWS, b, ost + 2 * i * TMA_ROWS);
                bulk_commit();
            }
        }
        __syncthreads();
    }
    if (a.tma && lt == 0) bulk_wait_all();
}

// Pass 2.  Staging: the column's n spectrum values (contiguous in W); one bulk copy (a.pf
// requires n sizeof(V) to be a multiple of 16 and W 16-byte aligned).
template <typename T, int E, int ED, bool TWS, bool PP = false>
__global__ void WSC_LBF(T, E, ED) kf_r2r_cols(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    // PP: two buffers per group, the transforms ping-pong between them (fft_static.cuh)
    V *buf = setup_smem<T, TWS>(a, twp, PP ? 2 * g : g);
    V *buf2 = PP ? buf + padded_len<T>(a.M) : buf;
    unsigned long long *bar;
    V *stg = stage_area<T, TWS, PP ? 2 : 1>(a, g, G, bar);
    const int n = a.n, M = a.M, h = a.h, stride = gridDim.x * G;
    const T *ghat = reinterpret_cast<const T *>(a.ghat);
    // column k2 of density b: read from a.in, written to a.out (the same array but for
    // conv_apply_multi, whose plans read one shared pass-1 spectrum)
    auto col_off = [&](int unit) -> size_t {
        const int k2 = unit / a.batch, b = unit - k2 * a.batch;
        return (size_t)b * h * n + (size_t)k2 * n;
    };
    auto fetch = [&](int unit) {
        if (!a.pf || lt != 0 || unit >= a.units) return;
        issue_bulk(stg, reinterpret_cast<const V *>(a.in) + col_off(unit), (unsigned)((size_t)n * sizeof(V)), bar);
    };
    unsigned par = 0;
    if (a.pf) {
        if (lt == 0) mbar_init(bar);
        __syncthreads();
        fetch(blockIdx.x * G + g);
    }
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf && !await_bulk(a, bar, par, valid)) return;
        const int k2 = valid ? unit / a.batch : 0, bq = valid ? unit - k2 * a.batch : 0;
        const size_t co = col_off(valid ? unit : 0);
        const V *cin = reinterpret_cast<const V *>(a.in) + co;
        V *col = reinterpret_cast<V *>(a.out) + co;
        const T *gc = (a.nsel ? reinterpret_cast<const T *>(a.gsel[bq]) : ghat) + (size_t)k2 * h;
        auto src = [&](int i) -> V {
            if (!valid || i >= n) return cmk<V>(0, 0);
            return a.pf ? stg[i] : cin[i];
        };
        auto mul = smem_hook([&](int o, V &x) {
            const int Lm = pruned<ED>() ? static_len<ED>() : M, k1 = o <= Lm / 2 ? o : Lm - o;
            x = a.odd ? odd_mul(x, __ldg(&gc[k1]), o, Lm) : cscale(x, __ldg(&gc[k1]));
        });
        fft_any2<T, E, ED, false, TWS, pruned<ED>(), false, PP>(buf, buf2, a.P, twp, a.tw, lt, a.tpt, src, mul,
                                                                [&]() { fetch(unit + stride); });
        auto dst = [&](int o, V x) {
            if (valid && o < n) col[o] = x;
        };
        // the inverse starts from the buffer the forward transform ended in
        if (final_in_b1<ED>() && PP)
            fft_any2<T, E, ED, true, TWS, false, pruned<ED>(), PP>(buf2, buf, a.P, twp, a.tw, lt, a.tpt, FromSmem{}, dst);
        else
            fft_any2<T, E, ED, true, TWS, false, pruned<ED>(), PP>(buf, buf2, a.P, twp, a.tw, lt, a.tpt, FromSmem{}, dst);
        __syncthreads();
    }
}

// Pass 3.  Staging: the row pair's spectra W[k][j1], W[k][j1+1] for k <= M/2, side by side;
// gathered by cp.async (a.pf requires W 16-byte aligned and, in FP32, n even).
template <typename T, int E, int ED, bool TWS, bool PP = false>
__global__ void WSC_LBF(T, E, ED) kf_r2r_rows_inv(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, PP ? 2 * g : g);
    V *buf2 = PP ? buf + padded_len<T>(a.M) : buf;
    unsigned long long *bar;
    V *stg = stage_area<T, TWS, PP ? 2 : 1>(a, g, G, bar);
    const int n = a.n, M = a.M, h = a.h, pairs = (n + 1) / 2, stride = gridDim.x * G;
    const bool pair_vec = (n & 1) == 0 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0;
    const T alpha = a.alpha.x, beta = a.beta;
    constexpr int WPE = (int)(sizeof(V) / 8);
    auto gather = [&](int unit) {
        if (!a.pf || unit >= a.units) return;
        const int b = unit / pairs, j1 = 2 * (unit - b * pairs);
        if (a.tma) {  // TMA boxes of TMA_ROWS pairs; rows k >= h arrive as zeros
            if (lt == 0) {
                const int nb = tma_boxes<T>(h);
                fence_proxy_async_smem();
                mbar_expect_tx(bar, (unsigned)(nb * 2 * TMA_ROWS * sizeof(V)));
                for (int i = 0; i < nb; ++i) tma_load_3d(stg + 2 * i * TMA_ROWS, &a.tmap, j1 * WPE, i * TMA_ROWS, b, bar);
            }
            return;
        }
        const V *Wp = reinterpret_cast<const V *>(a.in) + (size_t)b * h * n + j1;
        const bool two = j1 + 1 < n;
        for (int k = lt; k < h; k += a.tpt) {
            cp_async16(stg + 2 * k, Wp + (size_t)k * n);  // FP32: both spectra (n even)
            if constexpr (sizeof(T) == 8) {
                if (two) cp_async16(stg + 2 * k + 1, Wp + (size_t)k * n + 1);
            }
        }
    };
    unsigned par = 0;
    if (a.pf && a.tma) {
        if (lt == 0) mbar_init(bar);
        __syncthreads();
    }
    gather(blockIdx.x * G + g);
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf) {
            if (a.tma) {
                if (!await_bulk(a, bar, par, valid)) return;
            } else {
                cp_async_wait_all();
                __syncthreads();
            }
        }
        const int b = valid ? unit / pairs : 0, j1 = valid ? 2 * (unit - b * pairs) : 0;
        const bool has2 = valid && j1 + 1 < n;
        const V *Wb = reinterpret_cast<const V *>(a.in) + (size_t)b * h * n;
        // Z_k = A_k + i B_k (k <= M/2), Z_k = conj A_{M-k} + i conj B_{M-k} (k > M/2)
        auto src = [&](int i) -> V {
            if (!valid) return cmk<V>(0, 0);
            const bool lo = i <= M / 2;
            const int k = lo ? i : M - i;
            V A, B;
            if (a.pf) {
                if constexpr (sizeof(T) == 4) {
                    const float4 q = reinterpret_cast<const float4 *>(stg)[k];
                    A = make_float2(q.x, q.y);
                    B = make_float2(q.z, q.w);
                } else {
                    A = stg[2 * k];
                    B = has2 ? stg[2 * k + 1] : cmk<V>(0, 0);
                }
            } else {
                load_pair<T>(Wb + (size_t)k * n + j1, A, B, has2, pair_vec);
            }
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
        fft_any2<T, E, ED, true, TWS, false, pruned<ED>(), PP>(buf, buf2, a.P, twp, a.tw, lt, a.tpt, src, dst,
                                                               [&]() { gather(unit + stride); });
        __syncthreads();
    }
    if (a.pf) cp_async_wait_all();
}

// ============================================================================ R2C, complex ghat
// Real densities with a complex, even multiplier (the Helmholtz kernel): A_n u = conv(u, g_r) +
// i conv(u, g_i) with g_r, g_i the real, even kernels of Re ghat and Im ghat.  Pass 1 is the R2R
// pass 1 (row-pair spectra W[k2][j1], k2 <= M/2); pass 2 transforms each column of W once and
// multiplies it by Re ghat and by Im ghat, giving column k2 of the half spectra of both real
// convolutions, stored side by side as W2[k2][j1] = (Wr, Wi); pass 3 packs Z_k = Wr_k + i Wi_k,
// completes it to k < M by Hermitian symmetry of each part, and one inverse row transform gives
// the complex output row conv(u, g_r) + i conv(u, g_i) directly.  2.25 M length-M transforms per
// density instead of the C2C pipeline's 3 M.

// Pass 2.  Two transform buffers per group: Re ghat's product transforms in the first, Im ghat's
// in the second.  Staging: the column of W (one bulk copy, as in the R2R pass 2).
template <typename T, int E, int ED, bool TWS, bool ONE = false>
__global__ void WSC_LBF(T, E, ED) kf_r2c_cols(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    // ONE: a single buffer per group (two lines do not fit, FP64 at L = 8192); the Im-ghat
    // spectrum waits in the group's global scratch line, in L2, while the Re part is inverted
    V *bre = setup_smem<T, TWS>(a, twp, ONE ? g : 2 * g);
    V *bim = ONE ? nullptr : bre + padded_len<T>(a.M);
    V *tmp = ONE ? reinterpret_cast<V *>(a.scratch) + ((size_t)blockIdx.x * G + g) * a.M : nullptr;
    unsigned long long *bar;
    V *stg = stage_area<T, TWS, ONE ? 1 : 2>(a, g, G, bar);
    const int n = a.n, M = a.M, h = a.h, stride = gridDim.x * G;
    const V *cg = reinterpret_cast<const V *>(a.ghat);
    auto col_off = [&](int unit) -> size_t {
        const int k2 = unit / a.batch, b = unit - k2 * a.batch;
        return (size_t)b * h * n + (size_t)k2 * n;
    };
    auto fetch = [&](int unit) {
        if (!a.pf || lt != 0 || unit >= a.units) return;
        issue_bulk(stg, reinterpret_cast<const V *>(a.in) + col_off(unit), (unsigned)((size_t)n * sizeof(V)), bar);
    };
    unsigned par = 0;
    if (a.pf) {
        if (lt == 0) mbar_init(bar);
        __syncthreads();
        fetch(blockIdx.x * G + g);
    }
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf && !await_bulk(a, bar, par, valid)) return;
        const int k2 = valid ? unit / a.batch : 0, bq = valid ? unit - k2 * a.batch : 0;
        const size_t co = col_off(valid ? unit : 0);
        const V *cin = reinterpret_cast<const V *>(a.in) + co;
        auto src = [&](int i) -> V {
            if (!valid || i >= n) return cmk<V>(0, 0);
            return a.pf ? stg[i] : cin[i];
        };
        const V *gc = (a.nsel ? reinterpret_cast<const V *>(a.gsel[bq]) : cg) + (size_t)k2 * h;
        auto mul = smem_hook([&](int o, V &x) {
            const int Lm = pruned<ED>() ? static_len<ED>() : M, k1 = o <= Lm / 2 ? o : Lm - o;
            const V gk = __ldg(&gc[k1]);
            if constexpr (ONE) tmp[o] = cscale(x, gk.y);
            else bim[pidx<T>(o)] = cscale(x, gk.y);
            x = cscale(x, gk.x);
        });
        fft_any<T, E, ED, false, TWS, pruned<ED>(), false>(bre, a.P, twp, a.tw, lt, a.tpt, src, mul, [&]() { fetch(unit + stride); });
        V *cout = reinterpret_cast<V *>(a.out) + 2 * co;
        if constexpr (ONE) {
            // Wr straight to the output pairs' first halves; then Wi from the scratch line (its
            // stores by the whole group are visible after the barriers of the first inverse)
            auto dst_r = [&](int o, V xr) {
                if (valid && o < n) cout[2 * o] = xr;
            };
            fft_any<T, E, ED, true, TWS, false, pruned<ED>()>(bre, a.P, twp, a.tw, lt, a.tpt, FromSmem{}, dst_r);
            __syncthreads();
            auto src_i = [&](int i) -> V { return tmp[i]; };
            auto dst_i = [&](int o, V xi) {
                if (valid && o < n) cout[2 * o + 1] = xi;
            };
            fft_any<T, E, ED, true, TWS, false, pruned<ED>()>(bre, a.P, twp, a.tw, lt, a.tpt, src_i, dst_i);
            __syncthreads();
            continue;
        }
        fft_any<T, E, ED, true, TWS, false, pruned<ED>()>(bre, a.P, twp, a.tw, lt, a.tpt, FromSmem{}, ToSmem{});
        auto dst = [&](int o, V xi) {
            if (!valid || o >= n) return;
            const V xr = bre[pidx<T>(o)];
            if constexpr (sizeof(T) == 4) {
                if (a.vec) {
                    *reinterpret_cast<float4 *>(cout + 2 * o) = make_float4(xr.x, xr.y, xi.x, xi.y);
                    return;
                }
            }
            cout[2 * o] = xr;
            cout[2 * o + 1] = xi;
        };
        fft_any<T, E, ED, true, TWS, false, pruned<ED>()>(bim, a.P, twp, a.tw, lt, a.tpt, FromSmem{}, dst);
        __syncthreads();
    }
}

// Pass 3.  Staging: the row's pairs W2[k][j1] = (Wr, Wi), k <= M/2, gathered by cp.async
// (16-byte pieces; a.pf requires W2 16-byte aligned).
template <typename T, int E, int ED, bool TWS>
__global__ void WSC_LBF(T, E, ED) kf_r2c_rows_inv(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    unsigned long long *bar;
    V *stg = stage_area<T, TWS>(a, g, G, bar);
    const int n = a.n, M = a.M, h = a.h, stride = gridDim.x * G;
    constexpr int WPE = (int)(sizeof(V) / 8);
    auto gather = [&](int unit) {
        if (!a.pf || unit >= a.units) return;
        const int b = unit / n, j1 = unit - b * n;
        if (a.tma) {  // TMA boxes of TMA_ROWS (Wr, Wi) pairs; rows k >= h arrive as zeros
            if (lt == 0) {
                const int nb = tma_boxes<T>(h);
                fence_proxy_async_smem();
                mbar_expect_tx(bar, (unsigned)(nb * 2 * TMA_ROWS * sizeof(V)));
                for (int i = 0; i < nb; ++i)
                    tma_load_3d(stg + 2 * i * TMA_ROWS, &a.tmap, 2 * j1 * WPE, i * TMA_ROWS, b, bar);
            }
            return;
        }
        const V *Wp = reinterpret_cast<const V *>(a.in) + 2 * ((size_t)b * h * n + j1);
        for (int k = lt; k < h; k += a.tpt) {
            cp_async16(stg + 2 * k, Wp + 2 * (size_t)k * n);
            if constexpr (sizeof(T) == 8) cp_async16(stg + 2 * k + 1, Wp + 2 * (size_t)k * n + 1);
        }
    };
    unsigned par = 0;
    if (a.pf && a.tma) {
        if (lt == 0) mbar_init(bar);
        __syncthreads();
    }
    gather(blockIdx.x * G + g);
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf) {
            if (a.tma) {
                if (!await_bulk(a, bar, par, valid)) return;
            } else {
                cp_async_wait_all();
                __syncthreads();
            }
        }
        const int b = valid ? unit / n : 0, j1 = valid ? unit - b * n : 0;
        const V *Wb = reinterpret_cast<const V *>(a.in) + 2 * ((size_t)b * h * n + j1);
        // Z_k = Wr_k + i Wi_k (k <= M/2), Z_k = conj Wr_{M-k} + i conj Wi_{M-k} (k > M/2)
        auto src = [&](int i) -> V {
            if (!valid) return cmk<V>(0, 0);
            const bool lo = i <= M / 2;
            const int k = lo ? i : M - i;
            V A, B;
            if (a.pf) {
                A = stg[2 * k];
                B = stg[2 * k + 1];
            } else {
                A = Wb[2 * (size_t)k * n];
                B = Wb[2 * (size_t)k * n + 1];
            }
            return lo ? cmk<V>(A.x - B.y, A.y + B.x) : cmk<V>(A.x + B.y, B.x - A.y);
        };
        const size_t ro = (size_t)b * n * n + (size_t)j1 * n;
        V *o_ = reinterpret_cast<V *>(a.out) + ro;
        const T *ua = reinterpret_cast<const T *>(a.u) + ro;
        auto dst = [&](int o, V z) {
            if (!valid || o >= n) return;
            z = cmul(z, a.alpha);
            if (a.beta != (T)0) z.x += a.beta * ua[o];
            o_[o] = z;
        };
        fft_any<T, E, ED, true, TWS, false, pruned<ED>()>(buf, a.P, twp, a.tw, lt, a.tpt, src, dst, [&]() { gather(unit + stride); });
        __syncthreads();
    }
    if (a.pf) cp_async_wait_all();
}

// ============================================================================ C2C
// Pass 1.  Staging: row j1 of the input (n T real or n V complex); one bulk copy (a.pf requires
// its byte length to be a multiple of 16 and the input 16-byte aligned).
template <typename T, int E, int ED, bool TWS, bool IN_REAL>
__global__ void WSC_LBF(T, E, ED) kf_c2c_rows_fwd(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    typedef typename std::conditional<IN_REAL, T, V>::type I;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    unsigned long long *bar;
    I *stg = reinterpret_cast<I *>(stage_area<T, TWS>(a, g, G, bar));
    const int n = a.n, M = a.M, stride = gridDim.x * G;
    const I *in = reinterpret_cast<const I *>(a.in);
    auto fetch = [&](int unit) {
        if (!a.pf || lt != 0 || unit >= a.units) return;
        const int b = unit / n, j1 = unit - b * n;
        issue_bulk(stg, in + (size_t)b * n * n + (size_t)j1 * n, (unsigned)((size_t)n * sizeof(I)), bar);
    };
    unsigned par = 0;
    if (a.pf) {
        if (lt == 0) mbar_init(bar);
        __syncthreads();
        fetch(blockIdx.x * G + g);
    }
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf && !await_bulk(a, bar, par, valid)) return;
        const int b = valid ? unit / n : 0, j1 = valid ? unit - b * n : 0;
        const size_t ro = (size_t)b * n * n + (size_t)j1 * n;
        const T *mr = a.mask ? a.mask + (size_t)j1 * n : nullptr;
        auto src = [&](int i) -> V {
            if (!valid || i >= n) return cmk<V>(0, 0);
            const I x = a.pf ? stg[i] : in[ro + i];
            V z;
            if constexpr (IN_REAL) z = cmk<V>(x, (T)0);
            else z = x;
            return mr ? cscale(z, mr[i]) : z;
        };
        V *Wb = reinterpret_cast<V *>(a.out) + (size_t)b * M * n;
        auto dst = [&](int o, V z) {
            if (valid) Wb[(size_t)o * n + j1] = z;
        };
        fft_any<T, E, ED, false, TWS, pruned<ED>(), false>(buf, a.P, twp, a.tw, lt, a.tpt, src, dst, [&]() { fetch(unit + stride); });
        __syncthreads();
    }
}

// Pass 2.  Staging: the column's n spectrum values; one bulk copy (as in the R2R pass 2).
template <typename T, int E, int ED, bool TWS, bool CG>
__global__ void WSC_LBF(T, E, ED) kf_c2c_cols(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    unsigned long long *bar;
    V *stg = stage_area<T, TWS>(a, g, G, bar);
    const int n = a.n, M = a.M, h = a.h, stride = gridDim.x * G;
    auto col_at = [&](int unit) -> V * {
        const int k2 = unit / a.batch, b = unit - k2 * a.batch;
        return reinterpret_cast<V *>(a.out) + (size_t)b * M * n + (size_t)k2 * n;
    };
    auto fetch = [&](int unit) {
        if (!a.pf || lt != 0 || unit >= a.units) return;
        issue_bulk(stg, col_at(unit), (unsigned)((size_t)n * sizeof(V)), bar);
    };
    unsigned par = 0;
    if (a.pf) {
        if (lt == 0) mbar_init(bar);
        __syncthreads();
        fetch(blockIdx.x * G + g);
    }
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf && !await_bulk(a, bar, par, valid)) return;
        const int k2 = valid ? unit / a.batch : 0, bq = valid ? unit - k2 * a.batch : 0;
        V *col = col_at(valid ? unit : 0);
        const int k2q = k2 <= M / 2 ? k2 : M - k2;
        const void *gq = mult_of(a, bq);
        auto src = [&](int i) -> V {
            if (!valid || i >= n) return cmk<V>(0, 0);
            return a.pf ? stg[i] : col[i];
        };
        auto mul = smem_hook([&](int o, V &x) {
            const int Lm = pruned<ED>() ? static_len<ED>() : M, k1 = o <= Lm / 2 ? o : Lm - o;
            if (CG) x = cmul(x, __ldg(reinterpret_cast<const V *>(gq) + (size_t)k2q * h + k1));
            else x = cscale(x, __ldg(reinterpret_cast<const T *>(gq) + (size_t)k2q * h + k1));
        });
        fft_any<T, E, ED, false, TWS, pruned<ED>(), false>(buf, a.P, twp, a.tw, lt, a.tpt, src, mul, [&]() { fetch(unit + stride); });
        auto dst = [&](int o, V x) {
            if (valid && o < n) col[o] = x;
        };
        fft_any<T, E, ED, true, TWS, false, pruned<ED>()>(buf, a.P, twp, a.tw, lt, a.tpt, FromSmem{}, dst);
        __syncthreads();
    }
}

// Pass 3.  Staging: the row's spectrum W[i][j1], i < M, one element per i; gathered by cp.async
// (8-byte pieces in FP32, 16-byte in FP64; a.pf requires W aligned to the element size).
template <typename T, int E, int ED, bool TWS, bool IN_REAL>
__global__ void WSC_LBF(T, E, ED) kf_c2c_rows_inv(const __grid_constant__ PassArgs<T> a)
{
    typedef typename cvec<T>::t V;
    const int g = threadIdx.x / a.tpt, lt = threadIdx.x - g * a.tpt, G = blockDim.x / a.tpt;
    const V *twp;
    V *buf = setup_smem<T, TWS>(a, twp, g);
    unsigned long long *bar;
    V *stg = stage_area<T, TWS>(a, g, G, bar);
    const int n = a.n, M = a.M, stride = gridDim.x * G;
    auto gather = [&](int unit) {
        if (!a.pf || unit >= a.units) return;
        const int b = unit / n, j1 = unit - b * n;
        const V *Wp = reinterpret_cast<const V *>(a.in) + (size_t)b * M * n + j1;
        for (int i = lt; i < M; i += a.tpt) cp_async_elem<T>(stg + i, Wp + (size_t)i * n);
    };
    gather(blockIdx.x * G + g);
    for (int base = blockIdx.x * G; base < a.units; base += stride) {
        const int unit = base + g;
        const bool valid = unit < a.units;
        if (a.pf) {
            cp_async_wait_all();
            __syncthreads();
        }
        const int b = valid ? unit / n : 0, j1 = valid ? unit - b * n : 0;
        const V *Wb = reinterpret_cast<const V *>(a.in) + (size_t)b * M * n;
        auto src = [&](int i) -> V {
            if (!valid) return cmk<V>(0, 0);
            return a.pf ? stg[i] : Wb[(size_t)i * n + j1];
        };
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
        fft_any<T, E, ED, true, TWS, false, pruned<ED>()>(buf, a.P, twp, a.tw, lt, a.tpt, src, dst, [&]() { gather(unit + stride); });
        __syncthreads();
    }
    if (a.pf) cp_async_wait_all();
}

// ============================================================================ host glue
template <typename T, int E, int ED, bool TWS> conv_status set_attrs_fused(int smem)
{
#define WSC_ATTR(k) WSC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))
    WSC_ATTR((kf_r2r_rows_fwd<T, E, ED, TWS>));
    WSC_ATTR((kf_r2r_cols<T, E, ED, TWS>));
    WSC_ATTR((kf_r2r_rows_inv<T, E, ED, TWS>));
    if constexpr (pingpong_ok<T, ED>()) {
        WSC_ATTR((kf_r2r_rows_fwd<T, E, ED, TWS, true>));
        WSC_ATTR((kf_r2r_cols<T, E, ED, TWS, true>));
        WSC_ATTR((kf_r2r_rows_inv<T, E, ED, TWS, true>));
    }
    WSC_ATTR((kf_r2c_cols<T, E, ED, TWS>));
    if constexpr (split_one_ed(ED)) WSC_ATTR((kf_r2c_cols<T, E, ED, TWS, true>));
    WSC_ATTR((kf_r2c_rows_inv<T, E, ED, TWS>));
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

template <typename T, int E, int ED>
conv_status run_fused(conv_plan_s *p, const void *u, const void *mask, void *out, int batch, double are,
                      double aim, double beta, void *ws, cudaStream_t st)
{
    typedef typename cvec<T>::t V;
    const int n = p->n, M = p->M, h = p->h;
    const double sc = 1.0 / ((double)M * (double)M);
    PassArgs<T> a{};
    a.err = p->dev_err;
    a.give_up = fault_take(CONV_FAULT_WAIT) ? 1 : 0;
    a.nsel = p->nsel;
    for (int i = 0; i < p->nsel; ++i) a.gsel[i] = p->sel[i];
    a.odd = p->kern.family == CONV_K_DX1LOG ? 1 : 0;
    a.mask = reinterpret_cast<const T *>(mask);
    a.ghat = p->prec == CONV_P_FP64 ? (const void *)p->ghat64 : p->ghat32;
    a.u = u;
    a.tw = reinterpret_cast<const V *>(p->tw);
    a.tw_len = tw_split_ok<T, ED>() ? p->fft.toff[p->fft.nst - 1] : p->fft.tw_len;  // the shared-memory copy
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
    // prefetch needs the staged runs to start on 16 bytes (bulk copies, 16-byte cp.async) or on
    // their element size (8-byte cp.async), and bulk copy lengths that are multiples of 16
    auto al = [](const void *q, size_t m) { return (reinterpret_cast<uintptr_t>(q) % m) == 0; };
    const bool ws16 = al(ws, 16);
    const bool pf_cols = C.pf && ws16 && (n * sizeof(V)) % 16 == 0;
    // TMA over the spectrum pairs: W (pass 1 stores; R2R pass 3 loads) or W2 (split pass 3 loads),
    // n (or 2n) elements of sizeof(V) / 8 words per k2 row, h rows, `batch` densities
    constexpr unsigned WPE = (unsigned)(sizeof(V) / 8);
    auto tma_map = [&](const LaunchShape &S, const void *base, unsigned long long elems_per_row) {
        a.tma = S.tma && encode_rows_map(&a.tmap, base, elems_per_row * WPE, (unsigned long long)h,
                                         (unsigned long long)batch, 2 * WPE);
    };
    // one launch of kernel K<T, E, ED, tws[, X]> in shape S, with S's twiddle option
#define WSC_TARGS(T_, E_, ED_) T_, E_, ED_
#define WSC_LAUNCH(S, K, TA)                                                                   \
    do {                                                                                      \
        if ((S).tws) K<WSC_TARGS TA, true><<<grid(S, a.units), (S).tpt * (S).groups, (S).smem, st>>>(a);  \
        else K<WSC_TARGS TA, false><<<grid(S, a.units), (S).tpt * (S).groups, (S).smem, st>>>(a);      \
    } while (0)
#define WSC_LAUNCH2(S, K, TA, X)                                                                  \
    do {                                                                                         \
        if ((S).tws) K<WSC_TARGS TA, true, X><<<grid(S, a.units), (S).tpt * (S).groups, (S).smem, st>>>(a); \
        else K<WSC_TARGS TA, false, X><<<grid(S, a.units), (S).tpt * (S).groups, (S).smem, st>>>(a);     \
    } while (0)
    // kernels with a ping-pong variant: launched with it when the pass's shape holds two buffers
#define WSC_LAUNCH_PP(S, K)                                      \
    do {                                                         \
        if constexpr (pingpong_ok<T, ED>()) {                    \
            if ((S).pp) WSC_LAUNCH2(S, K, (T, E, ED), true);     \
            else WSC_LAUNCH(S, K, (T, E, ED));                   \
        } else {                                                 \
            WSC_LAUNCH(S, K, (T, E, ED));                        \
        }                                                        \
    } while (0)
    cudaEvent_t *ev = timing_slot(p);
    if (ev) cudaEventRecord(ev[0], st);
    // p->run_passes: the passes this launch runs (conv_apply_multi runs pass 1 once for several
    // plans, then passes 2 and 3 of each from the shared spectrum p->w_in)
    const int run = p->run_passes;
    if (p->io == CONV_IO_R2R) {
        a.tpt = R.tpt;
        a.in = u;
        a.out = ws;
        a.units = batch * ((n + 1) / 2);
        a.stage_len = R.stage;
        a.pf = R.pf && al(u, 16) && (n * sizeof(T)) % 16 == 0;
        tma_map(R, ws, n);
        if (run & 1) WSC_LAUNCH_PP(R, kf_r2r_rows_fwd);
        if (ev) cudaEventRecord(ev[1], st);
        a.tpt = C.tpt;
        a.in = p->w_in ? p->w_in : ws;
        a.out = ws;
        a.units = batch * h;
        a.stage_len = C.stage;
        a.pf = pf_cols && al(a.in, 16);
        a.tma = 0;
        if (run & 2) WSC_LAUNCH_PP(C, kf_r2r_cols);
        if (ev) cudaEventRecord(ev[2], st);
        if (!(run & 4)) goto launched;
        a.in = ws;
        a.tpt = I.tpt;
        a.out = out;
        a.units = batch * ((n + 1) / 2);
        a.stage_len = I.stage;
        a.pf = I.pf && ws16 && (sizeof(T) == 8 || n % 2 == 0);
        if (a.pf) tma_map(I, ws, n);
        else a.tma = 0;
        WSC_LAUNCH_PP(I, kf_r2r_rows_inv);
    } else if (p->r2c_split) {
        a.tpt = R.tpt;
        a.in = u;
        a.out = ws;
        a.units = batch * ((n + 1) / 2);
        a.stage_len = R.stage;
        a.pf = R.pf && al(u, 16) && (n * sizeof(T)) % 16 == 0;
        tma_map(R, ws, n);
        if (run & 1) WSC_LAUNCH_PP(R, kf_r2r_rows_fwd);
        if (ev) cudaEventRecord(ev[1], st);
        // W2 follows W on the next even element (the workspace holds batch (3 h n + 1) values)
        V *W2 = reinterpret_cast<V *>(ws) + (((size_t)batch * h * n + 1) & ~(size_t)1);
        a.tpt = C.tpt;
        a.in = p->w_in ? p->w_in : ws;
        a.out = W2;
        a.units = batch * h;
        a.stage_len = C.stage;
        a.pf = pf_cols && al(a.in, 16);
        a.tma = 0;
        a.vec = al(W2, 16);
        if constexpr (split_one_ed(ED)) {
            // one buffer per group: the scratch lines follow W2 (batch (3 h n + 1) values in all)
            a.scratch = reinterpret_cast<V *>(ws) + (((size_t)batch * (3 * (size_t)h * n + 1) + 1) & ~(size_t)1);
            if (run & 2) {
                if (C.one) WSC_LAUNCH2(C, kf_r2c_cols, (T, E, ED), true);
                else WSC_LAUNCH(C, kf_r2c_cols, (T, E, ED));
            }
        } else {
            if (run & 2) WSC_LAUNCH(C, kf_r2c_cols, (T, E, ED));
        }
        if (ev) cudaEventRecord(ev[2], st);
        if (!(run & 4)) goto launched;
        a.tpt = I.tpt;
        a.in = W2;
        a.out = out;
        a.units = batch * n;
        a.stage_len = I.stage;
        a.pf = I.pf && al(W2, 16);
        if (a.pf) tma_map(I, W2, 2 * (unsigned long long)n);
        else a.tma = 0;
        WSC_LAUNCH(I, kf_r2c_rows_inv, (T, E, ED));
    } else {
        const bool in_real = p->io == CONV_IO_R2C;
        a.tpt = R.tpt;
        a.in = u;
        a.out = ws;
        a.units = batch * n;
        a.stage_len = R.stage;
        a.pf = R.pf && al(u, 16) && (n * (in_real ? sizeof(T) : sizeof(V))) % 16 == 0;
        a.tma = 0;
        if (in_real)
            WSC_LAUNCH2(R, kf_c2c_rows_fwd, (T, E, ED), true);
        else
            WSC_LAUNCH2(R, kf_c2c_rows_fwd, (T, E, ED), false);
        if (ev) cudaEventRecord(ev[1], st);
        a.tpt = C.tpt;
        a.in = ws;
        a.units = batch * M;
        a.stage_len = C.stage;
        a.pf = pf_cols;
        if (p->complex_ghat)
            WSC_LAUNCH2(C, kf_c2c_cols, (T, E, ED), true);
        else
            WSC_LAUNCH2(C, kf_c2c_cols, (T, E, ED), false);
        if (ev) cudaEventRecord(ev[2], st);
        a.tpt = I.tpt;
        a.out = out;
        a.units = batch * n;
        a.stage_len = I.stage;
        a.pf = I.pf && al(ws, sizeof(V));
        a.tma = 0;
        if (in_real)
            WSC_LAUNCH2(I, kf_c2c_rows_inv, (T, E, ED), true);
        else
            WSC_LAUNCH2(I, kf_c2c_rows_inv, (T, E, ED), false);
    }
launched:
    if (ev) cudaEventRecord(ev[3], st);
#undef WSC_LAUNCH_PP
#undef WSC_LAUNCH2
#undef WSC_LAUNCH
#undef WSC_TARGS
    WSC_CUDA(cudaGetLastError());
    return CONV_OK;
}

}  // namespace wsc
