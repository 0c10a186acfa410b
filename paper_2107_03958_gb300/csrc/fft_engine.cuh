// fft_engine.cuh -- shared-memory Stockham FFT used by the three convolution passes.
//
// A CTA holds G independent length-L transforms in shared memory, each worked on by `tpt`
// threads.  Every radix-R stage (R in {2,3,4,5,8}) is the self-sorting Stockham step
//   y[(j / Ns) Ns R + (j mod Ns) + p Ns] = sum_q w^{pq}_R  t_q x[j + q L/R],
//   t_q = exp(-/+ 2 pi i q (j mod Ns) / (Ns R)),  j in [0, L/R),
// so the result comes out in natural order.  A stage reads its R inputs into registers, meets a
// barrier, then writes its R outputs, so one buffer suffices.  Shared memory is padded by one
// element per 128 bytes, which makes both the unit-stride reads and the stride-Ns writes
// bank-conflict free for Ns = 1 and Ns >= 32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wsc {

template <typename T> struct cvec;
template <> struct cvec<float> { typedef float2 t; };
template <> struct cvec<double> { typedef double2 t; };

template <typename V> __host__ __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return cmk<V>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V rot(V x) { return INV ? cmk<V>(-x.y, x.x) : cmk<V>(x.y, -x.x); }

// padding: one element per 128 bytes
template <typename T> struct pad_shift;
template <> struct pad_shift<float> { static const int v = 4; };   // 16 x 8 B
template <> struct pad_shift<double> { static const int v = 3; };  // 8 x 16 B
template <typename T> __device__ __forceinline__ int pidx(int e) { return e + (e >> pad_shift<T>::v); }
template <typename T> __host__ __device__ inline int padded_len(int L) { return L + (L >> (sizeof(T) == 4 ? 4 : 3)) + 1; }

#define WSC_MAX_STAGES 24

// Per-length stage table (device memory).  Twiddle table: for each stage s a block of 3 Ns entries,
// [w^k | w^{2k} | w^{4k}], k < Ns, w = exp(-2 pi i / (Ns R)), so that consecutive threads (consecutive
// k) read consecutive entries.
struct FFTDesc {
    int L;
    int nst;
    int R[WSC_MAX_STAGES];
    int Ns[WSC_MAX_STAGES];
    int tws[WSC_MAX_STAGES];                  // L / (Ns R)
    int toff[WSC_MAX_STAGES];                 // offset of stage s's twiddle block in the table
    int tw_len;                               // complex entries of the whole table
    int tw_full16;                            // radix-16 stages hold all fifteen powers (FP64)
    unsigned long long mag[WSC_MAX_STAGES];  // ceil(2^40 / Ns): j / Ns == (j * mag) >> 40 for j < 2^24, Ns < 2^16
};

// Compile-time lengths whose shared-memory twiddle table holds every stage's blocks but the last
// stage's: FP64 L = 2^13, whose full table (131 KB) does not fit beside the 139 KB line; the last,
// radix-2 stage (one power per butterfly) reads the global table.
__host__ __device__ constexpr bool tw_split_ed(int ed, int elem_bytes) { return elem_bytes == 8 && ed == 1013; }
template <typename T, int ED> __host__ __device__ constexpr bool tw_split_ok() { return tw_split_ed(ED, (int)sizeof(T)); }
// Compile-time lengths whose split R2C column pass may run with one buffer per CTA: those of the
// 512-thread kernels (at L = 2^14, 1024 threads of 64 registers, that kernel spills 600 B).
__host__ __device__ constexpr bool split_one_ed(int ed) { return ed >= 1000 && ed != 1014; }

// ---------------------------------------------------------------- small DFTs
template <bool INV, typename V> __device__ __forceinline__ void dft2(V *x) {
    V a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
}

template <bool INV, typename V> __device__ __forceinline__ void dft3(V *x) {
    typedef decltype(V::x) T;
    const T h = (T)0.8660254037844386467637231707529362;  // sin(2 pi / 3)
    V t = cadd(x[1], x[2]);
    V d = csub(x[1], x[2]);
    V y0 = cadd(x[0], t);
    V m = cmk<V>(x[0].x - (T)0.5 * t.x, x[0].y - (T)0.5 * t.y);
    V r = cscale(rot<INV>(d), h);
    x[0] = y0;
    x[1] = cadd(m, r);
    x[2] = csub(m, r);
}

template <bool INV, typename V> __device__ __forceinline__ void dft4(V *x) {
    V a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
    V a2 = cadd(x[1], x[3]), a3 = rot<INV>(csub(x[1], x[3]));
    x[0] = cadd(a0, a2);
    x[2] = csub(a0, a2);
    x[1] = cadd(a1, a3);
    x[3] = csub(a1, a3);
}

template <bool INV, typename V> __device__ __forceinline__ void dft5(V *x) {
    typedef decltype(V::x) T;
    const T c1 = (T)0.3090169943749474241022934171828191;   // cos(2 pi/5)
    const T c2 = (T)-0.8090169943749474241022934171828191;  // cos(4 pi/5)
    const T s1 = (T)0.9510565162951535721164393333793821;   // sin(2 pi/5)
    const T s2 = (T)0.5877852522924731291687059546390728;   // sin(4 pi/5)
    V t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
    V d1 = csub(x[1], x[4]), d2 = csub(x[2], x[3]);
    V y0 = cadd(x[0], cadd(t1, t2));
    V a1 = cmk<V>(x[0].x + c1 * t1.x + c2 * t2.x, x[0].y + c1 * t1.y + c2 * t2.y);
    V a2 = cmk<V>(x[0].x + c2 * t1.x + c1 * t2.x, x[0].y + c2 * t1.y + c1 * t2.y);
    V b1 = cmk<V>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
    V b2 = cmk<V>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
    V r1 = rot<INV>(b1), r2 = rot<INV>(b2);
    x[0] = y0;
    x[1] = cadd(a1, r1);
    x[4] = csub(a1, r1);
    x[2] = cadd(a2, r2);
    x[3] = csub(a2, r2);
}

template <bool INV, typename V> __device__ __forceinline__ void dft8(V *x) {
    typedef decltype(V::x) T;
    const T r2 = (T)0.7071067811865475244008443621048490;
    V e[4] = {x[0], x[2], x[4], x[6]};
    V o[4] = {x[1], x[3], x[5], x[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    // o[k] *= w8^{k} (forward w8 = e^{-i pi/4}; inverse conjugate)
    V o1 = INV ? cmk<V>((o[1].x - o[1].y) * r2, (o[1].x + o[1].y) * r2)
               : cmk<V>((o[1].x + o[1].y) * r2, (o[1].y - o[1].x) * r2);
    V o2 = rot<INV>(o[2]);
    V o3 = INV ? cmk<V>((-o[3].x - o[3].y) * r2, (o[3].x - o[3].y) * r2)
               : cmk<V>((o[3].y - o[3].x) * r2, (-o[3].x - o[3].y) * r2);
    x[0] = cadd(e[0], o[0]);
    x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[5] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], o3);
    x[7] = csub(e[3], o3);
}

// x w8^1 and x w8^3 (forward w8 = e^{-i pi/4}; inverse conjugate)
template <bool INV, typename V> __device__ __forceinline__ V w8_1(V x)
{
    typedef decltype(V::x) T;
    const T r2 = (T)0.7071067811865475244008443621048490;
    return INV ? cmk<V>((x.x - x.y) * r2, (x.x + x.y) * r2) : cmk<V>((x.x + x.y) * r2, (x.y - x.x) * r2);
}
template <bool INV, typename V> __device__ __forceinline__ V w8_3(V x)
{
    typedef decltype(V::x) T;
    const T r2 = (T)0.7071067811865475244008443621048490;
    return INV ? cmk<V>((-x.x - x.y) * r2, (x.x - x.y) * r2) : cmk<V>((x.y - x.x) * r2, (-x.x - x.y) * r2);
}

// Radix-8 DFT of x0, x1, x2 with x3 ... x7 zero (the first stage of a length-3m transform whose
// inputs beyond m are the zero extension): X_p = x0 + w^p x1 + w^2p x2.  The terms x0 + w^2p x2
// repeat with period 4 and w^(p+4) = -w^p, so X_p and X_(p+4) share them.
template <bool INV, typename V> __device__ __forceinline__ void dft8_in3(V *x)
{
    const V a = x[0], b = x[1], c = x[2], rc = rot<INV>(c);
    const V e0 = cadd(a, c), e1 = cadd(a, rc), e2 = csub(a, c), e3 = csub(a, rc);
    const V o1 = w8_1<INV>(b), o2 = rot<INV>(b), o3 = w8_3<INV>(b);
    x[0] = cadd(e0, b);
    x[4] = csub(e0, b);
    x[1] = cadd(e1, o1);
    x[5] = csub(e1, o1);
    x[2] = cadd(e2, o2);
    x[6] = csub(e2, o2);
    x[3] = cadd(e3, o3);
    x[7] = csub(e3, o3);
}

// Radix-8 DFT of x0, x1 with x2 ... x7 zero: X_p = x0 + w^p x1, X_(p+4) = x0 - w^p x1.
template <bool INV, typename V> __device__ __forceinline__ void dft8_in2(V *x)
{
    const V a = x[0], b = x[1];
    const V o1 = w8_1<INV>(b), o2 = rot<INV>(b), o3 = w8_3<INV>(b);
    x[0] = cadd(a, b);
    x[4] = csub(a, b);
    x[1] = cadd(a, o1);
    x[5] = csub(a, o1);
    x[2] = cadd(a, o2);
    x[6] = csub(a, o2);
    x[3] = cadd(a, o3);
    x[7] = csub(a, o3);
}

// x * (a + i b) for a constant unit root, conjugated for the inverse transform
template <bool INV, typename V> __device__ __forceinline__ V cmulc(V x, decltype(V::x) a, decltype(V::x) b)
{
    if (INV) b = -b;
    return cmk<V>(x.x * a - x.y * b, x.x * b + x.y * a);
}

// x (1 - i) (forward) or x (1 + i) (inverse): w16^2 without its 1/sqrt 2
template <bool INV, typename V> __device__ __forceinline__ V q1(V x)
{
    return INV ? cmk<V>(x.x - x.y, x.x + x.y) : cmk<V>(x.x + x.y, x.y - x.x);
}
// x (-1 - i) (forward) or x (-1 + i) (inverse): w16^6 without its 1/sqrt 2
template <bool INV, typename V> __device__ __forceinline__ V q3(V x)
{
    return INV ? cmk<V>(-(x.x + x.y), x.x - x.y) : cmk<V>(x.y - x.x, -(x.x + x.y));
}
// a + s b and a - s b, componentwise fused
template <typename V> __device__ __forceinline__ V cfma(V a, decltype(V::x) s, V b)
{
    return cmk<V>(fma(s, b.x, a.x), fma(s, b.y, a.y));
}
template <typename V> __device__ __forceinline__ V cfms(V a, decltype(V::x) s, V b)
{
    return cmk<V>(fma(-s, b.x, a.x), fma(-s, b.y, a.y));
}

// 16 points as 4 x 4: length-4 transforms over n = r + 4t (t), twiddles w16^{r m}, length-4
// transforms over r; X[m + 4 s] = sum_r w4^{r s} w16^{r m} sum_t w4^{t m} x[r + 4t].
// dft16_layer2 does the twiddles and the second layer from y[r][m].  Four of its twiddles,
// w16^2 and w16^6 (twice each), are (1 - i)/sqrt 2 and (-1 - i)/sqrt 2: their rotation is two
// additions (q1, q3) and their 1/sqrt 2 rides in the second layer's sums as fused multiply-adds,
// instead of two products and two multiply-adds each.
template <bool INV, typename V> __device__ __forceinline__ void dft16_layer2(V (*y)[4], V *x)
{
    typedef decltype(V::x) T;
    const T c = (T)0.9238795325112867561281831893967882;   // cos(pi/8)
    const T s = (T)0.3826834323650897717284599840303989;   // sin(pi/8)
    const T r2 = (T)0.7071067811865475244008443621048490;  // cos(pi/4)
    {   // m = 0: no twiddles
        V z[4] = {y[0][0], y[1][0], y[2][0], y[3][0]};
        dft4<INV>(z);
        x[0] = z[0];
        x[4] = z[1];
        x[8] = z[2];
        x[12] = z[3];
    }
    {   // m = 1: w16^{r}: (c, -s), (r2, -r2) = w16^2, (s, -c)
        const V z0 = y[0][1], z1 = cmulc<INV>(y[1][1], c, -s), z3 = cmulc<INV>(y[3][1], s, -c);
        const V u2 = q1<INV>(y[2][1]);
        const V a0 = cfma(z0, r2, u2), a1 = cfms(z0, r2, u2);
        const V a2 = cadd(z1, z3), a3 = rot<INV>(csub(z1, z3));
        x[1] = cadd(a0, a2);
        x[9] = csub(a0, a2);
        x[5] = cadd(a1, a3);
        x[13] = csub(a1, a3);
    }
    {   // m = 2: w16^{2r}: w16^2, -i, w16^6
        const V z0 = y[0][2], z2 = rot<INV>(y[2][2]);
        const V u1 = q1<INV>(y[1][2]), u3 = q3<INV>(y[3][2]);
        const V a0 = cadd(z0, z2), a1 = csub(z0, z2);
        const V v2 = cadd(u1, u3), v3 = rot<INV>(csub(u1, u3));
        x[2] = cfma(a0, r2, v2);
        x[10] = cfms(a0, r2, v2);
        x[6] = cfma(a1, r2, v3);
        x[14] = cfms(a1, r2, v3);
    }
    {   // m = 3: w16^{3r}: (s, -c), (-r2, -r2) = w16^6, (-c, s)
        const V z0 = y[0][3], z1 = cmulc<INV>(y[1][3], s, -c), z3 = cmulc<INV>(y[3][3], -c, s);
        const V u2 = q3<INV>(y[2][3]);
        const V a0 = cfma(z0, r2, u2), a1 = cfms(z0, r2, u2);
        const V a2 = cadd(z1, z3), a3 = rot<INV>(csub(z1, z3));
        x[3] = cadd(a0, a2);
        x[11] = csub(a0, a2);
        x[7] = cadd(a1, a3);
        x[15] = csub(a1, a3);
    }
}

template <bool INV, typename V> __device__ __forceinline__ void dft16(V *x) {
    V y[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        y[r][0] = x[r];
        y[r][1] = x[r + 4];
        y[r][2] = x[r + 8];
        y[r][3] = x[r + 12];
        dft4<INV>(y[r]);  // y[r][m], m = 0..3
    }
    dft16_layer2<INV>(y, x);
}

// dft16 of x[0..7] followed by eight zeros (the first stage of a zero-extended transform):
// the first layer's length-4 transforms see (x[r], x[r+4], 0, 0).
template <bool INV, typename V> __device__ __forceinline__ void dft16_half_in(V *x) {
    V y[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const V a = x[r], b = x[r + 4], rb = rot<INV>(b);
        y[r][0] = cadd(a, b);
        y[r][1] = cadd(a, rb);
        y[r][2] = csub(a, b);
        y[r][3] = csub(a, rb);
    }
    dft16_layer2<INV>(y, x);
}

template <int R, bool INV, typename V> __device__ __forceinline__ void dftR(V *x) {
    if (R == 2) dft2<INV>(x);
    else if (R == 3) dft3<INV>(x);
    else if (R == 4) dft4<INV>(x);
    else if (R == 5) dft5<INV>(x);
    else if (R == 8) dft8<INV>(x);
    else dft16<INV>(x);
}

// ---------------------------------------------------------------- twiddles
// x[q] *= w^{qk}, q = 1..R-1, from the stage's blocks (k < Ns): radices 2..8, and radix 16 in FP32,
// read [w^k | w^{2k} | w^{4k} (| w^{8k})] (the blocks they need) and form the other powers as
// products; FP64 radix 16 reads all fifteen powers [w^k | w^{2k} | ... | w^{15k}].
template <typename T, bool TWS>
__device__ __forceinline__ typename cvec<T>::t tw_load(const typename cvec<T>::t *__restrict__ tw, int t)
{
    if constexpr (TWS) return tw[t];
    else return __ldg(&tw[t]);
}

template <typename T, int R, bool INV, bool TWS>
__device__ __forceinline__ void apply_twiddles(typename cvec<T>::t *x, const typename cvec<T>::t *__restrict__ tab,
                                               int Ns, int k)
{
    typedef typename cvec<T>::t V;
    if constexpr (R == 16 && sizeof(T) == 8) {
        // FP64 radix 16 reads all fifteen powers (block q-1 holds w^{qk}): its FP64 units are the
        // bound, and loads cost less than eleven complex products
#pragma unroll
        for (int q = 1; q < 16; ++q) {
            V w = tw_load<T, TWS>(tab, (q - 1) * Ns + k);
            if (INV) w.y = -w.y;
            x[q] = cmul(x[q], w);
        }
        return;
    }
    V w1 = tw_load<T, TWS>(tab, k);
    if (INV) w1.y = -w1.y;
    x[1] = cmul(x[1], w1);
    if constexpr (R == 2) return;
    V w2 = tw_load<T, TWS>(tab, Ns + k);
    if (INV) w2.y = -w2.y;
    x[2] = cmul(x[2], w2);
    if constexpr (R == 3) return;
    V w3 = cmul(w1, w2);
    x[3] = cmul(x[3], w3);
    if constexpr (R == 4) return;
    V w4 = tw_load<T, TWS>(tab, 2 * Ns + k);
    if (INV) w4.y = -w4.y;
    x[4] = cmul(x[4], w4);
    if constexpr (R == 5) return;
    const V w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
    x[5] = cmul(x[5], w5);
    x[6] = cmul(x[6], w6);
    x[7] = cmul(x[7], w7);
    if constexpr (R == 8) return;
    // FP32 radix 16: a fourth block w^{8k}; powers 9..15 = (1..7) + 8
    V w8 = tw_load<T, TWS>(tab, 3 * Ns + k);
    if (INV) w8.y = -w8.y;
    x[8] = cmul(x[8], w8);
    x[9] = cmul(x[9], cmul(w1, w8));
    x[10] = cmul(x[10], cmul(w2, w8));
    x[11] = cmul(x[11], cmul(w3, w8));
    x[12] = cmul(x[12], cmul(w4, w8));
    x[13] = cmul(x[13], cmul(w5, w8));
    x[14] = cmul(x[14], cmul(w6, w8));
    x[15] = cmul(x[15], cmul(w7, w8));
}

// ---------------------------------------------------------------- one Stockham stage
// Every thread owns exactly E elements of a length-L transform (L = E * tpt); a radix-R stage
// gives it E/R butterflies j = lt + b tpt.  tw[t] = exp(-2 pi i t / L).
template <typename T, int E, int R, bool INV, bool TWS>
__device__ __forceinline__ void stockham_stage(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P, int s,
                                               const typename cvec<T>::t *__restrict__ tw, int lt,
                                               int tpt)
{
    typedef typename cvec<T>::t V;
    constexpr int NB = E / R;
    const int nbf = NB * tpt;
    const int Ns = __ldg(&P->Ns[s]), toff = __ldg(&P->toff[s]);
    const unsigned long long mg = __ldg(&P->mag[s]);
    V v[NB][R];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = lt + b * tpt;
#pragma unroll
        for (int q = 0; q < R; ++q) v[b][q] = buf[pidx<T>(j + q * nbf)];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = lt + b * tpt;
        const int jq = (int)(((unsigned long long)j * mg) >> 40);
        const int k = j - jq * Ns;
        if (Ns > 1) apply_twiddles<T, R, INV, TWS>(v[b], tw + toff, Ns, k);
        dftR<R, INV>(v[b]);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int p = 0; p < R; ++p) buf[pidx<T>(base + p * Ns)] = v[b][p];
        // keep the next butterfly's twiddle loads after these stores (bounds live registers)
        asm volatile("" ::: "memory");
    }
    __syncthreads();
}

// Generic stage for lengths without an exact per-thread split (E = 0 below): up to GMAXE elements
// per thread, butterflies guarded by j < L/R.
#define WSC_GMAXE 24
template <typename T, int R, bool INV, bool TWS>
__device__ __forceinline__ void stockham_stage_guarded(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P, int s,
                                                       const typename cvec<T>::t *__restrict__ tw, int lt,
                                                       int tpt)
{
    typedef typename cvec<T>::t V;
    constexpr int NB = WSC_GMAXE / R;
    const int nbf = __ldg(&P->L) / R;
    const int Ns = __ldg(&P->Ns[s]), toff = __ldg(&P->toff[s]);
    const unsigned long long mg = __ldg(&P->mag[s]);
    V v[NB][R];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = lt + b * tpt;
        if (j < nbf) {
#pragma unroll
            for (int q = 0; q < R; ++q) v[b][q] = buf[pidx<T>(j + q * nbf)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = lt + b * tpt;
        if (j < nbf) {
            const int jq = (int)(((unsigned long long)j * mg) >> 40);
            const int k = j - jq * Ns;
            if (Ns > 1) apply_twiddles<T, R, INV, TWS>(v[b], tw + toff, Ns, k);
            dftR<R, INV>(v[b]);
            const int base = jq * Ns * R + k;
#pragma unroll
            for (int p = 0; p < R; ++p) buf[pidx<T>(base + p * Ns)] = v[b][p];
        }
    }
    __syncthreads();
}

// Radices a given E supports: R must divide E (E = 0: the guarded generic stage takes any R).
template <int E, int R> struct radix_ok { static const bool v = E == 0 || (E % R) == 0; };

template <typename T, int E, int R, bool INV, bool TWS, bool OK = radix_ok<E, R>::v> struct stage_call;
template <typename T, int E, int R, bool INV, bool TWS> struct stage_call<T, E, R, INV, TWS, true> {
    static __device__ __forceinline__ void run(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P, int s,
                                               const typename cvec<T>::t *__restrict__ tw, int lt, int tpt)
    {
        if constexpr (E == 0) stockham_stage_guarded<T, R, INV, TWS>(buf, P, s, tw, lt, tpt);
        else stockham_stage<T, E, R, INV, TWS>(buf, P, s, tw, lt, tpt);
    }
};
template <typename T, int E, int R, bool INV, bool TWS> struct stage_call<T, E, R, INV, TWS, false> {
    static __device__ __forceinline__ void run(typename cvec<T>::t *, const FFTDesc *__restrict__, int,
                                               const typename cvec<T>::t *__restrict__, int, int) {}
};

// Whole transform (unnormalised).  All threads of the CTA must call it (barriers inside).  The
// host only builds radix sequences whose radices divide E.  TWS: tw points to shared memory.
template <typename T, int E, bool INV, bool TWS>
__device__ __forceinline__ void fft_smem(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P,
                                         const typename cvec<T>::t *__restrict__ tw, int lt, int tpt)
{
    const int nst = __ldg(&P->nst);
    for (int s = 0; s < nst; ++s) {
        // launder the thread index so per-stage address arithmetic is not hoisted out of the
        // stage loop (hoisting every radix's addresses keeps dozens of registers live)
        int lt_ = lt;
        asm volatile("" : "+r"(lt_));
        lt = lt_;
        switch (__ldg(&P->R[s])) {
        case 8: stage_call<T, E, 8, INV, TWS>::run(buf, P, s, tw, lt, tpt); break;
        case 4: stage_call<T, E, 4, INV, TWS>::run(buf, P, s, tw, lt, tpt); break;
        case 2: stage_call<T, E, 2, INV, TWS>::run(buf, P, s, tw, lt, tpt); break;
        case 3: stage_call<T, E, 3, INV, TWS>::run(buf, P, s, tw, lt, tpt); break;
        default: stage_call<T, E, 5, INV, TWS>::run(buf, P, s, tw, lt, tpt); break;
        }
    }
}

}  // namespace wsc
