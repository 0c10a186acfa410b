// fft_static.cuh -- the fused Stockham transform of fft_fused.cuh for a length fixed at compile
// time, in two families:
//   ED = 1000 + l: L = 2^l in radix-16 stages (and one radix-2, -4 or -8 stage for the remaining
//     factor): one shared-memory round trip per four bits, and no stage with Ns = 8, whose
//     stride-8 stores conflict in the padded layout;
//   ED = 2000 + l: L = 3 2^l (the period-3 grid, L = 3n) in radix-8 stages, one radix-4 or -2
//     stage for l mod 3, and a last radix-3 stage.
//
// With R, Ns and the thread count known, every shared-memory, twiddle and global index of a
// stage is a per-thread base plus a compile-time offset:
//   inputs   e = j + q L/R, j = lt + b tpt:   pidx(e) = pidx(lt) + c + (c >> PS),  c = b tpt + q L/R;
//   outputs  o = (j / Ns) R Ns + (j mod Ns) + p Ns, with j / Ns and j mod Ns split into a thread
//            part (jq0, k0) and a constant (cj, ck) of butterfly b, and pidx(o) = T0 + C(b) + C(p),
//            T0 from (jq0, k0), the constants from the padding period PAD = 2^PS (tpt, and so
//            b tpt, is a multiple of PAD).
// This needs every stage's Ns to be a power of two, which holds in both families: the radix-3
// stage, the one radix that is not a power of two, comes last.
// The runtime path recomputes these per element (shifts, magic-number divisions, stage-table
// loads); here each stage computes a handful of per-thread bases and the rest folds into the
// load/store immediates.
//
// Ping-pong (PP): with two transform buffers per line, stage s reads X_s and writes X_{s+1}
// (X_even = b0, X_odd = b1), so no thread can overwrite an input another thread has yet to read
// and each stage needs one barrier (after its stores) instead of two; the warps of a stage then
// overlap one another's loads, arithmetic and stores.  Without it b0 = b1 and every stage waits
// once after its loads and once after its stores.
#pragma once
#include "fft_fused.cuh"

namespace wsc {

__host__ __device__ constexpr int tw_blocks_c(int R, bool full16) { return R == 2 ? 1 : (R <= 4 ? 2 : (R <= 8 ? 3 : (full16 ? 15 : 4))); }

// Stage structure of compile-time length ED (the host's factorize gives the same sequence and
// twiddle table: with radix16 set for ED = 1000 + l, with E = 24 for ED = 2000 + l).
template <int ED, bool FULL16 = false> struct StaticStages {
    static constexpr bool X3 = ED >= 2000;                     // L = 3 2^L2
    static constexpr int L2 = X3 ? ED - 2000 : ED - 1000;      // log2 of the power-of-two factor
    static constexpr int L = X3 ? 3 << L2 : 1 << L2;
    static constexpr int LR = X3 ? 3 : 4;                      // log2 of the main radix
    static constexpr int NMAIN = L2 / LR, REM = L2 % LR;
    static constexpr int NST = NMAIN + (REM ? 1 : 0) + (X3 ? 1 : 0);
    __host__ __device__ static constexpr int R(int s) { return s < NMAIN ? 1 << LR : (s == NMAIN && REM ? 1 << REM : 3); }
    // log2 Ns of stage s: the radices before it are all powers of two
    __host__ __device__ static constexpr int lNs(int s)
    {
        int v = 0;
        for (int i = 0; i < s; ++i) v += i < NMAIN ? LR : REM;
        return v;
    }
    __host__ __device__ static constexpr int toff(int s)
    {
        int o = 0;
        for (int i = 0; i < s; ++i) o += tw_blocks_c(R(i), FULL16) << lNs(i);
        return o;
    }
};

// One radix-R stage S; every thread owns E/R butterflies j = lt + b tpt.
// HIN: the transform's inputs e >= n are zero (the zero extension; n = L/2 or L/3): stage 0 loads
// only the inputs below n and runs a butterfly with the others fixed at zero.
// HOUT: only outputs o < n are used (the crop): the last stage stores only p < R/2 (n = L/2) or
// p = 0 (n = L/3, the last radix is 3), and the arithmetic feeding the rest drops out.
template <typename T, int E, int ED, int S, bool INV, bool TWS, bool HIN, bool HOUT, bool PP, class Src, class Dst>
__device__ __forceinline__ void sstage(const typename cvec<T>::t *bin, typename cvec<T>::t *buf,
                                       const typename cvec<T>::t *__restrict__ tw, int lt, const Src &src,
                                       const Dst &dst)
{
    typedef typename cvec<T>::t V;
    typedef StaticStages<ED, sizeof(T) == 8> P;  // FP64 tables hold all fifteen radix-16 powers
    constexpr int R = P::R(S), lNs = P::lNs(S), Ns = 1 << lNs, RN = R * Ns;
    constexpr int TPT = P::L / E, NB = E / R, NBF = NB * TPT;
    constexpr int PS = pad_shift<T>::v, PAD = 1 << PS;
    static_assert(E % R == 0, "radix must divide the elements per thread");
    static_assert(TPT % PAD == 0, "threads per transform must be a multiple of the padding period");
    constexpr bool SRC_SMEM = std::is_same<Src, FromSmem>::value;
    constexpr bool DST_SMEM = writes_smem<Dst>::value;
    constexpr bool pin = HIN && S == 0, pout = HOUT && S == P::NST - 1;
    static_assert(!pin || R == (P::X3 ? 8 : 16), "the pruned-input butterflies are radix 16 (n = L/2) or 8 (n = L/3)");
    static_assert(!pout || !P::X3 || R == 3, "the period-3 family ends in its radix-3 stage");
    // input q of butterfly b (elements b tpt + q L/R + [0, tpt)) lies wholly below n or wholly
    // above it: n = L/2 is a multiple of L/R; for n = L/3, tpt = L/24 and R = 8 make the bound
    // 3q + b <= 7 an integer one
    constexpr int NIN = P::X3 ? P::L / 3 : P::L / 2;
    static_assert(!pin || !P::X3 || E == 24, "the period-3 input pruning assumes 24 elements per thread");
    constexpr int NOUT = pout ? (P::X3 ? 1 : R / 2) : R;
    __builtin_assume(lt >= 0 && lt < TPT);
    // per-thread bases of this stage
    const int pl = lt + (lt >> PS);
    int k0, jq0;
    if constexpr (Ns <= TPT) {
        k0 = lt & (Ns - 1);
        jq0 = lt >> lNs;
    } else {
        k0 = lt;
        jq0 = 0;
    }
    int T0;
    if constexpr (RN <= PAD) {
        const int x = jq0 * RN;
        T0 = x + (x >> PS) + k0;
    } else if constexpr (Ns < PAD) {
        T0 = jq0 * (RN + RN / PAD) + k0;
    } else {
        T0 = jq0 * (RN + RN / PAD) + k0 + (k0 >> PS);
    }
    const int O0 = jq0 * RN + k0;
    V v[NB][R];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int c = b * TPT + q * NBF;
            if (pin && c >= NIN) v[b][q] = cmk<V>(0, 0);
            else if constexpr (SRC_SMEM) v[b][q] = bin[pl + c + (c >> PS)];
            else v[b][q] = src(lt + c);
        }
    }
    if constexpr (SRC_SMEM && DST_SMEM && !PP) __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int cb = b * TPT, ck = cb & (Ns - 1), cj = cb >> lNs;
        if constexpr (Ns > 1) apply_twiddles<T, R, INV, TWS>(v[b], tw + P::toff(S) + ck, Ns, k0);
        if constexpr (pin && !P::X3) dft16_half_in<INV>(v[b]);
        else if constexpr (pin) {
            if (b * TPT + 2 * NBF < NIN) dft8_in3<INV>(v[b]);
            else dft8_in2<INV>(v[b]);
        } else dftR<R, INV>(v[b]);
        const int Cb = RN <= PAD ? cj * RN + ((cj * RN) >> PS) : cj * (RN + RN / PAD) + ck + (ck >> PS);
#pragma unroll
        for (int p = 0; p < NOUT; ++p) {
            const int Cp = RN <= PAD ? p * Ns : (Ns < PAD ? p * Ns + ((p * Ns) >> PS) : p * (Ns + Ns / PAD));
            const int o = O0 + cj * RN + ck + p * Ns;
            if constexpr (std::is_same<Dst, ToSmem>::value) {
                buf[T0 + Cb + Cp] = v[b][p];
            } else if constexpr (DST_SMEM) {
                V x = v[b][p];
                dst.f(o, x);
                buf[T0 + Cb + Cp] = x;
            } else {
                dst(o, v[b][p]);
            }
        }
        asm volatile("" ::: "memory");
    }
    if constexpr (DST_SMEM) __syncthreads();
}

template <typename T, int E, int ED, bool INV, bool TWS, bool HIN, bool HOUT, bool PP, class Src, class Dst, class After0,
          int S>
__device__ __forceinline__ void fft_static_from(typename cvec<T>::t *b0, typename cvec<T>::t *b1,
                                                const typename cvec<T>::t *__restrict__ tw,
                                                const typename cvec<T>::t *__restrict__ twg, int lt, const Src &src,
                                                const Dst &dst, const After0 &after0)
{
    constexpr int NST = StaticStages<ED>::NST;
    static_assert(NST >= 2, "at least two stages");
    // stage S reads X_S and writes X_{S+1}
    typename cvec<T>::t *bin = (S & 1) ? b1 : b0, *bout = (S & 1) ? b0 : b1;
    // a table split between shared and global memory: the last stage reads the global one
    constexpr bool GLOBAL_TW = TWS && S == NST - 1 && tw_split_ok<T, ED>();
    constexpr bool TWS_S = TWS && !GLOBAL_TW;
    const typename cvec<T>::t *tws = GLOBAL_TW ? twg : tw;
    // keep each stage's per-thread bases from being hoisted to the kernel start (register pressure)
    int lt_ = lt;
    asm volatile("" : "+r"(lt_));
    if constexpr (S == 0) {
        sstage<T, E, ED, 0, INV, TWS_S, HIN, HOUT, PP>(bin, bout, tws, lt_, src, ToSmem{});
        after0();
    } else if constexpr (S == NST - 1) {
        sstage<T, E, ED, S, INV, TWS_S, HIN, HOUT, PP>(bin, bout, tws, lt_, FromSmem{}, dst);
    } else {
        sstage<T, E, ED, S, INV, TWS_S, HIN, HOUT, PP>(bin, bout, tws, lt_, FromSmem{}, ToSmem{});
    }
    if constexpr (S + 1 < NST)
        fft_static_from<T, E, ED, INV, TWS, HIN, HOUT, PP, Src, Dst, After0, S + 1>(b0, b1, tw, twg, lt, src, dst,
                                                                                   after0);
}

// Whole transform of compile-time length ED; same contract as fft_fused.  Shared-memory inputs
// (FromSmem) are read from b0; shared-memory outputs end in X_NST (final_buf).  b1 = b0 without PP.
// tw: the twiddle table (shared memory with TWS); twg: the global table, which the last stage
// reads when the shared copy holds only the earlier stages' blocks (tw_split_ok).
template <typename T, int E, int ED, bool INV, bool TWS, bool HIN, bool HOUT, bool PP, class Src, class Dst, class After0>
__device__ __forceinline__ void fft_static(typename cvec<T>::t *b0, typename cvec<T>::t *b1,
                                           const typename cvec<T>::t *__restrict__ tw,
                                           const typename cvec<T>::t *__restrict__ twg, int lt, const Src &src,
                                           const Dst &dst, const After0 &after0)
{
    fft_static_from<T, E, ED, INV, TWS, HIN, HOUT, PP, Src, Dst, After0, 0>(b0, b1, tw, twg, lt, src, dst, after0);
}

// The buffer holding a compile-time transform's shared-memory outputs, X_NST, and the other one.
template <int ED> __device__ __forceinline__ bool final_in_b1() { return ED >= 1000 && (StaticStages<ED>::NST & 1); }

// The pass kernels' transform: ED >= 1000 selects the static path for length 2^(ED - 1000) or
// 3 2^(ED - 2000) (which the host picks only for n = L/2 or n = L/3 respectively, so HIN and HOUT
// hold there: zero-extended inputs, cropped outputs); otherwise the runtime-descriptor path of
// fft_fused with edge radices ED, which reads and writes every element.
template <typename T, int E, int ED, bool INV, bool TWS, bool HIN = false, bool HOUT = false, class Src, class Dst,
          class After0 = NoHook>
__device__ __forceinline__ void fft_any(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P,
                                        const typename cvec<T>::t *__restrict__ tw,
                                        const typename cvec<T>::t *__restrict__ twg, int lt, int tpt, const Src &src,
                                        const Dst &dst, const After0 &after0 = After0{})
{
    if constexpr (ED >= 1000) fft_static<T, E, ED, INV, TWS, HIN, HOUT, false>(buf, buf, tw, twg, lt, src, dst, after0);
    else fft_fused<T, E, ED, INV, TWS>(buf, P, tw, lt, tpt, src, dst, after0);
}

// fft_any with a second buffer: the compile-time lengths ping-pong between b0 and b1 when PP is
// set (outputs in X_NST, see final_in_b1); the runtime path uses b0 alone.
template <typename T, int E, int ED, bool INV, bool TWS, bool HIN, bool HOUT, bool PP, class Src, class Dst,
          class After0 = NoHook>
__device__ __forceinline__ void fft_any2(typename cvec<T>::t *b0, typename cvec<T>::t *b1, const FFTDesc *__restrict__ P,
                                         const typename cvec<T>::t *__restrict__ tw,
                                         const typename cvec<T>::t *__restrict__ twg, int lt, int tpt, const Src &src,
                                         const Dst &dst, const After0 &after0 = After0{})
{
    if constexpr (ED >= 1000) fft_static<T, E, ED, INV, TWS, HIN, HOUT, PP>(b0, PP ? b1 : b0, tw, twg, lt, src, dst, after0);
    else fft_fused<T, E, ED, INV, TWS>(b0, P, tw, lt, tpt, src, dst, after0);
}

// Transform length of the compile-time path (0 for the runtime path).
template <int ED> __host__ __device__ constexpr int static_len() { return ED >= 2000 ? 3 << (ED - 2000) : (ED >= 1000 ? 1 << (ED - 1000) : 0); }

}  // namespace wsc
