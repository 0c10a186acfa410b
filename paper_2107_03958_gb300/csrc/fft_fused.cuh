// fft_fused.cuh -- Stockham FFT whose first stage reads its inputs straight from global memory and
// whose last stage hands its outputs to the caller (global stores, or a per-element hook before the
// shared-memory store), so a pass never spends separate shared-memory sweeps on loading, zero-filling,
// multiplying or storing its data.
//
// Every stage dispatches on its radix (8, 4, 2 or 3; it must divide E).  Sources/destinations:
//   FromSmem / ToSmem          the transform buffer
//   a functor  V src(int i)    stage-0 input element i (global loads, zero beyond the data)
//   a functor  void dst(int i, V v)   last-stage output element i (global stores)
//   SmemHook{f}                last-stage output passes through f(i, v&), then to the buffer
#pragma once
#include <type_traits>

#include "fft_engine.cuh"

namespace wsc {

struct FromSmem {};
struct ToSmem {};
template <class F> struct SmemHook {
    F f;
};
template <class F> __device__ __forceinline__ SmemHook<F> smem_hook(F f) { return SmemHook<F>{f}; }

template <class D> struct writes_smem : std::false_type {};
template <> struct writes_smem<ToSmem> : std::true_type {};
template <class F> struct writes_smem<SmemHook<F>> : std::true_type {};

// One radix-R stage s; every thread owns E/R butterflies j = lt + b tpt.
template <typename T, int E, int R, bool INV, bool TWS, class Src, class Dst>
__device__ __forceinline__ void fstage(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P, int s,
                                       const typename cvec<T>::t *__restrict__ tw, int lt, int tpt,
                                       const Src &src, const Dst &dst)
{
    typedef typename cvec<T>::t V;
    constexpr int NB = E / R;
    constexpr bool SRC_SMEM = std::is_same<Src, FromSmem>::value;
    constexpr bool DST_SMEM = writes_smem<Dst>::value;
    const int nbf = NB * tpt;
    const int Ns = __ldg(&P->Ns[s]), toff = __ldg(&P->toff[s]);
    const unsigned long long mg = __ldg(&P->mag[s]);
    V v[NB][R];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = lt + b * tpt;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if constexpr (SRC_SMEM) v[b][q] = buf[pidx<T>(j + q * nbf)];
            else v[b][q] = src(j + q * nbf);
        }
    }
    if constexpr (SRC_SMEM && DST_SMEM) __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = lt + b * tpt;
        const int jq = (int)(((unsigned long long)j * mg) >> 40);
        const int k = j - jq * Ns;
        if (Ns > 1) apply_twiddles<T, R, INV, TWS>(v[b], tw + toff, Ns, k);
        dftR<R, INV>(v[b]);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int p = 0; p < R; ++p) {
            const int o = base + p * Ns;
            if constexpr (std::is_same<Dst, ToSmem>::value) {
                buf[pidx<T>(o)] = v[b][p];
            } else if constexpr (DST_SMEM) {
                V x = v[b][p];
                dst.f(o, x);
                buf[pidx<T>(o)] = x;
            } else {
                dst(o, v[b][p]);
            }
        }
        asm volatile("" ::: "memory");
    }
    if constexpr (DST_SMEM) __syncthreads();
}

// Interior stage: shared memory in and out, radix from the descriptor.
template <typename T, int E, bool INV, bool TWS>
__device__ __forceinline__ void fstage_mid(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P, int s,
                                           const typename cvec<T>::t *__restrict__ tw, int lt, int tpt)
{
    switch (__ldg(&P->R[s])) {
    case 8:
        if constexpr (E % 8 == 0) fstage<T, E, 8, INV, TWS>(buf, P, s, tw, lt, tpt, FromSmem{}, ToSmem{});
        break;
    case 4:
        if constexpr (E % 4 == 0) fstage<T, E, 4, INV, TWS>(buf, P, s, tw, lt, tpt, FromSmem{}, ToSmem{});
        break;
    case 2:
        if constexpr (E % 2 == 0) fstage<T, E, 2, INV, TWS>(buf, P, s, tw, lt, tpt, FromSmem{}, ToSmem{});
        break;
    default:
        if constexpr (E % 3 == 0) fstage<T, E, 3, INV, TWS>(buf, P, s, tw, lt, tpt, FromSmem{}, ToSmem{});
        break;
    }
}

// Edge stage (first or last) with the radix read from the descriptor.
template <typename T, int E, bool INV, bool TWS, class Src, class Dst>
__device__ __forceinline__ void fstage_edge(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P, int s,
                                            const typename cvec<T>::t *__restrict__ tw, int lt, int tpt,
                                            const Src &src, const Dst &dst)
{
    switch (__ldg(&P->R[s])) {
    case 8:
        if constexpr (E % 8 == 0) fstage<T, E, 8, INV, TWS>(buf, P, s, tw, lt, tpt, src, dst);
        break;
    case 4:
        if constexpr (E % 4 == 0) fstage<T, E, 4, INV, TWS>(buf, P, s, tw, lt, tpt, src, dst);
        break;
    case 2:
        if constexpr (E % 2 == 0) fstage<T, E, 2, INV, TWS>(buf, P, s, tw, lt, tpt, src, dst);
        break;
    default:
        if constexpr (E % 3 == 0) fstage<T, E, 3, INV, TWS>(buf, P, s, tw, lt, tpt, src, dst);
        break;
    }
}

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Whole transform, at least two stages.  All threads of the CTA call it.  If src is FromSmem the
// buffer must hold the input; if dst writes global memory, the caller must meet a barrier before
// the buffer is written again.  after0() runs on every thread once stage 0 has read all of its
// inputs and the CTA has met the barrier that ends the stage (the moment a prefetch may overwrite
// what src read).
// ED encodes the first and last radix at compile time as 16 R_first + R_last (0: read both from
// the descriptor).
template <typename T, int E, int ED, bool INV, bool TWS, class Src, class Dst, class After0 = NoHook>
__device__ __forceinline__ void fft_fused(typename cvec<T>::t *buf, const FFTDesc *__restrict__ P,
                                          const typename cvec<T>::t *__restrict__ tw, int lt, int tpt,
                                          const Src &src, const Dst &dst, const After0 &after0 = After0{})
{
    const int nst = __ldg(&P->nst);
    if constexpr (ED == 0) fstage_edge<T, E, INV, TWS>(buf, P, 0, tw, lt, tpt, src, ToSmem{});
    else fstage<T, E, ED / 16, INV, TWS>(buf, P, 0, tw, lt, tpt, src, ToSmem{});
    after0();
    for (int s = 1; s < nst - 1; ++s) {
        int lt_ = lt;
        asm volatile("" : "+r"(lt_));
        fstage_mid<T, E, INV, TWS>(buf, P, s, tw, lt_, tpt);
    }
    if constexpr (ED == 0) fstage_edge<T, E, INV, TWS>(buf, P, nst - 1, tw, lt, tpt, FromSmem{}, dst);
    else fstage<T, E, ED % 16, INV, TWS>(buf, P, nst - 1, tw, lt, tpt, FromSmem{}, dst);
}

}  // namespace wsc
