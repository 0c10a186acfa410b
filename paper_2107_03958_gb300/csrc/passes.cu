// passes.cu -- the three fused passes of the convolution A_n u = crop_n(ifft2(ghat . fft2(pad_M u)))
// (Sec. 2.1, eq. (An)).
//
// Workspace layout per density: the spectrum after the row transform, stored column-major,
// W[k2][j1] (k2 the x2-frequency, j1 < n the surviving rows), so the column pass reads and writes
// contiguous runs and the row passes touch one contiguous run of `rows` elements per frequency.
//
//   pass 1 (rows, forward): load row(s) of u (times the mask), zero-extend to M -- rows j1 >= n are
//          never formed -- forward length-M FFT along x2, write W[k2][j1].
//          R2R: two real rows share one complex FFT (z = u_a + i u_b) and are separated with the
//          Hermitian split; only k2 in [0, M/2] is kept.
//   pass 2 (columns): per column k2: forward length-M FFT along x1 over the n stored rows (the
//          others are zero), multiply by ghat(|k1|, |k2|) from the quadrant table, inverse FFT,
//          keep the first n outputs.
//   pass 3 (rows, inverse): gather W[.][j1], inverse length-M FFT along x2 (R2R: Hermitian
//          completion of two rows packed in one complex FFT), keep the first n outputs, scale by
//          1/M^2 and apply out = beta u + alpha (.).
#include <algorithm>
#include <cstdio>

#include <array>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

// ============================================================================ host side
// Per-thread element counts with exact (unguarded) kernels, in order of preference.  A count E
// admits radices dividing E; FP64 prefers radix-4 stages (E = 12 or 8), FP32 radix-8 (E = 24 or
// 16).  E = 0 is the generic guarded path (any 2^a 3^b 5^c).
// FP64 E = 16 exists only as the compile-time-length transforms (radix 16, 128 registers)
static const int kElems64[] = {16, 12, 24, 8, 0};
static const int kElems32[] = {24, 16, 0};

static int max_threads(conv_precision prec, int E)
{
    if (prec == CONV_P_FP64) {
        switch (E) {
        case 8: return maxt<double, 8>::v;
        case 12: return maxt<double, 12>::v;
        case 24: return maxt<double, 24>::v;
        default: return maxt<double, 0>::v;
        }
    }
    switch (E) {
    case 16: return maxt<float, 16>::v;
    case 24: return maxt<float, 24>::v;
    default: return maxt<float, 0>::v;
    }
}

// Dispatch on (precision, E, TWS) for the templated helpers.
#define WSC_DISPATCH(prec, E, tws, CALL)                                                      \
    do {                                                                                      \
        if ((prec) == CONV_P_FP64) {                                                          \
            if ((tws)) {                                                                      \
                switch (E) {                                                                  \
                case 8: { typedef double T_; constexpr int E_ = 8; constexpr bool W_ = true; CALL; } break;   \
                case 12: { typedef double T_; constexpr int E_ = 12; constexpr bool W_ = true; CALL; } break; \
                default: { typedef double T_; constexpr int E_ = 24; constexpr bool W_ = true; CALL; } break; \
                }                                                                             \
            } else {                                                                          \
                switch (E) {                                                                  \
                case 8: { typedef double T_; constexpr int E_ = 8; constexpr bool W_ = false; CALL; } break;   \
                case 12: { typedef double T_; constexpr int E_ = 12; constexpr bool W_ = false; CALL; } break; \
                case 24: { typedef double T_; constexpr int E_ = 24; constexpr bool W_ = false; CALL; } break; \
                default: { typedef double T_; constexpr int E_ = 0; constexpr bool W_ = false; CALL; } break;  \
                }                                                                             \
            }                                                                                 \
        } else {                                                                              \
            if ((tws)) {                                                                      \
                switch (E) {                                                                  \
                case 16: { typedef float T_; constexpr int E_ = 16; constexpr bool W_ = true; CALL; } break;   \
                default: { typedef float T_; constexpr int E_ = 24; constexpr bool W_ = true; CALL; } break;   \
                }                                                                             \
            } else {                                                                          \
                switch (E) {                                                                  \
                case 16: { typedef float T_; constexpr int E_ = 16; constexpr bool W_ = false; CALL; } break;  \
                case 24: { typedef float T_; constexpr int E_ = 24; constexpr bool W_ = false; CALL; } break;  \
                default: { typedef float T_; constexpr int E_ = 0; constexpr bool W_ = false; CALL; } break;   \
                }                                                                             \
            }                                                                                 \
        }                                                                                     \
    } while (0)

// Twiddle powers a radix-R butterfly reads from its stage's table: w^k (R = 2); w^k, w^2k (R = 3,
// 4; w^3k is their product); w^k, w^2k, w^4k (R = 5, 8; the other powers are products); all of
// w^k, w^2k, w^4k, w^8k (R = 16 in FP32) or all of w^k ... w^15k (R = 16 in FP64, whose FP64 units
// are the bound).
static inline int tw_blocks(int R, bool full16) { return R == 2 ? 1 : (R <= 4 ? 2 : (R <= 8 ? 3 : (full16 ? 15 : 4))); }
// power of w^k that block m holds: 2^m, or m + 1 for radix 16 with all fifteen powers
static inline long long tw_power(int R, bool full16, int m) { return R == 16 && full16 ? m + 1 : 1LL << m; }

// Radix sequence for L = 2^p 3^q 5^r whose radices divide E (E = 0: any of 8, 4, 2, 3, 5):
// power-of-two radices first (8s when allowed, else 4s), then 3s, then 5s.  radix16: a power of
// two as radix-16 stages and one stage for the remainder (the compile-time-length transforms).
static bool factorize(int L, int E, FFTDesc &d, bool radix16 = false, bool full16 = false)
{
    int rem = L, p2 = 0, p3 = 0, p5 = 0;
    while (rem % 2 == 0) { rem /= 2; ++p2; }
    while (rem % 3 == 0) { rem /= 3; ++p3; }
    while (rem % 5 == 0) { rem /= 5; ++p5; }
    if (rem != 1) return false;
    auto ok = [E](int r) { return E == 0 || E % r == 0; };
    if ((p3 && !ok(3)) || (p5 && !ok(5))) return false;
    std::vector<int> R;
    if (radix16 && p3 == 0 && p5 == 0 && E > 0 && E % 16 == 0) {
        for (int i = 0; i < p2 / 4; ++i) R.push_back(16);
        if (p2 % 4) R.push_back(1 << (p2 % 4));
    } else if (ok(8)) {
        for (int i = 0; i < p2 / 3; ++i) R.push_back(8);
        if (p2 % 3 == 2) R.push_back(4);
        if (p2 % 3 == 1) R.push_back(2);
    } else if (ok(4)) {
        for (int i = 0; i < p2 / 2; ++i) R.push_back(4);
        if (p2 % 2) R.push_back(2);
    } else {
        for (int i = 0; i < p2; ++i) R.push_back(2);
    }
    for (int i = 0; i < p3; ++i) R.push_back(3);
    for (int i = 0; i < p5; ++i) R.push_back(5);
    if ((int)R.size() > WSC_MAX_STAGES || R.empty()) return false;
    for (int r : R)
        if (!ok(r)) return false;
    d.L = L;
    d.nst = (int)R.size();
    long long Ns = 1;
    int off = 0;
    for (int s = 0; s < d.nst; ++s) {
        d.R[s] = R[s];
        d.Ns[s] = (int)Ns;
        d.tws[s] = (int)(L / (Ns * R[s]));
        d.toff[s] = off;
        off += tw_blocks(R[s], full16) * (int)Ns;
        d.mag[s] = ((1ULL << 40) + (unsigned long long)Ns - 1) / (unsigned long long)Ns;
        Ns *= R[s];
    }
    d.tw_len = off;
    d.tw_full16 = full16 ? 1 : 0;
    return true;
}

// Per-stage twiddle blocks [w^k | w^{2k} | w^{4k}] (the first tw_blocks(R) of them),
// w = exp(-2 pi i / (Ns R)), in long double.
void stage_twiddles(const FFTDesc &d, std::vector<double> &re_im)
{
    const long double PI_L = 3.141592653589793238462643383279502884L;
    re_im.assign(2 * (size_t)d.tw_len, 0.0);
    for (int s = 0; s < d.nst; ++s) {
        const long long Ns = d.Ns[s], NR = Ns * d.R[s];
        for (int m = 0; m < tw_blocks(d.R[s], d.tw_full16); ++m)
            for (long long k = 0; k < Ns; ++k) {
                const long long e = (tw_power(d.R[s], d.tw_full16, m) * k) % NR;
                const long double ang = 2.0L * PI_L * (long double)e / (long double)NR;
                const size_t i = (size_t)d.toff[s] + (size_t)m * Ns + (size_t)k;
                re_im[2 * i] = (double)cosl(ang);
                re_im[2 * i + 1] = (double)-sinl(ang);
            }
    }
}

// Threads per transform for the guarded path: every stage fits GMAXE/R butterflies per thread.
static int generic_tpt(const FFTDesc &P)
{
    int need = 1;
    for (int s = 0; s < P.nst; ++s) {
        int R = P.R[s], nb = WSC_GMAXE / R;
        need = std::max(need, (P.L / R + nb - 1) / nb);
    }
    return (need + 31) / 32 * 32;
}

// Fused-transform variants: (precision, E, ED = 16 R_first + R_last).
#define WSC_DISPATCH_FUSED(prec, E, ED, tws, CALL) \
    do { \
        if ((prec) == CONV_P_FP32 && (E) == 24 && (ED) == 131) { \
            if (tws) { typedef float T_; constexpr int E_ = 24, ED_ = 131; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 24, ED_ = 131; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 136) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 136; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 136; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 130) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 130; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 130; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 16 && (ED) == 1010) { \
            if (tws) { typedef double T_; constexpr int E_ = 16, ED_ = 1010; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 16, ED_ = 1010; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 16 && (ED) == 1011) { \
            if (tws) { typedef double T_; constexpr int E_ = 16, ED_ = 1011; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 16, ED_ = 1011; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 16 && (ED) == 1012) { \
            if (tws) { typedef double T_; constexpr int E_ = 16, ED_ = 1012; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 16, ED_ = 1012; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 16 && (ED) == 1013) { \
            if (tws) { typedef double T_; constexpr int E_ = 16, ED_ = 1013; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 16, ED_ = 1013; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 1008) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 1008; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 1008; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 1009) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 1009; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 1009; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 1010) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 1010; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 1010; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 1011) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 1011; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 1011; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 1012) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 1012; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 1012; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 1013) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 1013; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 1013; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 24 && (ED) == 2007) { \
            if (tws) { typedef float T_; constexpr int E_ = 24, ED_ = 2007; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 24, ED_ = 2007; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 24 && (ED) == 2008) { \
            if (tws) { typedef float T_; constexpr int E_ = 24, ED_ = 2008; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 24, ED_ = 2008; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 24 && (ED) == 2009) { \
            if (tws) { typedef float T_; constexpr int E_ = 24, ED_ = 2009; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 24, ED_ = 2009; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 24 && (ED) == 2010) { \
            if (tws) { typedef float T_; constexpr int E_ = 24, ED_ = 2010; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 24, ED_ = 2010; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 24 && (ED) == 2011) { \
            if (tws) { typedef float T_; constexpr int E_ = 24, ED_ = 2011; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 24, ED_ = 2011; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 24 && (ED) == 2012) { \
            if (tws) { typedef float T_; constexpr int E_ = 24, ED_ = 2012; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 24, ED_ = 2012; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 1014) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 1014; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 1014; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP32 && (E) == 16 && (ED) == 132) { \
            if (tws) { typedef float T_; constexpr int E_ = 16, ED_ = 132; constexpr bool W_ = true; CALL; } \
            else { typedef float T_; constexpr int E_ = 16, ED_ = 132; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 12 && (ED) == 67) { \
            if (tws) { typedef double T_; constexpr int E_ = 12, ED_ = 67; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 12, ED_ = 67; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 24 && (ED) == 131) { \
            if (tws) { typedef double T_; constexpr int E_ = 24, ED_ = 131; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 24, ED_ = 131; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 8 && (ED) == 136) { \
            if (tws) { typedef double T_; constexpr int E_ = 8, ED_ = 136; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 8, ED_ = 136; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 8 && (ED) == 130) { \
            if (tws) { typedef double T_; constexpr int E_ = 8, ED_ = 130; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 8, ED_ = 130; constexpr bool W_ = false; CALL; } \
        } \
        else if ((prec) == CONV_P_FP64 && (E) == 8 && (ED) == 132) { \
            if (tws) { typedef double T_; constexpr int E_ = 8, ED_ = 132; constexpr bool W_ = true; CALL; } \
            else { typedef double T_; constexpr int E_ = 8, ED_ = 132; constexpr bool W_ = false; CALL; } \
        } \
    } while (0)

static const int kFusedSets[][3] = {
    {0, 16, 1010},  // FP64 compile-time power-of-two lengths 2^10 ... 2^13
    {0, 16, 1011},
    {0, 16, 1012},
    {0, 16, 1013},
    {1, 16, 1008},  // FP32 compile-time power-of-two lengths 2^8 ... 2^14
    {1, 16, 1009},
    {1, 16, 1010},
    {1, 16, 1011},
    {1, 16, 1012},
    {1, 16, 1013},
    {1, 16, 1014},
    {1, 24, 2007},  // FP32 compile-time lengths 3 2^7 ... 3 2^12 (the period-3 grid, n = 128 ... 4096)
    {1, 24, 2008},
    {1, 24, 2009},
    {1, 24, 2010},
    {1, 24, 2011},
    {1, 24, 2012},
    {1, 24, 131},
    {1, 16, 136},
    {1, 16, 130},
    {1, 16, 132},
    {0, 12, 67},
    {0, 24, 131},
    {0, 8, 136},
    {0, 8, 130},
    {0, 8, 132},
};

// Fused passes exist for these (precision, E, ED): ED = 16 first radix + last radix with the
// stage structure read from the runtime descriptor, or the whole stage structure fixed at compile
// time (fft_static.cuh): ED = 1000 + log2 L for L = 2^l, chosen only when n = L/2, or
// ED = 2000 + log2(L/3) for L = 3 2^l, chosen only when n = L/3 (their transforms prune the zero
// extension and the crop).  Everything else runs the plain passes.  static_n = 0 skips the
// compile-time lengths.
static int fused_edges(conv_precision prec, int E, const FFTDesc &d, int static_n = 0)
{
    if (d.nst < 2) return 0;
    auto have = [&](int ed) {
        for (const auto &f : kFusedSets)
            if ((f[0] == 1) == (prec == CONV_P_FP32) && f[1] == E && f[2] == ed) return true;
        return false;
    };
    auto log2_of = [](int x) {  // log2 x for a power of two, else -1
        if (x <= 0 || (x & (x - 1))) return -1;
        int l = 0;
        while ((1 << l) < x) ++l;
        return l;
    };
    if (static_n > 0) {
        const int l2 = log2_of(d.L), l3 = d.L % 3 == 0 ? log2_of(d.L / 3) : -1;
        if (l2 >= 0 && 2 * static_n == d.L && have(1000 + l2)) return 1000 + l2;
        if (l3 >= 0 && 3 * static_n == d.L && have(2000 + l3)) return 2000 + l3;
    }
    const int ed = 16 * d.R[0] + d.R[d.nst - 1];
    for (const auto &f : kFusedSets)
        if ((f[0] == 1) == (prec == CONV_P_FP32) && f[1] == E && f[2] == ed) return ed;
    return 0;
}

int generic_threads(const FFTDesc &P) { return generic_tpt(P); }
bool factorize_any(int L, FFTDesc &d) { return factorize(L, 0, d); }

static conv_status set_all_attrs(int smem)
{
    conv_status rc = CONV_OK;
    for (int tws = 0; tws < 2 && rc == CONV_OK; ++tws) {
        for (const auto &f : kFusedSets)
            if (rc == CONV_OK)
                WSC_DISPATCH_FUSED(f[0] == 1 ? CONV_P_FP32 : CONV_P_FP64, f[1], f[2], tws,
                                   rc = (set_attrs_fused<T_, E_, ED_, W_>(smem)));
    }
    for (int prec = 0; prec < 2 && rc == CONV_OK; ++prec)
        for (int tws = 0; tws < 2 && rc == CONV_OK; ++tws)
            for (int E : {8, 12, 16, 24, 0}) {
                if (rc != CONV_OK) break;
                bool have = prec == CONV_P_FP64 ? (E == 8 || E == 12 || E == 24 || (E == 0 && !tws))
                                                : (E == 16 || E == 24 || (E == 0 && !tws));
                if (!have) continue;
                WSC_DISPATCH((conv_precision)prec, E, tws, rc = (set_attrs<T_, E_, W_>(smem)));
            }
    return rc;
}

static size_t round128(size_t x) { return (x + 127) & ~(size_t)127; }

// Shared memory of a pass CTA with G groups: [twiddles][G transform buffers][G staging areas]
// [G mbarriers], in the order stage_area() walks it on the device.
static size_t pass_smem(size_t twb, size_t per, size_t stage_bytes, int G)
{
    // staging: 128 bytes of slack to start it on a 128-byte shared address
    return twb + per * G + (stage_bytes ? 128 + (round128(stage_bytes) + 8) * G : 0);
}

// Most groups (<= 8, <= maxT / tpt) whose CTA fits `smem_optin`; 0 if not even one does.
static int max_groups(int maxT, int tpt, size_t twb, size_t per, size_t stage_bytes, int smem_optin)
{
    int G = std::min(8, std::max(1, maxT / tpt));
    while (G > 0 && pass_smem(twb, per, stage_bytes, G) > (size_t)smem_optin) --G;
    return G;
}

// Default options per pass (CFG_DEFAULT in a candidate), from FP32 measurements at n = 4096,
// batch 16 (per-pass ms of the R2R / split R2C plans in parentheses).
//   Runtime stage structure: prefetch pays in the row passes of the R2R and split R2C pipelines and
//   not in their column passes or in the C2C passes, where it costs a transform per CTA; TMA
//   copies of the strided spectrum pairs pay in both row passes (pass 1 2.15 -> 1.81, pass 3
//   2.07 -> 1.81).
//   Compile-time lengths (one transform per CTA, 128 registers): prefetch everywhere, twiddles
//   through L1; TMA loads in pass 3 (1.64 -> 1.35, split 3.20 -> 2.45) but not TMA stores in
//   pass 1: boxes of 16-byte runs drain at about 7 cycles per run per SM, slower than this
//   transform (1.72 -> 2.9).
static int default_options(const conv_plan_s *p, int ed, int pass)
{
    const bool pairs = p->io == CONV_IO_R2R || (p->io == CONV_IO_R2C && p->complex_ghat);
    // L = 2^14 at 1024 threads: 32 warps per SM hide the latency a prefetch would, and its staging
    // does not fit beside the 139 KB line (n = 8192, batch 8: 16.2 -> 15.4 ms per batch)
    if (ed == 1014) return 0;
    // FP64 column passes: twiddles in shared memory.  Read through L1, the fifteen powers a
    // radix-16 butterfly loads are hoisted into registers and the kernel spills (556 B a thread at
    // L = 2^13), whose write-backs doubled its DRAM writes (9.2 GB against 4.3 GB algorithmic per
    // launch at n = 4096, batch 16); from shared memory it does not spill, at +0.4 % time.  At
    // L = 2^13 only the radix-16 stages' blocks fit beside the line (tw_split_ed), without room for
    // the prefetch (which made no measurable difference there).
    if (ed >= 1000 && ed < 2000 && p->prec == CONV_P_FP64 && pass == 1)
        return tw_split_ed(ed, 8) ? CFG_TWS : CFG_TWS | CFG_PF;
    if (ed >= 1000) return pass == 2 ? (pairs ? CFG_PF | CFG_TMA : CFG_TWS) : CFG_PF;
    if (!pairs) return pass == 2 ? 0 : CFG_TWS;
    return pass == 1 ? CFG_TWS : CFG_TWS | CFG_PF | CFG_TMA;
}

// One launch configuration c = {E elements per thread, fused passes (1 when eligible, preferring a
// compile-time length; 2 when eligible, runtime stage structure; 0 never),
// options of pass 1, 2, 3 (CFG_* bits: shared-memory twiddles when they fit, prefetch when it
// fits (fused only), one transform per CTA)}.  An option that does not fit is dropped (twiddles
// first, then prefetch).  Returns false if the configuration does not exist for this plan.
static bool configure(conv_plan_s *p, const Candidate &c, int smem_optin, int sms)
{
    const int E = c[0], fused_pref = c[1];
    const int M = p->M, n = p->n;
    const size_t esz = p->prec == CONV_P_FP64 ? 16 : 8;
    const size_t per = (size_t)(p->prec == CONV_P_FP64 ? padded_len<double>(M) : padded_len<float>(M)) * esz;
    FFTDesc d;
    if (!factorize(M, E, d)) return false;
    int maxT = max_threads(p->prec, E);
    int tpt;
    if (E > 0) {
        if (M % E) return false;
        tpt = M / E;
    } else {
        tpt = generic_tpt(d);
    }
    if (tpt > maxT) return false;
    // compile-time lengths only for n = L/2 or n = L/3 (their transforms prune the zero
    // extension and the crop)
    const int ed = fused_pref != 0 ? fused_edges(p->prec, E, d, fused_pref == 1 ? n : 0) : 0;
    const bool fused = ed != 0;
    if (p->prec == CONV_P_FP64 && E == 16 && ed < 1000) return false;  // no runtime FP64 E = 16 kernels
    if (ed >= 1000) {
        // the compile-time-length kernels: radix-16 stages (L = 2^l; radix 8 and 3 for L = 3 2^l,
        // as factorize gives already), their launch bound
        if (ed < 2000 && !factorize(M, E, d, true, p->prec == CONV_P_FP64)) return false;
        maxT = std::min(maxT, static_max_threads(ed));
        if (tpt > maxT) return false;
    }
    // twiddle bytes in shared memory (TWS): the whole table, or all but the last stage's blocks
    const size_t twb = (size_t)(tw_split_ed(ed, (int)(esz / 2)) ? d.toff[d.nst - 1] : d.tw_len) * esz;
    // Staging per group (fused passes), by pass:
    //   pass 1: prefetched input rows (n elements V, rounded to 128 B), then with TMA stores the
    //           row pair's spectrum pairs, nbox x TMA_ROWS x 2 elements;
    //   pass 2: the prefetched column (n elements);
    //   pass 3: the row's spectrum: row-pair / (Wr, Wi) pairs for k <= M/2 (2 h, or the TMA boxes'
    //           nbox x TMA_ROWS x 2), or all M values (C2C).
    const size_t nbox_b = (size_t)((p->h + TMA_ROWS - 1) / TMA_ROWS) * TMA_ROWS * 2 * esz;
    auto stage_bytes = [&](int pass, bool pairs, bool pf, bool tma) -> size_t {
        if (pass == 0) return (pf ? round128((size_t)n * esz) : 0) + (tma ? nbox_b : 0);
        if (pass == 1) return pf ? (size_t)n * esz : 0;
        if (!pf) return 0;
        if (!pairs) return (size_t)M * esz;
        return tma ? nbox_b : 2 * (size_t)p->h * esz;
    };
    // pairs: the pass works on 16/32-byte spectrum pairs (R2R, split R2C) and may use TMA
    auto shape = [&](int cfg, int pass, bool pairs, int nbuf, LaunchShape &S) -> bool {
        const size_t pb = per * nbuf;
        bool tws = (cfg & CFG_TWS) && E > 0;
        bool pf = fused && (cfg & CFG_PF);
        bool tma = fused && pairs && (cfg & CFG_TMA) && (pass == 0 || (pass == 2 && pf));
        auto G_now = [&] { return max_groups(maxT, tpt, tws ? twb : 0, pb, stage_bytes(pass, pairs, pf, tma), smem_optin); };
        int G = G_now();
        if (G < 1 && tws) {
            tws = false;
            G = G_now();
        }
        if (G < 1 && tma) {
            tma = false;
            G = G_now();
        }
        if (G < 1 && pf) {
            pf = false;
            tma = false;
            G = G_now();
        }
        if (G < 1) return false;
        if (cfg & CFG_ONE) G = 1;
        const size_t sb = stage_bytes(pass, pairs, pf, tma);
        S.tpt = tpt;
        S.groups = G;
        S.pp = false;
        S.one = false;
        S.tws = tws;
        S.pf = pf;
        S.tma = tma;
        S.stage = (int)(sb / esz);
        S.smem = pass_smem(tws ? twb : 0, pb, sb, G);
        int bps = 1;
        if (fused)
            WSC_DISPATCH_FUSED(p->prec, E, ed, tws, bps = (blocks_per_sm_fused<T_, E_, ED_, W_>(tpt * G, S.smem)));
        else
            WSC_DISPATCH(p->prec, E, tws, bps = (blocks_per_sm<T_, E_, W_>(tpt * G, S.smem)));
        S.max_ctas = bps * sms;
        return true;
    };
    int opt[3];
    for (int k = 0; k < 3; ++k) opt[k] = c[2 + k] == CFG_DEFAULT ? default_options(p, ed, k) : c[2 + k];
    LaunchShape R, C, I;
    // R2C with complex ghat runs the split pipeline when its pass 2 fits two buffers per CTA.
    // Where two lines do not fit one CTA (FP64 at L = 8192), the compile-time lengths run it with
    // one buffer and a global scratch line per CTA group (after the spectra in the workspace:
    // workspace_bytes counts them).  Otherwise the C2C layout.
    const bool cplx_r2c = p->io == CONV_IO_R2C && p->complex_ghat;
    p->split_scratch_elems = 0;
    bool split = false;
    if (fused) {
        split = cplx_r2c && shape(opt[1], 1, false, 2, C);
        const char *one_env = getenv("WSCONV_SPLIT_ONE");  // 0: never, 1: even where two buffers fit
        const int one_mode = one_env ? atoi(one_env) : -1;
        if (cplx_r2c && split_one_ed(ed) && one_mode != 0 && (!split || one_mode == 1)) {
            LaunchShape C1;
            if (shape(opt[1], 1, false, 1, C1)) {
                C1.one = true;
                C = C1;
                split = true;
                p->split_scratch_elems = (size_t)C1.max_ctas * C1.groups * M;
            }
        }
        const bool pairs = p->io == CONV_IO_R2R || split;
        // the lengths with ping-pong kernels (R2R passes, and the split pipeline's pass 1): two
        // buffers per group when that costs none of the pass's options or groups.  By default
        // passes 1 and 2 (n = 4096, batch 16: pass 1 1.633 -> 1.595 ms, pass 2 3.221 -> 3.134 ms;
        // pass 3 1.342 -> 1.404 ms, so not pass 3).  WSCONV_PP selects the passes (bits 1, 2, 4
        // for passes 1, 2, 3; 0 turns it off).
        const char *pp_env = getenv("WSCONV_PP");
        const int pp_mask = pingpong_ed(ed, (int)(esz / 2)) ? (pp_env ? atoi(pp_env) : 3) : 0;
        auto shape_pp = [&](int cfg, int pass, bool prs, LaunchShape &S) -> bool {
            if (!shape(cfg, pass, prs, 1, S)) return false;
            LaunchShape two;
            if ((pp_mask >> pass) & 1 && shape(cfg, pass, prs, 2, two) && two.tws == S.tws && two.pf == S.pf &&
                two.tma == S.tma && two.groups == S.groups) {
                two.pp = true;
                S = two;
            }
            return true;
        };
        const bool r2r = p->io == CONV_IO_R2R;
        if (!(pairs ? shape_pp(opt[0], 0, pairs, R) : shape(opt[0], 0, pairs, 1, R)) ||
            (!split && !(r2r ? shape_pp(opt[1], 1, false, C) : shape(opt[1], 1, false, 1, C))) ||
            !(r2r ? shape_pp(opt[2], 2, pairs, I) : shape(opt[2], 2, pairs, 1, I)))
            return false;
    } else {
        if (!shape(opt[0], 0, false, 1, R)) return false;
        C = I = R;  // the plain kernels share one twiddle option and shape
    }
    p->r2c_split = split;
    p->elems = E;
    p->tws = R.tws;
    p->fft = d;
    p->ed = ed;
    p->fused = fused;
    p->rows = R;
    p->cols = C;
    p->inv = I;
    return true;
}


static conv_status device_limits(conv_plan_s *p, int &smem_optin, int &sms)
{
    const int dev = p->device;
    WSC_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    WSC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // once per device; plans may be created from several threads (the serving runtime's)
    static std::mutex mu;
    static bool attrs_set[64] = {false};
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(mu);
        if (!attrs_set[dev]) {
            conv_status rc = set_all_attrs(smem_optin);
            if (rc != CONV_OK) return rc;
            attrs_set[dev] = true;
        }
    }
    const int M = p->M;
    const size_t esz = p->prec == CONV_P_FP64 ? 16 : 8;
    const size_t per = (size_t)(p->prec == CONV_P_FP64 ? padded_len<double>(M) : padded_len<float>(M)) * esz;
    if (per > (size_t)smem_optin)
        return fail(CONV_EUNSUPPORTED, "transform length " + std::to_string(M) +
                                           " exceeds one CTA's shared memory at this precision");
    return CONV_OK;
}

// Default configuration: the first candidate E that exists, fused passes and the default options
// of each pass.  Environment overrides for experiments: WSCONV_ELEMS, WSCONV_FUSED (0/1),
// WSCONV_TWS (0: no pass keeps its table in shared memory), WSCONV_PF (0/1: prefetch in no / every
// pass), WSCONV_GROUPS (1: one transform per CTA), WSCONV_CFG ("r,c,i": the CFG_* bits per pass).
// Lines that one CTA cannot hold (or, with WSCONV_LONG_LINES=1, any line: tests) take the
// four-step FP64 line pipeline of fsmask.cu (p->long_lines).
static bool factor_235(int L)
{
    for (int f : {2, 3, 5})
        while (L % f == 0) L /= f;
    return L == 1;
}

conv_status select_transform(conv_plan_s *p)
{
    int smem_optin = 0, sms = 0;
    conv_status rc = device_limits(p, smem_optin, sms);
    const char *force_long = getenv("WSCONV_LONG_LINES");
    if ((rc == CONV_EUNSUPPORTED || (force_long && atoi(force_long) == 1)) && factor_235(p->M)) {
        p->long_lines = true;
        p->fused = false;
        return CONV_OK;
    }
    if (rc != CONV_OK) return rc;
    const int *cand = p->prec == CONV_P_FP64 ? kElems64 : kElems32;
    const int ncand = p->prec == CONV_P_FP64 ? (int)(sizeof kElems64 / sizeof(int)) : (int)(sizeof kElems32 / sizeof(int));
    auto env = [](const char *k, int dflt) {
        const char *v = getenv(k);
        return v ? atoi(v) : dflt;
    };
    const int force_e = env("WSCONV_ELEMS", -1), tws = env("WSCONV_TWS", 1), pf = env("WSCONV_PF", -1);
    const int one = env("WSCONV_GROUPS", 0) == 1;
    int cfg3[3] = {-1, -1, -1};
    if (const char *v = getenv("WSCONV_CFG")) sscanf(v, "%d,%d,%d", &cfg3[0], &cfg3[1], &cfg3[2]);
    for (int i = 0; i < ncand; ++i) {
        if (force_e >= 0 && cand[i] != force_e) continue;
        Candidate c = {cand[i], env("WSCONV_FUSED", 1), CFG_DEFAULT, CFG_DEFAULT, CFG_DEFAULT};
        for (int k = 0; k < 3; ++k) {
            int &o = c[2 + k];
            if (!tws || pf >= 0 || one) o = CFG_TWS;  // an override starts from twiddles in shared memory
            if (!tws) o &= ~CFG_TWS;
            if (pf == 1) o |= CFG_PF;
            if (one) o |= CFG_ONE;
            if (cfg3[k] >= 0) o = cfg3[k];
        }
        if (configure(p, c, smem_optin, sms)) return CONV_OK;
    }
    if (factor_235(p->M)) {  // fits shared memory but needs more threads than one CTA has
        p->long_lines = true;
        p->fused = false;
        return CONV_OK;
    }
    return fail(CONV_EUNSUPPORTED, "transform length " + std::to_string(p->M) + " is not 2^a 3^b 5^c");
}

// The autotuner's search space, as families that share E and fused: within a family the options
// of the three passes are chosen independently (each pass timed on its own), so a family lists
// the distinct per-pass option sets, all passes taking the same one.
std::vector<std::vector<Candidate>> transform_families(conv_plan_s *p)
{
    std::vector<std::vector<Candidate>> out;
    if (p->long_lines) return out;
    int smem_optin = 0, sms = 0;
    if (device_limits(p, smem_optin, sms) != CONV_OK) return out;
    const int *cand = p->prec == CONV_P_FP64 ? kElems64 : kElems32;
    const int ncand = p->prec == CONV_P_FP64 ? (int)(sizeof kElems64 / sizeof(int)) : (int)(sizeof kElems32 / sizeof(int));
    conv_plan_s probe = *p;
    probe.tev_used.clear();
    probe.tev_free.clear();
    for (int i = 0; i < ncand; ++i) {
        int ed_static = -1;
        for (int fu : {1, 2, 0}) {
            std::vector<Candidate> fam;
            std::vector<std::array<int, 12>> seen;  // distinct (tws, pf, tma, groups) of the three passes
            for (int cfg = 0; cfg < (fu ? 16 : 2); ++cfg) {
                const Candidate c = {cand[i], fu, cfg, cfg, cfg};
                if (!configure(&probe, c, smem_optin, sms) || probe.fused != (fu != 0)) continue;
                if (fu == 1) ed_static = probe.ed;
                if (fu == 2 && probe.ed == ed_static) break;  // no compile-time length: same as fu = 1
                const std::array<int, 12> key = {probe.rows.tws, probe.rows.pf, probe.rows.tma, probe.rows.groups,
                                                 probe.cols.tws, probe.cols.pf, probe.cols.tma, probe.cols.groups,
                                                 probe.inv.tws,  probe.inv.pf,  probe.inv.tma,  probe.inv.groups};
                bool dup = false;
                for (auto &k : seen) dup = dup || k == key;
                if (dup) continue;
                seen.push_back(key);
                fam.push_back(c);
            }
            if (!fam.empty()) out.push_back(fam);
        }
    }
    return out;
}

conv_status apply_candidate(conv_plan_s *p, const Candidate &c)
{
    int smem_optin = 0, sms = 0;
    conv_status rc = device_limits(p, smem_optin, sms);
    if (rc != CONV_OK) return rc;
    if (!configure(p, c, smem_optin, sms)) return fail(CONV_EINVAL, "candidate does not apply");
    return CONV_OK;
}

conv_status launch_pipeline(conv_plan_s *p, const void *u, const void *mask, void *out, int batch,
                            double alpha_re, double alpha_im, double beta, void *ws, cudaStream_t st)
{
    if (p->long_lines) return long_lines_apply(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
    conv_status rc = CONV_OK;
    if (p->fused)
        WSC_DISPATCH_FUSED(p->prec, p->elems, p->ed, false,
                           rc = (run_fused<T_, E_, ED_>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st)));
    else
        WSC_DISPATCH(p->prec, p->elems, p->tws,
                     rc = (run_pipeline<T_, E_, W_>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st)));
    return rc;
}

}  // namespace wsc
