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

#include <cstdlib>
#include <string>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

// ============================================================================ host side
// Per-thread element counts with exact (unguarded) kernels, in order of preference.  A count E
// admits radices dividing E; FP64 prefers radix-4 stages (E = 12 or 8, 1024 threads), FP32 radix-8
// (E = 24 or 16).  E = 0 is the generic guarded path (any 2^a 3^b 5^c).
static const int kElems64[] = {12, 8, 24, 0};
static const int kElems32[] = {24, 16, 12, 0};

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
    case 12: return maxt<float, 12>::v;
    case 16: return maxt<float, 16>::v;
    case 24: return maxt<float, 24>::v;
    default: return maxt<float, 0>::v;
    }
}

// Radix sequence for L = 2^p 3^q 5^r whose radices divide E (E = 0: any of 8, 4, 2, 3, 5):
// power-of-two radices first (8s when allowed, else 4s), then 3s, then 5s.
static bool factorize(int L, int E, FFTDesc &d)
{
    int rem = L, p2 = 0, p3 = 0, p5 = 0;
    while (rem % 2 == 0) { rem /= 2; ++p2; }
    while (rem % 3 == 0) { rem /= 3; ++p3; }
    while (rem % 5 == 0) { rem /= 5; ++p5; }
    if (rem != 1) return false;
    auto ok = [E](int r) { return E == 0 || E % r == 0; };
    if ((p3 && !ok(3)) || (p5 && !ok(5))) return false;
    std::vector<int> R;
    if (ok(8)) {
        for (int i = 0; i < p2 / 3; ++i) R.push_back(8);
        if (p2 % 3 == 2) R.push_back(ok(4) ? 4 : 2), (ok(4) ? (void)0 : R.push_back(2));
        if (p2 % 3 == 1) R.push_back(2);
    } else if (ok(4)) {
        for (int i = 0; i < p2 / 2; ++i) R.push_back(4);
        if (p2 % 2) R.push_back(2);
    } else {
        if (p2 && !ok(2)) return false;
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
    for (int s = 0; s < d.nst; ++s) {
        d.R[s] = R[s];
        d.Ns[s] = (int)Ns;
        d.tws[s] = (int)(L / (Ns * R[s]));
        d.mag[s] = ((1ULL << 40) + (unsigned long long)Ns - 1) / (unsigned long long)Ns;
        Ns *= R[s];
    }
    return true;
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

conv_status select_transform(conv_plan_s *p)
{
    int dev = p->device;
    int smem_optin = 0;
    WSC_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    static bool attrs_set[64] = {false};
    if (dev >= 0 && dev < 64 && !attrs_set[dev]) {
        conv_status rc = CONV_OK;
        for (int E : kElems64) {
            if (rc != CONV_OK) break;
            rc = E == 8 ? set_attrs<double, 8>(smem_optin) : E == 12 ? set_attrs<double, 12>(smem_optin)
               : E == 24 ? set_attrs<double, 24>(smem_optin) : set_attrs<double, 0>(smem_optin);
        }
        for (int E : kElems32) {
            if (rc != CONV_OK) break;
            rc = E == 12 ? set_attrs<float, 12>(smem_optin) : E == 16 ? set_attrs<float, 16>(smem_optin)
               : E == 24 ? set_attrs<float, 24>(smem_optin) : set_attrs<float, 0>(smem_optin);
        }
        if (rc != CONV_OK) return rc;
        attrs_set[dev] = true;
    }
    const int M = p->M;
    const size_t esz = p->prec == CONV_P_FP64 ? 16 : 8;
    const size_t per = (size_t)(p->prec == CONV_P_FP64 ? padded_len<double>(M) : padded_len<float>(M)) * esz;
    if (per > (size_t)smem_optin)
        return fail(CONV_EUNSUPPORTED, "transform length M=" + std::to_string(M) +
                                           " exceeds one CTA's shared memory at this precision");
    const int *cand = p->prec == CONV_P_FP64 ? kElems64 : kElems32;
    // optional overrides for tuning experiments: WSCONV_ELEMS (per-thread count), WSCONV_GROUPS
    const char *env_e = getenv("WSCONV_ELEMS"), *env_g = getenv("WSCONV_GROUPS");
    const int force_e = env_e ? atoi(env_e) : -1, force_g = env_g ? atoi(env_g) : 0;
    for (int i = 0; i < 4; ++i) {
        const int E = cand[i];
        if (force_e >= 0 && E != force_e) continue;
        FFTDesc d;
        if (!factorize(M, E, d)) continue;
        const int maxT = max_threads(p->prec, E);
        int tpt;
        if (E > 0) {
            if (M % E) continue;
            tpt = M / E;
        } else {
            tpt = generic_tpt(d);
        }
        if (tpt > maxT) continue;
        int G = std::max(1, maxT / tpt);
        G = std::min<int>(G, (int)(smem_optin / per));
        G = std::min(G, 8);
        if (force_g > 0 && force_g <= G) G = force_g;
        p->elems = E;
        p->fft = d;
        p->rows.tpt = p->cols.tpt = tpt;
        p->rows.groups = p->cols.groups = G;
        p->rows.smem = p->cols.smem = per * G;
        return CONV_OK;
    }
    return fail(CONV_EUNSUPPORTED, "M = " + std::to_string(M) +
                                       " is not 2^a 3^b 5^c or needs more threads than one CTA has");
}

conv_status launch_pipeline(conv_plan_s *p, const void *u, const void *mask, void *out, int batch,
                            double alpha_re, double alpha_im, double beta, void *ws, cudaStream_t st)
{
    if (p->prec == CONV_P_FP64) {
        switch (p->elems) {
        case 8: return run_pipeline<double, 8>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
        case 12: return run_pipeline<double, 12>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
        case 24: return run_pipeline<double, 24>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
        default: return run_pipeline<double, 0>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
        }
    }
    switch (p->elems) {
    case 12: return run_pipeline<float, 12>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
    case 16: return run_pipeline<float, 16>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
    case 24: return run_pipeline<float, 24>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
    default: return run_pipeline<float, 0>(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws, st);
    }
}

}  // namespace wsc
