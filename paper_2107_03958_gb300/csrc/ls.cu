// ls.cu -- Lippmann-Schwinger Nystrom solve (Sec. 3.3):  u + kappa^2 A_n(m u) = f on G_n
// (eq. (descretls)) by matrix-free restarted GMRES.
//
// The matvec is the convolution pipeline itself: L v = v + kappa^2 A_n(m v) is one
// conv_apply_axpby call (m applied at the row-pass load, the identity and kappa^2 at the final
// row-pass store).  Arnoldi uses classical Gram-Schmidt with one re-orthogonalisation; the
// Hessenberg matrix, Givens rotations and the triangular solve stay on the device in FP64, and
// the host reads one 8-byte residual estimate per iteration.  All reductions use a fixed
// partition and order, so a solve is bit-for-bit repeatable.
//
// Mixed precision (FP32 plan, refine != 0): iterative refinement
//   r = f - L64 x (FP64 operator),  solve L32 d = r to inner_tol by GMRES (FP32 matvec, FP64
//   Arnoldi),  x += d,  until ||r|| / ||f|| <= tol.
#include <cmath>
#include <mutex>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

#define LS_RED_BLOCKS 296  // 2 x 148..152 SMs: fixed partition for deterministic reductions
#define LS_RED_THREADS 256
#define LS_MAX_RESTART 1000  // Krylov basis (restart + 1) n^2 complex values; Hessenberg (restart + 1) restart

// Dot products of NV basis vectors V_i0 ... V_i0+NV-1 with w over this block's slice [lo, hi):
// one sweep that reads w once for the NV of them.  Each thread issues the loads of four elements
// (and of every vector) before it uses them, so enough reads are in flight to keep HBM busy;
// the sums still run over t in the order of a plain loop, so the result is the same bit for bit.
template <int NV>
__device__ __forceinline__ void dots_sweep(const double2 *__restrict__ V, size_t ldv, int i0,
                                           const double2 *__restrict__ w, long long lo, long long hi,
                                           double2 (*red)[LS_RED_THREADS / 32], double2 *__restrict__ partial)
{
    const long long S = blockDim.x;
    double sr[NV], si[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) sr[k] = si[k] = 0.0;
    long long t = lo + threadIdx.x;
    for (; t + 3 * S < hi; t += 4 * S) {
        double2 b[4], a[NV][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = w[t + u * S];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int u = 0; u < 4; ++u) a[k][u] = V[(size_t)(i0 + k) * ldv + t + u * S];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                sr[k] += a[k][u].x * b[u].x + a[k][u].y * b[u].y;
                si[k] += a[k][u].x * b[u].y - a[k][u].y * b[u].x;
            }
    }
    for (; t < hi; t += S) {
        const double2 b = w[t];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double2 a = V[(size_t)(i0 + k) * ldv + t];
            sr[k] += a.x * b.x + a.y * b.y;
            si[k] += a.x * b.y - a.y * b.x;
        }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            sr[k] += __shfl_down_sync(0xffffffffu, sr[k], o);
            si[k] += __shfl_down_sync(0xffffffffu, si[k], o);
        }
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = make_double2(sr[k], si[k]);
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        double ar = 0, ai = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            ar += red[k][q].x;
            ai += red[k][q].y;
        }
        partial[(size_t)(i0 + k) * gridDim.x + blockIdx.x] = make_double2(ar, ai);
    }
    __syncthreads();
}

// partial[i * nb + blk] = sum_{t in blk's slice} conj(V_i[t]) w[t], i < cnt; two vectors per sweep
__global__ void __launch_bounds__(LS_RED_THREADS) k_multidot(const double2 *__restrict__ V, size_t ldv, int cnt,
                                                             const double2 *__restrict__ w, long long N,
                                                             double2 *__restrict__ partial)
{
    __shared__ double2 red[2][LS_RED_THREADS / 32];
    const long long chunk = (N + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
    int i = 0;
    for (; i + 2 <= cnt; i += 2) dots_sweep<2>(V, ldv, i, w, lo, hi, red, partial);
    if (i < cnt) dots_sweep<1>(V, ldv, i, w, lo, hi, red, partial);
}

// out[i] = sum_blk partial[i * nb + blk] (+= if accumulate); one warp per i, fixed order.
__global__ void k_finalize_dots(const double2 *__restrict__ partial, int nb, int cnt,
                                double2 *__restrict__ out, int accumulate)
{
    int i = blockIdx.x;
    if (i >= cnt) return;
    double sr = 0, si = 0;
    for (int b = threadIdx.x; b < nb; b += 32) {
        sr += partial[(size_t)i * nb + b].x;
        si += partial[(size_t)i * nb + b].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (threadIdx.x == 0) {
        if (accumulate) {
            out[i].x += sr;
            out[i].y += si;
        } else out[i] = make_double2(sr, si);
    }
}

// w -= sum_{i<cnt} V_i h_i
__global__ void k_sub_combination(const double2 *__restrict__ V, size_t ldv, int cnt,
                                  const double2 *__restrict__ h, double2 *__restrict__ w, long long N)
{
    extern __shared__ double2 hs[];  // cnt coefficients
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        double2 acc = w[t];
        int i = 0;
        // four vectors' loads issued before their uses (same subtraction order as one at a time)
        for (; i + 4 <= cnt; i += 4) {
            double2 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = V[(size_t)(i + k) * ldv + t];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double2 c = hs[i + k];
                acc.x -= v[k].x * c.x - v[k].y * c.y;
                acc.y -= v[k].x * c.y + v[k].y * c.x;
            }
        }
        for (; i < cnt; ++i) {
            double2 v = V[(size_t)i * ldv + t], c = hs[i];
            acc.x -= v.x * c.x - v.y * c.y;
            acc.y -= v.x * c.y + v.y * c.x;
        }
        w[t] = acc;
    }
}

// x += sum_{i<cnt} V_i y_i
__global__ void k_add_combination(const double2 *__restrict__ V, size_t ldv, int cnt,
                                  const double2 *__restrict__ y, double2 *__restrict__ x, long long N)
{
    extern __shared__ double2 ys[];  // cnt coefficients
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        double2 acc = x[t];
        int i = 0;
        for (; i + 4 <= cnt; i += 4) {
            double2 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = V[(size_t)(i + k) * ldv + t];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double2 c = ys[i + k];
                acc.x += v[k].x * c.x - v[k].y * c.y;
                acc.y += v[k].x * c.y + v[k].y * c.x;
            }
        }
        for (; i < cnt; ++i) {
            double2 v = V[(size_t)i * ldv + t], c = ys[i];
            acc.x += v.x * c.x - v.y * c.y;
            acc.y += v.x * c.y + v.y * c.x;
        }
        x[t] = acc;
    }
}

// dst = src * (1/sqrt(nrm2->x)) where nrm2 holds a squared norm (x component)
__global__ void k_scale_by_invnorm(const double2 *__restrict__ src, double2 *__restrict__ dst,
                                   const double2 *__restrict__ nrm2, long long N)
{
    double nn = sqrt(nrm2->x);
    double s = nn > 0 ? 1.0 / nn : 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        double2 v = src[t];
        dst[t] = make_double2(v.x * s, v.y * s);
    }
}

// r = f - r (r holds L x on entry)
// x *= a (a real)
__global__ void k_scale_real(double2 *__restrict__ x, double a, long long N)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        const double2 v = x[t];
        x[t] = make_double2(v.x * a, v.y * a);
    }
}

__global__ void k_rsub(const double2 *__restrict__ f, double2 *__restrict__ r, long long N)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        double2 a = f[t], b = r[t];
        r[t] = make_double2(a.x - b.x, a.y - b.y);
    }
}

__global__ void k_axpy_real(double2 *__restrict__ x, const double2 *__restrict__ d, long long N)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        double2 a = x[t], b = d[t];
        x[t] = make_double2(a.x + b.x, a.y + b.y);
    }
}

__global__ void k_d2f(const double *__restrict__ in, float *__restrict__ out, long long N)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x)
        out[t] = (float)in[t];
}

__global__ void k_f2d(const float *__restrict__ in, double *__restrict__ out, long long N)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x)
        out[t] = (double)in[t];
}

// Small dense state of one GMRES cycle with restart R, device resident in one allocation of
// gmres_state_elems(R) complex values; the struct itself (its pointers into that allocation) is
// passed to the kernels by value.
struct GmresState {
    double2 *H;     // (R+1) x R, H[i * R + j], i <= j + 1 (rotated in place)
    double2 *cs, *sn;  // R rotations
    double2 *e;     // R + 1
    double2 *y;     // R
    double2 *hcol;  // R + 1: h of the current column (CGS accumulations)
    double2 *nrm2;  // squared norm scratch (x component)
    double *res;    // |e[j+1]|
    int R;
};

static size_t gmres_state_elems(int R) { return (size_t)(R + 1) * R + 2 * (size_t)R + (R + 1) + R + (R + 1) + 2; }

static GmresState gmres_state_view(double2 *base, int R)
{
    GmresState g;
    g.R = R;
    g.H = base;
    g.cs = g.H + (size_t)(R + 1) * R;
    g.sn = g.cs + R;
    g.e = g.sn + R;
    g.y = g.e + (R + 1);
    g.hcol = g.y + R;
    g.nrm2 = g.hcol + (R + 1);
    g.res = reinterpret_cast<double *>(g.nrm2 + 1);
    return g;
}

// e = [beta, 0, ...]; beta from the squared norm in st->nrm2
__global__ void k_gmres_init(GmresState st)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i <= st.R; ++i) st.e[i] = make_double2(0, 0);
        st.e[0] = make_double2(sqrt(st.nrm2->x), 0);
        *st.res = sqrt(st.nrm2->x);
    }
}

// Column j of H from hcol (j+1 entries) and the new norm; apply the previous rotations, form
// rotation j, update e and the residual estimate.
__global__ void k_gmres_givens(GmresState st, int j, int ldh)
{
    if (threadIdx.x != 0) return;
    for (int i = 0; i <= j; ++i) st.H[i * ldh + j] = st.hcol[i];
    double hn = sqrt(st.nrm2->x);
    st.H[(j + 1) * ldh + j] = make_double2(hn, 0);
    for (int i = 0; i < j; ++i) {
        double2 h0 = st.H[i * ldh + j], h1 = st.H[(i + 1) * ldh + j], c = st.cs[i], s = st.sn[i];
        // [h0; h1] <- [conj(c) h0 + conj(s) h1; -s h0 + c h1]
        double2 a = make_double2(c.x * h0.x + c.y * h0.y + s.x * h1.x + s.y * h1.y,
                                 c.x * h0.y - c.y * h0.x + s.x * h1.y - s.y * h1.x);
        double2 b = make_double2(-(s.x * h0.x - s.y * h0.y) + (c.x * h1.x - c.y * h1.y),
                                 -(s.x * h0.y + s.y * h0.x) + (c.x * h1.y + c.y * h1.x));
        st.H[i * ldh + j] = a;
        st.H[(i + 1) * ldh + j] = b;
    }
    double2 h0 = st.H[j * ldh + j], h1 = st.H[(j + 1) * ldh + j];
    double r = sqrt(h0.x * h0.x + h0.y * h0.y + h1.x * h1.x + h1.y * h1.y);
    double2 c = r > 0 ? make_double2(h0.x / r, h0.y / r) : make_double2(1, 0);
    double2 s = r > 0 ? make_double2(h1.x / r, h1.y / r) : make_double2(0, 0);
    st.cs[j] = c;
    st.sn[j] = s;
    st.H[j * ldh + j] = make_double2(r, 0);
    st.H[(j + 1) * ldh + j] = make_double2(0, 0);
    double2 ej = st.e[j];
    st.e[j + 1] = make_double2(-(s.x * ej.x - s.y * ej.y), -(s.x * ej.y + s.y * ej.x));
    st.e[j] = make_double2(c.x * ej.x + c.y * ej.y, c.x * ej.y - c.y * ej.x);
    *st.res = sqrt(st.e[j + 1].x * st.e[j + 1].x + st.e[j + 1].y * st.e[j + 1].y);
}

// back substitution H(0:k, 0:k) y = e(0:k)
__global__ void k_gmres_solve(GmresState st, int k, int ldh)
{
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = st.e[i];
        for (int t = i + 1; t < k; ++t) {
            double2 h = st.H[i * ldh + t], yt = st.y[t];
            acc.x -= h.x * yt.x - h.y * yt.y;
            acc.y -= h.x * yt.y + h.y * yt.x;
        }
        double2 d = st.H[i * ldh + i];
        double dd = d.x * d.x + d.y * d.y;
        st.y[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
}

struct LsWork {
    double2 *V = nullptr;     // (restart+1) x N
    double2 *w = nullptr, *r = nullptr, *d = nullptr, *x64 = nullptr;
    float2 *v32 = nullptr, *w32 = nullptr;
    float *m32 = nullptr;
    double2 *partial = nullptr;
    double2 *gsbuf = nullptr;  // the GMRES state's allocation
    GmresState gs{};
    double *host_res = nullptr;  // pinned
    // several right-hand sides: their normalised copies, and the matvecs' spectrum workspaces
    // when the batch exceeds the plans' own
    double2 *fsc = nullptr;
    void *cws = nullptr, *cws64 = nullptr;
};

// N: the (stacked) Krylov vector length, NN = n^2 (the contrast), batch: right-hand sides, with
// cws/cws64 bytes of matvec workspace (0: the plans' own suffices).
static bool alloc_work(LsWork &W, long long N, long long NN, int batch, size_t cws, size_t cws64, int restart,
                       bool mixed)
{
    bool ok = dev_alloc(&W.V, (size_t)(restart + 1) * N * sizeof(double2)) == cudaSuccess &&
              dev_alloc(&W.w, N * sizeof(double2)) == cudaSuccess &&
              dev_alloc(&W.r, N * sizeof(double2)) == cudaSuccess &&
              dev_alloc(&W.d, N * sizeof(double2)) == cudaSuccess &&
              dev_alloc(&W.partial, (size_t)(restart + 1) * LS_RED_BLOCKS * sizeof(double2)) == cudaSuccess &&
              dev_alloc(&W.gsbuf, gmres_state_elems(restart) * sizeof(double2)) == cudaSuccess &&
              (W.host_res = pinned_slot()) != nullptr;
    if (ok && mixed)
        ok = dev_alloc(&W.x64, N * sizeof(double2)) == cudaSuccess &&
             dev_alloc(&W.v32, N * sizeof(float2)) == cudaSuccess &&
             dev_alloc(&W.w32, N * sizeof(float2)) == cudaSuccess &&
             dev_alloc(&W.m32, NN * sizeof(float)) == cudaSuccess;
    if (ok && batch > 1) ok = dev_alloc(&W.fsc, N * sizeof(double2)) == cudaSuccess;
    if (ok && cws) ok = dev_alloc(&W.cws, cws) == cudaSuccess;
    if (ok && cws64) ok = dev_alloc(&W.cws64, cws64) == cudaSuccess;
    if (!ok) cudaGetLastError();
    if (ok) W.gs = gmres_state_view(W.gsbuf, restart);
    return ok;
}

static void free_work(LsWork &W)
{
    dev_free(W.V);
    dev_free(W.w);
    dev_free(W.r);
    dev_free(W.d);
    dev_free(W.x64);
    dev_free(W.v32);
    dev_free(W.w32);
    dev_free(W.m32);
    dev_free(W.fsc);
    dev_free(W.cws);
    dev_free(W.cws64);
    dev_free(W.partial);
    dev_free(W.gsbuf);
    pinned_slot_release(W.host_res);
    W = LsWork();
}

// A plan's Krylov workspace, kept from one solve to the next (allocation and the device-wide sync
// of cudaFree would otherwise cost each solve).  One solve at a time uses it; a solve that finds it
// in use allocates its own.
struct LsCache {
    std::mutex mu;
    LsWork W;
    long long N = 0;                       // Krylov vector length (batch n^2)
    int batch = 0;
    int restart = 0;
    bool mixed = false;
    double *m64 = nullptr;                 // the solve's contrast, copied in (the graphs read it here)
    std::vector<cudaGraphExec_t> iter;     // iteration j of a cycle, captured on first use
    cudaStream_t cap = nullptr;            // private stream the captures run on (any caller stream,
                                           // the legacy one included, can launch the graphs)
};

static void drop_graphs(LsCache *c)
{
    for (auto &g : c->iter)
        if (g) cudaGraphExecDestroy(g);
    c->iter.clear();
}
static std::mutex g_ls_cache_mu;

void destroy_ls_cache(conv_plan_s *p)
{
    if (!p->ls_cache) return;
    drop_graphs(p->ls_cache);
    free_work(p->ls_cache->W);
    dev_free(p->ls_cache->m64);
    if (p->ls_cache->cap) cudaStreamDestroy(p->ls_cache->cap);
    delete p->ls_cache;
    p->ls_cache = nullptr;
}

struct Solver {
    conv_plan_s *p;        // matvec plan of the Krylov iterations
    conv_plan_s *p64;      // FP64 operator for true residuals
    const double *m64;
    double kappa2;
    long long N;           // Krylov vector length: batch x n^2
    int batch;             // right-hand sides stacked in one vector (one batched matvec)
    int restart;
    LsWork W;
    cudaStream_t st;
    int grid_elem;
    std::vector<cudaGraphExec_t> *graphs = nullptr;  // the cached workspace's iteration graphs, or none
    cudaStream_t cap_stream = nullptr;               // where those graphs are captured

    // w = L v with the Krylov plan (FP64 or FP32 matvec), v and w FP64.
    conv_status matvec(const double2 *v, double2 *w)
    {
        if (p->prec == CONV_P_FP64)
            return conv_apply_axpby(p, v, m64, w, batch, kappa2, 0.0, 1.0, W.cws, st);
        k_d2f<<<grid_elem, 256, 0, st>>>(reinterpret_cast<const double *>(v), reinterpret_cast<float *>(W.v32), 2 * N);
        conv_status rc = conv_apply_axpby(p, W.v32, W.m32, W.w32, batch, kappa2, 0.0, 1.0, W.cws, st);
        if (rc != CONV_OK) return rc;
        k_f2d<<<grid_elem, 256, 0, st>>>(reinterpret_cast<const float *>(W.w32), reinterpret_cast<double *>(w), 2 * N);
        return CONV_OK;
    }

    conv_status true_residual(const double2 *f, const double2 *x, double2 *r)
    {
        conv_status rc = conv_apply_axpby(p64, x, m64, r, batch, kappa2, 0.0, 1.0, p64 == p ? W.cws : W.cws64, st);
        if (rc != CONV_OK) return rc;
        k_rsub<<<grid_elem, 256, 0, st>>>(f, r, N);
        return CONV_OK;
    }

    // squared norm of v (len elements, default the Krylov length) into st->nrm2
    void norm2(const double2 *v, long long len = -1)
    {
        k_multidot<<<LS_RED_BLOCKS, LS_RED_THREADS, 0, st>>>(v, 0, 1, v, len < 0 ? N : len, W.partial);
        k_finalize_dots<<<1, 32, 0, st>>>(W.partial, LS_RED_BLOCKS, 1, W.gs.nrm2, 0);
    }

    // ||v|| of len elements, waited for
    double norm_of(const double2 *v, long long len)
    {
        norm2(v, len);
        k_gmres_init<<<1, 32, 0, st>>>(W.gs);
        return read_scalar(W.gs.res);
    }

    double read_scalar(const double *dptr)
    {
        cudaMemcpyAsync(W.host_res, dptr, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return *W.host_res;
    }

    // Arnoldi step j of a cycle: v_{j+1} from L v_j by CGS2, the Givens update of the Hessenberg
    // column, and the new residual estimate copied to the pinned host word (not yet waited for).
    conv_status enqueue_iteration(int j, int ldh)
    {
        double2 *vj = W.V + (size_t)j * N, *vn = W.V + (size_t)(j + 1) * N;
        conv_status rc = matvec(vj, W.w);
        if (rc != CONV_OK) return rc;
        // CGS with one re-orthogonalisation: h = V^H w; w -= V h; h2 = V^H w; w -= V h2
        for (int pass = 0; pass < 2; ++pass) {
            k_multidot<<<LS_RED_BLOCKS, LS_RED_THREADS, 0, st>>>(W.V, N, j + 1, W.w, N, W.partial);
            k_finalize_dots<<<j + 1, 32, 0, st>>>(W.partial, LS_RED_BLOCKS, j + 1, W.gs.hcol, pass);
            // subtract with this pass's coefficients only: recompute them into y scratch
            k_finalize_dots<<<j + 1, 32, 0, st>>>(W.partial, LS_RED_BLOCKS, j + 1, W.gs.y, 0);
            k_sub_combination<<<grid_elem, 256, (j + 1) * sizeof(double2), st>>>(W.V, N, j + 1, W.gs.y, W.w, N);
        }
        norm2(W.w);
        k_scale_by_invnorm<<<grid_elem, 256, 0, st>>>(W.w, vn, W.gs.nrm2, N);
        k_gmres_givens<<<1, 32, 0, st>>>(W.gs, j, ldh);
        WSC_CUDA(cudaMemcpyAsync(W.host_res, W.gs.res, sizeof(double), cudaMemcpyDeviceToHost, st));
        return CONV_OK;
    }

    // Step j as one graph launch when the workspace is the plan's: the ~17 launches of a step are
    // captured once and replayed, so the GPU does not wait on the host's launches after every
    // residual check.  Every pointer the step uses belongs to the plan or its cached workspace.
    conv_status run_iteration(int j, int ldh)
    {
        if (!graphs || p->timing) return enqueue_iteration(j, ldh);
        if ((int)graphs->size() <= j) graphs->resize(j + 1, nullptr);
        cudaGraphExec_t &ex = (*graphs)[j];
        if (!ex) {
            // capture on the private stream, after the work the caller's stream holds
            cudaGraph_t g = nullptr;
            WSC_CUDA(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaStream_t user = st;
            st = cap_stream;
            conv_status rc = enqueue_iteration(j, ldh);
            st = user;
            cudaError_t ce = cudaStreamEndCapture(cap_stream, &g);
            if (rc != CONV_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ce != cudaSuccess) return cuda_fail(ce, "capture of a GMRES step");
            ce = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                ex = nullptr;
                return cuda_fail(ce, "instantiation of a GMRES step");
            }
        }
        WSC_CUDA(cudaGraphLaunch(ex, st));
        return CONV_OK;
    }

    // GMRES on L z = b from z (FP64 device vectors) to ||b - L z|| <= tol_abs (Arnoldi estimate,
    // confirmed by the residual of the Krylov operator at restarts).
    // trust_estimate: return once the Arnoldi residual estimate reaches tol_abs, without forming
    // b - L z again (the inner solves of the refinement, whose outer FP64 residual checks them)
    conv_status gmres(const double2 *b, double2 *z, double tol_abs, int maxit, bool z_is_zero,
                      int &iters, int &cycles, double &res_out, bool trust_estimate = false)
    {
        const int ldh = W.gs.R;  // the state's allocation, which the cached step graphs were captured with
        while (true) {
            // r = b - L z
            if (z_is_zero) {
                cudaMemcpyAsync(W.r, b, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
            } else {
                conv_status rc = matvec(z, W.r);
                if (rc != CONV_OK) return rc;
                k_rsub<<<grid_elem, 256, 0, st>>>(b, W.r, N);
            }
            z_is_zero = false;
            norm2(W.r);
            k_gmres_init<<<1, 32, 0, st>>>(W.gs);
            double beta = read_scalar(W.gs.res);
            res_out = beta;
            if (!(beta == beta)) return fail(CONV_ENONFINITE, "GMRES residual is not finite");
            if (beta <= tol_abs) return CONV_OK;
            if (iters >= maxit) return fail(CONV_ENOTCONVERGED, "GMRES reached its iteration limit");
            k_scale_by_invnorm<<<grid_elem, 256, 0, st>>>(W.r, W.V, W.gs.nrm2, N);
            ++cycles;
            int j = 0;
            bool reached = false;
            for (; j < restart && iters < maxit; ++j) {
                conv_status rc = run_iteration(j, ldh);
                if (rc != CONV_OK) return rc;
                ++iters;
                WSC_CUDA(cudaStreamSynchronize(st));
                double res = *W.host_res;
                res_out = res;
                if (!(res == res)) return fail(CONV_ENONFINITE, "GMRES residual is not finite");
                if (res <= tol_abs) {
                    ++j;
                    reached = true;
                    break;
                }
            }
            k_gmres_solve<<<1, 32, 0, st>>>(W.gs, j, ldh);
            k_add_combination<<<grid_elem, 256, std::max(j, 1) * sizeof(double2), st>>>(W.V, N, j, W.gs.y, z, N);
            WSC_CUDA(cudaGetLastError());
            if (reached && trust_estimate) return CONV_OK;
        }
    }
};

}  // namespace wsc

using namespace wsc;

// K right-hand sides with one operator (same plan and contrast): GMRES on the stacked system
// diag(L, ..., L) [x_1; ...; x_K] = [f_1; ...; f_K] / scales, each f_s scaled to unit norm, so
// that one stacked residual ||r|| <= tol / sqrt(K) ||[f]|| = tol bounds every system's relative
// residual ||r_s|| / ||f_s|| by tol.  Every matvec is one batched apply of K densities; the
// Krylov vectors are K n^2 long.  K = 1 is the plain solve.
static conv_status ls_solve_impl(conv_plan_t p, const double *m, const void *f, void *x, int K,
                                 const ls_opts *opts_in, ls_info *info, void *stream)
{
    if (!p || !m || !f || !x) return fail(CONV_EINVAL, "bad argument");
    if (K < 1) return fail(CONV_EINVAL, "count must be >= 1");
    if (p->kern.family != CONV_K_HELMHOLTZ || p->io != CONV_IO_C2C)
        return fail(CONV_EINVAL, "ls_solve needs a C2C Helmholtz plan");
    ls_opts o = {50, 2000, 1e-10, 0, 1e-5, 1};
    if (opts_in) o = *opts_in;
    if (o.restart < 1 || o.restart > LS_MAX_RESTART)
        return fail(CONV_EINVAL, "restart must be in [1, " + std::to_string(LS_MAX_RESTART) + "]");
    if (o.max_iters < 1) return fail(CONV_EINVAL, "max_iters must be >= 1");
    if (!(o.tol > 0)) return fail(CONV_EINVAL, "tol must be > 0");
    if (o.refine && !(o.inner_tol > 0 && o.inner_tol < 1)) return fail(CONV_EINVAL, "inner_tol must be in (0, 1)");
    if (K > 65535) return fail(CONV_EINVAL, "count must be <= 65535");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long NN = (long long)p->n * p->n, N = NN * K;

    // FP64 operator for true residuals
    conv_plan_s *p64 = p;
    if (p->prec != CONV_P_FP64) {
        if (!p->fp64_twin) {
            conv_plan_t twin = nullptr;
            conv_status rc = conv_plan_twin(p, &twin);
            if (rc != CONV_OK) return rc;
            p->fp64_twin = twin;
        }
        p64 = p->fp64_twin;
    }
    // matvec workspaces for a batch beyond the plans' own
    size_t cws = 0, cws64 = 0;
    if (K > p->batch_max) conv_workspace_size(p, K, &cws);
    if (p64 != p && K > p64->batch_max) conv_workspace_size(p64, K, &cws64);

    Solver S;
    S.p = p;
    S.p64 = p64;
    S.m64 = m;
    S.kappa2 = p->kern.kappa * p->kern.kappa;
    S.N = N;
    S.batch = K;
    S.restart = o.restart;
    S.st = st;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    S.grid_elem = (int)std::min<long long>((N + 255) / 256, (long long)sms * 8);
    // workspace: the plan's cached one when free (reallocated if it does not match), else a
    // private one
    const bool mixed = p->prec == CONV_P_FP32;
    LsCache *cache;
    {
        std::lock_guard<std::mutex> g(g_ls_cache_mu);
        if (!p->ls_cache) p->ls_cache = new LsCache();
        cache = p->ls_cache;
    }
    std::unique_lock<std::mutex> own(cache->mu, std::try_to_lock);
    const bool cached = own.owns_lock();
    if (cached) {
        if (cache->W.V && (cache->N != N || cache->batch != K || cache->restart < o.restart || (mixed && !cache->mixed))) {
            cudaStreamSynchronize(st);
            drop_graphs(cache);
            free_work(cache->W);
            dev_free(cache->m64);
            cache->m64 = nullptr;
        }
        if (!cache->W.V) {
            if (!alloc_work(cache->W, N, NN, K, cws, cws64, o.restart, mixed)) {
                free_work(cache->W);
                return fail(CONV_ENOMEM, "ls_solve workspace allocation failed");
            }
            cache->N = N;
            cache->batch = K;
            cache->restart = o.restart;
            cache->mixed = mixed;
        }
        S.W = cache->W;
        if (!mixed) {  // the FP64 matvec reads the contrast from the plan's copy
            if (!cache->m64 && dev_alloc(&cache->m64, NN * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                return fail(CONV_ENOMEM, "ls_solve contrast buffer");
            }
            WSC_CUDA(cudaMemcpyAsync(cache->m64, m, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
            S.m64 = cache->m64;
        }
        if (!cache->cap && cudaStreamCreateWithFlags(&cache->cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            cache->cap = nullptr;
        }
        if (cache->cap) {
            S.graphs = &cache->iter;
            S.cap_stream = cache->cap;
        }
    } else if (!alloc_work(S.W, N, NN, K, cws, cws64, o.restart, mixed)) {
        free_work(S.W);
        return fail(CONV_ENOMEM, "ls_solve workspace allocation failed");
    }
    if (p->prec == CONV_P_FP32) k_d2f<<<S.grid_elem, 256, 0, st>>>(m, S.W.m32, NN);

    const double2 *fb = reinterpret_cast<const double2 *>(f);
    double2 *xb = reinterpret_cast<double2 *>(x);
    if (o.zero_guess) cudaMemsetAsync(xb, 0, N * sizeof(double2), st);
    // several right-hand sides: unit-norm copies, the initial guesses scaled alike
    std::vector<double> scale(K, 1.0);
    double tol = o.tol;
    if (K > 1) {
        WSC_CUDA(cudaMemcpyAsync(S.W.fsc, fb, N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < K; ++k) {
            const double nk = S.norm_of(fb + (size_t)k * NN, NN);
            scale[k] = nk > 0 ? nk : 1.0;
            k_scale_real<<<S.grid_elem, 256, 0, st>>>(S.W.fsc + (size_t)k * NN, 1.0 / scale[k], NN);
            if (!o.zero_guess) k_scale_real<<<S.grid_elem, 256, 0, st>>>(xb + (size_t)k * NN, 1.0 / scale[k], NN);
        }
        fb = S.W.fsc;
        tol = o.tol / std::sqrt((double)K);
    }
    S.norm2(fb);
    k_gmres_init<<<1, 32, 0, st>>>(S.W.gs);
    double fn = S.read_scalar(S.W.gs.res);
    if (!(fn > 0)) fn = 1.0;

    int iters = 0, cycles = 0, refinements = 0;
    double res = 0;
    conv_status rc = CONV_OK;
    // the buffer holding f - L64 x for the current x, when the iteration has just formed it with the
    // FP64 operator (the final residual below is then that one, not a recomputation)
    const double2 *last_r = nullptr;
    if (!o.refine || p->prec == CONV_P_FP64) {
        rc = S.gmres(fb, xb, tol * fn, o.max_iters, o.zero_guess != 0, iters, cycles, res);
        // GMRES ends right after forming b - L z for its final z (its restart check); with the FP64
        // plan that is the true residual
        if (p->prec == CONV_P_FP64 && (rc == CONV_OK || rc == CONV_ENOTCONVERGED)) last_r = S.W.r;
    } else {
        // FP64 iterative refinement around an FP32-matvec GMRES
        bool first = o.zero_guess != 0;
        while (true) {
            if (first) cudaMemcpyAsync(S.W.d, fb, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
            else {
                rc = S.true_residual(fb, xb, S.W.d);
                if (rc != CONV_OK) break;
            }
            first = false;
            last_r = S.W.d;
            S.norm2(S.W.d);
            k_gmres_init<<<1, 32, 0, st>>>(S.W.gs);
            double rn = S.read_scalar(S.W.gs.res);
            res = rn;
            if (!(rn == rn)) {
                rc = fail(CONV_ENONFINITE, "residual is not finite");
                break;
            }
            if (rn <= tol * fn) break;
            if (iters >= o.max_iters) {
                rc = fail(CONV_ENOTCONVERGED, "GMRES-IR reached its iteration limit");
                break;
            }
            // inner solve L32 c = r from c = 0 to inner_tol relative (never tighter than the outer
            // target needs), then x += c
            cudaMemsetAsync(S.W.x64, 0, N * sizeof(double2), st);
            double inner_abs = std::max(o.inner_tol * rn, 0.5 * tol * fn);
            int it_before = iters;
            double inner_res = 0;
            conv_status irc = S.gmres(S.W.d, S.W.x64, inner_abs, o.max_iters, true, iters, cycles, inner_res, true);
            if (irc == CONV_OK || irc == CONV_ENOTCONVERGED) {
                k_axpy_real<<<S.grid_elem, 256, 0, st>>>(xb, S.W.x64, N);
                last_r = nullptr;  // x moved on
                ++refinements;
            }
            if (irc != CONV_OK && irc != CONV_ENOTCONVERGED) {
                rc = irc;
                break;
            }
            if (iters == it_before) {
                rc = fail(CONV_ENOTCONVERGED, "refinement made no progress");
                break;
            }
        }
    }
    // final true residual with the FP64 operator, per right-hand side
    std::vector<double> rel(K, 0.0);
    if (rc == CONV_OK || rc == CONV_ENOTCONVERGED) {
        conv_status r2 = CONV_OK;
        const double2 *r = last_r;
        if (!r) {
            r2 = S.true_residual(fb, xb, S.W.r);
            r = S.W.r;
        }
        if (r2 == CONV_OK) {
            if (K == 1) {
                S.norm2(r);
                k_gmres_init<<<1, 32, 0, st>>>(S.W.gs);
                rel[0] = S.read_scalar(S.W.gs.res) / fn;
            } else {
                for (int k = 0; k < K; ++k) rel[k] = S.norm_of(r + (size_t)k * NN, NN);  // ||f_s|| = 1
            }
        }
    }
    if (K > 1)
        for (int k = 0; k < K; ++k) k_scale_real<<<S.grid_elem, 256, 0, st>>>(xb + (size_t)k * NN, scale[k], NN);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (!cached) free_work(S.W);
    if (info)
        for (int k = 0; k < K; ++k) {
            info[k].iters = iters;
            info[k].restarts = cycles;
            info[k].refinements = refinements;
            info[k].rel_residual = rel[k];
        }
    if (ce != cudaSuccess) return cuda_fail(ce, "ls_solve");
    // a pass kernel that gave up on a bounded wait leaves the solve's matvecs incomplete
    const conv_status ds = conv_device_status(p, stream);
    return ds != CONV_OK ? ds : rc;
}

extern "C" conv_status ls_solve(conv_plan_t p, const double *m, const void *f, void *x, const ls_opts *opts,
                                ls_info *info, void *stream)
{
    return ls_solve_impl(p, m, f, x, 1, opts, info, stream);
}

extern "C" conv_status ls_solve_multi(conv_plan_t p, int count, const double *m, const void *f, void *x,
                                      const ls_opts *opts, ls_info *info, void *stream)
{
    return ls_solve_impl(p, m, f, x, count, opts, info, stream);
}
