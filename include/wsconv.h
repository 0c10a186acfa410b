/*
 * wsconv.h -- C ABI of the GB300 (sm_103a) library for the FFT convolution with weakly singular
 * kernels of Tiwari, Pandey, Paul & Anand (arXiv 2107.03958), and its use as the matvec of the
 * Lippmann-Schwinger Nystrom solver.
 *
 * Operation (Sec. 2.1, eq. (An)): for grid data u_j = u(j/n), j in G_n = [0,n)^2, on D = [0,1]^2,
 *     (A_n u)(x_j) = sum_{k in F_n} ghat(k) hat u_{e,n}(k) e^{2 pi i k.j/M},   M = n b,
 * with u_e the zero extension of u to the period-b square and hat u_{e,n} its trapezoidal Fourier
 * coefficients.  Equivalently A_n u = crop_n(ifft2(ghat (.) fft2(zero-extend_M(u)))) where ifft2
 * carries 1/M^2.  ghat(k) = int_{B_a(0)} g(y) e^{-2 pi i k.y/b} dy (eq. (bk), (ghat), Sec. 2.2).
 *
 * Conventions shared by every entry point:
 *   - Arrays are row-major, first index <-> x1.  A density batch is batch x n x n.
 *   - Complex data are interleaved (re, im) pairs of the plan's real type.
 *   - Data pointers (u, mask, out, workspace, m, f, x) are DEVICE pointers owned by the caller,
 *     unless the name says host.  The plan owns ghat, the twiddle table and a default workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  conv_apply is
 *     asynchronous; ls_solve synchronises at restart boundaries.
 *   - No exception or abort crosses the ABI.  On failure a status is returned and
 *     conv_last_error() gives a message (thread-local).
 */
#ifndef WSCONV_H
#define WSCONV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CONV_OK = 0,
    CONV_EINVAL = 1,          /* bad argument, or a (b, a) pair outside eq. (io)'s admissible range */
    CONV_EUNSUPPORTED = 2,    /* valid but not implemented: e.g. M = n b odd or with a prime factor > 5,
                                 or a transform length beyond one CTA's shared memory */
    CONV_ENOMEM = 3,          /* device allocation failed */
    CONV_ECUDA = 4,           /* a CUDA call or kernel launch failed */
    CONV_ETIMEOUT = 5,        /* a bounded device-side wait gave up */
    CONV_ENOTCONVERGED = 6,   /* GMRES hit its iteration limit */
    CONV_ENONFINITE = 7,      /* NaN/Inf detected */
    CONV_ECANCELLED = 8       /* a serving request was cancelled before it ran (srv_cancel) */
} conv_status;

/* Kernel families (Sec. 2.2, Sec. 3.2).  g(x) = scale * log|x|, scale * |x|^gamma (gamma > -2; the
 * closed-form moments need 2 gamma an integer, the quadrature moments of conv_plan_moments do not),
 * scale * (i/4) H0^(1)(kappa |x|), or scale * K0(kappa |x|) / (2 pi) (the Yukawa kernel of
 * -Delta + kappa^2, Sec. 3.2).  The paper's Laplace kernel is LOG with scale = -1/(2 pi). */
typedef enum {
    CONV_K_LOG = 0,
    CONV_K_POW = 1,
    CONV_K_HELMHOLTZ = 2,
    CONV_K_YUKAWA = 3,
    /* the non-radial kernel of Sec. 3.1: g(x) = scale * (-x1 / (2 pi |x|^2)) = scale * d/dx1 of
     * -(1/2pi) log|x|; ghat(k) = i scale xi1 (1 - J0(|xi| a)) / |xi|^2, xi = 2 pi k / b, odd in k1
     * (the unpaired Nyquist mode k1 = -M/2 is given multiplier 0, so real u gives real A_n u).
     * R2R plans on the period-b grid with closed-form moments only (CONV_EUNSUPPORTED otherwise). */
    CONV_K_DX1LOG = 4
} conv_kernel_family;

typedef struct {
    int family;      /* conv_kernel_family */
    double gamma;    /* CONV_K_POW exponent */
    double kappa;    /* CONV_K_HELMHOLTZ wavenumber, CONV_K_YUKAWA decay rate (> 0) */
    double scale;    /* multiplies g; 0 is read as 1 */
} conv_kernel;

/* Arithmetic of the transform passes.  ghat is always built in FP64; an FP32 plan keeps an FP32
 * copy.  FP64 meets 1e-12 relative L-infinity against the FP64 oracle; FP32 about 1e-6. */
typedef enum { CONV_P_FP64 = 0, CONV_P_FP32 = 1 } conv_precision;

/* Input/output types.  R2R needs a real ghat (LOG, POW). */
typedef enum {
    CONV_IO_R2R = 0,   /* real u -> real A_n u */
    CONV_IO_R2C = 1,   /* real u -> complex A_n u (any kernel) */
    CONV_IO_C2C = 2    /* complex u -> complex A_n u (any kernel) */
} conv_io;

typedef struct conv_plan_s *conv_plan_t;

/* Build a plan: validates the period b = period_num/period_den and the truncation radius a
 * (eq. (io), Sec. 2.1: sqrt 2 <= a <= b - 1 for support D), computes the FP64 moment table
 * ghat(|k1|, |k2|) for 0 <= k1, k2 <= M/2 on the GPU (Sec. 2.2; the Helmholtz k = 0 value with the
 * sign of its 2/(kappa pi) term corrected), the twiddle table, and allocates a workspace for
 * batch_max densities.
 *   trunc_a <= 0 selects the midpoint (sqrt 2 + b - 1)/2 and requires b >= 1 + sqrt 2.
 *   An explicit trunc_a > 0 is accepted as given (the caller vouches that the density's support
 *   keeps B_a(x) inside the period for all x in D).
 * Returns CONV_EINVAL for bad arguments, CONV_EUNSUPPORTED for M odd, M with a prime factor > 5, a
 * transform beyond shared memory, or POW with 2 gamma not an integer. */
conv_status conv_plan(const conv_kernel *kernel, int period_num, int period_den, int n,
                      double trunc_a, conv_precision precision, conv_io io, int batch_max,
                      conv_plan_t *plan);

/* Plan flags for conv_plan_ex. */
enum {
    /* Compact embedding: the passes run on the 2n-periodic lattice instead of the period-b one.
     * A_n u is the quadrature of eq. (quad), (A_n u)_i = sum_j w(i - j) u_j, whose weights
     * w(d) (eq. (quad_wts), |d1|, |d2| <= n - 1) are built once from the moments ghat (period b,
     * Sec. 2.2) by an FP64 M x M inverse DFT; placed on the period-2n lattice they make A_n u a
     * cyclic convolution of length L = 2n, so the passes transform 2n points per line with the
     * L x L DFT of w as multiplier.  Same A_n u up to rounding, fewer points (2n vs n b per line). */
    CONV_PLAN_COMPACT = 1,
    /* Autotune the launch configuration (elements per thread, twiddles in shared memory or not,
     * fused or plain passes): time each on zero densities at batch_max and keep the fastest
     * (results cached per shape for the process).  Allocates temporary buffers. */
    CONV_PLAN_AUTOTUNE = 2
};

conv_status conv_plan_ex(const conv_kernel *kernel, int period_num, int period_den, int n,
                         double trunc_a, conv_precision precision, conv_io io, int batch_max,
                         int flags, conv_plan_t *plan);

/* How the moment table ghat is computed (Sec. 2.2, 2.3).
 *   CONV_MOMENTS_CLOSED:     the closed forms of Sec. 2.2 (and of the Yukawa kernel, Sec. 3.2), with
 *                            quadrature where they lose digits (conv_plan's default).
 *   CONV_MOMENTS_QUADRATURE: Sec. 2.3: ghat(k) = 2 pi p int_0^{a^{1/p}} g(tau^p) J0(2 pi |k| tau^p/b)
 *                            tau^{2p-1} d tau by a high-order rule, for any family (a kernel without
 *                            closed-form moments; |x|^gamma with any gamma > -2).
 *   CONV_MOMENTS_LOCALIZED:  Sec. 2.3, eq. (io_split): the moments of g eta_beta by the trapezoidal
 *                            rule in tau, plus the classical trapezoidal rule for g (1 - eta_beta),
 *                            whose weights h^2 g(|d|h)(1 - eta_beta(|d|h)) enter as their DFT.
 *                            eta_beta = 1 on [0, beta/2], 0 beyond beta, the half-window varkappa of
 *                            eq. (halfwindow1) in between.
 * The quadrature rules cost O((M/2)^2 z) Bessel evaluations at plan time, z = pi sqrt2 M R / b
 * (R = a, or beta when localized): seconds at n = 1024, minutes at n = 4096. */
typedef enum { CONV_MOMENTS_CLOSED = 0, CONV_MOMENTS_QUADRATURE = 1, CONV_MOMENTS_LOCALIZED = 2 } conv_moment_method;
typedef struct {
    int method;      /* conv_moment_method */
    int p;           /* substitution rho = tau^p, 1..16 (<= 0: 4) */
    int nodes;       /* quadrature nodes (<= 0: chosen from the table's largest phase 2 pi |k| R / b) */
    double beta;     /* LOCALIZED: localization radius, 0 < beta <= a (<= 0: 1) */
} conv_moments;

/* conv_plan_ex with the moment table computed as `moments` says (NULL: closed forms). */
conv_status conv_plan_moments(const conv_kernel *kernel, int period_num, int period_den, int n,
                              double trunc_a, conv_precision precision, conv_io io, int batch_max,
                              int flags, const conv_moments *moments, conv_plan_t *plan);

/* Bytes of workspace conv_apply needs for `batch` densities (the n x (L/2+1) or n x L spectra,
 * L the transform length). */
conv_status conv_workspace_size(conv_plan_t plan, int batch, size_t *bytes);

/* out = A_n(u . mask) for `batch` densities (Sec. 2.1, eq. (An)).
 *   u:    batch x n x n, real (R2R, R2C) or complex (C2C), plan precision.
 *   mask: NULL or an n x n real array (plan precision) shared by the batch; it multiplies u at the
 *         load (the Fourier-smoothed indicator chi^n psi of Sec. 2.4, or a contrast).
 *   out:  batch x n x n, real (R2R) or complex (R2C, C2C); must not alias u.
 *   workspace: NULL (use the plan's, valid for batch <= batch_max) or conv_workspace_size bytes,
 *              16-byte aligned.
 * u, out and mask must be aligned to their element type (CONV_EINVAL otherwise).
 * Asynchronous on `stream`.  Three kernel launches. */
conv_status conv_apply(conv_plan_t plan, const void *u, const void *mask, void *out, int batch,
                       void *workspace, void *stream);

/* conv_apply for densities in HOST memory (no counterpart in the paper; the host link is slower
 * than the passes, so the copies have to overlap them).  The batch runs in chunks of
 * ceil(batch_max / 4) densities: chunk i's upload, passes and download overlap chunk i+1's upload
 * and chunk i-1's download, on three streams the plan creates at the first call together with
 * two device slots of a chunk's densities and results.
 *   u_host:   batch x n x n, layout and type as conv_apply's u, host memory.
 *   out_host: batch x n x n, layout and type as conv_apply's out, host memory.
 *   mask:     NULL or a DEVICE n x n array, as in conv_apply.
 * Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister): pageable memory works,
 * but its copies do not overlap.  Ordered on `stream` like conv_apply: it starts after earlier
 * work on `stream`, later work on `stream` starts after out_host is complete, and the call
 * returns without waiting.  It uses the plan's workspace and device slots: calls on one plan
 * must not overlap (on different streams or threads).  Returns CONV_EINVAL for bad arguments or
 * while per-pass timing is on, CONV_ENOMEM when the slots cannot be allocated. */
conv_status conv_apply_host(conv_plan_t plan, const void *u_host, const void *mask, void *out_host, int batch,
                            void *stream);

/* conv_apply_host for several plans on ONE batch of host densities (no counterpart in the paper;
 * e.g. the same densities convolved with several kernels of Sec. 2.2).  Each chunk of densities
 * (ceil(min batch_max / 4)) is uploaded once; the plans' passes run on it in list order, each
 * with its own workspace, and plan k's result chunk downloads while plan k+1's passes run.
 *   plans:    `count` distinct plans with the same n, precision, device and input type (R2R and
 *             R2C take real densities, C2C complex ones); per-pass timing off.
 *   u_host:   batch x n x n densities, host memory, as conv_apply's u.
 *   mask:     NULL or a DEVICE n x n array (plan precision) shared by every plan.
 *   out_host: `count` host arrays, out_host[k] batch x n x n in plans[k]'s output layout.
 * Host buffers should be page-locked.  Ordered on `stream` like conv_apply_host; returns without
 * waiting.  The device slots (four chunks of densities, four of each plan's results) and three
 * streams are created at the first call and kept on plans[0] until conv_destroy, or rebuilt when
 * a later call's chunk or result sizes differ.  Calls on any of these plans must not overlap.
 * Returns CONV_EINVAL for bad or mismatched arguments, CONV_ENOMEM when the slots cannot be
 * allocated. */
conv_status conv_apply_host_multi(int count, const conv_plan_t *plans, const void *u_host, const void *mask,
                                  void *const *out_host, int batch, void *stream);

/* Densities of one batch convolved with DIFFERENT kernels that share one transform shape (no
 * counterpart in the paper; a serving aid for Sec. 2.1, eq. (An)):
 *     out[b] = A_n(u[b] . mask) with the moment table of plans[b],  b < batch,
 * in one launch of each pass on `shape` (its workspace and launch configuration).  Every
 * plans[b] must share the shape plan's n, period, precision, io, embedding and multiplier type
 * (real or complex); their kernels, kappa and truncation radius may differ.  Each result is
 * bitwise the one conv_apply gives on plans[b] alone.
 *   batch <= 32; workspace as for conv_apply on `shape` (NULL: the shape plan's, batch <= its
 *   batch_max).  Asynchronous on `stream`; the plans must outlive the launch.
 * Returns CONV_EINVAL for what conv_apply rejects and for plans of another shape,
 * CONV_EUNSUPPORTED for lines beyond one CTA (plans whose info.long_lines is set). */
conv_status conv_apply_kernels(conv_plan_t shape, const conv_plan_t *plans, const void *u, const void *mask,
                               void *out, int batch, void *workspace, void *stream);

/* The same densities convolved with several kernels, A_n^(k)(u . mask) for each plan k, with the
 * row transforms of pass 1 computed once (Sec. 2.1, eq. (An): the forward row transform of the
 * zero-extended density does not depend on the kernel; the paper's Tables 1-3 apply four
 * kernels to one density):
 *     outs[k][b] = A_n^(k)(u[b] . mask),   k < count, b < batch.
 *   plans:  `count` distinct plans running the fused R2R or split R2C passes (real densities; a
 *           plan whose info.fused is 0 or info.long_lines is 1 is refused), sharing n, period,
 *           precision, embedding and the row pass's launch configuration; kernels may differ.
 *   u, mask: as for conv_apply (real densities of the plans' precision).
 *   outs:   `count` device arrays, outs[k] batch x n x n in plans[k]'s output layout, distinct
 *           and not aliasing u.
 *   workspace: NULL (then batch <= every plan's batch_max; a workspace comes from the library's
 *           memory pool and returns to it in stream order) or conv_multi_workspace_size bytes,
 *           16-byte aligned, owned by the caller.
 * Each result is bitwise the one conv_apply gives on plans[k] alone.  Asynchronous on `stream`.
 * The call sets per-plan launch state for its duration: calls on the same plans must not
 * overlap (from several threads).
 * Returns CONV_EINVAL for what conv_apply rejects and for mismatched plans, CONV_EUNSUPPORTED for
 * plans outside the fused R2R / split R2C pipelines, CONV_ENOMEM when the pool cannot supply
 * the workspace. */
conv_status conv_apply_multi(const conv_plan_t *plans, int count, const void *u, const void *mask,
                             void *const *outs, int batch, void *workspace, void *stream);

/* Bytes of the caller's workspace conv_apply_multi needs for `batch` densities: the shared row
 * spectrum (batch x n x (L/2 + 1) complex, rounded to 256 bytes) plus the largest of the plans'
 * own conv_workspace_size.  CONV_EINVAL / CONV_EUNSUPPORTED as conv_apply_multi. */
conv_status conv_multi_workspace_size(const conv_plan_t *plans, int count, int batch, size_t *bytes);

/* conv_apply without any allocation (the paper has no counterpart; this is a deployment aid).
 * For callers that cannot call cudaMalloc when they run the convolution: code under a device
 * memory budget that forbids new allocations, real-time loops where an allocation may block, or
 * host frameworks that own all device memory and pass this library only inputs and outputs.
 * The plan must exist already (conv_plan allocates its tables once); this call uses neither the
 * plan's workspace nor a caller's, but a fixed 32 MiB device array inside the library.  The array
 * is placed on a device when the first plan is built there (conv_plan looks up its device address
 * and keeps it in the plan) and stays until the process exits; this call looks nothing up, loads
 * nothing and allocates nothing.
 *   Same arguments, argument checks and result as conv_apply (workspace and stream aside); the
 *   batch is limited by the array's size, not by the plan's batch_max.
 *   Returns CONV_EINVAL for whatever conv_apply rejects (NULL or aliased pointers, u, out or mask
 *   not aligned to its element size), with a message giving both sizes when the plan and batch
 *   need more than 32 MiB of workspace (conv_workspace_size), and when per-pass timing is enabled
 *   on the plan.  Returns CONV_ECUDA when the array's address could not be looked up at plan
 *   creation.
 *   All calls share the one array: calls that overlap on the GPU (other streams, other threads)
 *   race and corrupt each other's results; serialise them.  The array keeps the last call's
 *   contents; nothing in it needs to start at zero, since each call writes every element it
 *   later reads. */
conv_status conv_apply_noalloc(conv_plan_t plan, const void *u, const void *mask, void *out,
                               int batch, void *stream);

/* Mixed-size batching (no counterpart in the paper; a serving aid for the convolutions of
 * Sec. 2.1, eq. (An)).  A group is a fixed list of `count` applies,
 *     out[i] = A_n(u[i] . mask[i])   on plans[i], batch[i] densities,
 * whose plans may differ in n, kernel, period, precision and io.  conv_group_create captures the
 * items' pass kernels into one CUDA graph and instantiates it; each conv_group_launch then runs
 * every item with one graph launch on `stream`.
 *   Items on different plans are concurrent branches of the graph, so the passes of small grids,
 *   which do not fill the GPU alone, run side by side.  Items on one plan share its workspace
 *   and run in list order on one branch.
 *   plans, u, out, batch: arrays of `count` entries; u[i], out[i] as in conv_apply for plans[i];
 *   mask: NULL, or an array of `count` entries each NULL or as conv_apply's mask;
 *   batch[i] in [0, batch_max of plans[i]] (0 skips the item).
 *   The pointers are fixed in the graph: every launch reads u[i] and writes out[i] as given at
 *   creation (their contents may change between launches).  The plans and buffers must outlive
 *   the group, and no other call on one of its plans may overlap a launch.
 *   Every plan must be on the current device, with per-pass timing off.
 *   A pass kernel's given-up bounded wait is reported in its plan's status word
 *   (conv_device_status on that plan).
 * Returns CONV_EINVAL for bad arguments: count < 1, an item conv_apply would reject, an out[i]
 * equal to another item's u or out (ranges are not checked for partial overlap).  Returns
 * CONV_ECUDA when capture or instantiation fails. */
typedef struct conv_group_s *conv_group_t;
conv_status conv_group_create(int count, const conv_plan_t *plans, const void *const *u, const void *const *mask,
                              void *const *out, const int *batch, conv_group_t *group);
/* One graph launch of every item, ordered on `stream` like conv_apply.  Returns CONV_EINVAL when
 * the current device is not the group's. */
conv_status conv_group_launch(conv_group_t group, void *stream);
/* Frees the graph (the plans and buffers stay the caller's).  Call it with no launch in flight. */
void conv_group_destroy(conv_group_t group);

/* Generalised apply used by the Lippmann-Schwinger operator (Sec. 3.3, eq. (descretls)):
 *     out = beta * u + alpha * A_n(u . mask)
 * with complex alpha (alpha_re, alpha_im) and real beta; C2C/R2C plans only when beta != 0 needs a
 * complex u.  conv_apply is the case alpha = 1, beta = 0. */
conv_status conv_apply_axpby(conv_plan_t plan, const void *u, const void *mask, void *out,
                             int batch, double alpha_re, double alpha_im, double beta,
                             void *workspace, void *stream);

typedef struct {
    int n, M, period_num, period_den;
    double b, a;
    int precision, io, family, batch_max;
    int nstages;
    int radices[16];
    size_t ghat_bytes, workspace_bytes;
    int threads_rows, groups_rows, threads_cols, groups_cols;
    int transform_len;   /* points per line in the passes: M = n b, or 2n when compact */
    int compact;         /* CONV_PLAN_COMPACT was set */
    int elems;           /* complex elements per thread in the transform kernels (0: generic) */
    int smem_twiddles;   /* twiddle table staged in shared memory */
    int fused;           /* fused passes (global-memory first/last stages) */
    int static_log2;     /* log2 of the transform length when it is a power of two whose stage
                          * structure is fixed at compile time (fused passes), else 0 */
    int r2c_split;       /* R2C with complex ghat on the split pipeline (Re/Im ghat columns) */
    int static_len;      /* the transform length when its stage structure is fixed at compile
                          * time (2^l with n = L/2, or 3 2^l with n = L/3), else 0 */
    int long_lines;      /* 1: transform lines exceed one CTA (n = 8192 in FP64, or on the
                            period-3 grid): the passes run as four-step FP64 line transforms */
    int cols_pingpong;   /* 1: the R2R column pass holds two buffers per line and alternates
                            between them stage by stage (one barrier per stage) */
} conv_plan_info;

conv_status conv_get_info(conv_plan_t plan, conv_plan_info *info);

/* Copy the FP64 moment table ghat(|k1|, |k2|), 0 <= k1, k2 <= M/2, to host memory:
 * (M/2+1)^2 doubles (real kernels) or (M/2+1)^2 interleaved complex doubles (Helmholtz),
 * index [k2 * (M/2+1) + k1].  Synchronous. */
conv_status conv_ghat_to_host(conv_plan_t plan, double *host_out);

void conv_destroy(conv_plan_t plan);

/* Message for the last failing call on this thread ("" if none). */
const char *conv_last_error(void);

/* ------------------------------------------------------------------------------------------
 * Lippmann-Schwinger solve (Sec. 3.3, eq. (lippsch) discretised as eq. (descretls)):
 *     u + kappa^2 A_n(m u) = f   on G_n,
 * by restarted GMRES with matrix-free matvecs (Arnoldi by classical Gram-Schmidt with one
 * re-orthogonalisation, Givens rotations, all in FP64 on the device).
 *   plan: a C2C Helmholtz plan (its precision is the matvec precision of the inner solve).
 *   m:    n x n real contrast m = 1 - mu, FP64, device.
 *   f:    n x n complex128 right-hand side (u_inc on the grid), device.
 *   x:    n x n complex128, device: initial guess on entry (ignored when opts->zero_guess),
 *         solution on exit.
 * With an FP32 plan and opts->refine != 0 the solve is mixed precision: an outer FP64 residual
 * r = f - L x (FP64 matvec built internally), an inner FP32-matvec GMRES on L d = r to
 * opts->inner_tol, x += d, until ||r|| / ||f|| <= opts->tol.
 * The first solve on a plan allocates its Krylov workspace ((restart + 1) n^2 complex128 and a few
 * vectors) and keeps it with the plan, for later solves of the same n, until conv_destroy; a solve
 * that starts while another uses it (another thread) allocates and frees its own.
 * Returns CONV_ENOTCONVERGED (with info filled) when max_iters is reached. */
typedef struct {
    int restart;       /* Krylov dimension per cycle, 1..1000 (default 50) */
    int max_iters;     /* total matvec limit (default 2000) */
    double tol;        /* relative residual target ||f - L x||_2 / ||f||_2 (default 1e-10) */
    int refine;        /* mixed precision: 1 = FP64 iterative refinement around an FP32 inner solve */
    double inner_tol;  /* inner relative tolerance for refinement (default 1e-5) */
    int zero_guess;    /* 1: start from x = 0 */
} ls_opts;

typedef struct {
    int iters;            /* matvecs in the Krylov iterations */
    int restarts;         /* GMRES cycles */
    int refinements;      /* outer refinement steps (mixed precision) */
    double rel_residual;  /* final true relative residual (FP64 operator) */
} ls_info;

conv_status ls_solve(conv_plan_t plan, const double *m, const void *f, void *x, const ls_opts *opts,
                     ls_info *info, void *stream);

/* ls_solve for `count` right-hand sides with one operator (the same plan, contrast m and kappa;
 * e.g. several incident plane waves on one scatterer, Sec. 3.3).
 *   f, x: count x n x n complex128, contiguous (x: initial guesses unless opts->zero_guess; on
 *         return the solutions).  info: NULL or `count` entries.
 * GMRES runs on the stacked block-diagonal system with each f_s scaled to unit norm, so every
 * matvec is one batched apply of `count` densities.  The stacked target tol / sqrt(count) bounds
 * each system's relative residual by tol; info[s].rel_residual is system s's own, from the FP64
 * operator, and iters / restarts / refinements are the shared iteration's.
 * Workspace: the Krylov basis grows with count ((restart + 1) x count x n^2 complex128), kept with
 * the plan like ls_solve's; matvec workspaces for count beyond the plans' batch_max are allocated
 * with it.  Returns as ls_solve, CONV_EINVAL also for count < 1 or > 65535. */
conv_status ls_solve_multi(conv_plan_t plan, int count, const double *m, const void *f, void *x,
                           const ls_opts *opts, ls_info *info, void *stream);

/* Fourier-smoothed indicator mask for discontinuous densities (Sec. 2.4, eq. (tfs)):
 *     mask_j = Re chi^n_Omega(x_j) * psi(x_j),  x_j = j/n,
 *     chi^n_Omega(x) = sum_{k in F_n} chihat_b(k) e^{2 pi i k.x/b},
 *     chihat_b(k) = (1/b^2) int_Omega e^{-2 pi i k.y/b} dy   (closed forms for a disk and a rectangle),
 * i.e. eq. (tfs) read with the plan's period b and index set F_n.  psi(x) = w(x1) w(x2) is the
 * smooth window: w = 1 on [delta, 1 - delta], ramping to 0 at the edges of D through the
 * half-window varkappa(t) = exp(2 e^{-1/t}/(t - 1)) of eq. (halfwindow1); delta <= 0 omits psi.
 * The approximation of A u is then A_n(u~ . mask) with u~ a smooth extension of u (pass the mask
 * to conv_apply).
 *   shape: 0 = disk, geom = {c1, c2, r}; 1 = rectangle [x0, x1] x [y0, y1], geom = {x0, x1, y0, y1}
 *          (HOST array).
 *   mask:  device, n x n, the plan's real type.
 * Computed in FP64 by one pruned M x M inverse transform; allocates temporary device buffers and
 * synchronises `stream` (geometry-time operation). */
conv_status conv_fs_mask(conv_plan_t plan, int shape, const double *geom, double delta, void *mask,
                         void *stream);

/* Device status of the plan's pass kernels (no counterpart in the paper).  The fused passes fetch
 * their next work item into shared memory with asynchronous copies while transforming the current
 * one; every wait for such a copy is bounded (one second of wall time).  A wait that gives up
 * makes its kernel record CONV_ETIMEOUT in the plan's device status word and leave without
 * finishing, so the applies since then are incomplete.  conv_device_status synchronises `stream`,
 * reads and clears that word (and the FP64 twin's of a mixed-precision LS plan) and returns it:
 * CONV_OK, or CONV_ETIMEOUT.  ls_solve and the serving layer call it for their own work. */
conv_status conv_device_status(conv_plan_t plan, void *stream);

/* Per-pass device timing (benchmark instrumentation; no counterpart in the paper).  While enabled,
 * every apply on this plan records CUDA events around its three kernel launches on the apply's
 * stream (no synchronisation).  conv_timing_read waits for the recorded events, returns the summed
 * milliseconds of pass 1 (rows forward), pass 2 (columns) and pass 3 (rows inverse) and the number
 * of applies recorded, and clears the record. */
conv_status conv_timing_enable(conv_plan_t plan, int enable);
conv_status conv_timing_read(conv_plan_t plan, double ms_out[3], long long *applies);

/* ------------------------------------------------------------------------------------------
 * Serving (no counterpart in the paper): a request loop with continuous batching around
 * conv_apply (Sec. 2.1) and ls_solve (Sec. 3.3).  Requests may be submitted at any time from any
 * thread.  A dispatcher admits them first-fit against a device-memory budget (plan tables,
 * workspaces and batching buffers, Krylov bases), keeps plans resident (evicting idle ones
 * oldest-first when the budget requires), batches waiting convolutions that share a plan into one
 * launch on that plan's stream, and runs Lippmann-Schwinger solves on worker threads with their
 * own streams, so the work of different requests overlaps on the GPU.  Every result equals the one
 * the same request gets alone (same kernels, fixed-order reductions).
 * The caller owns every request buffer (device memory) until srv_wait returns for that ticket. */
typedef struct srv_s *srv_t;
typedef enum { SRV_CONV = 0, SRV_LS = 1 } srv_kind;

typedef struct {
    int kind;                      /* SRV_CONV or SRV_LS */
    conv_kernel kernel;            /* SRV_LS: a Helmholtz kernel */
    int n, period_num, period_den;
    int precision;                 /* conv: plan precision; LS: CONV_P_FP64, or CONV_P_FP32 = FP32
                                      matvecs inside FP64 iterative refinement */
    int io;                        /* conv: conv_io (ignored for LS) */
    const void *in;                /* conv: u (n x n, plan types); LS: f (complex128 n x n) */
    const void *mask;              /* conv: optional n x n mask (plan real type) */
    const double *m;               /* LS: contrast (FP64 n x n) */
    void *out;                     /* conv: A_n(u . mask); LS: solution (complex128), zero start */
    double tol;                    /* LS: relative residual target (<= 0: 1e-10) */
    int restart, max_iters;        /* LS: (<= 0: 50, 2000) */
} srv_request;

typedef struct {
    int status;                    /* conv_status of the request */
    double t_submit, t_start, t_done;  /* seconds, one monotonic host clock */
    int batched_with;              /* requests in the launch that carried this one */
    int iters;                     /* LS: matvecs */
    double rel_residual;           /* LS: final true relative residual */
} srv_result;

typedef struct {
    long long submitted, completed, failed, batches, batched_requests, plans_built, plans_evicted;
    size_t bytes_in_use;
    int plans_cached;
} srv_stats;

/* mem_budget_bytes: device bytes the server may hold; max_inflight: admitted requests at once;
 * conv_batch_max: convolutions per batched launch; ls_workers: concurrent LS solves;
 * plan_flags: conv_plan_ex flags for every plan the server builds (CONV_PLAN_COMPACT, ...). */
conv_status srv_create(size_t mem_budget_bytes, int max_inflight, int conv_batch_max, int ls_workers,
                       int plan_flags, srv_t *server);
/* Non-blocking; returns a ticket.  CONV_EINVAL for malformed requests. */
conv_status srv_submit(srv_t server, const srv_request *request, long long *ticket);
/* Blocks until the request finished (timeout_s <= 0: no limit); CONV_ETIMEOUT if the limit
 * passed first.  On CONV_OK the ticket is released and *result filled. */
conv_status srv_wait(srv_t server, long long ticket, double timeout_s, srv_result *result);
conv_status srv_get_stats(srv_t server, srv_stats *stats);
/* Stops admitting, finishes what is on the GPU, frees every cached plan. */
void srv_destroy(srv_t server);

/* Cancel a request that has not been admitted yet (still waiting for memory or a slot, or lost
 * by an injected CONV_FAULT_DROP).  Its result then reads status CONV_ECANCELLED; srv_wait on the
 * ticket returns at once and releases it.  CONV_EINVAL for an unknown ticket or a request that
 * already runs (wait for it instead). */
conv_status srv_cancel(srv_t server, long long ticket);

/* ------------------------------------------------------------------------------------------
 * Host-side fault injection (no counterpart in the paper; a test aid for the failure paths).
 * Nothing here faults, traps or hangs a GPU.  Each call arms `count` occurrences of one fault
 * (count 0 disarms it); the environment variable CONV_FAULT="alloc:N,wait:N,drop:N" arms the same
 * when the library loads.
 *   CONV_FAULT_ALLOC: the next plan builds fail their workspace allocation (CONV_ENOMEM), after
 *                     the plan's tables were allocated, so the clean-up path runs.
 *   CONV_FAULT_WAIT:  in the next applies, every pass kernel that prefetches its work items treats
 *                     its first bounded wait as given up: it records CONV_ETIMEOUT in the plan's
 *                     status word, waits (bounded) for the copy it issued to land, and leaves.
 *                     The applies' results are incomplete; conv_device_status reports it.
 *                     Plans whose passes do not prefetch never wait, so nothing is recorded.
 *   CONV_FAULT_DROP:  the next srv_submit calls return a ticket but the request is lost before
 *                     the dispatcher sees it (srv_wait with a limit times out; srv_cancel ends it).
 * Returns CONV_EINVAL for an unknown kind or a negative count. */
typedef enum { CONV_FAULT_ALLOC = 1, CONV_FAULT_WAIT = 2, CONV_FAULT_DROP = 3 } conv_fault_kind;
conv_status conv_fault_inject(int kind, int count);

/* ------------------------------------------------------------------------------------------
 * Roofline denominators measured on the running GPU (no counterpart in the paper):
 *   copy:  bytes read + written per second by a grid-stride float4 copy of `bytes` bytes;
 *   fma:   FP64 and FP32 fused multiply-add throughput (flops/s, an FMA counts 2).
 * Synchronous; allocates and frees its own buffers. */
conv_status conv_measure_peaks(size_t bytes, double *copy_gbs, double *fp64_tflops,
                               double *fp32_tflops);

/* The tensor-core alternative for the passes' butterflies, measured (no counterpart in the paper;
 * the FFTs of Sec. 2.1): one radix-16 Stockham stage (Ns = 16) of an FP32 length-8192 column, one
 * column per SM held in shared memory, computed (a) on the CUDA cores and (b) as a DFT-matrix
 * product on the tensor cores (tcgen05.mma, M = 128 butterflies x N = 32 x K = 32, BF16 operands
 * split hi + lo, three products, FP32 accumulation in tensor memory).
 *   us_cuda_core, us_tensor: microseconds per stage per column (each SM one column), over reps
 *   stages; max_rel_err: max |(b) - (a)| / max |(a)| over one stage.
 * Synchronous; allocates and frees its own buffers.  CONV_ETIMEOUT if the bounded wait for the
 * products gave up. */
conv_status conv_measure_tc_stage(int reps, double *us_cuda_core, double *us_tensor, double *max_rel_err);

#ifdef __cplusplus
}
#endif
#endif /* WSCONV_H */
