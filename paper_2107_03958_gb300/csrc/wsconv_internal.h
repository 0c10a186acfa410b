// wsconv_internal.h -- plan object and helpers shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/wsconv.h"
#include "fft_engine.cuh"

struct conv_plan_s;
namespace wsc {
struct LsCache;
struct LongLines;
}

namespace wsc {

// Error message of the last failing call on this thread.
void set_error(const std::string &msg);
conv_status fail(conv_status st, const std::string &msg);
conv_status cuda_fail(cudaError_t e, const char *what);

#define WSC_CUDA(call)                                              \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return ::wsc::cuda_fail(_e, #call);  \
    } while (0)

// Threads-per-CTA bound of the pass kernels for E complex elements per thread (E = 0: generic
// guarded stages): keeps the E values in registers.
template <typename T, int E> struct maxt { static const int v = (E == 0 || (int)(2 * sizeof(T) * E) > 160) ? 512 : 1024; };
// Fused passes: the compile-time-length transforms (ED >= 1000) unroll every stage into straight-
// line code, one transform of L/E threads per CTA: at most 512 threads (128 registers each), except
// L = 2^14 at 16 elements per thread, whose 1024 threads get 64 registers.
#define WSC_STATIC_MAXT 512
__host__ __device__ constexpr int static_max_threads(int ed) { return ed == 1014 ? 1024 : WSC_STATIC_MAXT; }
template <typename T, int E, int ED> struct maxt_fused {
    static const int v = ED >= 1000 ? static_max_threads(ED) : maxt<T, E>::v;
};
// Compile-time lengths whose R2R column pass may hold two buffers per line and ping-pong between
// them (one barrier per stage): FP32 L = 2^12, 2^13 (two 66 KB buffers at L = 2^13 beside the
// prefetched column).
__host__ __device__ constexpr bool pingpong_ed(int ed, int elem_bytes) { return elem_bytes == 4 && (ed == 1012 || ed == 1013); }
template <typename T, int ED> __host__ __device__ constexpr bool pingpong_ok() { return pingpong_ed(ED, (int)sizeof(T)); }

template <typename T, int E, bool TWS>
conv_status run_pipeline(conv_plan_s *p, const void *u, const void *mask, void *out, int batch,
                         double are, double aim, double beta, void *ws, cudaStream_t st);
template <typename T, int E, bool TWS> conv_status set_attrs(int smem);
template <typename T, int E, bool TWS> int blocks_per_sm(int threads, size_t smem);
template <typename T, int E, int ED>
conv_status run_fused(conv_plan_s *p, const void *u, const void *mask, void *out, int batch, double are,
                      double aim, double beta, void *ws, cudaStream_t st);
template <typename T, int E, int ED, bool TWS> conv_status set_attrs_fused(int smem);
template <typename T, int E, int ED, bool TWS> int blocks_per_sm_fused(int threads, size_t smem);

// Launch shape of one pass family (rows or columns).
// Per-pass launch options (bits): twiddle table in shared memory, prefetch of the next work item
// (fused passes), one transform per CTA instead of the most that fit, TMA tiled copies for the
// row passes' strided spectrum accesses (R2R and split R2C: pass 1 stores, pass 3 loads).
enum { CFG_TWS = 1, CFG_PF = 2, CFG_ONE = 4, CFG_TMA = 8, CFG_DEFAULT = -1 };

// panel quadratures of the moment tables (ghat.cu, moments.cu): Clenshaw-Curtis rules of CC_N + 1 points
#define CC_N 16

// densities of a conv_apply_kernels batch (each its own multiplier, passed in the kernel parameters)
#define WSC_MAX_SEL 32

// rows (k2 values) per TMA box
#define TMA_ROWS 256
// tma.cu
bool encode_rows_map(CUtensorMap *m, const void *base, unsigned long long words, unsigned long long rows,
                     unsigned long long batch, unsigned box_words);
// A launch configuration: {E, fused passes, options of pass 1, of pass 2, of pass 3}.  Unfused
// passes share pass 1's twiddle option.
typedef std::array<int, 5> Candidate;

struct LaunchShape {
    int tpt;       // threads per transform
    int groups;    // transforms per CTA
    size_t smem;   // dynamic shared memory bytes
    int max_ctas;  // persistent grid size (CTAs resident at once)
    int stage;     // fused passes: elements of each group's prefetch staging area (0: no prefetch)
    bool tws;      // twiddle table in shared memory
    bool pf;       // fused passes: prefetch of the next work item into the staging area
    bool tma;      // pass 1: TMA stores of the spectra; pass 3: TMA loads into the staging area
    bool pp;       // R2R column pass: two transform buffers per group (ping-pong stages)
    bool one;      // split R2C column pass: one buffer per group, the Im part via a global line
};

}  // namespace wsc

struct conv_plan_s {
    conv_kernel kern;
    int pnum, pden, n;
    int Mb;                   // n b: the period-b grid of eq. (An), on which the moments live
    int M, h;                 // transform length of the passes (Mb, or 2n for the compact embedding), h = M/2 + 1
    bool compact = false;     // passes use the 2n-periodic embedding of the quadrature weights
    double b, a;
    conv_precision prec;
    conv_io io;
    int batch_max;
    bool complex_ghat;
    conv_moments moments{};  // how ghat is computed (closed forms by default)
    bool r2c_split = false;  // R2C with complex ghat on the split pipeline (fused passes)
    size_t split_scratch_elems = 0;  // split pass 2 with one buffer per CTA: its global lines
    int run_passes = 7;              // passes a launch runs (bits 1, 2, 4); conv_apply_multi only
    const void *w_in = nullptr;      // pass 2's input spectrum when not the workspace (conv_apply_multi)
    int device;
    cudaStream_t setup_stream = nullptr;  // private stream for plan-time device work
    int elems;  // complex elements per thread in the transform kernels
    bool tws;   // twiddle table staged in shared memory
    bool fused; // passes on the fused transform (global-memory first/last stages)
    bool long_lines = false;                 // lines beyond one CTA: four-step FP64 pipeline (fsmask.cu)
    wsc::LongLines *longl = nullptr;
    // conv_apply_kernels: for the duration of one launch, each density's multiplier table
    int nsel = 0;
    const void *sel[WSC_MAX_SEL] = {};
    int ed = 0; // fused: 16 * first radix + last radix
    wsc::FFTDesc fft;
    wsc::FFTDesc *fft_dev = nullptr;  // device copy read by the pass kernels
    int *dev_err = nullptr;           // device status word, in the stage-table allocation
    // FP64 moment quadrant [k2][k1], k1, k2 <= Mb/2: real or complex (ghat_bytes)
    double *ghat_paper = nullptr;
    // FP64 multiplier of the passes, quadrant [k2][k1], k1, k2 < h: the moments (aliases ghat_paper)
    // or the compact-embedding table (table_bytes)
    double *ghat64 = nullptr;
    size_t table_bytes = 0;
    // FP32 copy for FP32 plans (float or float2)
    void *ghat32 = nullptr;
    size_t ghat_bytes = 0;
    // twiddle table exp(-2 pi i t / M), t in [0, M), plan precision
    void *tw = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    wsc::LaunchShape rows, cols, inv;  // inv: fused pass 3 (twiddles always from global memory)
    // FP64 companion plan used as the outer operator of mixed-precision refinement (owned)
    conv_plan_s *fp64_twin = nullptr;
    // per-pass timing instrumentation
    bool timing = false;
    std::vector<std::array<cudaEvent_t, 4>> tev_used, tev_free;
    // host-buffer pipeline (host_io.cu), created by the first conv_apply_host
    struct HostPipe *hostpipe = nullptr;
    struct HostMulti *hostmulti = nullptr;  // conv_apply_host_multi's slots (on its first plan)
    // Krylov workspace of ls_solve (ls.cu), created by the first solve
    wsc::LsCache *ls_cache = nullptr;
    // device address of conv_apply_noalloc's fixed scratch array (noalloc.cu), looked up when the
    // plan is built; NULL with the reason in noalloc_error when the lookup failed
    void *noalloc_scratch = nullptr;
    std::string noalloc_error;
};

namespace wsc {
// plan.cu: timing marks; returns the event set for this apply (nullptr when timing is off)
cudaEvent_t *timing_slot(conv_plan_s *p);
// plan.cu: the argument checks of every apply entry point
conv_status check_apply(conv_plan_s *p, const void *u, const void *mask, const void *out, int batch,
                        double alpha_im, void *workspace, void **ws);
// passes.cu
conv_status launch_pipeline(conv_plan_s *p, const void *u, const void *mask, void *out, int batch,
                            double alpha_re, double alpha_im, double beta, void *ws,
                            cudaStream_t st);
conv_status select_transform(conv_plan_s *p);
// ghat.cu
conv_status build_ghat(conv_plan_s *p);
conv_status copy_ghat(conv_plan_s *p, const conv_plan_s *src);  // src's FP64 tables, no recomputation
// moments.cu: the Sec. 2.3 quadrature or localized moments into the plan's moment quadrant
conv_status build_moments_numeric(conv_plan_s *p, double scale, double *table, cudaStream_t st);
void bessel_k01_host(double x, double *k0, double *k1);
// plan.cu: the FP64 C2C twin of an FP32 plan (refinement residuals), tables copied from it
conv_status conv_plan_twin(const conv_plan_s *p, conv_plan_s **twin);
size_t spectrum_elems(const conv_plan_s *p);  // complex elements of the workspace per density
void destroy_hostpipe(conv_plan_s *p);          // host_io.cu (both host pipelines)
void destroy_ls_cache(conv_plan_s *p);          // ls.cu
void noalloc_lookup(conv_plan_s *p);             // noalloc.cu: address of the fixed scratch array
// fsmask.cu: the pipeline for transform lines beyond one CTA
conv_status long_lines_init(conv_plan_s *p);
void long_lines_destroy(conv_plan_s *p);
size_t long_lines_ws_bytes(const conv_plan_s *p);
conv_status long_lines_apply(conv_plan_s *p, const void *u, const void *mask, void *out, int batch, double are,
                             double aim, double beta, void *ws, cudaStream_t st);
size_t workspace_bytes(const conv_plan_s *p, int batch);  // plan.cu: conv_workspace_size
bool fault_take(int kind);                      // plan.cu: consume one armed injected fault
// plan.cu: free a plan; wait_device = false only when no queued or running work uses it
void plan_release(conv_plan_s *p, bool wait_device);
// dmem.cu: device memory from a stream-ordered pool (no implicit synchronisation); dev_free only
// for memory no queued or running work reads or writes
cudaError_t dev_alloc(void **ptr, size_t bytes);
template <class P> cudaError_t dev_alloc(P **ptr, size_t bytes) { return dev_alloc(reinterpret_cast<void **>(ptr), bytes); }
void dev_free(void *ptr);
void dev_pool_trim(int dev);
double *pinned_slot();                          // one page-locked double (64-byte slot)
void pinned_slot_release(double *slot);
}  // namespace wsc
