// tc_stage.cu -- one radix-16 Stockham stage of an FP32 length-8192 column transform computed as a
// DFT-matrix product on the 5th-generation tensor cores (tcgen05, BF16 operands split in two,
// three products, FP32 accumulation in tensor memory), timed against the same stage on the CUDA
// cores (no counterpart in the paper: this measures the tensor-core alternative for the passes'
// butterflies, Sec. 2.1's FFTs).
//
// One CTA of 512 threads holds one column (8192 complex FP32 values) in shared memory; thread j
// owns butterfly j of the stage with Ns = 16 (the column passes' second stage):
//   inputs  x[j + q 512], q < 16, times the twiddles w^{(j mod 16) q}, w = e^{-2 pi i / 256};
//   outputs y[(j / 16) 256 + (j mod 16) + 16 p] = (1/4) sum_q e^{-2 pi i p q / 16} x'_q.
// Tensor-core path: the 512 butterflies are four 128-row tiles of A (K = 32: the 16 real parts,
// then the 16 imaginary parts, as BF16 hi and lo halves); B (N = 32 outputs x K = 32) is the real
// form [[C, S], [-S, C]] / 4 of the DFT matrix, also split hi + lo.  Per tile: D = Ah Bh^T +
// Ah Bl^T + Al Bh^T in two K = 16 steps each (six tcgen05.mma, M = 128, N = 32), D in 32 columns of
// tensor memory; each warp reads its 32 rows back with tcgen05.ld.  Operands sit in shared memory
// in the canonical no-swizzle K-major layout: 8 x 16-byte core matrices, 128 bytes apart along K,
// 512 bytes apart along M (N).
// The wait for the products is an mbarrier wait bounded by one second; a wait that gives up
// records an error, waits (bounded again) for the products in flight, frees the tensor memory and
// leaves the loop.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

#define TCS_L 8192
#define TCS_THREADS 512
#define TCS_NS 16
#define TCS_WAIT_NS 1000000000ull

__device__ __forceinline__ unsigned tcs_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tcs_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool tcs_try(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tcs_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool tcs_wait(unsigned long long *bar, unsigned parity)
{
    const unsigned long long t0 = tcs_now();
    while (!tcs_try(bar, parity))
        if (tcs_now() - t0 > TCS_WAIT_NS) return false;
    return true;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets of the
// core matrices, the fixed version bits, no swizzle.
__device__ __forceinline__ unsigned long long tcs_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
           ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

// byte offset of element (row, k) in a K-major no-swizzle tile of 32 K values per row
__device__ __forceinline__ unsigned tcs_off(int row, int k)
{
    return (unsigned)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N = 32, M = 128.
#define TCS_IDESC ((1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24))

struct TcsSmem {
    float2 x[TCS_L];
    float2 y[TCS_L];
    __align__(1024) unsigned char ahi[4 * 128 * 64];
    __align__(1024) unsigned char alo[4 * 128 * 64];
    __align__(1024) unsigned char bhi[32 * 64];
    __align__(1024) unsigned char blo[32 * 64];
    float2 tw[256];
    unsigned long long bar;
    unsigned tmem;
};

// The stage's inputs of butterfly j, twiddled.
__device__ __forceinline__ void tcs_load(const TcsSmem &S, int j, float2 *v)
{
    const int k = j & (TCS_NS - 1);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float2 a = S.x[j + q * (TCS_L / 16)];
        const float2 w = S.tw[(k * q) & 255];
        v[q] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
    }
}

__device__ __forceinline__ int tcs_out(int j, int p) { return (j / TCS_NS) * (16 * TCS_NS) + (j & (TCS_NS - 1)) + p * TCS_NS; }

// mode 0: CUDA-core butterflies; mode 1: tensor cores.  reps stages, x and y swapped after each;
// check != 0: one stage, y left in place for the caller.
__global__ void __launch_bounds__(TCS_THREADS, 1) k_tc_stage(const float2 *__restrict__ in, float2 *__restrict__ out,
                                                           int reps, int mode, int *err)
{
    extern __shared__ __align__(1024) unsigned char raw[];
    TcsSmem &S = *reinterpret_cast<TcsSmem *>(raw);
    const int j = threadIdx.x, warp = j >> 5;
    const float2 *src = in + (size_t)blockIdx.x * TCS_L;
    for (int i = j; i < TCS_L; i += TCS_THREADS) S.x[i] = src[i];
    if (j < 256) {
        float sn, cs;
        sincospif(-2.0f * j / 256.0f, &sn, &cs);
        S.tw[j] = make_float2(cs, sn);
    }
    if (mode == 1) {
        // B = the real form of the 16-point DFT matrix / 4, rows n (outputs), columns k (inputs)
        for (int e = j; e < 32 * 32; e += TCS_THREADS) {
            const int n = e >> 5, k = e & 31, p = n & 15, q = k & 15;
            float sn, cs;
            sincospif(2.0f * (float)((p * q) & 15) / 16.0f, &sn, &cs);
            float b;
            if (n < 16) b = k < 16 ? cs : sn;  // Yr = sum Xr c + Xi s
            else b = k < 16 ? -sn : cs;        // Yi = sum Xi c - Xr s
            b *= 0.25f;
            const __nv_bfloat16 h = __float2bfloat16_rn(b);
            const __nv_bfloat16 l = __float2bfloat16_rn(b - __bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16 *>(S.bhi + tcs_off(n, k)) = h;
            *reinterpret_cast<__nv_bfloat16 *>(S.blo + tcs_off(n, k)) = l;
        }
        if (j == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcs_smem(&S.bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(tcs_smem(&S.tmem))
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = mode == 1 ? S.tmem : 0u;
    unsigned parity = 0;
    bool failed = false;
    float2 *X = S.x, *Y = S.y;
    for (int r = 0; r < reps && !failed; ++r) {
        float2 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float2 a = X[j + q * (TCS_L / 16)];
            const float2 w = S.tw[((j & (TCS_NS - 1)) * q) & 255];
            v[q] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
        }
        if (mode == 0) {
            dftR<16, false>(v);
            __syncthreads();  // every input read before any output lands (in-place ping-pong)
#pragma unroll
            for (int p = 0; p < 16; ++p) Y[tcs_out(j, p)] = make_float2(0.25f * v[p].x, 0.25f * v[p].y);
        } else {
            // A rows: tile j / 128, row j % 128; K = 32 (re 0..15, im 16..31), hi and lo halves
            const int t = j >> 7, row = j & 127;
            unsigned char *ah = S.ahi + t * (128 * 64), *al = S.alo + t * (128 * 64);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const __nv_bfloat16 hr = __float2bfloat16_rn(v[q].x), hi = __float2bfloat16_rn(v[q].y);
                const __nv_bfloat16 lr = __float2bfloat16_rn(v[q].x - __bfloat162float(hr));
                const __nv_bfloat16 li = __float2bfloat16_rn(v[q].y - __bfloat162float(hi));
                *reinterpret_cast<__nv_bfloat16 *>(ah + tcs_off(row, q)) = hr;
                *reinterpret_cast<__nv_bfloat16 *>(ah + tcs_off(row, 16 + q)) = hi;
                *reinterpret_cast<__nv_bfloat16 *>(al + tcs_off(row, q)) = lr;
                *reinterpret_cast<__nv_bfloat16 *>(al + tcs_off(row, 16 + q)) = li;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (j == 0) {
                for (int tt = 0; tt < 4; ++tt) {
                    const unsigned d = tmem + 32u * tt;  // columns 32 tt .. 32 tt + 31, lanes 0..127
                    for (int c = 0; c < 2; ++c) {
                        const unsigned a_h = tcs_smem(S.ahi + tt * (128 * 64)) + c * 256,
                                       a_l = tcs_smem(S.alo + tt * (128 * 64)) + c * 256;
                        const unsigned b_h = tcs_smem(S.bhi) + c * 256, b_l = tcs_smem(S.blo) + c * 256;
                        const unsigned long long da[3] = {tcs_desc(a_h, 128, 512), tcs_desc(a_h, 128, 512),
                                                          tcs_desc(a_l, 128, 512)};
                        const unsigned long long db[3] = {tcs_desc(b_h, 128, 512), tcs_desc(b_l, 128, 512),
                                                          tcs_desc(b_h, 128, 512)};
                        for (int m = 0; m < 3; ++m) {
                            const unsigned acc = (c | m) ? 1u : 0u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                                "l"(da[m]), "l"(db[m]), "r"(TCS_IDESC), "r"(acc)
                                : "memory");
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tcs_smem(&S.bar))
                             : "memory");
            }
            const bool ok = tcs_wait(&S.bar, parity);
            if (__syncthreads_or(!ok)) {
                if (j == 0) atomicExch(err, (int)CONV_ETIMEOUT);
                if (!ok) tcs_wait(&S.bar, parity);  // the products in flight, bounded again
                failed = true;
                break;
            }
            parity ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // this warp's 32 rows of its tile: lanes 32 (warp % 4) .., columns 32 (warp / 4) ..
            unsigned d[32];
            const unsigned taddr = tmem + ((unsigned)(32 * (warp & 3)) << 16) + 32u * (warp >> 2);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
                  "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]),
                  "=r"(d[15]), "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]), "=r"(d[21]),
                  "=r"(d[22]), "=r"(d[23]), "=r"(d[24]), "=r"(d[25]), "=r"(d[26]), "=r"(d[27]), "=r"(d[28]),
                  "=r"(d[29]), "=r"(d[30]), "=r"(d[31])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int p = 0; p < 16; ++p) Y[tcs_out(j, p)] = make_float2(__uint_as_float(d[p]), __uint_as_float(d[16 + p]));
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        __syncthreads();
        float2 *tmp = X;
        X = Y;
        Y = tmp;
    }
    // the last stage's result is in X after the swap
    float2 *dst = out + (size_t)blockIdx.x * TCS_L;
    for (int i = j; i < TCS_L; i += TCS_THREADS) dst[i] = X[i];
    if (mode == 1) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
    }
}

}  // namespace wsc

using namespace wsc;

extern "C" conv_status conv_measure_tc_stage(int reps, double *us_cuda_core, double *us_tensor, double *max_rel_err)
{
    if (reps < 1) return fail(CONV_EINVAL, "reps must be >= 1");
    int dev = 0, sms = 0;
    WSC_CUDA(cudaGetDevice(&dev));
    WSC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sizeof(TcsSmem) + 1024;
    WSC_CUDA(cudaFuncSetAttribute(k_tc_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const size_t N = (size_t)sms * TCS_L;
    std::vector<float2> h(N);
    unsigned s = 12345u;
    for (auto &v : h) {
        s = s * 1664525u + 1013904223u;
        const float a = (float)((s >> 8) & 0xFFFF) / 65536.0f - 0.5f;
        s = s * 1664525u + 1013904223u;
        const float b = (float)((s >> 8) & 0xFFFF) / 65536.0f - 0.5f;
        v = make_float2(a, b);
    }
    float2 *in = nullptr, *o0 = nullptr, *o1 = nullptr;
    int *err = nullptr;
    if (cudaMalloc(&in, N * sizeof(float2)) != cudaSuccess || cudaMalloc(&o0, N * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&o1, N * sizeof(float2)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(in);
        cudaFree(o0);
        cudaFree(o1);
        return fail(CONV_ENOMEM, "tensor-core stage buffers");
    }
    conv_status rc = CONV_OK;
    cudaMemcpy(in, h.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemset(err, 0, sizeof(int));
    // one stage both ways, compared
    k_tc_stage<<<sms, TCS_THREADS, smem>>>(in, o0, 1, 0, err);
    k_tc_stage<<<sms, TCS_THREADS, smem>>>(in, o1, 1, 1, err);
    cudaError_t e = cudaDeviceSynchronize();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "tensor-core stage");
    else if (herr) rc = fail((conv_status)herr, "the tensor-core stage's bounded wait gave up");
    if (rc == CONV_OK) {
        std::vector<float2> a(N), b(N);
        cudaMemcpy(a.data(), o0, N * sizeof(float2), cudaMemcpyDeviceToHost);
        cudaMemcpy(b.data(), o1, N * sizeof(float2), cudaMemcpyDeviceToHost);
        double mx = 0.0, md = 0.0;
        for (size_t i = 0; i < N; ++i) {
            mx = std::max(mx, (double)std::hypot(a[i].x, a[i].y));
            md = std::max(md, (double)std::hypot(a[i].x - b[i].x, a[i].y - b[i].y));
        }
        if (max_rel_err) *max_rel_err = mx > 0 ? md / mx : md;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        double us[2] = {0.0, 0.0};
        for (int mode = 0; mode < 2; ++mode) {
            k_tc_stage<<<sms, TCS_THREADS, smem>>>(in, o0, 2, mode, err);  // warm-up
            cudaEventRecord(e0);
            k_tc_stage<<<sms, TCS_THREADS, smem>>>(in, o0, reps, mode, err);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            us[mode] = 1e3 * ms / reps;  // one stage of one column per SM
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        e = cudaDeviceSynchronize();
        if (e == cudaSuccess) cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "tensor-core stage timing");
        else if (herr) rc = fail((conv_status)herr, "the tensor-core stage's bounded wait gave up");
        if (us_cuda_core) *us_cuda_core = us[0];
        if (us_tensor) *us_tensor = us[1];
    }
    cudaFree(in);
    cudaFree(o0);
    cudaFree(o1);
    cudaFree(err);
    return rc;
}
