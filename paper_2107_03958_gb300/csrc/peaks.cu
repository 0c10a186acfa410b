// peaks.cu -- measured roofline denominators on the running GPU: HBM copy bandwidth and FP64/FP32
// FMA throughput (no counterpart in the paper; used to report achieved fractions).
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

__global__ void k_copy4(const float4 *__restrict__ a, float4 *__restrict__ b, size_t n4)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// Independent FMA chains per thread; the result is stored so nothing is optimised away.
template <typename T>
__global__ void k_fma(T *out, int iters, T seed)
{
    T x0 = seed + threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    const T m = (T)0.9999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            x0 = x0 * m + c; x1 = x1 * m + c; x2 = x2 * m + c; x3 = x3 * m + c;
            x4 = x4 * m + c; x5 = x5 * m + c; x6 = x6 * m + c; x7 = x7 * m + c;
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace wsc

using namespace wsc;

extern "C" conv_status conv_measure_peaks(size_t bytes, double *copy_gbs, double *fp64_tflops,
                                          double *fp32_tflops)
{
    int dev = 0, sms = 0;
    WSC_CUDA(cudaGetDevice(&dev));
    WSC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaEvent_t e0, e1;
    WSC_CUDA(cudaEventCreate(&e0));
    WSC_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    if (copy_gbs) {
        size_t n4 = bytes / 2 / 16;
        if (n4 < 1024) n4 = 1024;
        float4 *a = nullptr, *b = nullptr;
        if (cudaMalloc(&a, n4 * 16) != cudaSuccess || cudaMalloc(&b, n4 * 16) != cudaSuccess) {
            cudaGetLastError();
            if (a) cudaFree(a);
            return fail(CONV_ENOMEM, "peak buffers");
        }
        cudaMemset(a, 0, n4 * 16);
        int blocks = sms * 8;
        double best = 0.0;
        for (int rep = 0; rep < 12; ++rep) {
            cudaEventRecord(e0);
            k_copy4<<<blocks, 512>>>(a, b, n4);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 2) best = std::max(best, 2.0 * n4 * 16 / (ms * 1e-3) / 1e9);
        }
        *copy_gbs = best;
        cudaFree(a);
        cudaFree(b);
    }
    const int threads = 256, blocks = sms * 16, iters = 2048;
    void *out = nullptr;
    if (cudaMalloc(&out, (size_t)threads * blocks * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(CONV_ENOMEM, "peak buffers");
    }
    if (fp64_tflops) {
        double best = 0;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0);
            k_fma<double><<<blocks / 4, threads>>>((double *)out, iters / 8, 1.0);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            double flops = 2.0 * 64.0 * (iters / 8) * (double)threads * (blocks / 4);
            if (rep >= 1) best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
        *fp64_tflops = best;
    }
    if (fp32_tflops) {
        double best = 0;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0);
            k_fma<float><<<blocks, threads>>>((float *)out, iters, 1.0f);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            double flops = 2.0 * 64.0 * iters * (double)threads * blocks;
            if (rep >= 1) best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
        *fp32_tflops = best;
    }
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    WSC_CUDA(cudaGetLastError());
    return CONV_OK;
}
