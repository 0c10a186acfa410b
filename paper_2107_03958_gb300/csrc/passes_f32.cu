// passes_f32.cu -- FP32, twiddles from global memory instantiations of the convolution pass kernels.
#include "passes.cuh"

namespace wsc {
template conv_status run_pipeline<float, 16, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 16, false>(int);
template int blocks_per_sm<float, 16, false>(int, size_t);
template conv_status run_pipeline<float, 24, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 24, false>(int);
template int blocks_per_sm<float, 24, false>(int, size_t);
template conv_status run_pipeline<float, 0, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 0, false>(int);
template int blocks_per_sm<float, 0, false>(int, size_t);
}  // namespace wsc
