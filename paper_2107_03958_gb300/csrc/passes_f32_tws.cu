// passes_f32_tws.cu -- FP32, twiddles staged in shared memory instantiations of the convolution pass kernels.
#include "passes.cuh"

namespace wsc {
template conv_status run_pipeline<float, 16, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 16, true>(int);
template int blocks_per_sm<float, 16, true>(int, size_t);
template conv_status run_pipeline<float, 24, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 24, true>(int);
template int blocks_per_sm<float, 24, true>(int, size_t);
}  // namespace wsc
