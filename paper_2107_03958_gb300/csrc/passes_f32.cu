// passes_f32.cu -- FP32 instantiations of the convolution pass kernels.
#include "passes.cuh"

namespace wsc {
template conv_status run_pipeline<float, 12>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 12>(int);
template conv_status run_pipeline<float, 16>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 16>(int);
template conv_status run_pipeline<float, 24>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 24>(int);
template conv_status run_pipeline<float, 0>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<float, 0>(int);
}  // namespace wsc
