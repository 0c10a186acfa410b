// passes_f64.cu -- FP64 instantiations of the convolution pass kernels.
#include "passes.cuh"

namespace wsc {
template conv_status run_pipeline<double, 8>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 8>(int);
template conv_status run_pipeline<double, 12>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 12>(int);
template conv_status run_pipeline<double, 24>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 24>(int);
template conv_status run_pipeline<double, 0>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 0>(int);
}  // namespace wsc
