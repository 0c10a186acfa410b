// passes_f64.cu -- FP64, twiddles from global memory instantiations of the convolution pass kernels.
#include "passes.cuh"

namespace wsc {
template conv_status run_pipeline<double, 8, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 8, false>(int);
template int blocks_per_sm<double, 8, false>(int, size_t);
template conv_status run_pipeline<double, 12, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 12, false>(int);
template int blocks_per_sm<double, 12, false>(int, size_t);
template conv_status run_pipeline<double, 24, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 24, false>(int);
template int blocks_per_sm<double, 24, false>(int, size_t);
template conv_status run_pipeline<double, 0, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 0, false>(int);
template int blocks_per_sm<double, 0, false>(int, size_t);
}  // namespace wsc
