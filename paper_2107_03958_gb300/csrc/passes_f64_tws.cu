// passes_f64_tws.cu -- FP64, twiddles staged in shared memory instantiations of the convolution pass kernels.
#include "passes.cuh"

namespace wsc {
template conv_status run_pipeline<double, 8, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 8, true>(int);
template int blocks_per_sm<double, 8, true>(int, size_t);
template conv_status run_pipeline<double, 12, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 12, true>(int);
template int blocks_per_sm<double, 12, true>(int, size_t);
template conv_status run_pipeline<double, 24, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs<double, 24, true>(int);
template int blocks_per_sm<double, 24, true>(int, size_t);
}  // namespace wsc
