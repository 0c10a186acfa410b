// passes_fused_f32_s14.cu -- FP32, 16 elements per thread, transform length 2^14 fixed at compile
// time (1024 threads of 64 registers): instantiations of the fused-transform pass kernels.
#include "passes_fused.cuh"

namespace wsc {
template conv_status run_fused<float, 16, 1014>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<float, 16, 1014, true>(int);
template int blocks_per_sm_fused<float, 16, 1014, true>(int, size_t);
template conv_status set_attrs_fused<float, 16, 1014, false>(int);
template int blocks_per_sm_fused<float, 16, 1014, false>(int, size_t);
}  // namespace wsc
