// passes_fused_f32_s8.cu -- FP32, 16 elements per thread, transform length 2^8 fixed at compile time:
// instantiations of the fused-transform pass kernels.
#include "passes_fused.cuh"

namespace wsc {
template conv_status run_fused<float, 16, 1008>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<float, 16, 1008, true>(int);
template int blocks_per_sm_fused<float, 16, 1008, true>(int, size_t);
template conv_status set_attrs_fused<float, 16, 1008, false>(int);
template int blocks_per_sm_fused<float, 16, 1008, false>(int, size_t);
}  // namespace wsc
