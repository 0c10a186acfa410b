// passes_fused_f32_e16.cu -- FP32, 16 elements per thread: instantiations of the fused-transform pass kernels.
#include "passes_fused.cuh"

namespace wsc {
template conv_status run_fused<float, 16, 136>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<float, 16, 136, true>(int);
template int blocks_per_sm_fused<float, 16, 136, true>(int, size_t);
template conv_status set_attrs_fused<float, 16, 136, false>(int);
template int blocks_per_sm_fused<float, 16, 136, false>(int, size_t);
template conv_status run_fused<float, 16, 130>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<float, 16, 130, true>(int);
template int blocks_per_sm_fused<float, 16, 130, true>(int, size_t);
template conv_status set_attrs_fused<float, 16, 130, false>(int);
template int blocks_per_sm_fused<float, 16, 130, false>(int, size_t);
template conv_status run_fused<float, 16, 132>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<float, 16, 132, true>(int);
template int blocks_per_sm_fused<float, 16, 132, true>(int, size_t);
template conv_status set_attrs_fused<float, 16, 132, false>(int);
template int blocks_per_sm_fused<float, 16, 132, false>(int, size_t);
}  // namespace wsc
