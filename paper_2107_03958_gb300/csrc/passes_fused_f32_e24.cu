// passes_fused_f32_e24.cu -- FP32, 24 elements per thread: instantiations of the fused-transform pass kernels.
#include "passes_fused.cuh"

namespace wsc {
template conv_status run_fused<float, 24, 131>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<float, 24, 131, true>(int);
template int blocks_per_sm_fused<float, 24, 131, true>(int, size_t);
template conv_status set_attrs_fused<float, 24, 131, false>(int);
template int blocks_per_sm_fused<float, 24, 131, false>(int, size_t);
}  // namespace wsc
