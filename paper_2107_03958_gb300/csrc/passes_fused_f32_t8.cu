// passes_fused_f32_t8.cu -- FP32, 24 elements per thread, transform length 3 x 2^8 = 768 fixed at
// compile time (the period-3 grid of n = 256): instantiations of the fused-transform pass kernels.
#include "passes_fused.cuh"

namespace wsc {
template conv_status run_fused<float, 24, 2008>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<float, 24, 2008, true>(int);
template int blocks_per_sm_fused<float, 24, 2008, true>(int, size_t);
template conv_status set_attrs_fused<float, 24, 2008, false>(int);
template int blocks_per_sm_fused<float, 24, 2008, false>(int, size_t);
}  // namespace wsc
