// passes_fused_f64_s11.cu -- FP64, 16 elements per thread, transform length 2^11 fixed at compile time:
// instantiations of the fused-transform pass kernels.
#include "passes_fused.cuh"

namespace wsc {
template conv_status run_fused<double, 16, 1011>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<double, 16, 1011, true>(int);
template int blocks_per_sm_fused<double, 16, 1011, true>(int, size_t);
template conv_status set_attrs_fused<double, 16, 1011, false>(int);
template int blocks_per_sm_fused<double, 16, 1011, false>(int, size_t);
}  // namespace wsc
