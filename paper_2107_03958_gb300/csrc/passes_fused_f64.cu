// passes_fused_f64.cu -- FP64 instantiations of the fused-transform pass kernels.
#include "passes_fused.cuh"

namespace wsc {
template conv_status run_fused<double, 12, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<double, 12, true>(int);
template int blocks_per_sm_fused<double, 12, true>(int, size_t);
template conv_status run_fused<double, 12, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<double, 12, false>(int);
template int blocks_per_sm_fused<double, 12, false>(int, size_t);
template conv_status run_fused<double, 24, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<double, 24, true>(int);
template int blocks_per_sm_fused<double, 24, true>(int, size_t);
template conv_status run_fused<double, 24, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<double, 24, false>(int);
template int blocks_per_sm_fused<double, 24, false>(int, size_t);
template conv_status run_fused<double, 8, true>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<double, 8, true>(int);
template int blocks_per_sm_fused<double, 8, true>(int, size_t);
template conv_status run_fused<double, 8, false>(conv_plan_s *, const void *, const void *, void *, int, double, double, double, void *, cudaStream_t);
template conv_status set_attrs_fused<double, 8, false>(int);
template int blocks_per_sm_fused<double, 8, false>(int, size_t);
}  // namespace wsc
