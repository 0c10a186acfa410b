// tma.cu -- tensor maps for the row passes' strided spectrum accesses (TMA tiled copies).
//
// The spectra of a row pair (or the Wr/Wi pair of one row) sit as one 16-byte (FP32) or 32-byte
// (FP64) run per k2 in W[batch][k2][j1]; a 3-D map over (inner 8-byte words, k2, batch) with box
// {words of one run, 256, 1} moves 256 such runs per copy, zero-filling (loads) or clipping
// (stores) at k2 >= h.  cuTensorMapEncodeTiled comes from the driver through the runtime's entry-
// point query, so the library does not link libcuda.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "wsconv_internal.h"

namespace wsc {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Map over `batch` x `rows` x `words` 8-byte words at `base` (rows contiguous), box
// {box_words, TMA_ROWS, 1}.  False if the driver refuses it or an alignment rule fails (16-byte
// base and strides).
bool encode_rows_map(CUtensorMap *m, const void *base, unsigned long long words, unsigned long long rows,
                     unsigned long long batch, unsigned box_words)
{
    auto fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (words * 8) % 16) return false;
    const cuuint64_t dim[3] = {words, rows, batch};
    const cuuint64_t stride[2] = {words * 8, words * 8 * rows};
    const cuuint32_t box[3] = {box_words, TMA_ROWS, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void *>(base), dim, stride, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace wsc
