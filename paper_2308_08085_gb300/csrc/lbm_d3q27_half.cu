// D3Q27 kernels with 16-bit shifted storage (BF16, FP16) and FP32 arithmetic.
#include "../../include/amr.h"
#include "lbm_kernels.cuh"

namespace amr {
const LbmOps* lbm_ops_d3q27_half(int storage) {
  switch (storage) {
    case AMR_F32_BF16: return Launch<3, 27, __nv_bfloat16>::ops();
    case AMR_F32_F16: return Launch<3, 27, __half>::ops();
    default: return nullptr;
  }
}
}  // namespace amr
