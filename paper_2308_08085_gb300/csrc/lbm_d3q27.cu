// D3Q27 kernels with FP64 and FP32 storage.
#include "../../include/amr.h"
#include "lbm_kernels.cuh"

namespace amr {
const LbmOps* lbm_ops_d3q27_half(int storage);
const LbmOps* lbm_ops_d3q27(int storage) {
  switch (storage) {
    case AMR_F64: return Launch<3, 27, double>::ops();
    case AMR_F32: return Launch<3, 27, float>::ops();
    default: return lbm_ops_d3q27_half(storage);
  }
}
}  // namespace amr
