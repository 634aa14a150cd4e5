// D3Q19 kernels with FP64 and FP32 storage.
#include "../../include/amr.h"
#include "lbm_kernels.cuh"

namespace amr {
const LbmOps* lbm_ops_d3q19_half(int storage);
const LbmOps* lbm_ops_d3q19(int storage) {
  switch (storage) {
    case AMR_F64: return Launch<3, 19, double>::ops();
    case AMR_F32: return Launch<3, 19, float>::ops();
    default: return lbm_ops_d3q19_half(storage);
  }
}
}  // namespace amr
