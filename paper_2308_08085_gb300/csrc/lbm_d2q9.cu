// D2Q9 kernels (FP64 and FP32 storage).
#include "../../include/amr.h"
#include "lbm_kernels.cuh"

namespace amr {
const LbmOps* lbm_ops_d2q9(int storage) {
  switch (storage) {
    case AMR_F64: return Launch<2, 9, double>::ops();
    case AMR_F32: return Launch<2, 9, float>::ops();
    default: return nullptr;
  }
}
}  // namespace amr
