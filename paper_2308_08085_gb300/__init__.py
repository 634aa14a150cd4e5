"""GB300-native block-forest AMR lattice Boltzmann library (method of arXiv
2308.08085).  The compute path is the CUDA library libamr.so (C ABI in
include/amr.h); this package holds its build script and ctypes binding."""
from .amr import (AMR_BLOCKS, AMR_COORDS, AMR_COUNTS, AMR_F, AMR_FORCE, AMR_GAPS, AMR_IDSETS,
                  AMR_MASKS, AMR_MASS, AMR_NBR, AMR_NBR_CHILD, AMR_RHO_U, AmrBatch, AmrError,
                  AmrLBM, Cells, Mlp, cells_table, load_library)

__all__ = ["AmrLBM", "AmrBatch", "Mlp", "Cells", "cells_table", "AmrError", "load_library", "AMR_RHO_U", "AMR_F", "AMR_BLOCKS",
           "AMR_COORDS", "AMR_NBR", "AMR_NBR_CHILD", "AMR_IDSETS", "AMR_GAPS", "AMR_MASKS",
           "AMR_COUNTS", "AMR_MASS", "AMR_FORCE"]
