// rhs_fp64_m1_prim.cu -- the FP64 RHS kernel, tile capacity 8x4, 256 threads, primitive reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(fp64_m1_prim, double, false, 8, 4, 2, true, 256)
