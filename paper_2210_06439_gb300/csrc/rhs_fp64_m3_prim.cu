// rhs_fp64_m3_prim.cu -- the FP64 RHS kernel, tile capacity 8x8, 1024 threads, primitive reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(fp64_m3_prim, double, false, 8, 8, 1, true, 1024)
