// rhs_fp64_m1.cu -- the FP64 RHS kernel, tile capacity 8x4, 256 threads, conserved-field reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(fp64_m1, double, false, 8, 4, 2, false, 256)
