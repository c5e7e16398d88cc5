// rhs_fp64_m2.cu -- the FP64 RHS kernel, tile capacity 8x8, 512 threads, conserved-field reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(fp64_m2, double, false, 8, 8, 1, false, 512)
