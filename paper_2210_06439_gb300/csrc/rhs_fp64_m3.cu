// rhs_fp64_m3.cu -- the FP64 RHS kernel, tile capacity 8x8, 1024 threads, conserved-field reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(fp64_m3, double, false, 8, 8, 1, false, 1024)
