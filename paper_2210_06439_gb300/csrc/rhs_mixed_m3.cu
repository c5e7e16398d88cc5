// rhs_mixed_m3.cu -- the mixed RHS kernel, tile capacity 8x8, 1024 threads, conserved-field reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(mixed_m3, float, true, 8, 8, 1, false, 1024)
