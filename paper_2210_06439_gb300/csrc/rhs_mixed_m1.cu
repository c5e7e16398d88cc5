// rhs_mixed_m1.cu -- the mixed RHS kernel, tile capacity 8x4, 256 threads, conserved-field reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(mixed_m1, float, true, 8, 4, 3, false, 256)
