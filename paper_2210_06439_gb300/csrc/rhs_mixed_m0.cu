// rhs_mixed_m0.cu -- the mixed RHS kernel, tile capacity 8x8, 256 threads, conserved-field reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(mixed_m0, float, true, 8, 8, 1, false, 256)
