// rhs_mixed_m2.cu -- the mixed RHS kernel, tile capacity 8x8, 512 threads, conserved-field reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(mixed_m2, float, true, 8, 8, 1, false, 512)
