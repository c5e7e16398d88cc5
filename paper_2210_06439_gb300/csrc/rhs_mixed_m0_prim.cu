// rhs_mixed_m0_prim.cu -- the mixed RHS kernel, tile capacity 8x8, 256 threads, primitive reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(mixed_m0_prim, float, true, 8, 8, 1, true, 256)
