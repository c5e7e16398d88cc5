// rhs_mixed_m1_prim.cu -- the mixed RHS kernel, tile capacity 8x4, 256 threads, primitive reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(mixed_m1_prim, float, true, 8, 4, 3, true, 256)
