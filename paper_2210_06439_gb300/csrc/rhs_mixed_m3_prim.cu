// rhs_mixed_m3_prim.cu -- the mixed RHS kernel, tile capacity 8x8, 1024 threads, primitive reconstruction.
#include "rhs_instance.cuh"

OCT_RHS_INSTANCE(mixed_m3_prim, float, true, 8, 8, 1, true, 1024)
