// rhs_instance.cuh -- host entry points of one RHS kernel instance.  Each
// instance (FP64 or mixed form; launch shape: 8x8 tiles with 256, 512 or 1024
// threads, or 8x4 tiles with 256; conserved or primitive reconstruction) is
// compiled in a translation unit of its own so that the instances build in
// parallel; each unit uploads its own copy of the line-group tables into its
// constant memory.
#pragma once
#include "rhs_kernel.cuh"
#include "rhs_launch.h"

#define OCT_RHS_INSTANCE(NAME, T, STAGED, TXM, TYM, MINB, PRIM, NT)                                               \
    namespace octh {                                                                                          \
    cudaError_t rhs_prepare_##NAME(int nf, int *ctas_per_sm)                                                  \
    {                                                                                                         \
        GroupTab gs[NGROUPS];                                                                                 \
        if (!build_group_tables(gs))                                                                          \
            return cudaErrorInvalidValue;                                                                     \
        cudaError_t t = cudaMemcpyToSymbol(c_groups, gs, sizeof gs);                                          \
        if (t != cudaSuccess)                                                                                 \
            return t;                                                                                         \
        /* the attribute is process-wide: it is set to the plan of the largest field                       \
           count, never lowered, so that handles of any field count (and the                                \
           allocation-free call) launch under it; the occupancy follows this nf */                          \
        const size_t sm = smem_plan(nf, sizeof(T), STAGED, TXM, TYM).total;                                   \
        const size_t sm_max = smem_plan(MAXNF, sizeof(T), STAGED, TXM, TYM).total;                            \
        cudaError_t e = cudaFuncSetAttribute(rhs_kernel<T, STAGED, TXM, TYM, MINB, PRIM, NT>,                     \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_max);       \
        if (e != cudaSuccess)                                                                                 \
            return e;                                                                                         \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm,                                     \
                                                             rhs_kernel<T, STAGED, TXM, TYM, MINB, PRIM, NT>,     \
                                                             NT, sm);                                         \
    }                                                                                                         \
    cudaError_t rhs_launch_##NAME(int grid, cudaStream_t stream, const RhsArgs &args)                         \
    {                                                                                                         \
        const size_t sm = smem_plan(args.nf, sizeof(T), STAGED, TXM, TYM).total;                              \
        rhs_kernel<T, STAGED, TXM, TYM, MINB, PRIM, NT><<<grid, NT, sm, stream>>>(args);                          \
        return cudaGetLastError();                                                                            \
    }                                                                                                         \
    }
