// rhs_mixed_m1.cu -- the mixed RHS kernel with tile capacity 8x4 (three CTAs per SM).
#include "rhs_kernel.cuh"
#include "rhs_launch.h"

namespace octh {

cudaError_t rhs_prepare_mixed_m1(int nf, int *ctas_per_sm)
{
    // this unit's copy of the line-group tables
    GroupTab gs[NGROUPS];
    if (!build_group_tables(gs))
        return cudaErrorInvalidValue;
    cudaError_t t = cudaMemcpyToSymbol(c_groups, gs, sizeof gs);
    if (t != cudaSuccess)
        return t;
    const size_t sm = smem_plan(nf, sizeof(float), true, 8, 4).total;
    cudaError_t e = cudaFuncSetAttribute(rhs_kernel<float, true, 8, 4, 3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, rhs_kernel<float, true, 8, 4, 3>,
                                                         NTHREADS, sm);
}

cudaError_t rhs_launch_mixed_m1(int grid, cudaStream_t stream, const RhsArgs &args)
{
    const size_t sm = smem_plan(args.nf, sizeof(float), true, 8, 4).total;
    rhs_kernel<float, true, 8, 4, 3><<<grid, NTHREADS, sm, stream>>>(args);
    return cudaGetLastError();
}

}  // namespace octh
