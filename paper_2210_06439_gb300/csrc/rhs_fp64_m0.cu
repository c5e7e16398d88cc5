// rhs_fp64_m0.cu -- the fp64 RHS kernel with tile capacity 8x8.
#include "rhs_kernel.cuh"
#include "rhs_launch.h"

namespace octh {

cudaError_t rhs_prepare_fp64_m0(int nf, int *ctas_per_sm)
{
    // this unit's copy of the line-group tables
    GroupTab gs[NGROUPS];
    if (!build_group_tables(gs))
        return cudaErrorInvalidValue;
    cudaError_t t = cudaMemcpyToSymbol(c_groups, gs, sizeof gs);
    if (t != cudaSuccess)
        return t;
    const size_t sm = smem_plan(nf, sizeof(double), false, 8, 8).total;
    cudaError_t e = cudaFuncSetAttribute(rhs_kernel<double, false, 8, 8, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, rhs_kernel<double, false, 8, 8, 1>,
                                                         NTHREADS, sm);
}

cudaError_t rhs_launch_fp64_m0(int grid, cudaStream_t stream, const RhsArgs &args)
{
    const size_t sm = smem_plan(args.nf, sizeof(double), false, 8, 8).total;
    rhs_kernel<double, false, 8, 8, 1><<<grid, NTHREADS, sm, stream>>>(args);
    return cudaGetLastError();
}

}  // namespace octh
