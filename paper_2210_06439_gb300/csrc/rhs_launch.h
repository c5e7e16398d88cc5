// rhs_launch.h -- host launchers of the RHS kernel instances.  Each instance
// (FP64 or mixed, tile capacity 8x8 or 8x4, conserved or primitive
// reconstruction) is compiled in a translation unit of its own
// (rhs_<form>_m<mode>[_prim].cu) so that they build in parallel.
#pragma once
#include <cuda_runtime.h>

#include "oct_common.cuh"

namespace octh {

// form: precision (0 FP64, 1 mixed) + 2 for primitive reconstruction; mode
// (the launch shape): 0 tile capacity 8x8 with 256 threads (one CTA per SM),
// 1 capacity 8x4 with 256 threads (two CTAs per SM for FP64, three for the
// mixed form), 2 capacity 8x8 with 512 threads (one CTA per SM), 3 capacity
// 8x8 with 1024 threads (one CTA per SM, at most 64 registers a thread).
constexpr int RHS_MODES = 4;
size_t rhs_smem_bytes(int nf, int form, int mode);
bool build_group_tables(GroupTab *groups);
cudaError_t rhs_prepare(int form, int mode, int nf, int *ctas_per_sm);
cudaError_t rhs_launch(int form, int mode, int grid, cudaStream_t stream, const RhsArgs &args);
// uniform_subgrid_kernel of a precision (0 FP64, 1 mixed) over n_sub subgrids
cudaError_t uniform_launch(int precision, int n_sub, cudaStream_t stream, const RhsArgs &args, const int *item_begin,
                           int *sub_uniform, bool write_rhs, bool only_unknown = false);
// live_items_kernel (one CTA)
cudaError_t live_items_launch(int n_sub, cudaStream_t stream, const int *sub_uniform, const int *item_begin,
                              const WorkItem *items, int grid, bool split, WorkItem *live, int *live_slot,
                              int *n_live, double *amax_tile);
// interior_record_kernel over n_sub subgrids of args.U
cudaError_t interior_record_launch(int n_sub, cudaStream_t stream, const RhsArgs &args, int *rec_uni,
                                   double *rec_val);
// uniform_from_record_kernel of a precision (item_begin: also a_max)
cudaError_t record_test_launch(int precision, int n_sub, cudaStream_t stream, const RhsArgs &args, const int *nbr,
                               const int *rec_uni, const double *rec_val, int *sub_uniform, const int *item_begin);

}  // namespace octh
