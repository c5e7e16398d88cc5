// rhs_dispatch.cu -- selects the RHS kernel instance of a precision and tile mode.
#include <cstring>

#include "rhs_kernel.cuh"
#include "rhs_launch.h"

namespace octh {

static void canon(const int *d, int *line, int *end)
{
    int first = d[0] ? d[0] : (d[1] ? d[1] : d[2]);
    int sg = first > 0 ? 1 : -1;
    for (int a = 0; a < 3; a++)
        line[a] = d[a] * sg;
    *end = first > 0 ? 1 : 0;
}

// The 13 PPM lines in 4 groups (the axis lines x, y, z; the xy and xz
// diagonals; the yz diagonals; the body diagonals) and,
// per group, its face quadrature points, per-axis point lists and the +z ends
// it carries to the next plane (see rhs_kernel.cuh).
bool build_group_tables(GroupTab *gs)
{
    static const int L[13][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1},
                                 {0, 1, 1}, {0, 1, -1}, {1, 1, 1}, {1, -1, -1}, {1, -1, 1}, {1, 1, -1}};
    static const int GL[NGROUPS][5] = {{3, 0, 1, 2}, {4, 3, 4, 5, 6}, {2, 7, 8}, {4, 9, 10, 11, 12}};
    for (int g = 0; g < NGROUPS; g++) {
        GroupTab &G = gs[g];
        memset(&G, 0, sizeof G);
        G.nl = GL[g][0];
        for (int l = 0; l < G.nl; l++)
            for (int a = 0; a < 3; a++) {
                G.line[l][a] = L[GL[g][1 + l]][a];
                if (G.line[l][a])
                    G.has[a] = 1;
            }
        auto find = [&](const int *d) -> int {
            int ln[3], e;
            canon(d, ln, &e);
            for (int l = 0; l < G.nl; l++)
                if (ln[0] == G.line[l][0] && ln[1] == G.line[l][1] && ln[2] == G.line[l][2])
                    return 2 * l + e;
            return -1;
        };
        for (int k = 0; k < 3; k++) {
            int a1 = (k == 0) ? 1 : 0, a2 = (k == 2) ? 1 : 2;
            for (int t2 = -1; t2 <= 1; t2++)
                for (int t1 = -1; t1 <= 1; t1++) {
                    int dL[3] = {0, 0, 0}, dR[3] = {0, 0, 0};
                    dL[k] = 1;
                    dR[k] = -1;
                    dL[a1] = dR[a1] = t1;
                    dL[a2] = dR[a2] = t2;
                    int ls = find(dL), rs = find(dR);
                    if (ls < 0 || rs < 0)
                        continue;
                    int p = G.npt++;
                    G.axis[p] = (signed char)k;
                    G.wcls[p] = (signed char)((t1 != 0) + (t2 != 0));
                    G.rslot[p] = (signed char)rs;
                    G.lslot[p] = (signed char)(k == 2 ? 16 + (t2 + 1) * 3 + (t1 + 1) : ls);
                }
        }
        int cnt[3] = {0, 0, 0};
        for (int p = 0; p < G.npt; p++) {
            int k = G.axis[p];
            G.apt[k][cnt[k]++] = (signed char)p;
        }
        G.napt = cnt[0] > cnt[1] ? (cnt[0] > cnt[2] ? cnt[0] : cnt[2]) : (cnt[1] > cnt[2] ? cnt[1] : cnt[2]);
        for (int k = 0; k < 3; k++)
            G.nax[k] = cnt[k];
        for (int l = 0; l < G.nl; l++) {
            if (!G.line[l][2])
                continue;
            int end = G.line[l][2] > 0 ? 1 : 0;
            int sg = end ? 1 : -1;
            int dxe = G.line[l][0] * sg, dye = G.line[l][1] * sg;
            G.zp_src[G.nzp] = (signed char)(2 * l + end);
            G.zp_dst[G.nzp] = (signed char)((dye + 1) * 3 + (dxe + 1));
            G.nzp++;
        }
    }
    return true;
}

#define OCT_DECLARE(NAME)                                         \
    cudaError_t rhs_prepare_##NAME(int nf, int *ctas_per_sm); \
    cudaError_t rhs_launch_##NAME(int grid, cudaStream_t stream, const RhsArgs &args);
OCT_DECLARE(fp64_m0)
OCT_DECLARE(fp64_m1)
OCT_DECLARE(fp64_m2)
OCT_DECLARE(mixed_m0)
OCT_DECLARE(mixed_m1)
OCT_DECLARE(mixed_m2)
OCT_DECLARE(fp64_m0_prim)
OCT_DECLARE(fp64_m1_prim)
OCT_DECLARE(fp64_m2_prim)
OCT_DECLARE(mixed_m0_prim)
OCT_DECLARE(mixed_m1_prim)
OCT_DECLARE(mixed_m2_prim)
OCT_DECLARE(fp64_m3)
OCT_DECLARE(mixed_m3)
OCT_DECLARE(fp64_m3_prim)
OCT_DECLARE(mixed_m3_prim)
#undef OCT_DECLARE

namespace {
using prepare_fn = cudaError_t (*)(int, int *);
using launch_fn = cudaError_t (*)(int, cudaStream_t, const RhsArgs &);
// [form][mode]; form = precision + 2 * (primitive reconstruction)
const prepare_fn k_prepare[4][RHS_MODES] = {
    {rhs_prepare_fp64_m0, rhs_prepare_fp64_m1, rhs_prepare_fp64_m2, rhs_prepare_fp64_m3},
    {rhs_prepare_mixed_m0, rhs_prepare_mixed_m1, rhs_prepare_mixed_m2, rhs_prepare_mixed_m3},
    {rhs_prepare_fp64_m0_prim, rhs_prepare_fp64_m1_prim, rhs_prepare_fp64_m2_prim, rhs_prepare_fp64_m3_prim},
    {rhs_prepare_mixed_m0_prim, rhs_prepare_mixed_m1_prim, rhs_prepare_mixed_m2_prim, rhs_prepare_mixed_m3_prim}};
const launch_fn k_launch[4][RHS_MODES] = {
    {rhs_launch_fp64_m0, rhs_launch_fp64_m1, rhs_launch_fp64_m2, rhs_launch_fp64_m3},
    {rhs_launch_mixed_m0, rhs_launch_mixed_m1, rhs_launch_mixed_m2, rhs_launch_mixed_m3},
    {rhs_launch_fp64_m0_prim, rhs_launch_fp64_m1_prim, rhs_launch_fp64_m2_prim, rhs_launch_fp64_m3_prim},
    {rhs_launch_mixed_m0_prim, rhs_launch_mixed_m1_prim, rhs_launch_mixed_m2_prim, rhs_launch_mixed_m3_prim}};
}  // namespace

size_t rhs_smem_bytes(int nf, int form, int mode)
{
    const int precision = form & 1;
    return smem_plan(nf, precision == 0 ? 8 : 4, precision != 0, 8, mode == 1 ? 4 : 8).total;
}

cudaError_t rhs_prepare(int form, int mode, int nf, int *ctas_per_sm)
{
    if (form < 0 || form > 3 || mode < 0 || mode >= RHS_MODES)
        return cudaErrorInvalidValue;
    return k_prepare[form][mode](nf, ctas_per_sm);
}

cudaError_t rhs_launch(int form, int mode, int grid, cudaStream_t stream, const RhsArgs &args)
{
    if (form < 0 || form > 3 || mode < 0 || mode >= RHS_MODES)
        return cudaErrorInvalidValue;
    return k_launch[form][mode](grid, stream, args);
}

cudaError_t uniform_launch(int precision, int n_sub, cudaStream_t stream, const RhsArgs &args, const int *item_begin,
                           int *sub_uniform, bool write_rhs, bool only_unknown)
{
    if (n_sub <= 0)
        return cudaSuccess;
    if (precision == 0)
        uniform_subgrid_kernel<double><<<n_sub, UNI_THREADS, 0, stream>>>(args, item_begin, sub_uniform, write_rhs,
                                                                          only_unknown);
    else
        uniform_subgrid_kernel<float><<<n_sub, UNI_THREADS, 0, stream>>>(args, item_begin, sub_uniform, write_rhs,
                                                                         only_unknown);
    return cudaGetLastError();
}

cudaError_t live_items_launch(int n_sub, cudaStream_t stream, const int *sub_uniform, const int *item_begin,
                              const WorkItem *items, int grid, bool split, WorkItem *live, int *live_slot,
                              int *n_live, double *amax_tile)
{
    live_items_kernel<<<1, LIVE_THREADS, 0, stream>>>(n_sub, sub_uniform, item_begin, items, grid, split ? 1 : 0,
                                                      live, live_slot, n_live, amax_tile);
    return cudaGetLastError();
}

cudaError_t interior_record_launch(int n_sub, cudaStream_t stream, const RhsArgs &args, int *rec_uni,
                                   double *rec_val)
{
    if (n_sub <= 0)
        return cudaSuccess;
    constexpr int per = REC_THREADS / 32;  // one warp per subgrid
    interior_record_kernel<<<(n_sub + per - 1) / per, REC_THREADS, 0, stream>>>(args.U, args.edge, args.off, args.nf,
                                                                                 n_sub, rec_uni, rec_val);
    return cudaGetLastError();
}

cudaError_t record_test_launch(int precision, int n_sub, cudaStream_t stream, const RhsArgs &args, const int *nbr,
                               const int *rec_uni, const double *rec_val, int *sub_uniform, const int *item_begin)
{
    if (n_sub <= 0)
        return cudaSuccess;
    const int grid = (n_sub + 255) / 256;
    if (precision == 0)
        uniform_from_record_kernel<double><<<grid, 256, 0, stream>>>(args, n_sub, nbr, rec_uni, rec_val, sub_uniform,
                                                                      item_begin);
    else
        uniform_from_record_kernel<float><<<grid, 256, 0, stream>>>(args, n_sub, nbr, rec_uni, rec_val, sub_uniform,
                                                                     item_begin);
    return cudaGetLastError();
}

}  // namespace octh
