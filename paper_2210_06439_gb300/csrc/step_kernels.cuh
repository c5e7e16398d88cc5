// step_kernels.cuh -- the memory-bound kernels around the RHS: per-subgrid
// signal-speed reduction, the CFL dt reduction, the SSP-RK3 combine with
// floors and dual-energy re-synchronisation, and the uniform-level ghost fill.
#pragma once
#include "oct_common.cuh"

namespace octh {

// a_max of each subgrid = max over its work items (the items of subgrid s
// are item_begin[s] .. item_begin[s+1]-1).
__global__ void amax_subgrid_kernel(int n_sub, const int *item_begin, const double *amax_tile, double *amax)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sub)
        return;
    double m = 0.0;
    for (int t = item_begin[s]; t < item_begin[s + 1]; t++)
        m = fmax(m, amax_tile[t]);
    amax[s] = m;
}

// dt = cfl * min over items of dx_s / a_max,item (Sec. V-A, time-step size);
// min_t dx/a_t = dx / max_t a_t exactly because correctly rounded division is
// monotone.  One block of 1024 threads; writes dt[0].
// dt = cfl * min over work items of dx / a_max, capped by *dt_cap when
// dt_cap is not null and *dt_cap > 0 (the cap lives in device memory so that a
// captured step graph follows later changes of it).
__global__ void dt_kernel(int n_items, const WorkItem *items, const double *dx, const double *amax_tile, double cfl,
                          const double *dt_cap, double *dt)
{
    __shared__ double red[32];
    double m = INFINITY;
    for (int t = threadIdx.x; t < n_items; t += blockDim.x)
        m = fmin(m, dx[items[t].s] / amax_tile[t]);
    for (int o = 16; o > 0; o >>= 1)
        m = fmin(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : INFINITY;
        for (int o = 16; o > 0; o >>= 1)
            m = fmin(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if (threadIdx.x == 0) {
            double d = cfl * m;
            const double cap = dt_cap ? *dt_cap : 0.0;
            if (cap > 0.0 && cap < d)
                d = cap;
            dt[0] = d;
        }
    }
}

// dt as dt_kernel gives it, from many blocks: each block takes the min of
// dx / a_max over a strided share of the items and stores it in part[b];
// the last block to finish (a counter in device memory, returned to zero
// for the next launch) takes the min of the parts.  The min does not depend
// on the order in which the values are combined.
constexpr int DT_THREADS = 256;
constexpr int DT_MAX_BLOCKS = 304;  // two per SM of a full GB300
__global__ void __launch_bounds__(DT_THREADS) dt_blocks_kernel(int n_items, const WorkItem *items, const double *dx,
                                                               const double *amax_tile, double cfl,
                                                               const double *dt_cap, double *part, int *count,
                                                               double *dt)
{
    __shared__ double red[DT_THREADS / 32];
    __shared__ bool last;
    double m = INFINITY;
    for (int t = blockIdx.x * DT_THREADS + threadIdx.x; t < n_items; t += gridDim.x * DT_THREADS)
        m = fmin(m, dx[items[t].s] / amax_tile[t]);
    for (int o = 16; o > 0; o >>= 1)
        m = fmin(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < DT_THREADS / 32; w++)
            m = fmin(m, red[w]);
        part[blockIdx.x] = m;
        __threadfence();
        last = atomicAdd(count, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0)
        return;
    __threadfence();
    double r = INFINITY;
    for (int b = 0; b < (int)gridDim.x; b++)
        r = fmin(r, *(volatile double *)(part + b));
    double d = cfl * r;
    const double cap = dt_cap ? *dt_cap : 0.0;
    if (cap > 0.0 && cap < d)
        d = cap;
    dt[0] = d;
    *count = 0;
}

struct CombineArgs {
    int stage;            // 1, 2, 3
    const double *U0;     // state at the start of the step (ghosted layout)
    const double *X;      // stage input (ghosted layout)
    double *out;          // stage output (ghosted layout); may alias X
    const double *L;      // RHS of X (RHS layout)
    const double *dt;     // device scalar
    const int *edge;
    const long long *off, *doff;
    int nf;
    double gamma, rho_floor, eps2;
    unsigned *flags;
    // Optional (null: every subgrid cell by cell): per subgrid, 1 when the
    // ghosted block of X (uni_x) and of U0 (uni_u0) held one value per field
    // at this stage's RHS (its L is then -0.0 everywhere), and the per-subgrid
    // "interior of out changed" flags this combine writes (stages 2 and 3,
    // whose out aliases X or U0; null otherwise).
    const int *uni_x, *uni_u0;
    int *changed;
    int out_is_x, out_is_u0;
    // optional record of out (null: none): per subgrid whether the uniform
    // pass gave it one value per field, and that value ([s * MAXNF + f]).
    // In stage 1 it describes out (W) as left by the last step, on entry.
    int *out_uni;
    double *out_val;
};

// One SSP-RK3 combine (Shu-Osher) on the interior:
//   stage 1: out = X + dt L                     (X = U0)
//   stage 2: out = 3/4 U0 + 1/4 (X + dt L)
//   stage 3: out = 1/3 U0 + 2/3 (X + dt L)
// then the floors rho >= rho_floor, rho_i >= 0, the tau re-synchronisation
// tau = e_int^(1/gamma) where e_int = E - |s|^2/(2 rho) > eps2 E, and tau >= 0.
// The arithmetic of one cell (xv, lv, u0: its X, L and U0 values; u0 unused
// in stage 1); returns true when a floor fired.
template <bool S1>
__device__ __forceinline__ bool combine_cell(const CombineArgs &A, int nf, double a, double b, double dt,
                                             const double (&xv)[MAXNF], const double (&lv)[MAXNF],
                                             const double (&u0)[MAXNF], double (&u)[MAXNF])
{
#pragma unroll
    for (int f = 0; f < MAXNF; f++)
        if (f < nf) {
            const double x1 = xv[f] + dt * lv[f];
            u[f] = S1 ? x1 : a * u0[f] + b * x1;
        }
    bool fired = false;
    if (u[F_RHO] < A.rho_floor) {
        u[F_RHO] = A.rho_floor;
        fired = true;
    }
#pragma unroll
    for (int f = F_SPC; f < MAXNF; f++)
        if (f < nf) {
            const int hi = __double2hiint(u[f]);
            if (hi < 0 && ((hi & 0x7FFFFFFF) | __double2loint(u[f])) != 0) {  // negative, not -0
                u[f] = 0.0;
                fired = true;
            }
        }
    const double ei =
        u[F_EGAS] - 0.5 * (u[F_SX] * u[F_SX] + u[F_SY] * u[F_SY] + u[F_SZ] * u[F_SZ]) * rcp_nr(u[F_RHO]);
    if (ei > A.eps2 * u[F_EGAS])
        u[F_TAU] = tau_of_eint(ei, A.gamma);
    if (u[F_TAU] < 0.0) {
        u[F_TAU] = 0.0;
        fired = true;
    }
    return fired;
}

__device__ __forceinline__ int nb_slot(int dx, int dy, int dz)
{
    int n = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
    return n > 13 ? n - 1 : n;
}

// The cells of one thread of the persistent combine grid: items
// blockIdx.x, blockIdx.x + gridDim.x, ... of n_items = n_sub * parts (item i:
// subgrid i / parts, part i % parts), and within an item the interior cells
// c = part * blockDim + threadIdx + k * parts * blockDim (x fastest, so a warp
// reads whole interior rows).
// Whether subgrid s takes the combine's uniform pass: its X and (for stages
// 2 and 3) U0 blocks were found to hold one value per field, so every cell
// of it has the same inputs (L = -0.0 included) and the same result.
__device__ __forceinline__ bool uniform_item(const CombineArgs &A, int s)
{
    return A.uni_x != nullptr && A.uni_x[s] != 0 && (A.stage == 1 || A.uni_u0[s] != 0);
}

struct CombineCursor {
    int item, c, E, E3, B;
    unsigned mE;
    long long gbase, lbase, FS;
    __device__ bool next(const CombineArgs &A, int parts, int n_items)
    {
        if (c >= 0) {
            c += parts * (int)blockDim.x;
            if (c < E3)
                return true;
            item += gridDim.x;
        }
        for (; item < n_items; item += gridDim.x) {
            const int s = item / parts, part = item - s * parts;
            if (uniform_item(A, s))
                continue;  // done by the uniform pass
            E = A.edge[s];
            E3 = E * E * E;
            B = E + 2 * NG;
            FS = (long long)B * B * B;
            mE = rcp_div(E);
            gbase = A.off[s];
            lbase = A.doff[s];
            c = part * (int)blockDim.x + (int)threadIdx.x;
            if (c < E3)
                return true;
        }
        return false;
    }
    __device__ long long gi() const
    {
        const int zy = div_by(c, mE), z = div_by(zy, mE);
        return gbase + ((long long)(z + NG) * B + (zy - z * E + NG)) * B + (c - zy * E + NG);
    }
};

constexpr int COMBINE_THREADS = 256;

// The combine over all interior cells, software-pipelined: a thread issues
// the loads of its next cell before the arithmetic of the current one, so
// that each CTA keeps its memory traffic and its FP64 work in flight at the
// same time (with one cell per thread and CTA, the CTAs of an SM load, then
// compute, then store in step with each other, and the launch takes the sum
// of its memory time and its FP64 time).  Persistent grid of as many CTAs as
// fit on the GPU, whole subgrids as items.
template <bool S1>
__global__ void __launch_bounds__(COMBINE_THREADS, 1) combine_kernel(CombineArgs A, int n_items)
{
    const double dt = A.dt[0];
    const double a = A.stage == 2 ? 0.75 : 1.0 / 3.0;
    const double b = A.stage == 2 ? 0.25 : 2.0 / 3.0;
    const int nf = A.nf;
    CombineCursor cur;
    cur.item = blockIdx.x;
    cur.c = -1;
    bool have = false;
    double xp[MAXNF], lp[MAXNF], vp[MAXNF], xq[MAXNF], lq[MAXNF], vq[MAXNF];
    long long gp = 0, fsp = 0, gq = 0, fsq = 0;
    auto load = [&](double (&xv)[MAXNF], double (&lv)[MAXNF], double (&u0)[MAXNF], long long &g, long long &fs) {
        g = cur.gi();
        fs = cur.FS;
        const long long li = cur.lbase + cur.c;
#pragma unroll
        for (int f = 0; f < MAXNF; f++)
            if (f < nf) {
                xv[f] = A.X[g + f * fs];
                lv[f] = A.L[li + f * cur.E3];
                if (!S1)
                    u0[f] = A.U0[g + f * fs];
            }
    };
    bool fired = false;
    // uniform pass: the subgrids whose cells all have the same inputs get the
    // result of one cell, computed by the lanes of warp 0 for 32 of the CTA's
    // subgrids at a time; where out aliases X or U0 and the result equals the
    // value already there, nothing is written and the subgrid counts as
    // unchanged (the ghost fill after this combine then skips subgrids whose
    // whole neighbourhood is unchanged)
    __shared__ double s_u[32][MAXNF];
    __shared__ int s_todo[32];
    for (int base = blockIdx.x; base < n_items; base += 32 * gridDim.x) {
        if (threadIdx.x < 32) {
            const int item = base + (int)threadIdx.x * (int)gridDim.x;
            int todo = 0;
            if (item < n_items && uniform_item(A, item)) {
                const int E = A.edge[item], B = E + 2 * NG;
                const long long FS = (long long)B * B * B;
                const long long g0 = A.off[item] + ((long long)NG * B + NG) * B + NG;  // first interior cell
                double xv[MAXNF], lv[MAXNF], u0[MAXNF], u[MAXNF];
#pragma unroll
                for (int f = 0; f < MAXNF; f++)
                    if (f < nf) {
                        xv[f] = A.X[g0 + f * FS];
                        lv[f] = -0.0;
                        u0[f] = S1 ? 0.0 : A.U0[g0 + f * FS];
                    }
                fired |= combine_cell<S1>(A, nf, a, b, dt, xv, lv, u0, u);
                bool same = false;
                if (A.out_is_x || A.out_is_u0) {
                    same = true;
#pragma unroll
                    for (int f = 0; f < MAXNF; f++)
                        if (f < nf)
                            same &= __double_as_longlong(u[f]) == __double_as_longlong(A.out_is_x ? xv[f] : u0[f]);
                } else if (A.out_uni != nullptr && A.out_uni[item] != 0) {
                    // stage 1: out (W) still holds what the last combine that
                    // wrote it recorded
                    same = true;
#pragma unroll
                    for (int f = 0; f < MAXNF; f++)
                        if (f < nf)
                            same &= __double_as_longlong(u[f]) ==
                                    __double_as_longlong(A.out_val[(long long)item * MAXNF + f]);
                }
#pragma unroll
                for (int f = 0; f < MAXNF; f++)
                    s_u[threadIdx.x][f] = u[f];
                todo = same ? 0 : 1;
                if (A.changed != nullptr)
                    A.changed[item] = todo;
                if (A.out_uni != nullptr) {
                    A.out_uni[item] = 1;
#pragma unroll
                    for (int f = 0; f < MAXNF; f++)
                        if (f < nf)
                            A.out_val[(long long)item * MAXNF + f] = u[f];
                }
            } else if (item < n_items) {
                // done cell by cell below
                if (A.changed != nullptr)
                    A.changed[item] = 1;
                if (A.out_uni != nullptr)
                    A.out_uni[item] = 0;
            }
            s_todo[threadIdx.x] = todo;
        }
        __syncthreads();
        for (int j = 0; j < 32; j++) {
            if (!s_todo[j])
                continue;
            const int item = base + j * (int)gridDim.x;
            const int E = A.edge[item], B = E + 2 * NG, E3 = E * E * E;
            const long long FS = (long long)B * B * B;
            const unsigned mE = rcp_div(E);
            for (int c = threadIdx.x; c < E3; c += blockDim.x) {
                const int zy = div_by(c, mE), z = div_by(zy, mE);
                const long long gi =
                    A.off[item] + ((long long)(z + NG) * B + (zy - z * E + NG)) * B + (c - zy * E + NG);
#pragma unroll
                for (int f = 0; f < MAXNF; f++)
                    if (f < nf)
                        A.out[gi + f * FS] = s_u[j][f];
            }
        }
        __syncthreads();
    }
    // the other subgrids cell by cell
    have = cur.next(A, 1, n_items);
    if (have)
        load(xp, lp, vp, gp, fsp);
    while (have) {
        // the next cell's loads, then this cell's arithmetic and stores
        const bool more = cur.next(A, 1, n_items);
        if (more)
            load(xq, lq, vq, gq, fsq);
        double u[MAXNF];
        fired |= combine_cell<S1>(A, nf, a, b, dt, xp, lp, vp, u);
#pragma unroll
        for (int f = 0; f < MAXNF; f++)
            if (f < nf)
                A.out[gp + f * fsp] = u[f];
        if (more) {
#pragma unroll
            for (int f = 0; f < MAXNF; f++) {
                xp[f] = xq[f];
                lp[f] = lq[f];
                vp[f] = vq[f];
            }
            gp = gq;
            fsp = fsq;
        }
        have = more;
    }
    if (fired)
        atomicOr(A.flags, 2u);
}

// The ghost shell of a subgrid of edge E, enumerated as: the two z slabs
// (3 planes of B x B each, lower first), then the two y slabs within the
// interior z range (3 rows of B each per plane), then the two x slabs within
// the interior y and z ranges (3 columns each); coords(q) gives entry q's
// position (x, y, z), relative to the interior origin.
struct GhostShell {
    int E, B, nzs, nys, nxs, total;
    unsigned m_B, m_E, m_nzs, m_nys, m_nxs;  // reciprocals for div_by
    __device__ explicit GhostShell(int e)
        : E(e), B(e + 2 * NG), nzs(NG * B * B), nys(NG * B * e), nxs(NG * e * e),
          total(2 * nzs + 2 * nys + 2 * nxs), m_B(rcp_div(B)), m_E(rcp_div(e)), m_nzs(rcp_div(nzs)),
          m_nys(rcp_div(nys)), m_nxs(rcp_div(nxs))
    {
    }
    __device__ void coords(int q, int g[3]) const
    {
        if (q < 2 * nzs) {
            const int side = div_by(q, m_nzs), r = q - side * nzs;
            const int a = div_by(r, m_B), b = div_by(a, m_B);
            g[0] = r - a * B - NG;
            g[1] = a - b * B - NG;
            g[2] = b + (side ? E : -NG);
        } else if (q < 2 * nzs + 2 * nys) {
            const int r0 = q - 2 * nzs, side = div_by(r0, m_nys), r = r0 - side * nys;
            const int a = div_by(r, m_B);
            g[0] = r - a * B - NG;
            g[1] = a % NG + (side ? E : -NG);
            g[2] = a / NG;
        } else {
            const int r0 = q - 2 * nzs - 2 * nys, side = div_by(r0, m_nxs), r = r0 - side * nxs;
            const int a = r / NG, b = div_by(a, m_E);
            g[0] = r - a * NG + (side ? E : -NG);
            g[1] = a - b * E;
            g[2] = b;
        }
    }
};

// Ghost fill on a uniform level, one block per subgrid: each ghost cell
// copies the matching interior cell of the neighbour subgrid; along an axis
// whose face neighbour is missing (-1, a domain edge) the nearest interior
// cell is copied instead (zero-gradient outflow).  Interiors are only read.
// Ghost cells are enumerated directly (z slabs below and above the interior,
// then y slabs, then x slabs of the remaining rows); a thread loads all fields
// of its cell before storing them.
// The ghost cells of subgrid s, by all threads of the block.
__device__ __forceinline__ void ghost_fill_block(double *U, int E, const long long *off, int nf, const int *nbr,
                                                 unsigned *flags, int s)
{
    const int B = E + 2 * NG;
    const long long FS = (long long)B * B * B;
    const int *nb = nbr + 26 * (long long)s;
    const GhostShell sh(E);
    bool err = false;
    for (int q = threadIdx.x; q < sh.total; q += blockDim.x) {
        int g[3];
        sh.coords(q, g);
        const long long di = off[s] + ((long long)(g[2] + NG) * B + (g[1] + NG)) * B + (g[0] + NG);
        int d[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            d[a] = g[a] < 0 ? -1 : (g[a] >= E ? 1 : 0);
            if (d[a] != 0) {
                int dd[3] = {0, 0, 0};
                dd[a] = d[a];
                if (nb[nb_slot(dd[0], dd[1], dd[2])] < 0) {
                    g[a] = d[a] < 0 ? 0 : E - 1;
                    d[a] = 0;
                }
            }
        }
        int src = s;
        if (d[0] || d[1] || d[2]) {
            src = nb[nb_slot(d[0], d[1], d[2])];
            if (src < 0) {
                err = true;
                continue;
            }
        }
        const long long si = off[src] + ((long long)(g[2] - d[2] * E + NG) * B + (g[1] - d[1] * E + NG)) * B +
                             (g[0] - d[0] * E + NG);
        double v[MAXNF];
#pragma unroll
        for (int f = 0; f < MAXNF; f++)
            if (f < nf)
                v[f] = U[si + f * FS];
#pragma unroll
        for (int f = 0; f < MAXNF; f++)
            if (f < nf)
                U[di + f * FS] = v[f];
    }
    if (err)
        atomicOr(flags, 4u);  // OCT_FLAG_NO_SOURCE
}

// With `changed` (per subgrid: its interior may have changed since U's
// ghosts were last valid), a subgrid whose own and 26 neighbours' interiors
// are all unchanged keeps its ghosts as they are.
__global__ void ghost_fill_kernel(double *U, int E, const long long *off, int nf, const int *nbr, unsigned *flags,
                                  const int *changed)
{
    const int s = blockIdx.x;
    if (changed != nullptr) {
        int ch = 0;
        if (threadIdx.x < 27) {
            const int t = threadIdx.x == 26 ? s : nbr[26 * (long long)s + threadIdx.x];
            ch = t >= 0 && changed[t] != 0;
        }
        if (!__syncthreads_or(ch))
            return;
    }
    ghost_fill_block(U, E, off, nf, nbr, flags, s);
}

// Ghost fill across refinement levels from a host-built plan: entry q of
// subgrid s (ghost cells enumerated as in ghost_fill_kernel) holds the source
// subgrid in x -- bit 31 set: the mean of the 2x2x2 cells starting at the
// source index; bit 30 set: limited linear prolongation from that coarse
// cell; neither: a copy -- and in y the source cell's index in its ghosted
// block (bits 0..15), for a prolongation also the upper-half flags of the
// fine cell per axis (bits 16..18) and the usable-slope axes (bits 19..21).
// Pass 0 does the copies and means (they read interiors only), pass 1 the
// prolongations (they also read coarse ghosts of pass 0).  The 8 cells of a
// mean are summed in z, y, x order; a prolongation is u + t/4 with
// t = s_x d_x + s_y d_y + s_z d_z summed in that order, d the minmod slope.
__global__ void amr_ghost_kernel(double *U, int E, const long long *off, int nf, const int2 *plan, int pass)
{
    const int s = blockIdx.x;
    const int B = E + 2 * NG;
    const long long FS = (long long)B * B * B;
    const GhostShell sh(E);
    const int2 *pl = plan + (long long)s * sh.total;
    for (int q = threadIdx.x; q < sh.total; q += blockDim.x) {
        const int2 e = pl[q];
        const bool prolong = (e.x & 0x40000000) && e.x >= 0;
        if (prolong != (pass == 1))
            continue;
        int g[3];
        sh.coords(q, g);
        const long long di = off[s] + ((long long)(g[2] + NG) * B + (g[1] + NG)) * B + (g[0] + NG);
        const int t = e.x & 0x3FFFFFFF;
        double v[MAXNF];
        if (prolong) {
            const long long si = off[t] + (e.y & 0xFFFF);
            const int par = (e.y >> 16) & 7, mask = (e.y >> 19) & 7;
            const long long step[3] = {1, B, (long long)B * B};
#pragma unroll
            for (int f = 0; f < MAXNF; f++)
                if (f < nf) {
                    const double *c = U + si + f * FS;
                    const double u = c[0];
                    double acc = 0.0;
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        double d = 0.0;
                        if ((mask >> a) & 1) {
                            const double up = __dsub_rn(c[step[a]], u), dn = __dsub_rn(u, c[-step[a]]);
                            d = __dmul_rn(up, dn) > 0.0 ? (fabs(up) < fabs(dn) ? up : dn) : 0.0;
                        }
                        const double sd = ((par >> a) & 1) ? d : -d;
                        acc = a == 0 ? sd : __dadd_rn(acc, sd);
                    }
                    v[f] = __dadd_rn(u, __dmul_rn(acc, 0.25));
                }
        } else if (e.x < 0) {
            const long long si = off[t] + e.y;
#pragma unroll
            for (int f = 0; f < MAXNF; f++)
                if (f < nf) {
                    const double *c = U + si + f * FS;
                    double sum = 0.0;
                    for (int dz = 0; dz < 2; dz++)
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++)
                                sum += c[(long long)dz * B * B + dy * B + dx];
                    v[f] = sum / 8.0;
                }
        } else {
            const long long si = off[t] + e.y;
#pragma unroll
            for (int f = 0; f < MAXNF; f++)
                if (f < nf)
                    v[f] = U[si + f * FS];
        }
#pragma unroll
        for (int f = 0; f < MAXNF; f++)
            if (f < nf)
                U[di + f * FS] = v[f];
    }
}

// One flux correction at a coarse-fine face: the coarse cell's RHS entry d
// (field 0, in the dU/dt array) of subgrid s, its own flux on the face at fc
// and the first of the 2x2 fine fluxes at ff (field 0, in the face array),
// side 1 for the coarse cell's upper face.
struct RefluxCorr {
    long long d, fc, ff;
    int s, side;
};

// Flux correction at coarse-fine faces: one thread per coarse cell, which
// applies its corrections (first[i] .. first[i+1]-1, in axis order) field by
// field: the coarse flux is replaced by the mean of the 4 fine fluxes, added
// first-tangential-index fastest and scaled by 1/4.
__global__ void reflux_kernel(double *dUdt, const double *faces, const RefluxCorr *corr, const int *first, int ncell,
                              int nf, int E, const double *dx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell)
        return;
    const long long EE = (long long)E * E, E3 = EE * E;
    const int c0 = first[i], c1 = first[i + 1];
    for (int f = 0; f < nf; f++) {
        double *dp = dUdt + corr[c0].d + f * E3;
        double d = *dp;
        for (int c = c0; c < c1; c++) {
            const RefluxCorr C = corr[c];
            const double *q = faces + C.ff + f * EE;
            const double Ff = (((q[0] + q[1]) + q[E]) + q[E + 1]) * 0.25;
            const double Fc = faces[C.fc + f * EE];
            const double h = dx[C.s];
            d += C.side ? (Fc - Ff) / h : (Ff - Fc) / h;
        }
        *dp = d;
    }
}

// Primitive variables for reconstruction, one ghosted block per CTA:
// w = (rho, v, p, tau, X_i = rho_i / rho) of every cell, ghosts included,
// in the layout of the state.  p comes from the dual-energy switch: the
// kinetic remainder e = E - |s|^2 / (2 rho), or tau^gamma when e < eps1 E.
// A cell with rho not positive and finite, or p negative or not finite,
// raises the non-physical flag (bit 0).
__global__ void prim_cells_kernel(const double *U, double *W, const int *edge, const long long *off, int nf,
                                  double gamma, double eps1, unsigned *flags)
{
    const int s = blockIdx.x;
    const int B = edge[s] + 2 * NG;
    const long long FS = (long long)B * B * B;
    const double *u = U + off[s];
    double *w = W + off[s];
    bool bad = false;
    for (long long c = threadIdx.x; c < FS; c += blockDim.x) {
        const double rho = u[c], sx = u[FS + c], sy = u[2 * FS + c], sz = u[3 * FS + c];
        const double E = u[4 * FS + c], tau = u[5 * FS + c];
        const double ir = rcp_nr(rho);
        const double vx = sx * ir, vy = sy * ir, vz = sz * ir;
        double ei = fma(-0.5, fma(sz, vz, fma(sy, vy, sx * vx)), E);
        if (ei < eps1 * E)
            ei = eint_of_tau(tau, gamma);
        const double p = (gamma - 1.0) * ei;
        w[c] = rho;
        w[FS + c] = vx;
        w[2 * FS + c] = vy;
        w[3 * FS + c] = vz;
        w[4 * FS + c] = p;
        w[5 * FS + c] = tau;
        for (int f = F_SPC; f < nf; f++)
            w[f * FS + c] = u[f * FS + c] * ir;
        const int rh = __double2hiint(rho), ph = __double2hiint(p);
        bad |= !(rh > 0 && rh < 0x7FF00000) || !(ph >= 0 && ph < 0x7FF00000);
    }
    if (bad)
        atomicOr(flags, 1u);  // non-physical state
}

}  // namespace octh
