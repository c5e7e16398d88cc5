/*
 * oct_hydro.h -- C ABI of the GB300 (sm_103a) batched hydro right-hand side.
 *
 * The method is the hydro solver of Octo-Tiger (arXiv 2210.06439, Sec. II
 * "Solvers"): finite volumes for the inviscid Euler equations with the
 * Kurganov-Tadmor central flux, piecewise-parabolic reconstruction of the
 * evolved variables to 26 points per cell, Newton-Cotes quadrature of the
 * flux over each face; each kernel call works on sub-grids of 8^3 cells with
 * their ghost layers (Sec. II "Data-Structure", Sec. III-D), and a time step
 * takes three hydro iterations (Sec. V-B).  The paper gives no equations; the
 * readings used here are:
 *   - the conserved fields (rho, s_x, s_y, s_z, E_gas, tau, rho_1..rho_ns)
 *     are reconstructed (primitive variables on request, see
 *     oct_hydro_set_reconstruction);
 *   - PPM: Colella-Woodward 1984 interface values with monotonised-central
 *     slopes and the CW84 monotonicity constraints;
 *   - the 26 points are the 6 face centres, 12 edge midpoints and 8 corners of
 *     a cell; the value at x + d/2 comes from 1-D PPM along cells x + m d;
 *   - Newton-Cotes = tensor Simpson over the 3x3 points of a face (weights
 *     16, 4, 1 over 36);
 *   - KT flux with the local speed a_q = max(|v_n| + c) over both sides of
 *     each quadrature point; a subgrid's a_max is the max over its faces;
 *   - ideal gas with dual energy: e_int = E - |s|^2/(2 rho), replaced by
 *     tau^gamma when e_int < de_switch1 * E;
 *   - SSP-RK3 (Shu-Osher) with dt = cfl * min_s dx_s / a_max,s from the state
 *     at the start of the step; after each stage rho >= rho_floor,
 *     rho_i >= 0, tau re-synchronised when e_int > de_switch2 * E, tau >= 0.
 *
 * Data layout (all device pointers unless stated otherwise):
 *   state U  : one ghosted block per subgrid, doubles, [field][z][y][x] with
 *              B = edge + 6 cells per side (3 ghost layers), block s starting
 *              at element offsets[s]; every offset a multiple of 4 (32 bytes).
 *   dUdt     : interior only, doubles, [subgrid][field][z][y][x] with edge^3
 *              cells per field, subgrids packed in index order.
 *   neighbour table (host): 26 int32 per subgrid; direction (dx,dy,dz) in
 *              {-1,0,1}^3 \ {0} at (dz+1)*9 + (dy+1)*3 + (dx+1), minus one
 *              when that exceeds 13; -1 means a domain edge.
 *
 * Ownership: the caller owns every state, RHS and host buffer passed in.  The
 * handle owns its scratch (the RK stage state, the RHS register, per-tile
 * signal speeds, the dt slot, the work list, error flags) and its captured
 * CUDA graphs; it allocates them with cudaMalloc on the current device at
 * set-up and frees them in oct_hydro_destroy.
 *
 * Errors: every call returns an oct_status; nothing is thrown across the ABI.
 * Arguments are validated on the host before any launch.  A non-physical
 * state met on the device (rho <= 0 or a non-finite point value) sets a flag
 * that oct_hydro_get_error_flags reads; no kernel traps.  oct_hydro_last_error
 * gives the text of the calling thread's last failure.
 *
 * Streams: every call is ordered on the given CUDA stream (NULL = the legacy
 * default stream).  Only the calls that return a value to the host
 * (oct_hydro_max_dt, oct_hydro_rk_step with a non-NULL dt pointer,
 * oct_hydro_get_error_flags, the *_host calls) synchronise that stream.
 * A handle is not thread-safe: one host thread at a time per handle.  Its
 * scratch buffers and the RHS kernel's scheduling counters are per handle,
 * so work on one handle must not overlap on the GPU: issue it on one stream,
 * or order the streams with events.
 *
 * Device: a handle belongs to the device that is current at
 * oct_hydro_create; every call on it makes that device current for its
 * duration and restores the caller's device afterwards.  Streams and
 * pointers passed in must belong to that device.
 */
#ifndef OCT_HYDRO_H
#define OCT_HYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oct_hydro *oct_hydro_t;

typedef enum {
    OCT_OK = 0,
    OCT_E_ARG = -1,     /* invalid argument (size, pointer, alignment, value) */
    OCT_E_CUDA = -2,    /* a CUDA runtime call failed                         */
    OCT_E_NONPHYS = -3, /* a non-physical state was met on the device         */
    OCT_E_TIMEOUT = -4, /* a bounded device wait ran out                      */
    OCT_E_NOMEM = -5,   /* device or host allocation failed                   */
    OCT_E_STATE = -6    /* call out of order (e.g. no layout set)             */
} oct_status;

typedef enum { OCT_FP64 = 0, OCT_MIXED = 1 } oct_precision;

typedef enum { OCT_BC_GIVEN = 0, OCT_BC_PERIODIC = 1, OCT_BC_OUTFLOW = 2, OCT_BC_AMR = 3 } oct_bc;
typedef enum { OCT_RECON_CONSERVED = 0, OCT_RECON_PRIMITIVE = 1 } oct_recon;

/* Device error flags (oct_hydro_get_error_flags). */
#define OCT_FLAG_NONPHYS 0x1u  /* rho <= 0 or non-finite value at a point   */
#define OCT_FLAG_FLOOR 0x2u    /* a density, species or tau floor fired      */
/* The uniform-level ghost fill met a ghost cell with no source (a diagonal
 * neighbour missing where its face neighbours exist: an inconsistent
 * neighbour table); that cell is left as it was. */
#define OCT_FLAG_NO_SOURCE 0x4u

/* Creates a handle for n_subgrids subgrids (Sec. II "Data-Structure": one
 * kernel invocation per set of subgrids with ghost layers).
 *   edge      : 8, 12 or 16 for a uniform batch; 0 when per-subgrid edges are
 *               given to oct_hydro_set_layout.
 *   ghost     : number of ghost layers; must be 3.
 *   n_species : 0..5 (fields = 6 + n_species).
 *   gamma     : ratio of specific heats, > 1.
 * For a uniform batch the default layout is packed blocks, dx = 1/edge per
 * subgrid and ghosts given (OCT_BC_GIVEN).  Returns OCT_E_ARG for bad values,
 * OCT_E_CUDA/OCT_E_NOMEM when the device cannot be set up; *out is NULL then.
 */
oct_status oct_hydro_create(int n_subgrids, int edge, int ghost, int n_species, double gamma, oct_hydro_t *out);

/* Sets the batch layout (Sec. II "Data-Structure": the octree's leaves are
 * subgrids of 8^3 cells with ghost layers, handed to the kernels in sets;
 * Sec. III-D: one kernel call per set of subgrids).  All pointers are HOST
 * pointers and are copied.
 *   edges      : n_subgrids edges in {8, 12, 16}; NULL = the create-time edge.
 *   offsets    : n_subgrids state offsets in doubles (multiples of 4, blocks
 *                not overlapping); NULL = packed in index order.
 *   dx         : n_subgrids cell widths (> 0); NULL keeps the current ones.
 *   level      : refinement levels (informational, may be NULL).
 *   neighbours : 26 * n_subgrids int32 (see above); required when bc is
 *                OCT_BC_PERIODIC or OCT_BC_OUTFLOW, which need one common edge.
 *   bc         : oct_bc.
 * Rebuilds the work list and drops captured graphs. */
oct_status oct_hydro_set_layout(oct_hydro_t h, const int32_t *edges, const int64_t *offsets, const double *dx,
                                const int32_t *level, const int32_t *neighbours, int bc);

/* Ghost exchange across refinement levels (Sec. II "Data-Structure": an
 * adaptive octree with one subgrid per leaf).  All subgrids share one even
 * edge E; subgrid s sits at level level[s] >= 0 and covers the cells
 * origin[3s..3s+2] .. +E-1 of its level (HOST arrays, origins multiples of E),
 * in a root box of root_cells cells per side at level 0 (root_cells * 2^l at
 * level l), periodic (periodic != 0) or with outflow edges.  Each ghost cell
 * then takes: the covering cell of a subgrid at the same level (a copy); else
 * the covering cell one level coarser (prolongation by injection); else the
 * mean of the 8 cells one level finer (restriction).  In this mode the RHS
 * (oct_hydro_rhs, oct_hydro_rhs_host and every stage of oct_hydro_rk_step)
 * also applies the flux correction at coarse-fine faces: the coarse cell's
 * flux through such a face is replaced by the mean of the 4 fine fluxes on
 * it, which makes the update conservative across levels.  Sets the boundary
 * mode to OCT_BC_AMR (used by oct_hydro_fill_ghosts and oct_hydro_rk_step);
 * OCT_E_ARG when a ghost cell has no source (levels not properly nested),
 * subgrids overlap, or the arrays are invalid.  Device buffers: the ghost
 * plan (8 bytes per ghost cell) and the face fluxes of the subgrids next to
 * a level change (48 nf E^2 bytes each), held until the layout changes. */
oct_status oct_hydro_set_amr(oct_hydro_t h, const int32_t *level, const int32_t *origin, int root_cells,
                             int periodic);

/* Prolongation order of the ghost fill across levels (the order of the fine
 * ghost cells under a coarse cell; the paper does not state it): 0 (the
 * default) injection -- the coarse value; 1 limited linear -- the coarse value
 * plus, per axis, a quarter of the minmod slope of the coarse cell and its
 * two neighbours along that axis (neighbours that are themselves prolonged
 * ghosts give no slope), signed + for the upper half: t = s_x d_x + s_y d_y
 * + s_z d_z in that order, u + t/4.  The 8 children of a coarse cell average
 * to its value and no new extremum appears.  Rebuilds the ghost plan when
 * levels are set.  OCT_E_ARG for another order. */
oct_status oct_hydro_set_prolongation(oct_hydro_t h, int order);

/* Which variables PPM reconstructs (Sec. II "Solvers": the reconstruct
 * kernel yields point values of the evolved variables at 26 points per cell;
 * which variables it interpolates is not stated).  OCT_RECON_CONSERVED (the
 * default): the conserved fields themselves.  OCT_RECON_PRIMITIVE: w = (rho, v, p, tau, X_i = rho_i / rho)
 * of every cell (p from the dual-energy switch), each point turned back into
 * conserved fields (s = rho v, E = p / (gamma - 1) + rho |v|^2 / 2,
 * rho_i = rho X_i) with its reconstructed v and p used in the flux; this
 * costs one extra pass over the state per RHS and a device buffer of
 * oct_hydro_state_len doubles (allocated here or with the layout).
 * OCT_E_ARG for another value.  Both precisions support both choices; the
 * allocation-free entry point reconstructs the conserved fields only. */
oct_status oct_hydro_set_reconstruction(oct_hydro_t h, int variables);

/* Numerical parameters (Sec. II "Solvers": the explicit finite-volume
 * scheme and its CFL time step, Sec. V-A; the paper runs everything in FP64,
 * Sec. V; the mixed form and the floors and dual-energy switches are
 * readings of this library): precision (oct_precision: FP64 everywhere, or
 * reconstruction/flux arithmetic in FP32 with FP64 divergence, update,
 * floors and dt), CFL number (0 < cfl <= 1, default 0.4), density floor
 * (>= 0, default 1e-12) and the two dual-energy switches (default 1e-3 for
 * the pressure recovery and 0.1 for the tau re-synchronisation). */
oct_status oct_hydro_set_params(oct_hydro_t h, int precision, double cfl, double rho_floor, double de_switch1,
                                double de_switch2);

/* Caps dt in oct_hydro_rk_step (dt_cap > 0), e.g. to land on an output time;
 * dt_cap <= 0 removes the cap.  Waits for the device to be idle (so that no
 * step in flight sees the change), then stores the cap in device memory,
 * where the captured step graphs read it: changing it costs no recapture. */
oct_status oct_hydro_set_dt_cap(oct_hydro_t h, double dt_cap);

/* Number of doubles of the state array the layout spans, and of dUdt. */
int64_t oct_hydro_state_len(oct_hydro_t h);
int64_t oct_hydro_rhs_len(oct_hydro_t h);

/* One RHS evaluation (Sec. II "Solvers": the reconstruct and flux kernels
 * plus the finite-volume divergence): reads U (ghosts used as they are),
 * writes dUdt = -sum_k (F_k,+ - F_k,-)/dx for every interior cell and, when
 * amax is not NULL, each subgrid's max signal speed (n_subgrids doubles).
 * After oct_hydro_set_amr the coarse-fine flux correction is part of it.
 * U and dUdt must not overlap. */
oct_status oct_hydro_rhs(oct_hydro_t h, const double *U, double *dUdt, double *amax, void *cuda_stream);

/* CFL time step of state U (Sec. V-A "determination of time-step size"):
 * dt = cfl * min_s dx_s / a_max,s.  Writes it to *dt_host_out (host) and
 * synchronises the stream. */
oct_status oct_hydro_max_dt(oct_hydro_t h, const double *U, double *dt_host_out, void *cuda_stream);

/* Fills the ghost layers of U: on a uniform level from the neighbour table
 * (periodic or outflow), across levels after oct_hydro_set_amr; does
 * nothing for OCT_BC_GIVEN. */
oct_status oct_hydro_fill_ghosts(oct_hydro_t h, double *U, void *cuda_stream);

/* One SSP-RK3 time step in place (three hydro iterations per time step,
 * Sec. V-B): dt from U's signal speeds, three RHS evaluations, combines,
 * floors and dual-energy re-synchronisation, and a ghost fill after each
 * stage (unless OCT_BC_GIVEN; across levels, with the flux correction in
 * each RHS, after oct_hydro_set_amr).  On entry U's ghosts must be valid.  The
 * sequence is replayed from a CUDA graph captured on first use for this U (on
 * a non-default stream; up to 16 state pointers are remembered).
 * When dt_used_host_out is not NULL the stream is synchronised and the dt
 * used is written there. */
oct_status oct_hydro_rk_step(oct_hydro_t h, double *U, double *dt_used_host_out, void *cuda_stream);

/* End-to-end variants on HOST buffers: copy the host state in, run n_steps
 * RK3 steps (or one RHS), copy the result back.  U_host: oct_hydro_state_len
 * doubles (page-locked memory gives full copy speed); dUdt_host:
 * oct_hydro_rhs_len doubles.  The device copy of the state is owned by the
 * handle.  Synchronous.  On a uniform level (periodic or outflow, every ghost
 * cell with a source) in the default contiguous layout, oct_hydro_rk_steps_host
 * copies in only the interior z-planes of each field block and fills the
 * ghosts on the device from the interiors: the step requires U's ghosts to be
 * those copies anyway, and the ghost layers are most of the state's bytes.
 * The whole state, ghosts included, is copied back. */
oct_status oct_hydro_rk_steps_host(oct_hydro_t h, double *U_host, int n_steps, double *dt_last_out,
                                   void *cuda_stream);
oct_status oct_hydro_rhs_host(oct_hydro_t h, const double *U_host, double *dUdt_host, void *cuda_stream);

/* Bytes oct_hydro_rk_steps_host copies host to device and device to host
 * per call for the current layout (either pointer may be NULL).  OCT_E_ARG
 * for a NULL handle or one without a layout. */
oct_status oct_hydro_host_copy_bytes(oct_hydro_t h, int64_t *h2d_bytes, int64_t *d2h_bytes);

/* Chooses the work decomposition of the RHS kernel for this GPU (Sec. V-B:
 * the paper splits its largest kernels into several tasks so that every
 * core has work; here the unit is a column of cells of a subgrid, and the
 * split is chosen by measurement).  Times the candidate launch shapes of the
 * RHS kernel on U_sample -- tile
 * capacity and threads (8x8 cells per work item with 256, 512 or 1024
 * threads, or 8x4 with 256) x resident CTAs per SM (1 up to the occupancy
 * limit) -- and keeps the fastest for this layout, precision and
 * reconstruction choice.  Drops captured graphs.  When the environment
 * variable OCT_HYDRO_TUNE_CACHE names a file, a result stored there for the
 * same GPU model, SM count, form, field count and edge counts is applied
 * without trial launches, and a new result is appended (one text line per
 * result; a file that cannot be read or written only disables the cache). */
oct_status oct_hydro_autotune(oct_hydro_t h, const double *U_sample, void *cuda_stream);

/* Allocation-free RHS + CFL dt (the paper has no counterpart: this is a
 * calling convention of this library, not a step of the method).
 * For callers that cannot call cudaMalloc on their hot path: host programs
 * whose device memory is all handed out by their own pool allocator, and
 * programs that must not take the implicit device-wide synchronisation that
 * cudaMalloc/cudaFree can cause.  The call needs no handle and allocates
 * nothing; its scratch (work list, per-item signal speeds, flag word) is one
 * fixed device array of 475,392 bytes in the library, reserved on every GPU
 * that loads it and held until the process exits.
 *   n_subgrids : 1..4096 (larger batches fail with OCT_E_ARG);
 *   edge, n_species, gamma, precision, cfl, de_switch1 : as for
 *                oct_hydro_create / oct_hydro_set_params;
 *   U          : device, packed ghosted blocks (block s at element
 *                s * round_up(nf * (edge+6)^3, 4)), ghosts valid;
 *   dx         : device, n_subgrids cell widths;
 *   dUdt       : device output, RHS layout (n_subgrids * nf * edge^3);
 *   dt         : device output, one double, cfl * min_s dx_s / a_max,s.
 * Results equal oct_hydro_rhs and oct_hydro_max_dt of a handle with the same
 * layout and parameters.  The first call on a device sets that device up
 * (scratch address, line tables, kernel attributes) and should come before
 * any stream capture.  Every call shares the scratch array, which keeps the
 * last call's contents: calls that overlap on the GPU (other streams, other
 * host threads) race on it and must be serialised by the caller.  Device
 * error flags of this call are not reported. */
oct_status oct_hydro_rhs_dt_noalloc(int n_subgrids, int edge, int n_species, double gamma, int precision, double cfl,
                                    double de_switch1, const double *U, const double *dx, double *dUdt, double *dt,
                                    void *cuda_stream);

/* Gravity, same-level monopole interactions (Sec. II "Solvers": the gravity
 * solver's most compute-intensive step is the interaction between close-by
 * cells of one level; for non-refined cells it is the monopole kernel).  The
 * paper gives no equations; the reading used: every interior cell i receives
 * from each cell j of its level within r_s cell widths (0 < |d| <= r_s,
 * d = j - i in cells) the potential and acceleration of a point mass
 * m_j = rho_j dx^3 at the cell centre,
 *     phi_i = -G sum_j m_j / r_ij,   g_i = -G sum_j m_j (x_i - x_j) / r_ij^3,
 * with rho field 0 of the state U (interiors only: the subgrid's own and its
 * neighbours' through the neighbour table; a missing neighbour holds no
 * mass).  For the paper's opening angle theta = 0.34, r_s = 2 / theta.
 * Needs the periodic or outflow layout (one edge, a neighbour table) and one
 * cell width for every subgrid; 1 <= r_s <= edge, and the subgrid with its
 * halo of floor(r_s) cells plus the stencil must fit in shared memory
 * (edge 8: r_s < 9; OCT_E_ARG otherwise).  G > 0.
 * Output (device): phi [subgrid][edge^3], g [subgrid][3][edge^3] (x, y, z).
 * A call with a new r_s rebuilds the stencil (a synchronous copy); the
 * launch itself is stream-ordered. */
oct_status oct_hydro_gravity_monopole(oct_hydro_t h, const double *U, double G, double r_s, double *phi, double *g,
                                      void *cuda_stream);

/* Diagnostics (the paper has no counterpart: they serve the measurements
 * and tests of this library).
 *
 * oct_hydro_pipe_peaks: FP64 and FP32 FMA throughput of the current GPU in
 * TFLOP/s (an FMA counts as two flops), each from one launch of independent
 * FMA chains on a full grid lasting at least target_ms (0 < target_ms <=
 * 10000), timed with CUDA events on the stream; synchronises it.  These are
 * the measured peaks against which the benchmark reports its arithmetic-bound
 * kernels.
 *
 * oct_hydro_eval_math: y[i] = fn(x[i]) for i < n on DEVICE arrays of doubles,
 * stream-ordered, with fn the FP64 helpers the kernels use -- 0 the
 * reciprocal, 1 the square root, 2 tau^gamma, 3 e^(1/gamma) -- or, for
 * comparison, CUDA's own 1.0 / x (16), sqrt (17), pow(x, gamma) (18) and
 * pow(x, 1.0 / gamma) (19).  OCT_E_ARG for another fn or NULL arrays. */
oct_status oct_hydro_pipe_peaks(double target_ms, double *fp64_tflops, double *fp32_tflops, void *cuda_stream);
oct_status oct_hydro_eval_math(int fn, const double *x, double *y, int64_t n, double gamma, void *cuda_stream);

/* Launch shape of the RHS kernel for the current layout and precision
 * (the paper's Sec. V-B splits big kernels into tasks for the same reason:
 * enough independent work per core): tile mode (0: 8x8-cell columns with
 * 256 threads, 1: 8x4 with 256, 2: 8x8 with 512, 3: 8x8 with 1024), CTAs
 * resident per SM, and work items.  The items are the tiles of every
 * subgrid, the last round's tiles cut in half along y when they would leave
 * at least half the persistent grid idle; CTAs draw items in order of
 * decreasing work from a counter on the device.  Any pointer may be NULL. */
oct_status oct_hydro_launch_info(oct_hydro_t h, int *tile_mode, int *ctas_per_sm, int *n_items);

/* Kernel launches of one oct_hydro_rk_step for the current layout and
 * settings (the three stages of Sec. V-B's "3 hydro solver iterations"):
 * per stage the RHS kernel (plus the primitive pass with primitive
 * reconstruction and the flux correction across levels), the combine, and
 * the ghost fill (none with given ghosts, two passes across levels with
 * prolongation); plus one dt reduction.  -1 for a NULL handle or one
 * without a layout. */
int oct_hydro_step_launches(oct_hydro_t h);

/* Reads and clears the device error flags (OCT_FLAG_*); synchronises.  The
 * paper states no error handling; the flags report what readings R6 and R7
 * of the floors and a non-physical point (rho <= 0, non-finite values) meet
 * on the device, since a kernel does not trap. */
oct_status oct_hydro_get_error_flags(oct_hydro_t h, uint32_t *flags);

/* Text of the calling thread's last failed call ("" if none). */
const char *oct_hydro_last_error(void);

/* Releases the handle's device memory and graphs.  NULL is ignored. */
void oct_hydro_destroy(oct_hydro_t h);

#ifdef __cplusplus
}
#endif

#endif /* OCT_HYDRO_H */
