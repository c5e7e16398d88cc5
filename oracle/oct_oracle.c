/*
 * oct_oracle.c -- plain, slow FP64 CPU oracle of the Octo-Tiger hydro
 * right-hand side, as the paper describes it (arXiv 2210.06439, Sec. II
 * "Solvers" and "Data-Structure"): finite-volume Euler equations with the
 * Kurganov-Tadmor central flux, piecewise-parabolic reconstruction to 26
 * points per cell, Newton-Cotes quadrature over each face, the flux
 * divergence, a three-stage Runge-Kutta step (Sec. V-B: three hydro solver
 * iterations per time step) and the CFL time-step reduction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Style: every quantity is computed directly from its definition, in the
 * order the method states it, with no blocking, fusion or reuse of partial
 * results between faces.  Compile with -O2 -ffp-contract=off (no FMA
 * contraction) so that every operation is one IEEE-754 round-to-nearest
 * FP64 operation; the bitwise mirror-symmetry property relies on that.
 *
 * The paper names the methods but prints no equations, so the following
 * readings of it are fixed here (each is listed in the design notes):
 *   R1  the conserved fields themselves are reconstructed;
 *   R2  PPM = Colella-Woodward (1984) interface interpolant with
 *       monotonised-central slopes and the CW84 monotonicity fix-up; no
 *       steepening or flattening;
 *   R3  the 26 points of a cell are its 6 face centres, 12 edge midpoints and
 *       8 corners; the value at x + d/2 comes from 1-D PPM along the line of
 *       cells x + m d, m = -2..2 (13 lines, two ends each);
 *   R4  Newton-Cotes = tensor Simpson rule on the 3x3 face points, weights
 *       16/36 centre, 4/36 edge midpoints, 1/36 corners;
 *   R5  KT flux with a local speed a_q per quadrature point,
 *       a_q = max(|v_n,L| + c_L, |v_n,R| + c_R); the face's maximum signal
 *       speed is max_q a_q and feeds the dt reduction;
 *   R6  dual energy: e_int = E - |s|^2/(2 rho); if e_int < eps1 * E then
 *       e_int = tau^gamma; after each RK stage tau is re-synchronised when
 *       E - |s|^2/(2 rho) > eps2 * E;
 *   R7  floors after each RK stage: rho >= rho_floor, tau >= 0, rho_i >= 0;
 *   R8  Shu-Osher SSP-RK3, dt from the state at the start of the step,
 *       dt = cfl * min over subgrids of dx / a_max;
 *   R9  ghost fill on a uniform level: copy from the neighbour subgrid's
 *       interior; at a domain edge with no neighbour, copy the nearest
 *       interior cell (zero-gradient outflow);
 *   R14 ghost fill across refinement levels: the same-level cell if one
 *       covers the ghost, else the covering coarser cell (injection), else
 *       the mean of the 8 finer cells (restriction);
 *   R15 flux correction at coarse-fine faces: the coarse flux through such
 *       a face is replaced by the mean of the 4 fine fluxes on it;
 *   R17 (optional) limited linear prolongation instead of injection: the
 *       coarse value plus a quarter of each axis's minmod slope, signed by
 *       the fine cell's side;
 *   R16 (optional, recon = 1) primitive reconstruction: PPM acts on
 *       w = (rho, v, p, tau, X_i = rho_i / rho) of every cell, and each point
 *       is turned back into conserved fields (s = rho v,
 *       E = p / (gamma - 1) + rho |v|^2 / 2, rho_i = rho X_i) with its v, p
 *       taken as reconstructed; the cell's p uses the dual-energy switch;
 *   R18 gravity, same-level monopole interactions: each cell receives
 *       -G m_j / r and -G m_j (x_i - x_j) / r^3 from every cell j of its
 *       level within r_s cell widths, m_j = rho_j dx^3 at the cell centre.
 *
 * Field order: rho, s_x, s_y, s_z, E_gas, tau, rho_1 .. rho_ns.
 * State layout: one ghosted block per subgrid, structure of arrays
 * [field][z][y][x], B = E + 6 cells per side, starting at element offset
 * off[s].  RHS layout: interior only, [subgrid][field][z][y][x] with E cells
 * per side, subgrids packed in order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 3 /* ghost layers */

enum { F_RHO = 0, F_SX = 1, F_SY = 2, F_SZ = 3, F_EGAS = 4, F_TAU = 5, F_SPC = 6 };

/* ------------------------------------------------------------------------ */
/* 1-D piecewise-parabolic reconstruction (reading R2)                       */
/* ------------------------------------------------------------------------ */

/* Monotonised-central slope of cell j from its neighbours: the minmod of the
 * centred difference and twice the one-sided differences; zero unless all
 * three have the same strict sign. */
static double mc_slope(double um, double u0, double up)
{
    double c = 0.5 * (up - um);
    double l = 2.0 * (u0 - um);
    double r = 2.0 * (up - u0);
    if (c > 0.0 && l > 0.0 && r > 0.0)
        return fmin(c, fmin(l, r));
    if (c < 0.0 && l < 0.0 && r < 0.0)
        return fmax(c, fmax(l, r));
    return 0.0;
}

/* PPM on the 5-cell stencil u[0..4] = u_{-2..2}.  Returns the limited values
 * at the two ends of the centre cell: *um at -1/2 and *up at +1/2.
 * CW84 interface value: u_{j+1/2} = (u_j + u_{j+1})/2 - (du_{j+1} - du_j)/6,
 * then the CW84 monotonicity constraints on (um, u0, up). */
void oco_ppm(const double *u, double *um_out, double *up_out)
{
    double dm = mc_slope(u[0], u[1], u[2]);
    double d0 = mc_slope(u[1], u[2], u[3]);
    double dp = mc_slope(u[2], u[3], u[4]);
    double u0 = u[2];
    double up = 0.5 * (u[2] + u[3]) - (dp - d0) / 6.0;
    double um = 0.5 * (u[1] + u[2]) - (d0 - dm) / 6.0;
    /* The constraints are conditions on signs and on ratios of magnitudes,
     * the same at every scale of u; they are written without products of two
     * differences, which underflow for |u| below about 1e-154. */
    if (!((up - u0 > 0.0 && u0 - um > 0.0) || (up - u0 < 0.0 && u0 - um < 0.0))) {
        /* local extremum, (up - u0)(u0 - um) <= 0: flat profile */
        um = u0;
        up = u0;
    } else {
        /* overshoot: du (u0 - (up + um)/2) > du^2/6, or < -du^2/6; divided
         * by |du| > 0 these read 6 sgn(du) x > |du| and < -|du| */
        double du = up - um;
        double x = u0 - 0.5 * (up + um);
        double t = du > 0.0 ? 6.0 * x : -6.0 * x;
        double a = fabs(du);
        if (t > a)
            um = 3.0 * u0 - 2.0 * up;
        else if (t < -a)
            up = 3.0 * u0 - 2.0 * um;
    }
    *um_out = um;
    *up_out = up;
}

/* ------------------------------------------------------------------------ */
/* Equation of state and point primitives (reading R6)                       */
/* ------------------------------------------------------------------------ */

/* From one point's conserved fields q[0..5]: velocity v[3], pressure, sound
 * speed.  Returns 0, or 1 when the state is not physical (rho <= 0 or a
 * non-finite result). */
int oco_prim(const double *q, double gamma, double eps1, double *v, double *p_out, double *c_out)
{
    double rho = q[F_RHO];
    double sx = q[F_SX], sy = q[F_SY], sz = q[F_SZ];
    double E = q[F_EGAS], tau = q[F_TAU];
    v[0] = sx / rho;
    v[1] = sy / rho;
    v[2] = sz / rho;
    double ek = 0.5 * (sx * sx + sy * sy + sz * sz) / rho;
    double ei = E - ek;
    if (ei < eps1 * E)
        ei = pow(tau, gamma);
    double p = (gamma - 1.0) * ei;
    double c = sqrt(gamma * p / rho);
    *p_out = p;
    *c_out = c;
    if (!(rho > 0.0) || !isfinite(c) || !isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2]))
        return 1;
    return 0;
}

/* Physical Euler flux along axis k of field f, for a point with conserved
 * fields q, velocity v and pressure p. */
static double phys_flux(int k, int f, const double *q, const double *v, double p)
{
    double vk = v[k];
    if (f == F_SX + k)
        return q[f] * vk + p;
    if (f == F_EGAS)
        return (q[F_EGAS] + p) * vk;
    return q[f] * vk;
}

/* Kurganov-Tadmor central flux at one quadrature point (reading R5):
 * F = (F_k(qL) + F_k(qR))/2 - a (qR - qL)/2 with the local speed
 * a = max(|v_k,L| + c_L, |v_k,R| + c_R), from both sides' conserved fields
 * q and primitives v, p, c.  Writes F[0..nf-1]; returns a. */
static double kt_flux(int k, int nf, const double *qL, const double *vL, double pL, double cL, const double *qR,
                      const double *vR, double pR, double cR, double *F)
{
    double aL = fabs(vL[k]) + cL;
    double aR = fabs(vR[k]) + cR;
    double a = fmax(aL, aR);
    for (int f = 0; f < nf; f++) {
        double FL = phys_flux(k, f, qL, vL, pL);
        double FR = phys_flux(k, f, qR, vR, pR);
        F[f] = 0.5 * (FL + FR) - 0.5 * a * (qR[f] - qL[f]);
    }
    return a;
}

/* The same from the conserved fields alone (primitives by oco_prim).
 * Writes F[0..nf-1] and *a_out. */
int oco_kt_point(int k, int nf, const double *qL, const double *qR, double gamma, double eps1,
                 double *F, double *a_out)
{
    double vL[3], vR[3], pL, pR, cL, cR;
    int bad = oco_prim(qL, gamma, eps1, vL, &pL, &cL);
    bad |= oco_prim(qR, gamma, eps1, vR, &pR, &cR);
    *a_out = kt_flux(k, nf, qL, vL, pL, cL, qR, vR, pR, cR, F);
    return bad;
}

/* Reading R16, cell side: the variables reconstructed in primitive mode,
 * w = (rho, v_x, v_y, v_z, p, tau, X_1 .. X_ns) with X_i = rho_i / rho, from
 * a cell's conserved fields q (p by oco_prim, with the dual-energy switch).
 * Returns 1 for a non-physical cell. */
static int cell_prim(const double *q, int nf, double gamma, double eps1, double *w)
{
    double v[3], p, c;
    int bad = oco_prim(q, gamma, eps1, v, &p, &c);
    w[F_RHO] = q[F_RHO];
    w[F_SX] = v[0];
    w[F_SY] = v[1];
    w[F_SZ] = v[2];
    w[F_EGAS] = p;
    w[F_TAU] = q[F_TAU];
    for (int f = F_SPC; f < nf; f++)
        w[f] = q[f] / q[F_RHO];
    return bad;
}

/* Reading R16, point side: conserved fields q and primitives v, p, c of a
 * point from its reconstructed w.  Returns 1 for a non-physical point
 * (rho <= 0 or a non-finite sound speed). */
static int point_from_prim(const double *w, int nf, double gamma, double *q, double *v, double *p_out, double *c_out)
{
    double rho = w[F_RHO], p = w[F_EGAS];
    v[0] = w[F_SX];
    v[1] = w[F_SY];
    v[2] = w[F_SZ];
    q[F_RHO] = rho;
    q[F_SX] = rho * v[0];
    q[F_SY] = rho * v[1];
    q[F_SZ] = rho * v[2];
    q[F_EGAS] = p / (gamma - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    q[F_TAU] = w[F_TAU];
    for (int f = F_SPC; f < nf; f++)
        q[f] = rho * w[f];
    double c = sqrt(gamma * p / rho);
    *p_out = p;
    *c_out = c;
    return (!(rho > 0.0) || !isfinite(c)) ? 1 : 0;
}

/* Tensor Simpson (closed Newton-Cotes, degree 2) over the 3x3 face points
 * (reading R4).  Fq holds 9 values in the order of QPT below.  The sums pair
 * mirror-image points first so that reflecting the face permutes only
 * commutative operands. */
static const int QPT[9][2] = {
    {0, 0},                                     /* centre          */
    {-1, 0}, {1, 0}, {0, -1}, {0, 1},           /* edge midpoints  */
    {-1, -1}, {1, -1}, {-1, 1}, {1, 1}          /* corners         */
};

double oco_simpson(const double *Fq)
{
    double edges = (Fq[1] + Fq[2]) + (Fq[3] + Fq[4]);
    double corners = (Fq[5] + Fq[6]) + (Fq[7] + Fq[8]);
    return (16.0 * Fq[0] + 4.0 * edges + corners) / 36.0;
}

/* ------------------------------------------------------------------------ */
/* Reconstruction at a cell point (reading R3)                               */
/* ------------------------------------------------------------------------ */

static inline int64_t cidx(int B, int x, int y, int z)
{
    return ((int64_t)z * B + y) * B + x;
}

/* Value of field block Uf at the point x + d/2 of ghosted cell (x, y, z):
 * the +1/2 end of PPM along the line of cells (x, y, z) + m d. */
static double point_value(const double *Uf, int B, int x, int y, int z, const int *d)
{
    double s[5], um, up;
    for (int m = -2; m <= 2; m++)
        s[m + 2] = Uf[cidx(B, x + m * d[0], y + m * d[1], z + m * d[2])];
    oco_ppm(s, &um, &up);
    return up;
}

/* ------------------------------------------------------------------------ */
/* RHS of one subgrid                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nf;
    double gamma, eps1;
    int recon; /* 0: conserved fields (R1), 1: primitive variables (R16) */
} hydro_par;

/* Transverse axes of face normal k, in increasing order. */
static void transverse(int k, int *a1, int *a2)
{
    *a1 = (k == 0) ? 1 : 0;
    *a2 = (k == 2) ? 1 : 2;
}

/* Direction index of d in {-1,0,1}^3: (dz+1)*9 + (dy+1)*3 + (dx+1); 13 is
 * the (unused) centre. */
static inline int dir_index(const int *d)
{
    return (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1);
}

/* Face flux array index: face position p in [0, E] along the normal
 * (between interior cells p-1 and p), transverse interior indices t1, t2. */
static inline int64_t fidx(int E, int f, int p, int t1, int t2)
{
    return (((int64_t)f * E + t2) * E + t1) * (E + 1) + p;
}

/* Computes dU/dt for the interior of one subgrid and its max signal speed,
 * in the two steps the paper names (Sec. II "Solvers"): reconstruct (point
 * values at the 26 points of every cell next to a face) then flux (KT at the
 * 9 Newton-Cotes points of every face), followed by the divergence.
 * Optional cell mask (NULL = all cells): only the faces of masked cells are
 * evaluated and only masked cells are written. */
static int rhs_subgrid(const double *U, int E, double dx, const hydro_par *hp, double *dU, double *amax_out,
                       const uint8_t *mask, double *faces_out)
{
    int nf = hp->nf;
    int B = E + 2 * NG;
    int64_t fs = (int64_t)B * B * B;
    int nc = E + 2; /* reconstructed cells: interior index -1 .. E */
    int64_t ncell = (int64_t)nc * nc * nc;
    int64_t nfa = (int64_t)nf * E * E * (E + 1);
    double *Ff[3];
    uint8_t *need[3];
    for (int k = 0; k < 3; k++) {
        Ff[k] = (double *)calloc((size_t)nfa, sizeof(double));
        need[k] = (uint8_t *)calloc((size_t)E * E * (E + 1), 1);
    }
    uint8_t *needc = (uint8_t *)calloc((size_t)ncell, 1);
    double *Q = (double *)calloc((size_t)(ncell * 27 * nf), sizeof(double));

    /* which faces are needed, and which cells border them */
    for (int z = 0; z < E; z++)
        for (int y = 0; y < E; y++)
            for (int x = 0; x < E; x++) {
                if (mask && !mask[((int64_t)z * E + y) * E + x])
                    continue;
                int c[3] = {x, y, z};
                for (int k = 0; k < 3; k++) {
                    int a1, a2;
                    transverse(k, &a1, &a2);
                    for (int p = c[k]; p <= c[k] + 1; p++) {
                        need[k][((int64_t)c[a2] * E + c[a1]) * (E + 1) + p] = 1;
                        int l[3] = {c[0], c[1], c[2]};
                        l[k] = p - 1;
                        needc[((int64_t)(l[2] + 1) * nc + (l[1] + 1)) * nc + (l[0] + 1)] = 1;
                        l[k] = p;
                        needc[((int64_t)(l[2] + 1) * nc + (l[1] + 1)) * nc + (l[0] + 1)] = 1;
                    }
                }
            }

    /* primitive mode (R16): the reconstructed variables w of every cell of
     * the ghosted block, and which cells are not physical */
    const double *R = U;
    double *Wb = NULL;
    uint8_t *badc = NULL;
    int bad = 0;
    if (hp->recon) {
        int64_t B3 = (int64_t)B * B * B;
        Wb = (double *)malloc(sizeof(double) * (size_t)(nf * B3));
        badc = (uint8_t *)calloc((size_t)B3, 1);
        double q[64], w[64];
        for (int64_t c = 0; c < B3; c++) {
            for (int f = 0; f < nf; f++)
                q[f] = U[f * fs + c];
            badc[c] = (uint8_t)cell_prim(q, nf, hp->gamma, hp->eps1, w);
            for (int f = 0; f < nf; f++)
                Wb[f * fs + c] = w[f];
        }
        R = Wb;
    }

    /* step 1, reconstruct: point value of every field at x + d/2 for all 26
     * directions d of every needed cell */
    for (int z = -1; z <= E; z++)
        for (int y = -1; y <= E; y++)
            for (int x = -1; x <= E; x++) {
                int64_t ci = ((int64_t)(z + 1) * nc + (y + 1)) * nc + (x + 1);
                if (!needc[ci])
                    continue;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int ddx = -1; ddx <= 1; ddx++) {
                            int d[3] = {ddx, dy, dz};
                            if (!ddx && !dy && !dz)
                                continue;
                            for (int f = 0; f < nf; f++)
                                Q[(ci * 27 + dir_index(d)) * nf + f] =
                                    point_value(R + f * fs, B, x + NG, y + NG, z + NG, d);
                            if (badc)
                                for (int m = -2; m <= 2; m++)
                                    bad |= badc[cidx(B, x + NG + m * ddx, y + NG + m * dy, z + NG + m * dz)];
                        }
            }

    /* step 2, flux: KT at the 9 quadrature points of each needed face, then
     * the Simpson face average */
    double amax = 0.0;
    double Fq[9][64];
    for (int k = 0; k < 3; k++) {
        int a1, a2;
        transverse(k, &a1, &a2);
        for (int t2 = 0; t2 < E; t2++)
            for (int t1 = 0; t1 < E; t1++)
                for (int p = 0; p <= E; p++) {
                    if (!need[k][((int64_t)t2 * E + t1) * (E + 1) + p])
                        continue;
                    int cL[3], cR[3];
                    cL[k] = p - 1;
                    cL[a1] = t1;
                    cL[a2] = t2;
                    cR[0] = cL[0], cR[1] = cL[1], cR[2] = cL[2];
                    cR[k] = p;
                    int64_t iL = ((int64_t)(cL[2] + 1) * nc + (cL[1] + 1)) * nc + (cL[0] + 1);
                    int64_t iR = ((int64_t)(cR[2] + 1) * nc + (cR[1] + 1)) * nc + (cR[0] + 1);
                    for (int q = 0; q < 9; q++) {
                        int dL[3], dR[3];
                        dL[k] = 1;
                        dR[k] = -1;
                        dL[a1] = dR[a1] = QPT[q][0];
                        dL[a2] = dR[a2] = QPT[q][1];
                        const double *qL = Q + (iL * 27 + dir_index(dL)) * nf;
                        const double *qR = Q + (iR * 27 + dir_index(dR)) * nf;
                        double a;
                        if (hp->recon) {
                            double uL[64], uR[64], vL[3], vR[3], pL, pR, cL, cR;
                            bad |= point_from_prim(qL, nf, hp->gamma, uL, vL, &pL, &cL);
                            bad |= point_from_prim(qR, nf, hp->gamma, uR, vR, &pR, &cR);
                            a = kt_flux(k, nf, uL, vL, pL, cL, uR, vR, pR, cR, Fq[q]);
                        } else {
                            bad |= oco_kt_point(k, nf, qL, qR, hp->gamma, hp->eps1, Fq[q], &a);
                        }
                        amax = fmax(amax, a);
                    }
                    for (int f = 0; f < nf; f++) {
                        double w[9];
                        for (int q = 0; q < 9; q++)
                            w[q] = Fq[q][f];
                        Ff[k][fidx(E, f, p, t1, t2)] = oco_simpson(w);
                    }
                }
    }

    /* the face-averaged fluxes of the subgrid's own boundary faces, when
     * asked for: face 2k (+1 for the upper side) of axis k, field f, at
     * (t1, t2) = the two other coordinates in increasing axis order */
    if (faces_out && !mask)
        for (int k = 0; k < 3; k++)
            for (int side = 0; side < 2; side++)
                for (int f = 0; f < nf; f++)
                    for (int t2 = 0; t2 < E; t2++)
                        for (int t1 = 0; t1 < E; t1++)
                            faces_out[(((int64_t)(2 * k + side) * nf + f) * E + t2) * E + t1] =
                                Ff[k][fidx(E, f, side ? E : 0, t1, t2)];

    /* divergence: dU/dt = -sum_k (F_{k,+} - F_{k,-}) / dx */
    for (int f = 0; f < nf; f++)
        for (int z = 0; z < E; z++)
            for (int y = 0; y < E; y++)
                for (int x = 0; x < E; x++) {
                    int64_t ci = ((int64_t)z * E + y) * E + x;
                    if (mask && !mask[ci])
                        continue;
                    double Dx = Ff[0][fidx(E, f, x + 1, y, z)] - Ff[0][fidx(E, f, x, y, z)];
                    double Dy = Ff[1][fidx(E, f, y + 1, x, z)] - Ff[1][fidx(E, f, y, x, z)];
                    double Dz = Ff[2][fidx(E, f, z + 1, x, y)] - Ff[2][fidx(E, f, z, x, y)];
                    dU[(int64_t)f * E * E * E + ci] = -(Dx + Dy + Dz) / dx;
                }
    for (int k = 0; k < 3; k++) {
        free(Ff[k]);
        free(need[k]);
    }
    free(needc);
    free(Q);
    free(Wb);
    free(badc);
    if (amax_out)
        *amax_out = amax;
    return bad;
}

static int valid_edge(int E)
{
    return E == 8 || E == 12 || E == 16;
}

static void rhs_offsets(int n_sub, const int32_t *edge, int nf, int64_t *doff)
{
    int64_t o = 0;
    for (int s = 0; s < n_sub; s++) {
        doff[s] = o;
        o += (int64_t)nf * edge[s] * edge[s] * edge[s];
    }
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Number of threads the OpenMP build would use (1 without OpenMP). */
int oco_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* dU/dt for all subgrids.  amax (may be NULL) receives each subgrid's max
 * signal speed; faces (may be NULL) each subgrid's boundary face fluxes,
 * [s][6][nf][E][E] packed in subgrid order.  Returns the number of subgrids
 * that met a non-physical point state, or -1 on bad arguments. */
static int rhs_all(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                   double eps1, int recon, const double *U, double *dUdt, double *amax, double *faces, int nthreads)
{
    if (n_sub < 0 || nf < 6 || nf > 64)
        return -1;
    for (int s = 0; s < n_sub; s++)
        if (!valid_edge(edge[s]))
            return -1;
    hydro_par hp = {nf, gamma, eps1, recon};
    int64_t *doff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_sub > 0 ? n_sub : 1));
    int64_t *foff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_sub > 0 ? n_sub : 1));
    rhs_offsets(n_sub, edge, nf, doff);
    int64_t o = 0;
    for (int s = 0; s < n_sub; s++) {
        foff[s] = o;
        o += 6 * nf * edge[s] * edge[s];
    }
    int nbad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad)
    for (int s = 0; s < n_sub; s++) {
        double a;
        nbad += rhs_subgrid(U + off[s], edge[s], dx[s], &hp, dUdt + doff[s], &a, NULL,
                            faces ? faces + foff[s] : NULL);
        if (amax)
            amax[s] = a;
    }
    free(doff);
    free(foff);
    return nbad;
}

int oco_rhs_faces(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                  double eps1, const double *U, double *dUdt, double *amax, double *faces, int nthreads)
{
    return rhs_all(n_sub, edge, off, dx, nf, gamma, eps1, 0, U, dUdt, amax, faces, nthreads);
}

/* oco_rhs_faces with the reconstructed variables chosen by recon. */
int oco_rhs_faces_recon(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                        double eps1, int recon, const double *U, double *dUdt, double *amax, double *faces,
                        int nthreads)
{
    return rhs_all(n_sub, edge, off, dx, nf, gamma, eps1, recon, U, dUdt, amax, faces, nthreads);
}

/* dU/dt with the reconstructed variables chosen by recon (0: conserved
 * fields, reading R1; 1: primitive variables, reading R16). */
int oco_rhs_recon(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                  double eps1, int recon, const double *U, double *dUdt, double *amax, int nthreads)
{
    return rhs_all(n_sub, edge, off, dx, nf, gamma, eps1, recon, U, dUdt, amax, NULL, nthreads);
}

int oco_rhs(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
            double eps1, const double *U, double *dUdt, double *amax, int nthreads)
{
    return rhs_all(n_sub, edge, off, dx, nf, gamma, eps1, 0, U, dUdt, amax, NULL, nthreads);
}

/* dU/dt at a list of sampled cells only: samples[2*i] = subgrid index,
 * samples[2*i+1] = interior linear cell index z*E*E + y*E + x.
 * out[i*nf + f] receives dU_f/dt of sample i. */
int oco_rhs_cells(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                  double eps1, const double *U, int n_samples, const int64_t *samples, double *out, int nthreads)
{
    if (nf < 6 || nf > 64)
        return -1;
    hydro_par hp = {nf, gamma, eps1, 0};
    int nbad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad)
    for (int i = 0; i < n_samples; i++) {
        int64_t s = samples[2 * i], ci = samples[2 * i + 1];
        int E = edge[s];
        uint8_t *mask = (uint8_t *)calloc((size_t)E * E * E, 1);
        double *dU = (double *)calloc((size_t)nf * E * E * E, sizeof(double));
        mask[ci] = 1;
        nbad += rhs_subgrid(U + off[s], E, dx[s], &hp, dU, NULL, mask, NULL);
        for (int f = 0; f < nf; f++)
            out[(int64_t)i * nf + f] = dU[(int64_t)f * E * E * E + ci];
        free(mask);
        free(dU);
    }
    return nbad;
}

/* dt = cfl * min_s dx_s / amax_s (reading R8). */
double oco_dt_from_amax(int n_sub, const double *dx, const double *amax, double cfl)
{
    double m = INFINITY;
    for (int s = 0; s < n_sub; s++)
        m = fmin(m, dx[s] / amax[s]);
    return cfl * m;
}

/* ------------------------------------------------------------------------ */
/* Ghost fill on a uniform level (reading R9)                                */
/* ------------------------------------------------------------------------ */

/* Neighbour table: 26 int32 per subgrid, direction (dx, dy, dz) in
 * {-1,0,1}^3 \ {0} at index n = (dz+1)*9 + (dy+1)*3 + (dx+1), minus one
 * for n > 13.  -1 = no neighbour (domain edge).  All subgrids share edge E. */
static int nb_index(int dx, int dy, int dz)
{
    int n = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
    return n > 13 ? n - 1 : n;
}

int oco_ghost_fill(int n_sub, int E, const int64_t *off, int nf, const int32_t *nbr, double *U)
{
    if (!valid_edge(E))
        return -1;
    int B = E + 2 * NG;
    int64_t fs = (int64_t)B * B * B;
    int err = 0;
    for (int s = 0; s < n_sub; s++) {
        for (int z = -NG; z < E + NG; z++)
            for (int y = -NG; y < E + NG; y++)
                for (int x = -NG; x < E + NG; x++) {
                    if (x >= 0 && x < E && y >= 0 && y < E && z >= 0 && z < E)
                        continue;
                    int g[3] = {x, y, z}, d[3];
                    for (int a = 0; a < 3; a++) {
                        d[a] = g[a] < 0 ? -1 : (g[a] >= E ? 1 : 0);
                        if (d[a] != 0) {
                            int dd[3] = {0, 0, 0};
                            dd[a] = d[a];
                            if (nbr[26 * (int64_t)s + nb_index(dd[0], dd[1], dd[2])] < 0) {
                                /* domain edge: zero-gradient copy of the nearest interior cell */
                                g[a] = d[a] < 0 ? 0 : E - 1;
                                d[a] = 0;
                            }
                        }
                    }
                    int src = s;
                    if (d[0] || d[1] || d[2]) {
                        src = nbr[26 * (int64_t)s + nb_index(d[0], d[1], d[2])];
                        if (src < 0) {
                            err = 1;
                            continue;
                        }
                    }
                    int sx = g[0] - d[0] * E, sy = g[1] - d[1] * E, sz = g[2] - d[2] * E;
                    for (int f = 0; f < nf; f++)
                        U[off[s] + f * fs + cidx(B, x + NG, y + NG, z + NG)] =
                            U[off[src] + f * fs + cidx(B, sx + NG, sy + NG, sz + NG)];
                }
    }
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Floors and dual-energy re-synchronisation (readings R6, R7)               */
/* ------------------------------------------------------------------------ */

/* Applies the floors to the interior of every subgrid.  Returns the number of
 * floor firings (rho or species raised, tau clipped). */
int64_t oco_floors(int n_sub, const int32_t *edge, const int64_t *off, int nf, double gamma, double rho_floor,
                   double eps2, double *U)
{
    int64_t fired = 0;
    for (int s = 0; s < n_sub; s++) {
        int E = edge[s], B = E + 2 * NG;
        int64_t fs = (int64_t)B * B * B;
        double *u = U + off[s];
        for (int z = 0; z < E; z++)
            for (int y = 0; y < E; y++)
                for (int x = 0; x < E; x++) {
                    int64_t c = cidx(B, x + NG, y + NG, z + NG);
                    if (u[c] < rho_floor) {
                        u[c] = rho_floor;
                        fired++;
                    }
                    for (int f = F_SPC; f < nf; f++)
                        if (u[f * fs + c] < 0.0) {
                            u[f * fs + c] = 0.0;
                            fired++;
                        }
                    double rho = u[c];
                    double sx = u[F_SX * fs + c], sy = u[F_SY * fs + c], sz = u[F_SZ * fs + c];
                    double E0 = u[F_EGAS * fs + c];
                    double ei = E0 - 0.5 * (sx * sx + sy * sy + sz * sz) / rho;
                    if (ei > eps2 * E0)
                        u[F_TAU * fs + c] = pow(ei, 1.0 / gamma);
                    if (u[F_TAU * fs + c] < 0.0) {
                        u[F_TAU * fs + c] = 0.0;
                        fired++;
                    }
                }
    }
    return fired;
}

/* One SSP-RK3 combine on the interior (reading R8):
 *   stage 1: U = U0 + dt L
 *   stage 2: U = 3/4 U0 + 1/4 (U + dt L)
 *   stage 3: U = 1/3 U0 + 2/3 (U + dt L)
 * U0 and U are ghosted blocks; L is in RHS layout. */
int oco_rk_combine(int stage, int n_sub, const int32_t *edge, const int64_t *off, int nf, double dt,
                   const double *U0, const double *L, double *U)
{
    if (stage < 1 || stage > 3)
        return -1;
    int64_t *doff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_sub > 0 ? n_sub : 1));
    rhs_offsets(n_sub, edge, nf, doff);
    for (int s = 0; s < n_sub; s++) {
        int E = edge[s], B = E + 2 * NG;
        int64_t fs = (int64_t)B * B * B;
        for (int f = 0; f < nf; f++)
            for (int z = 0; z < E; z++)
                for (int y = 0; y < E; y++)
                    for (int x = 0; x < E; x++) {
                        int64_t c = off[s] + f * fs + cidx(B, x + NG, y + NG, z + NG);
                        double l = L[doff[s] + (int64_t)f * E * E * E + ((int64_t)z * E + y) * E + x];
                        if (stage == 1)
                            U[c] = U0[c] + dt * l;
                        else if (stage == 2)
                            U[c] = 0.75 * U0[c] + 0.25 * (U[c] + dt * l);
                        else
                            U[c] = (1.0 / 3.0) * U0[c] + (2.0 / 3.0) * (U[c] + dt * l);
                    }
    }
    free(doff);
    return 0;
}

int oco_amr_ghost_fill(int n_sub, int E, const int64_t *off, int nf, const int32_t *lev, const int32_t *org,
                       int n0, int periodic, double *U);
int oco_amr_reflux(int n_sub, int E, const double *dx, int nf, const int32_t *lev, const int32_t *org, int n0,
                   int periodic, const double *faces, double *dUdt);

/* amr (may be NULL): when bc == 3, the ghosts are refreshed by the ghost
 * fill across levels with amr->lev, amr->org, amr->n0, amr->periodic. */
typedef struct {
    const int32_t *lev, *org;
    int n0, periodic;
    int order; /* prolongation order (reading R17): 0 injection, 1 limited linear */
} oco_amr;
int oco_amr_ghost_fill_order(int n_sub, int E, const int64_t *off, int nf, const int32_t *lev, const int32_t *org,
                             int n0, int periodic, int order, double *U);

static int rk3_step_impl(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                         double eps1, double eps2, double rho_floor, double cfl, double dt_cap, int bc,
                         const int32_t *nbr, const oco_amr *amr, int recon, double *U, int64_t total_len,
                         double *dt_out, int64_t *floors_out, int nthreads);

/* One full SSP-RK3 step (reading R8) on n_sub subgrids of a common edge E.
 * dt_cap > 0 caps the CFL time step (to land on an output time).
 * bc: 0 = ghosts given (left as they are), 1/2 = ghosts refreshed from the
 * neighbour table after every stage (periodic or outflow tables are both
 * expressed by nbr).  On entry U's ghosts must be valid.  *dt_out receives
 * the dt used; *floors_out (may be NULL) the number of floor firings.
 * Returns 0, 1 if a non-physical state was met, or a negative error. */
int oco_rk3_step(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                 double eps1, double eps2, double rho_floor, double cfl, double dt_cap, int bc, const int32_t *nbr,
                 double *U, int64_t total_len, double *dt_out, int64_t *floors_out, int nthreads)
{
    return rk3_step_impl(n_sub, edge, off, dx, nf, gamma, eps1, eps2, rho_floor, cfl, dt_cap, bc, nbr, NULL, 0, U,
                         total_len, dt_out, floors_out, nthreads);
}

/* oco_rk3_step with the reconstructed variables chosen by recon (0:
 * conserved fields, reading R1; 1: primitive variables, reading R16). */
int oco_rk3_step_recon(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                       double eps1, double eps2, double rho_floor, double cfl, double dt_cap, int bc,
                       const int32_t *nbr, int recon, double *U, int64_t total_len, double *dt_out,
                       int64_t *floors_out, int nthreads)
{
    return rk3_step_impl(n_sub, edge, off, dx, nf, gamma, eps1, eps2, rho_floor, cfl, dt_cap, bc, nbr, NULL, recon,
                         U, total_len, dt_out, floors_out, nthreads);
}

/* One SSP-RK3 step across refinement levels (readings R14, R15): after each
 * RHS the coarse side of every coarse-fine face takes the fine fluxes, and
 * after each stage the ghosts are refreshed by the fill across levels. */
int oco_rk3_step_amr(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                     double eps1, double eps2, double rho_floor, double cfl, double dt_cap, const int32_t *lev,
                     const int32_t *org, int n0, int periodic, double *U, int64_t total_len, double *dt_out,
                     int64_t *floors_out, int nthreads)
{
    oco_amr a = {lev, org, n0, periodic, 0};
    return rk3_step_impl(n_sub, edge, off, dx, nf, gamma, eps1, eps2, rho_floor, cfl, dt_cap, 3, NULL, &a, 0, U,
                         total_len, dt_out, floors_out, nthreads);
}

/* oco_rk3_step_amr with the prolongation order of the ghost fill (R17). */
int oco_rk3_step_amr_order(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf,
                           double gamma, double eps1, double eps2, double rho_floor, double cfl, double dt_cap,
                           const int32_t *lev, const int32_t *org, int n0, int periodic, int order, double *U,
                           int64_t total_len, double *dt_out, int64_t *floors_out, int nthreads)
{
    oco_amr a = {lev, org, n0, periodic, order};
    return rk3_step_impl(n_sub, edge, off, dx, nf, gamma, eps1, eps2, rho_floor, cfl, dt_cap, 3, NULL, &a, 0, U,
                         total_len, dt_out, floors_out, nthreads);
}

static int rk3_step_impl(int n_sub, const int32_t *edge, const int64_t *off, const double *dx, int nf, double gamma,
                         double eps1, double eps2, double rho_floor, double cfl, double dt_cap, int bc,
                         const int32_t *nbr, const oco_amr *amr, int recon, double *U, int64_t total_len,
                         double *dt_out, int64_t *floors_out, int nthreads)
{
    if (n_sub <= 0)
        return -1;
    for (int s = 0; s < n_sub; s++)
        if (edge[s] != edge[0] && bc != 0)
            return -1;
    int64_t nl = 0;
    for (int s = 0; s < n_sub; s++)
        nl += (int64_t)nf * edge[s] * edge[s] * edge[s];
    double *U0 = (double *)malloc(sizeof(double) * (size_t)total_len);
    double *L = (double *)malloc(sizeof(double) * (size_t)nl);
    double *amax = (double *)malloc(sizeof(double) * (size_t)n_sub);
    double *faces = bc == 3 ? (double *)malloc(sizeof(double) * (size_t)n_sub * 6 * nf * edge[0] * edge[0]) : NULL;
    memcpy(U0, U, sizeof(double) * (size_t)total_len);
    int bad = 0;
    int64_t fired = 0;
    double dt = 0.0;
    for (int stage = 1; stage <= 3; stage++) {
        int nb = rhs_all(n_sub, edge, off, dx, nf, gamma, eps1, recon, U, L, amax, faces, nthreads);
        if (nb < 0) {
            bad = -1;
            break;
        }
        if (bc == 3 &&
            oco_amr_reflux(n_sub, edge[0], dx, nf, amr->lev, amr->org, amr->n0, amr->periodic, faces, L) != 0) {
            bad = -2;
            break;
        }
        if (nb > 0)
            bad = 1;
        if (stage == 1) {
            dt = oco_dt_from_amax(n_sub, dx, amax, cfl);
            if (dt_cap > 0.0 && dt_cap < dt)
                dt = dt_cap;
        }
        oco_rk_combine(stage, n_sub, edge, off, nf, dt, U0, L, U);
        fired += oco_floors(n_sub, edge, off, nf, gamma, rho_floor, eps2, U);
        if (bc == 3) {
            if (oco_amr_ghost_fill_order(n_sub, edge[0], off, nf, amr->lev, amr->org, amr->n0, amr->periodic,
                                         amr->order, U) != 0) {
                bad = -2;
                break;
            }
        } else if (bc != 0 && oco_ghost_fill(n_sub, edge[0], off, nf, nbr, U) != 0) {
            bad = -2;
            break;
        }
    }
    free(U0);
    free(L);
    free(amax);
    free(faces);
    *dt_out = dt;
    if (floors_out)
        *floors_out = fired;
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Ghost fill across refinement levels (reading R14)                         */
/* ------------------------------------------------------------------------ */

/* Subgrids of a common edge E sit on an octree-like set of levels: subgrid s
 * at level lev[s] covers the cells org[3s..3s+2] .. +E-1 of its level, in a
 * root box of n0 cells per side at level 0 (n0 * 2^l cells at level l);
 * periodic != 0 wraps the root box, else its edges are outflow (zero
 * gradient).  Each ghost cell takes, by geometric search:
 *   - the cell of a subgrid at the same level that covers it (a copy);
 *   - else the covering cell one level coarser (prolongation by injection:
 *     the fine ghost takes the coarse cell's value);
 *   - else the mean of the 8 cells one level finer that cover it
 *     (restriction).
 * At an outflow edge the ghost cell's position is first clamped into the
 * root box.  Returns 0, or -2 when some ghost cell has no source. */
static int find_cover(int n_sub, int E, const int32_t *lev, const int32_t *org, int l, const int64_t *c)
{
    for (int s = 0; s < n_sub; s++) {
        if (lev[s] != l)
            continue;
        int in = 1;
        for (int a = 0; a < 3; a++)
            if (c[a] < org[3 * s + a] || c[a] >= org[3 * s + a] + E)
                in = 0;
        if (in)
            return s;
    }
    return -1;
}

int oco_amr_ghost_fill(int n_sub, int E, const int64_t *off, int nf, const int32_t *lev, const int32_t *org,
                       int n0, int periodic, double *U)
{
    if (!valid_edge(E))
        return -1;
    int B = E + 2 * NG;
    int64_t fs = (int64_t)B * B * B;
    int err = 0;
    for (int s = 0; s < n_sub; s++) {
        int l = lev[s];
        int64_t nl = (int64_t)n0 << l; /* cells per side at this level */
        for (int z = -NG; z < E + NG; z++)
            for (int y = -NG; y < E + NG; y++)
                for (int x = -NG; x < E + NG; x++) {
                    if (x >= 0 && x < E && y >= 0 && y < E && z >= 0 && z < E)
                        continue;
                    int64_t g[3] = {org[3 * s] + x, org[3 * s + 1] + y, org[3 * s + 2] + z};
                    for (int a = 0; a < 3; a++) {
                        if (periodic)
                            g[a] = ((g[a] % nl) + nl) % nl;
                        else
                            g[a] = g[a] < 0 ? 0 : (g[a] >= nl ? nl - 1 : g[a]);
                    }
                    int64_t dst = off[s] + cidx(B, x + NG, y + NG, z + NG);
                    /* same level */
                    int t = find_cover(n_sub, E, lev, org, l, g);
                    if (t >= 0) {
                        int64_t src = off[t] + cidx(B, (int)(g[0] - org[3 * t]) + NG, (int)(g[1] - org[3 * t + 1]) + NG,
                                                    (int)(g[2] - org[3 * t + 2]) + NG);
                        for (int f = 0; f < nf; f++)
                            U[dst + f * fs] = U[src + f * fs];
                        continue;
                    }
                    /* one level coarser: the coarse cell containing this one */
                    if (l > 0) {
                        int64_t gc[3] = {g[0] >> 1, g[1] >> 1, g[2] >> 1};
                        t = find_cover(n_sub, E, lev, org, l - 1, gc);
                        if (t >= 0) {
                            int64_t src = off[t] + cidx(B, (int)(gc[0] - org[3 * t]) + NG,
                                                        (int)(gc[1] - org[3 * t + 1]) + NG,
                                                        (int)(gc[2] - org[3 * t + 2]) + NG);
                            for (int f = 0; f < nf; f++)
                                U[dst + f * fs] = U[src + f * fs];
                            continue;
                        }
                    }
                    /* one level finer: mean of the 8 children */
                    {
                        int64_t gf[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
                        t = find_cover(n_sub, E, lev, org, l + 1, gf);
                        if (t < 0) {
                            err = 1;
                            continue;
                        }
                        for (int f = 0; f < nf; f++) {
                            double sum = 0.0;
                            for (int dz = 0; dz < 2; dz++)
                                for (int dy = 0; dy < 2; dy++)
                                    for (int dx = 0; dx < 2; dx++) {
                                        int64_t ch[3] = {gf[0] + dx, gf[1] + dy, gf[2] + dz};
                                        int u = find_cover(n_sub, E, lev, org, l + 1, ch);
                                        if (u < 0) {
                                            err = 1;
                                            continue;
                                        }
                                        sum += U[off[u] + f * fs +
                                                 cidx(B, (int)(ch[0] - org[3 * u]) + NG, (int)(ch[1] - org[3 * u + 1]) + NG,
                                                      (int)(ch[2] - org[3 * u + 2]) + NG)];
                                    }
                            U[dst + f * fs] = sum / 8.0;
                        }
                    }
                }
    }
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Flux correction at coarse-fine faces (reading R15)                        */
/* ------------------------------------------------------------------------ */

/* With faces = the boundary face fluxes of oco_rhs_faces, replaces in dUdt
 * the flux through every face between a cell and a finer neighbour region by
 * the mean of the 4 fine fluxes on that face, so that what leaves the fine
 * cells enters the coarse cell and the total is conserved.  For the coarse
 * cell's upper face along axis k the RHS changes by (F_c - F_fine)/dx, for
 * its lower face by (F_fine - F_c)/dx.  The fine mean adds the 4 fluxes with
 * the first tangential index fastest, then scales by 1/4.  Cells are visited
 * subgrid by subgrid, axis x, y, z, lower side first.  Returns 0, or -2 when
 * a finer neighbour region does not start at a fine subgrid's face (levels
 * overlapping). */
int oco_amr_reflux(int n_sub, int E, const double *dx, int nf, const int32_t *lev, const int32_t *org, int n0,
                   int periodic, const double *faces, double *dUdt)
{
    int64_t EE = (int64_t)E * E, E3 = EE * E;
    int64_t fsz = 6 * (int64_t)nf * EE; /* one subgrid's face block */
    int err = 0;
    for (int s = 0; s < n_sub; s++) {
        int l = lev[s];
        int64_t nl = (int64_t)n0 << l;
        for (int k = 0; k < 3; k++) {
            int a1, a2;
            transverse(k, &a1, &a2);
            if (a1 > a2) {
                int t = a1;
                a1 = a2;
                a2 = t;
            }
            for (int side = 0; side < 2; side++)
                for (int t2 = 0; t2 < E; t2++)
                    for (int t1 = 0; t1 < E; t1++) {
                        int c[3];
                        c[k] = side ? E - 1 : 0;
                        c[a1] = t1;
                        c[a2] = t2;
                        /* the neighbour cell across the face, at this level */
                        int64_t g[3] = {org[3 * s] + c[0], org[3 * s + 1] + c[1], org[3 * s + 2] + c[2]};
                        g[k] += side ? 1 : -1;
                        if (g[k] < 0 || g[k] >= nl) {
                            if (!periodic)
                                continue; /* root-box edge */
                            g[k] = ((g[k] % nl) + nl) % nl;
                        }
                        if (find_cover(n_sub, E, lev, org, l, g) >= 0)
                            continue;
                        /* the finer cells on the far side of the face */
                        int64_t fc[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
                        if (!side)
                            fc[k] += 1;
                        int t = find_cover(n_sub, E, lev, org, l + 1, fc);
                        if (t < 0)
                            continue; /* a coarser neighbour: the fine side keeps its own flux */
                        int64_t nk = fc[k] - org[3 * t + k];
                        if (nk != (side ? 0 : E - 1)) {
                            err = 1;
                            continue;
                        }
                        int64_t u1 = fc[a1] - org[3 * t + a1], u2 = fc[a2] - org[3 * t + a2];
                        const double *Ft = faces + t * fsz + (int64_t)(2 * k + (side ? 0 : 1)) * nf * EE;
                        const double *Fs = faces + s * fsz + (int64_t)(2 * k + side) * nf * EE;
                        int64_t ci = ((int64_t)c[2] * E + c[1]) * E + c[0];
                        for (int f = 0; f < nf; f++) {
                            const double *q = Ft + f * EE;
                            double Ff = (((q[u2 * E + u1] + q[u2 * E + u1 + 1]) + q[(u2 + 1) * E + u1]) +
                                         q[(u2 + 1) * E + u1 + 1]) *
                                        0.25;
                            double Fc = Fs[f * EE + (int64_t)t2 * E + t1];
                            double *d = dUdt + (int64_t)s * nf * E3 + f * E3 + ci;
                            *d += side ? (Fc - Ff) / dx[s] : (Ff - Fc) / dx[s];
                        }
                    }
        }
    }
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Ghost fill across levels with limited linear prolongation (reading R17)   */
/* ------------------------------------------------------------------------ */

/* minmod of the two one-sided differences a = u(+1) - u(0), b = u(0) - u(-1):
 * the smaller in magnitude when both have the same strict sign, else 0. */
static double minmod2(double a, double b)
{
    if (!(a * b > 0.0))
        return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* As oco_amr_ghost_fill, with the prolongation order chosen by order:
 * 0 = injection (the fine ghost takes the covering coarse cell's value);
 * 1 = limited linear: the coarse value plus, per axis, a quarter of the
 *     minmod slope of the coarse cell and its two neighbours along that axis
 *     in the coarse subgrid's ghosted block, with the sign of the fine cell's
 *     offset from the coarse centre (+ for the upper child).  Sum order:
 *     t = s_x d_x; t = t + s_y d_y; t = t + s_z d_z; value = u + t / 4.
 *     A neighbour that is itself a ghost cell filled by prolongation is not
 *     used (zero slope on that axis), so the result does not depend on the
 *     order in which ghost cells are filled.
 * Copies and restrictions are done first, prolongations second (they read
 * the coarse blocks' ghost cells).  The 8 children of a coarse cell average
 * to its value.  Returns 0, or -2 when some ghost cell has no source. */
int oco_amr_ghost_fill_order(int n_sub, int E, const int64_t *off, int nf, const int32_t *lev, const int32_t *org,
                             int n0, int periodic, int order, double *U)
{
    if (!valid_edge(E) || order < 0 || order > 1)
        return -1;
    int B = E + 2 * NG;
    int64_t fs = (int64_t)B * B * B;
    /* kind of every cell of every block: 0 interior, 1 copy, 2 restriction,
     * 3 prolongation; and, for prolongations, the coarse source */
    uint8_t *kind = (uint8_t *)calloc((size_t)n_sub * fs, 1);
    int32_t *src_t = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_sub * fs);
    int64_t *src_c = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_sub * fs);
    uint8_t *par = (uint8_t *)calloc((size_t)n_sub * fs, 1);
    int err = 0;
    for (int pass = 1; pass <= 2; pass++)
        for (int s = 0; s < n_sub; s++) {
            int l = lev[s];
            int64_t nl = (int64_t)n0 << l;
            for (int z = -NG; z < E + NG; z++)
                for (int y = -NG; y < E + NG; y++)
                    for (int x = -NG; x < E + NG; x++) {
                        if (x >= 0 && x < E && y >= 0 && y < E && z >= 0 && z < E)
                            continue;
                        int64_t dl = cidx(B, x + NG, y + NG, z + NG);
                        int64_t dst = off[s] + dl;
                        if (pass == 2) {
                            if (kind[(int64_t)s * fs + dl] != 3)
                                continue;
                            /* limited linear prolongation from the coarse cell */
                            int t = src_t[(int64_t)s * fs + dl];
                            int64_t cl = src_c[(int64_t)s * fs + dl];
                            int p = par[(int64_t)s * fs + dl];
                            int64_t step[3] = {1, B, (int64_t)B * B};
                            for (int f = 0; f < nf; f++) {
                                const double *u = U + off[t] + f * fs;
                                double acc = 0.0;
                                for (int a = 0; a < 3; a++) {
                                    int64_t up = cl + step[a], dn = cl - step[a];
                                    double d = 0.0;
                                    if (kind[(int64_t)t * fs + up] != 3 && kind[(int64_t)t * fs + dn] != 3)
                                        d = minmod2(u[up] - u[cl], u[cl] - u[dn]);
                                    double sd = (p >> a) & 1 ? d : -d;
                                    acc = a == 0 ? sd : acc + sd;
                                }
                                U[dst + f * fs] = u[cl] + acc / 4.0;
                            }
                            continue;
                        }
                        int64_t g[3] = {org[3 * s] + x, org[3 * s + 1] + y, org[3 * s + 2] + z};
                        for (int a = 0; a < 3; a++) {
                            if (periodic)
                                g[a] = ((g[a] % nl) + nl) % nl;
                            else
                                g[a] = g[a] < 0 ? 0 : (g[a] >= nl ? nl - 1 : g[a]);
                        }
                        int t = find_cover(n_sub, E, lev, org, l, g);
                        if (t >= 0) {
                            int64_t src = off[t] + cidx(B, (int)(g[0] - org[3 * t]) + NG, (int)(g[1] - org[3 * t + 1]) + NG,
                                                        (int)(g[2] - org[3 * t + 2]) + NG);
                            for (int f = 0; f < nf; f++)
                                U[dst + f * fs] = U[src + f * fs];
                            kind[(int64_t)s * fs + dl] = 1;
                            continue;
                        }
                        if (l > 0) {
                            int64_t gc[3] = {g[0] >> 1, g[1] >> 1, g[2] >> 1};
                            t = find_cover(n_sub, E, lev, org, l - 1, gc);
                            if (t >= 0) {
                                int64_t cl = cidx(B, (int)(gc[0] - org[3 * t]) + NG, (int)(gc[1] - org[3 * t + 1]) + NG,
                                                  (int)(gc[2] - org[3 * t + 2]) + NG);
                                if (order == 0) {
                                    for (int f = 0; f < nf; f++)
                                        U[dst + f * fs] = U[off[t] + cl + f * fs];
                                    kind[(int64_t)s * fs + dl] = 1;
                                } else {
                                    kind[(int64_t)s * fs + dl] = 3;
                                    src_t[(int64_t)s * fs + dl] = t;
                                    src_c[(int64_t)s * fs + dl] = cl;
                                    par[(int64_t)s * fs + dl] =
                                        (uint8_t)((g[0] & 1) | ((g[1] & 1) << 1) | ((g[2] & 1) << 2));
                                }
                                continue;
                            }
                        }
                        int64_t gf[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
                        t = find_cover(n_sub, E, lev, org, l + 1, gf);
                        if (t < 0) {
                            err = 1;
                            continue;
                        }
                        for (int f = 0; f < nf; f++) {
                            double sum = 0.0;
                            for (int dz = 0; dz < 2; dz++)
                                for (int dy = 0; dy < 2; dy++)
                                    for (int dx = 0; dx < 2; dx++)
                                        sum += U[off[t] + f * fs +
                                                 cidx(B, (int)(gf[0] + dx - org[3 * t]) + NG,
                                                      (int)(gf[1] + dy - org[3 * t + 1]) + NG,
                                                      (int)(gf[2] + dz - org[3 * t + 2]) + NG)];
                            U[dst + f * fs] = sum / 8.0;
                        }
                        kind[(int64_t)s * fs + dl] = 2;
                    }
        }
    free(kind);
    free(src_t);
    free(src_c);
    free(par);
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Gravity: same-level monopole interactions (reading R18)                   */
/* ------------------------------------------------------------------------ */

/* The gravity solver's most compute-intensive step is the same-level
 * interaction between close-by cells; for non-refined cells it is the
 * "monopole" kernel (Sec. II "Solvers", Sec. IV).  Reading R18: on one level
 * of cell width dx, every interior cell i receives the potential and the
 * acceleration of every cell j of the same level within the interaction
 * radius, 0 < |x_j - x_i| <= r_s dx, each taken as a point mass
 * m_j = rho_j dx^3 at its centre (Newtonian gravity, constant G):
 *     phi_i = -G sum_j m_j / r_ij,
 *     g_i   = -G sum_j m_j (x_i - x_j) / r_ij^3,   r_ij = |x_i - x_j|.
 * Cells j are integer offsets d = (j - i) with d.d <= r_s^2, visited z
 * outermost, then y, then x, each from -R to R (R = floor(r_s) <= E); a
 * source cell is found in the subgrid itself or through the neighbour table
 * (as for the ghost fill; a missing neighbour holds no mass).  rho is field 0
 * of the ghosted state; all subgrids share edge E and the cell width dx.
 * Output: phi [subgrid][E^3], g [subgrid][3][E^3] (x, y, z).
 * Returns 0, or -1 for bad arguments. */
int oco_gravity_monopole(int n_sub, int E, const int64_t *off, int nf, const int32_t *nbr, double dx, double G,
                         double r_s, const double *U, double *phi, double *g)
{
    if (!valid_edge(E) || !(r_s >= 1.0) || (int)floor(r_s) > E || !(dx > 0.0))
        return -1;
    const int R = (int)floor(r_s);
    const int B = E + 2 * NG;
    const int64_t E3 = (int64_t)E * E * E;
    const double r2max = r_s * r_s;
    const double dx3 = dx * dx * dx;
    (void)nf;
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < n_sub; s++) {
        for (int z = 0; z < E; z++)
            for (int y = 0; y < E; y++)
                for (int x = 0; x < E; x++) {
                    double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
                    for (int dz = -R; dz <= R; dz++)
                        for (int dy = -R; dy <= R; dy++)
                            for (int ddx = -R; ddx <= R; ddx++) {
                                if (dz == 0 && dy == 0 && ddx == 0)
                                    continue;
                                const double d2 = (double)(ddx * ddx + dy * dy + dz * dz);
                                if (d2 > r2max)
                                    continue;
                                /* the source cell: its subgrid and local coordinates */
                                int c[3] = {x + ddx, y + dy, z + dz}, o[3];
                                for (int a = 0; a < 3; a++) {
                                    o[a] = c[a] < 0 ? -1 : (c[a] >= E ? 1 : 0);
                                    c[a] -= o[a] * E;
                                }
                                int src = s;
                                if (o[0] || o[1] || o[2]) {
                                    src = nbr[26 * (int64_t)s + nb_index(o[0], o[1], o[2])];
                                    if (src < 0)
                                        continue;
                                }
                                const double rho = U[off[src] + cidx(B, c[0] + NG, c[1] + NG, c[2] + NG)];
                                const double m = rho * dx3;
                                const double r = sqrt(d2) * dx;
                                const double r3 = r * r * r;
                                p -= G * m / r;
                                /* x_i - x_j = -d dx */
                                gx -= G * m * (-ddx * dx) / r3;
                                gy -= G * m * (-dy * dx) / r3;
                                gz -= G * m * (-dz * dx) / r3;
                            }
                    const int64_t q = ((int64_t)z * E + y) * E + x;
                    phi[(int64_t)s * E3 + q] = p;
                    g[(int64_t)s * 3 * E3 + q] = gx;
                    g[(int64_t)s * 3 * E3 + E3 + q] = gy;
                    g[(int64_t)s * 3 * E3 + 2 * E3 + q] = gz;
                }
    }
    return 0;
}
