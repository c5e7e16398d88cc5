// oct_common.cuh -- shared device definitions of the GB300 hydro kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace octh {

constexpr int NG = 3;       // ghost layers
constexpr int MAXNF = 11;   // 6 hydro fields + up to 5 species
constexpr int MAXT = 8;     // max tile edge (x and y) of one work item
constexpr int NTHREADS = 256;


enum { F_RHO = 0, F_SX = 1, F_SY = 2, F_SZ = 3, F_EGAS = 4, F_TAU = 5, F_SPC = 6 };

// One work item of the RHS kernel: a column of a subgrid, tx * ty cells in
// x-y, all E cells in z (the kernel streams through z planes).
struct WorkItem {
    int s;        // subgrid index
    int x0, y0;   // tile origin (interior coordinates)
    int txty;     // tx | ty << 8
};

// Line groups: the 13 PPM lines grouped so that both sides of every face
// quadrature point come from lines of one group (the L point of x-face point
// (t1,t2) lies on line (1,t1,t2), the R point on line (1,-t1,-t2)).
// Face point entries: axis, Simpson weight class, L (slot), R (slot); a slot
// is 2*line+end (end 1 = the x + d/2 end of canonical line d, end 0 = x - d/2)
// or, for the L side of a z face, 16 + index of the +z direction in the
// saved-plane buffer ((dy+1)*3 + (dx+1)).
struct GroupTab {
    int nl;
    int line[4][3];
    int npt;
    signed char axis[12], wcls[12], lslot[12], rslot[12];
    int nzp;                       // +z ends this group leaves for the next plane
    signed char zp_src[4], zp_dst[4];
    int has[3];                    // group has lines with a nonzero x / y / z step
    int napt;                      // face points per face, the most over the axes
    int nax[3];                    // face points per face of each axis
    signed char apt[3][4];         // indices into the point arrays, per face axis
};
constexpr int NGROUPS = 4;

struct RhsArgs {
    const double *U;
    double *dUdt;
    double *amax_tile;             // per work item
    const int *edge;
    const long long *off;          // state offsets (doubles)
    const long long *doff;         // RHS offsets (doubles)
    const double *dx;
    const WorkItem *items;
    int n_items;
    int nf;
    double gamma, eps1;
    double inv_gm1;                // 1 / (gamma - 1)
    unsigned *flags;
    // optional boundary face fluxes (null: none): subgrid s with
    // face_slot[s] >= 0 writes its 6 faces at faces + face_slot[s]*6*nf*E*E,
    // [face 2k+side][f][t2][t1] with (t1, t2) its other axes in increasing order
    double *faces;
    const int *face_slot;
    // execution order of the items (null: in index order) and the ticket
    // counter of dynamic scheduling ([0] next ticket, [1] CTAs done; both zero
    // between launches; null: static round robin)
    const int *order;
    int *ticket;
    // per subgrid: 1 when its ghosted block holds one value per field and
    // uniform_subgrid_kernel has written its RHS and a_max (null: no such test)
    const int *sub_uniform;
    // optional (null: the static items): the items of the subgrids left
    // after the uniform test, n_live[0] of them, and per item the slot of
    // amax_tile it reports to (~slot: half of a static item, reported by
    // atomic max into a slot zeroed beforehand)
    const WorkItem *live_items;
    const int *live_slot;
    const int *n_live;
    // optional (null: none): per subgrid, bit f set when field f of its
    // ghosted block holds one value.  Written by uniform_subgrid_kernel for
    // every subgrid it tests, read by the FP64 RHS kernel (conserved
    // reconstruction) for the subgrids that kernel takes
    unsigned *field_uni;
};

// q / d for the small divisors of the kernels' index arithmetic (tile widths,
// edges, cell and ghost-cell counts; 2 <= d < 2^12) as a multiply-high by
// m = ceil(2^32 / d): exact for q < 2^16, since the rounding error of m adds
// less than q d / 2^32 < 1/d to q / d.  A plain 32-bit division costs about
// twenty integer instructions.
__device__ __forceinline__ unsigned rcp_div(int d) { return 0xFFFFFFFFu / (unsigned)d + 1u; }
__device__ __forceinline__ int div_by(int q, unsigned m) { return (int)__umulhi((unsigned)q, m); }

// FP32-estimate helpers shared by the kernels (FP64 arithmetic on this GPU
// runs at about 1/64 of the FP32 rate).
__device__ __forceinline__ long long dbits_c(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd_c(long long b) { return __longlong_as_double(b); }

// double -> float for operands known to be in the normal float range,
// truncating the mantissa (an estimate only); returns false otherwise.
__device__ __forceinline__ bool d2f_est(double x, float &f)
{
    long long b = dbits_c(x);
    int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    unsigned int m = (unsigned int)((b >> 29) & 0x7FFFFF);
    f = __uint_as_float(((unsigned int)(b >> 32) & 0x80000000u) | ((unsigned int)e << 23) | m);
    return e > 1 && e < 253;
}

__device__ __forceinline__ double f2d_normal(float f)
{
    unsigned int b = __float_as_uint(f);
    unsigned long long e = ((b >> 23) & 0xFF) - 127 + 1023;
    return bitsd_c((long long)(((unsigned long long)(b & 0x80000000u) << 32) | (e << 52) |
                             ((unsigned long long)(b & 0x7FFFFF) << 29)));
}

// 1/x: FP32 reciprocal estimate (rcp.approx, about 2^-22 relative), then two
// Newton-Raphson steps r <- r + r (1 - x r), each squaring the relative error.
__device__ __forceinline__ double rcp_nr(double x)
{
    float xf;
    if (!d2f_est(x, xf))
        return 1.0 / x;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
    double r = f2d_normal(rf);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// sqrt(q): FP32 reciprocal-square-root estimate y (about 2^-22), s = q y,
// then two Newton (Heron) corrections s <- s + (q - s^2) y / 2.
__device__ __forceinline__ double sqrt_nr(double q)
{
    float qf;
    if (!d2f_est(q, qf) || __double2hiint(q) < 0)  // negative: sqrt gives NaN
        return sqrt(q);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(qf));
    double y = f2d_normal(yf);
    double h = f2d_normal(0.5f * yf);
    double s = q * y;
    double r = fma(-s, s, q);
    s = fma(r, h, s);
    r = fma(-s, s, q);
    return fma(r, h, s);
}

// tau^gamma, the internal energy that the entropy tracer gives where the
// dual-energy switch selects it.  For gamma = 5/3 (the ideal monatomic gas of
// every workload here): with tau = m 2^(3k), m in [1, 8) (exact, on the
// exponent field), tau^(5/3) = m^(5/3) 2^(5k), and y = m^(5/3) solves
// y^3 = m^5.  An FP32 estimate y0 = 2^(5/3 log2 m) (the hardware log2 and
// exp2 approximations; relative error below 1e-6) is refined by two Newton
// steps y <- y - (y^3 - m^5) r in FP64, r = 1/(3 y0^2) from FP32: each step
// multiplies the relative error by max(error, error of r), about 1e-6, so the
// result is within a few ulp.  Nine FP64 operations instead of a pow.  Other
// gamma, tau <= 0, tau outside [2^-600, 2^601) and inf or NaN: pow, in a call
// of its own so that warps without such a point do not issue it.
static __device__ __noinline__ double pow_rare(double x, double y) { return pow(x, y); }
__device__ __forceinline__ double eint_of_tau(double tau, double gamma)
{
    const int th = __double2hiint(tau);
    const int eb = (th >> 20) - 1023;  // unbiased exponent (th > 0: positive)
    if (__double_as_longlong(gamma) != __double_as_longlong(5.0 / 3.0) || th <= 0 || eb < -600 || eb > 600)
        return pow_rare(tau, gamma);
    // k = floor(eb / 3), j = eb - 3k in {0, 1, 2}
    const int k = (eb >= 0 ? eb : eb - 2) / 3;
    const int j = eb - 3 * k;
    const double m = __hiloint2double((th & 0x000FFFFF) | ((j + 1023) << 20), __double2loint(tau));
    const double m2 = m * m;
    const double T = m2 * m2 * m;
    float mf;
    d2f_est(m, mf);
    float lf, yf, rf;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lf) : "f"(mf));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(lf * (5.0f / 3.0f)));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(3.0f * yf * yf));
    const double r = f2d_normal(rf);
    double y = f2d_normal(yf);
    y = fma(-fma(y * y, y, -T), r, y);
    y = fma(-fma(y * y, y, -T), r, y);
    // y in [1, 32): scale by 2^(5k) on the exponent field (the result stays normal)
    return __hiloint2double(__double2hiint(y) + 5 * k * (1 << 20), __double2loint(y));
}

// e^(1/gamma), the entropy tracer of an internal energy e (the tau
// re-synchronisation).  For gamma = 5/3 (the ideal monatomic gas of every
// workload here): with e = m 2^(5k), m in [1, 32) (exact, on the exponent
// field), e^(3/5) = m^(3/5) 2^(3k), and y = m^(3/5) solves y^5 = m^3 = T.
// An FP32 estimate y0 = 2^(3/5 log2 m) (the hardware log2 and exp2
// approximations; relative error below 1e-6 for every m) is refined by two
// chord-Newton steps y <- y - (y^5 - T) r in FP64 with r = 1/(5 y0^4) from
// FP32: each multiplies the relative error by about 1e-6, so the result is
// within a couple of ulp whatever the magnitude of e.  Other gamma, e <= 0,
// zero, subnormal, inf or NaN: pow, in a call of its own.
static __device__ __noinline__ double pow_inv_rare(double x, double g) { return pow(x, 1.0 / g); }
__device__ __forceinline__ double tau_of_eint(double e, double gamma)
{
    const int eh = __double2hiint(e);
    if (__double_as_longlong(gamma) != __double_as_longlong(5.0 / 3.0) || eh < 0x00100000 || eh >= 0x7FF00000)
        return pow_inv_rare(e, gamma);
    const int eb = (eh >> 20) - 1023;  // unbiased exponent of a positive normal e
    // k = floor(eb / 5), j = eb - 5k in 0..4
    const int k = (eb >= 0 ? eb : eb - 4) / 5;
    const int j = eb - 5 * k;
    const double m = __hiloint2double((eh & 0x000FFFFF) | ((j + 1023) << 20), __double2loint(e));
    const double T = m * m * m;
    float mf;
    d2f_est(m, mf);
    float lf, yf, rf;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lf) : "f"(mf));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(lf * 0.6f));
    const float y2f = yf * yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(5.0f * y2f * y2f));
    const double r = f2d_normal(rf);
    double y = f2d_normal(yf);
#pragma unroll
    for (int it = 0; it < 2; it++) {
        const double y2 = y * y;
        y = fma(-fma(y2 * y2, y, -T), r, y);
    }
    // y in [1, 8): scale by 2^(3k) on the exponent field (the result stays normal)
    return __hiloint2double(__double2hiint(y) + 3 * k * (1 << 20), __double2loint(y));
}

}  // namespace octh
