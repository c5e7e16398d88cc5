// rhs_kernel.cuh -- fused hydro right-hand side on sm_103a (one template,
// instantiated for FP64 and for the mixed form).
//
// Method (Octo-Tiger hydro solver, arXiv 2210.06439 Sec. II "Solvers"):
// PPM reconstruction of every conserved field (or, on request, of the
// primitive variables) to the 26 points of each cell
// (6 face centres, 12 edge midpoints, 8 corners; the value at x + d/2 comes
// from 1-D PPM along the cells x + m d), the Kurganov-Tadmor flux at the 9
// Newton-Cotes (tensor Simpson) points of every face with a local speed per
// point, the face average, and the finite-volume divergence.
//
// GPU organisation.  A persistent CTA takes work items one after another (the
// first by block index, the rest from a device counter); an item is a tx * ty
// column of a subgrid (tx, ty <= 8), and the CTA streams through its z planes
// kz = -1 .. E.  For each plane
// the 13 lines are processed in 4 groups (the axis lines x, y, z; the xy and
// xz diagonals; the yz diagonals; the body diagonals); within a group both sides of each
// face quadrature point are available, so the flux of that point is formed as
// soon as the group's point values exist and no plane ever holds all 26
// points of all fields:
//   phase A  every (line, cell, field) of the group: 1-D PPM -> both ends
//            into the group buffer (shared memory);
//   phase B1 (FP64) the primitives of every needed point, once;
//   phase B2 one thread per face: the group's quadrature points of that face,
//            primitives on both sides, KT flux, Simpson-weighted sum into the
//            face accumulator; the z faces below the plane take their L side
//            from the +z ends the previous plane left in the saved buffer, and
//            the same thread then replaces those with this plane's +z ends.
// After the 4 groups the in-plane (x, y) face fluxes are complete; the
// divergence of a plane is finished one plane later, once its upper z face
// is known.  The signal speed max over all face points is reduced per item.
#pragma once
#include <utility>

#include "oct_common.cuh"

namespace octh {

// line-group tables, filled by the host at handle creation
__constant__ GroupTab c_groups[NGROUPS];

template <class T> struct Num;
template <> struct Num<double> {
    __device__ static __forceinline__ double from_d(double x) { return x; }
    __device__ static __forceinline__ double to_d(double x) { return x; }
};
// The mixed form converts with the hardware cvt (exact, round to nearest
// even): it issues on the FP64 pipe, which this form leaves idle, in one issue
// slot where a conversion in integer code takes about fifteen.
template <> struct Num<float> {
    __device__ static __forceinline__ float from_d(double x) { return __double2float_rn(x); }
    __device__ static __forceinline__ double to_d(float x) { return (double)x; }
};

// ---------------------------------------------------------------------------
// FP64 helpers that keep work off the FP64 pipe.  GB300 retires FP64
// arithmetic, compares, min/max and f64<->f32 conversions at about 1/64 of
// the FP32 rate, so sign tests, magnitude comparisons and power-of-two
// scalings are done on the bit patterns with integer operations (valid for
// normal numbers; the rare zero/subnormal/huge operands take a plain FP64
// path), and reciprocals and square roots start from an FP32 estimate and
// are refined by Newton-Raphson steps in FP64.
// ---------------------------------------------------------------------------

// The sign, zero and magnitude tests below work on the two 32-bit halves of
// a double: written on the 64-bit pattern they would be recognised and issued
// as FP64 compares and min/max, which is what they are meant to avoid.
struct HL {
    int h;           // high word (sign, exponent, top 20 mantissa bits)
    unsigned int l;  // low word
};
__device__ __forceinline__ HL hl(double x) { return HL{__double2hiint(x), (unsigned int)__double2loint(x)}; }
__device__ __forceinline__ double from_hl(int h, unsigned int l) { return __hiloint2double(h, (int)l); }
// |x| as (high word without sign, low word)
__device__ __forceinline__ bool is_zero(HL a) { return ((a.h & 0x7FFFFFFF) | a.l) == 0u; }
// |a| < |b| for the magnitude words (high words already without sign)
__device__ __forceinline__ bool mag_lt(int ah, unsigned int al, int bh, unsigned int bl)
{
    return ((unsigned int)ah < (unsigned int)bh) || (ah == bh && al < bl);
}

// Nonzero unless a and b have the same bit pattern (integer operations only).
__device__ __forceinline__ unsigned bit_diff(double a, double b)
{
    const HL A = hl(a), B = hl(b);
    return (unsigned)(A.h ^ B.h) | (A.l ^ B.l);
}
__device__ __forceinline__ unsigned bit_diff(float a, float b) { return __float_as_uint(a) ^ __float_as_uint(b); }

// max of two non-negative (or NaN) doubles by their bit patterns
__device__ __forceinline__ double max_nonneg(double x, double y)
{
    const HL X = hl(x), Y = hl(y);
    return mag_lt(X.h, X.l, Y.h, Y.l) ? y : x;
}
__device__ __forceinline__ float max_nonneg(float x, float y) { return fmaxf(x, y); }

// Monotonised-central slope from the two one-sided differences a = u0 - u-1
// and b = u1 - u0: minmod((a + b)/2, 2a, 2b), zero unless a and b share a
// strict sign.
// The rare cases (an operand or result outside the normal range) in calls
// of their own: a real branch, so that no warp issues their FP64 operations
// unless one of its lanes needs them.
static __device__ __noinline__ double mc_slope_rare(double s, int mh, unsigned int ml)
{
    return fmin(0.5 * fabs(s), 2.0 * from_hl(mh, ml));
}

__device__ __forceinline__ double mc_slope(double a, double b)
{
    // the common case without branches: the one FP64 operation (a + b) for
    // every lane, the case analysis on the integer words by selects
    const double s = a + b;
    const HL A = hl(a), Bv = hl(b), S = hl(s);
    const bool same = ((A.h ^ Bv.h) >= 0) && !is_zero(A) && !is_zero(Bv);
    const int ah = A.h & 0x7FFFFFFF, bh = Bv.h & 0x7FFFFFFF, sh = S.h & 0x7FFFFFFF;
    // m = min(|a|, |b|)
    const bool alb = mag_lt(ah, A.l, bh, Bv.l);
    const int mh = alb ? ah : bh;
    const unsigned int ml = alb ? A.l : Bv.l;
    const int em = mh >> 20, es = sh >> 20;
    // |s|/2 <= 2 m  <=>  |s| <= 4 m: compare with m's exponent raised by 2
    const bool half_s = !mag_lt(mh + (2 << 20), ml, sh, S.l);
    int rh = half_s ? sh - (1 << 20) : mh + (1 << 20);  // |s| / 2 or 2 m
    unsigned int rl = half_s ? S.l : ml;
    if (__builtin_expect(same && !(em >= 1 && em <= 2043 && es >= 2 && es <= 2046), 0)) {
        const HL R = hl(mc_slope_rare(s, mh, ml));
        rh = R.h;
        rl = R.l;
    }
    rh = same ? (rh | (A.h & (int)0x80000000)) : 0;
    rl = same ? rl : 0u;
    return from_hl(rh, rl);
}
__device__ __forceinline__ float mc_slope(float a, float b)
{
    // same strict sign <=> a b > 0 (a product below the FP32 range counts as
    // a sign change: such differences are far below the form's resolution)
    const float s = a + b;
    const float r = fminf(0.5f * fabsf(s), 2.0f * fminf(fabsf(a), fabsf(b)));
    return a * b > 0.f ? copysignf(r, s) : 0.f;
}

// x/2 exactly: on the exponent field of the high word for normal results;
// zero, infinity and NaN stay as they are; subnormal inputs or results by a
// multiply in a call of its own.
static __device__ __noinline__ double half_rare(double x) { return 0.5 * x; }
__device__ __forceinline__ double half_d(double x)
{
    const HL X = hl(x);
    const int e = (X.h >> 20) & 0x7FF;
    if (__builtin_expect(e == 1 || (e == 0 && !is_zero(X)), 0))
        return half_rare(x);
    return (e > 1 && e < 2047) ? from_hl(X.h - (1 << 20), X.l) : x;
}

// The CW84 constraints in FP64 for half-widths outside the normal range.
static __device__ __noinline__ void cw84_rare(double &d1, double &d2)
{
    if (fabs(d2) > 2.0 * fabs(d1))
        d2 = 2.0 * d1;
    else if (fabs(d1) > 2.0 * fabs(d2))
        d1 = 2.0 * d2;
}

// CW84 PPM on u_{-2..2}: limited values at the cell's two ends.  The
// parabola is carried as d1 = up - u0 and d2 = u0 - um, where up, um are the
// interface values (u0 + u+-1)/2 - (du+-1 - du0)/6:
//   d1 = (u1 - u0)/2 + (du0 - du1)/6,   d2 = (u0 - u-1)/2 + (du0 - du-1)/6.
// The CW84 monotonicity constraints then act on (d1, d2): flat at an
// extremum (d1 d2 <= 0); when |d2| > 2|d1| the parabola overshoots on the
// minus side and d2 becomes 2 d1; when |d1| > 2|d2|, d1 becomes 2 d2.
// Finally up = u0 + d1, um = u0 - d2.  The FP64 operations run for every
// lane; the constraints choose on the integer words.
// Returns true when the stencil's five values are bitwise equal (the cell
// value returned at both ends without arithmetic).
__device__ __forceinline__ bool ppm5(double um2, double um1, double u0, double up1, double up2, double &vm,
                                     double &vp)
{
    // a stencil of five bitwise-equal values (uniform regions such as an
    // atmosphere) is its own reconstruction: tested on the integer words
    // before any FP64 operation, a branch so that warps with no other lanes
    // skip the rest
    {
        const HL M2 = hl(um2), M1 = hl(um1), Z = hl(u0), Q1 = hl(up1), Q2 = hl(up2);
        const unsigned d = (unsigned)((M2.h ^ Z.h) | (M1.h ^ Z.h) | (Q1.h ^ Z.h) | (Q2.h ^ Z.h)) |
                           (M2.l ^ Z.l) | (M1.l ^ Z.l) | (Q1.l ^ Z.l) | (Q2.l ^ Z.l);
        if (d == 0u) {
            vm = u0;
            vp = u0;
            return true;
        }
    }
    const double am2 = um1 - um2, am1 = u0 - um1, ap1 = up1 - u0, ap2 = up2 - up1;
    // a constant stencil whose values differ only in the sign of zero
    const HL A2 = hl(am2), A1 = hl(am1), P1 = hl(ap1), P2 = hl(ap2);
    if (is_zero(A2) && is_zero(A1) && is_zero(P1) && is_zero(P2)) {
        vm = u0;
        vp = u0;
        return false;
    }
    const double dm = mc_slope(am2, am1);
    const double d0 = mc_slope(am1, ap1);
    const double dp = mc_slope(ap1, ap2);
    const double s6 = 1.0 / 6.0;
    double d1 = fma(d0 - dp, s6, half_d(ap1));
    double d2 = fma(d0 - dm, s6, half_d(am1));
    HL D1 = hl(d1), D2 = hl(d2);
    const bool flat = ((D1.h ^ D2.h) < 0) || is_zero(D1) || is_zero(D2);
    const int h1 = D1.h & 0x7FFFFFFF, h2 = D2.h & 0x7FFFFFFF;
    const int e1 = h1 >> 20, e2 = h2 >> 20;
    if (__builtin_expect(!flat && !(e1 >= 1 && e1 <= 2045 && e2 >= 1 && e2 <= 2045), 0)) {
        cw84_rare(d1, d2);
        D1 = hl(d1);
        D2 = hl(d2);
    } else {
        const bool A = mag_lt(h1 + (1 << 20), D1.l, h2, D2.l);         // |d2| > 2|d1|: d2 = 2 d1
        const bool Bp = !A && mag_lt(h2 + (1 << 20), D2.l, h1, D1.l);  // |d1| > 2|d2|: d1 = 2 d2
        const HL N2 = {A ? D1.h + (1 << 20) : D2.h, A ? D1.l : D2.l};
        const HL N1 = {Bp ? D2.h + (1 << 20) : D1.h, Bp ? D2.l : D1.l};
        D1 = N1;
        D2 = N2;
    }
    // flat: both half-widths zero, so that up = um = u0
    vp = u0 + from_hl(flat ? 0 : D1.h, flat ? 0u : D1.l);
    vm = u0 - from_hl(flat ? 0 : D2.h, flat ? 0u : D2.l);
    return false;
}

// The FP32 form: the interface values first, then the constraints on
// d1 = up - u0 and d2 = u0 - um formed from them.
// No test for stencils of one value here: a constant stencil already gives
// u0 at both ends through the arithmetic below, the FP32 form has no phase B1
// to feed, and whole uniform columns never reach this phase; on data without
// uniform regions the test cost about 4% of the RHS.
__device__ __forceinline__ bool ppm5(float um2, float um1, float u0, float up1, float up2, float &vm, float &vp)
{
    const float am2 = um1 - um2, am1 = u0 - um1, ap1 = up1 - u0, ap2 = up2 - up1;
    const float dm = mc_slope(am2, am1);
    const float d0 = mc_slope(am1, ap1);
    const float dp = mc_slope(ap1, ap2);
    const float s6 = 1.0f / 6.0f;
    const float up = fmaf(d0 - dp, s6, fmaf(0.5f, ap1, u0));
    const float um = fmaf(d0 - dm, -s6, fmaf(-0.5f, am1, u0));
    const float d1 = up - u0, d2 = u0 - um;
    // the constraints by selects: FP32 arithmetic is cheap, divergence is not
    const bool flat = d1 * d2 <= 0.f;
    const bool A = fabsf(d2) > 2.f * fabsf(d1);
    const bool Bp = !A && fabsf(d1) > 2.f * fabsf(d2);
    const float umc = fmaf(-2.f, d1, u0), upc = fmaf(2.f, d2, u0);
    vm = flat ? u0 : (A ? umc : um);
    vp = flat ? u0 : (Bp ? upc : up);
    return false;
}

// Point primitives: velocity, pressure (dual energy) and sound speed.
__device__ __forceinline__ void prim_point(const double *q, double gamma, double gm1, double ggm1, double eps1,
                                           double *v, double &p, double &c, bool &bad)
{
    const double rho = q[F_RHO];
    const double ir = rcp_nr(rho);
    const double vx = q[F_SX] * ir, vy = q[F_SY] * ir, vz = q[F_SZ] * ir;
    const double sv = fma(q[F_SZ], vz, fma(q[F_SY], vy, q[F_SX] * vx));
    double ei = fma(-0.5, sv, q[F_EGAS]);
    double c2;
    if (ei < eps1 * q[F_EGAS]) {
        ei = eint_of_tau(q[F_TAU], gamma);
        p = gm1 * ei;
        c2 = gamma * p * ir;
    } else {
        p = gm1 * ei;
        c2 = ggm1 * ei * ir;
    }
    // c2 > 0 (and finite) on the high word; zero gives c = 0; a negative or
    // non-finite c2 or rho is reported as non-physical
    const int ch = __double2hiint(c2), rh = __double2hiint(rho);
    c = (ch > 0 && ch < 0x7FF00000) ? sqrt_nr(c2) : (is_zero(hl(c2)) ? 0.0 : sqrt(c2));
    v[0] = vx;
    v[1] = vy;
    v[2] = vz;
    bad |= !(rh > 0 && rh < 0x7FF00000) || !(ch >= 0 && ch < 0x7FF00000);
}
__device__ __forceinline__ void prim_point(const float *q, float gamma, float gm1, float ggm1, float eps1,
                                           float *v, float &p, float &c, bool &bad)
{
    const float rho = q[F_RHO];
    const float ir = __fdividef(1.f, rho);
    const float vx = q[F_SX] * ir, vy = q[F_SY] * ir, vz = q[F_SZ] * ir;
    const float sv = fmaf(q[F_SZ], vz, fmaf(q[F_SY], vy, q[F_SX] * vx));
    float ei = fmaf(-0.5f, sv, q[F_EGAS]);
    float c2;
    if (ei < eps1 * q[F_EGAS]) {
        ei = powf(q[F_TAU], gamma);
        p = gm1 * ei;
        c2 = gamma * p * ir;
    } else {
        p = gm1 * ei;
        c2 = ggm1 * ei * ir;
    }
    c = c2 > 0.f ? c2 * rsqrtf(c2) : sqrtf(c2);
    v[0] = vx;
    v[1] = vy;
    v[2] = vz;
    bad |= !(rho > 0.f) || !(c == c);
}

// Primitive reconstruction (the optional variable choice): the point holds
// w = (rho, v, p, tau, X_i); its sound speed c = sqrt(gamma p / rho) and
// whether it is physical (rho > 0, c finite).
__device__ __forceinline__ double sound_from_w(double rho, double p, double gamma, bool &bad)
{
    const double c2 = gamma * p * rcp_nr(rho);
    const int ch = __double2hiint(c2), rh = __double2hiint(rho);
    bad |= !(rh > 0 && rh < 0x7FF00000) || !(ch >= 0 && ch < 0x7FF00000);
    return (ch > 0 && ch < 0x7FF00000) ? sqrt_nr(c2) : (is_zero(hl(c2)) ? 0.0 : sqrt(c2));
}
__device__ __forceinline__ float sound_from_w(float rho, float p, float gamma, bool &bad)
{
    const float c2 = gamma * p * __fdividef(1.f, rho);
    const float c = c2 > 0.f ? c2 * rsqrtf(c2) : sqrtf(c2);
    bad |= !(rho > 0.f) || !(c == c);
    return c;
}

// Shared-memory plan of one CTA (dynamic shared memory) for a tile capacity
// of txm x tym cells and nf fields.
struct SmemPlan {
    int nc;          // cells per plane buffer row: interior + ring
    size_t temp, saved, pr, prs, cpr, faccx, faccy, zacc, dxy, raw, red, lists, total;
};

__host__ __device__ inline SmemPlan smem_plan(int nf, int elem, bool staged, int txm, int tym)
{
    SmemPlan p;
    const int cin = txm * tym;
    p.nc = cin + 2 * txm + 2 * tym;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o += (bytes + 15) / 16 * 16; return at; };
    p.temp = take((size_t)8 * nf * p.nc * elem);
    p.saved = take((size_t)9 * nf * cin * elem);
    const bool shared_prims = elem == 8;  // FP32 recomputes primitives per face point
    p.pr = shared_prims ? take((size_t)8 * 5 * p.nc * elem) : 0;
    p.prs = shared_prims ? take((size_t)9 * 5 * cin * elem) : 0;
    p.cpr = shared_prims ? take((size_t)5 * p.nc * elem) : 0;
    p.faccx = take((size_t)nf * (txm + 1) * tym * elem);
    p.faccy = take((size_t)nf * txm * (tym + 1) * elem);
    p.zacc = take((size_t)2 * nf * cin * elem);
    p.dxy = take((size_t)nf * cin * sizeof(double));
    p.raw = staged ? take((size_t)5 * nf * (tym + 2 * NG) * (txm + 2 * NG) * sizeof(float)) : 0;
    p.red = take(64 * sizeof(double));
    p.lists = take((size_t)4 * p.nc * sizeof(int));
    p.total = o;
    return p;
}

// Compact index of plane cell (i, j) of a tx * ty tile: interior first, then
// the x ring (i = -1, i = tx), then the y ring (j = -1, j = ty).
__device__ __forceinline__ int cidx(int i, int j, int tx, int ty)
{
    if (i >= 0 && i < tx && j >= 0 && j < ty)
        return j * tx + i;
    if (i == -1)
        return tx * ty + j;
    if (i == tx)
        return tx * ty + ty + j;
    if (j == -1)
        return tx * ty + 2 * ty + i;
    return tx * ty + 2 * ty + tx + i;
}

// Compile-time line geometry of group g (the same grouping as the host's
// table): 0 the three axis lines x, y, z; 1 the xy and xz diagonals; 2 the yz
// diagonals; 3 the body diagonals.
__host__ __device__ constexpr int gnl(int g) { return g == 0 ? 3 : (g == 2 ? 2 : 4); }
__host__ __device__ constexpr int gline(int g, int l, int a)
{
    return g == 0   ? (a == l ? 1 : 0)
           : g == 1 ? (a == 0 ? 1 : a == 1 ? (l == 0 ? 1 : l == 1 ? -1 : 0) : (l == 2 ? 1 : l == 3 ? -1 : 0))
           : g == 2 ? (a == 1 ? 1 : a == 2 ? (l == 0 ? 1 : -1) : 0)
                    : (a == 0 ? 1 : a == 1 ? ((l == 0 || l == 3) ? 1 : -1) : ((l == 0 || l == 2) ? 1 : -1));
}

template <class F, int... I>
__device__ __forceinline__ void sfor_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
// calls f(integral_constant<int, i>) for i = 0 .. N-1
template <int N, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// Phase A of line group G: 1-D PPM of every (line, field, cell), both ends
// into the group buffer.  The line steps are compile-time constants; the
// mixed form orders the items line, field, cell, the FP64 form field, line,
// cell (its stencils come through L1, and the lines of one field then reuse
// that field's planes: RHS 6.91 -> 6.82 ms on the 256^3 binary star, 3.41 ->
// 3.38 ms on the 64^3 box).  The mixed form takes three fields per
// item: its integer work (item decoding, addressing) outweighs the FP32
// arithmetic, and the fields of an item share it (RHS 0.82 -> 0.77 ms on the
// 64^3 box; two fields 0.78, four 0.82); the FP64 form keeps one field per
// item (registers).
//
// The FP64 form takes only the nfa fields listed in fmap (the others hold one
// value over the subgrid's whole ghosted block, and their group slots were
// filled with it once for the item).  Its items read their stencils from the
// state through L1; with up to 512 threads (128 registers) each thread loads
// the stencil of its next item before the PPM of the current one, so that the
// load latency overlaps the arithmetic.
template <class T, bool STAGED, int G, int NT>
__device__ __forceinline__ bool phase_a(T *temp, const float *raw, const double *Ub, long long FS, int B, int x0,
                                        int y0, int kz, bool inplane, int nf, int NC, int RWX, int plane,
                                        const int *lists, const int *nlist, const unsigned *magic, const int *so,
                                        int tid, const unsigned char *fmap, int nfa)
{
    constexpr int NL = gnl(G);
    constexpr int FPI = STAGED ? 3 : 1;  // fields per item
    const int nfi = STAGED ? (nf + FPI - 1) / FPI : nfa;
    // per line: its cell list (the x / y ring only for lines with a nonzero x /
    // y step, in planes that own x / y faces) and its item count; lines without
    // a z step have nothing to do in the boundary planes
    bool sawc = false;  // a stencil of one value met
    int beg[NL + 1];
    beg[0] = 0;
    sfor<NL>([&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        constexpr int t = (gline(G, L, 0) != 0) | ((gline(G, L, 1) != 0) << 1);
        const int n = inplane ? nlist[t] : (gline(G, L, 2) != 0 ? nlist[0] : 0);
        beg[L + 1] = beg[L] + n * nfi;
    });
    if constexpr (!STAGED) {
        // items field-major: every line of one field, then the next field, so
        // that the lines of a field reuse its planes while they are in L1
        int cum[NL + 1];
        cum[0] = 0;
        sfor<NL>([&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            constexpr int t = (gline(G, L, 0) != 0) | ((gline(G, L, 1) != 0) << 1);
            cum[L + 1] = cum[L] + (inplane ? nlist[t] : (gline(G, L, 2) != 0 ? nlist[0] : 0));
        });
        const int S = cum[NL];
        const unsigned mS = S > 0 ? rcp_div(S) : 0u;
        // item q: its slot offset o in temp and its stencil (centre ub, step st)
        auto item = [&](int q, int &o, const double *&ub, long long &st) {
            const int fq = __umulhi((unsigned)q, mS);
            const int rq = q - fq * S;
            sfor<NL>([&](auto Lc) {
                constexpr int L = decltype(Lc)::value;
                if (rq >= cum[L] && rq < cum[L + 1]) {
                    constexpr int dx = gline(G, L, 0), dy = gline(G, L, 1), dz = gline(G, L, 2);
                    const int t = inplane ? ((dx != 0) | ((dy != 0) << 1)) : 0;
                    const int c = rq - cum[L];
                    const int info = lists[t * NC + c];
                    const int i = (info & 0xFF) - 1, j = ((info >> 8) & 0xFF) - 1;
                    const int f = fmap[fq];
                    o = ((2 * L) * nf + f) * NC + (info >> 16);
                    st = (long long)dz * B * B + (long long)dy * B + dx;
                    ub = Ub + f * FS + (long long)(kz + NG) * B * B + (long long)(y0 + j + NG) * B + (x0 + i + NG);
                }
            });
        };
        if constexpr (NT <= 512) {
            double un[5];
            int on = 0;
            if (tid < beg[NL]) {
                const double *ub = Ub;
                long long st = 0;
                item(tid, on, ub, st);
#pragma unroll
                for (int m = -2; m <= 2; m++)
                    un[m + 2] = __ldg(ub + m * st);
            }
            for (int q = tid; q < beg[NL]; q += NT) {
                double u[5];
#pragma unroll
                for (int m = 0; m < 5; m++)
                    u[m] = un[m];
                const int o = on;
                if (q + NT < beg[NL]) {
                    const double *ub = Ub;
                    long long st = 0;
                    item(q + NT, on, ub, st);
#pragma unroll
                    for (int m = -2; m <= 2; m++)
                        un[m + 2] = __ldg(ub + m * st);
                }
                double vm, vp;
                sawc |= ppm5(u[0], u[1], u[2], u[3], u[4], vm, vp);
                temp[o] = vm;
                temp[o + nf * NC] = vp;
            }
        } else {
            for (int q = tid; q < beg[NL]; q += NT) {
                int o = 0;
                const double *ub = Ub;
                long long st = 0;
                item(q, o, ub, st);
                double u[5];
#pragma unroll
                for (int m = -2; m <= 2; m++)
                    u[m + 2] = __ldg(ub + m * st);
                double vm, vp;
                sawc |= ppm5(u[0], u[1], u[2], u[3], u[4], vm, vp);
                temp[o] = vm;
                temp[o + nf * NC] = vp;
            }
        }
        return sawc;
    } else {
        for (int q = tid; q < beg[NL]; q += NT) {
            sfor<NL>([&](auto Lc) {
                constexpr int L = decltype(Lc)::value;
                if (q >= beg[L] && q < beg[L + 1]) {
                    constexpr int dx = gline(G, L, 0), dy = gline(G, L, 1), dz = gline(G, L, 2);
                    const int t = inplane ? ((dx != 0) | ((dy != 0) << 1)) : 0;
                    const int n = nlist[t];
                    const int r = q - beg[L];
                    const int fq = __umulhi((unsigned)r, magic[t]);
                    const int c = r - fq * n;
                    const int info = lists[t * NC + c];
                    const int i = (info & 0xFF) - 1, j = ((info >> 8) & 0xFF) - 1, ci = info >> 16;
#pragma unroll
                    for (int k = 0; k < FPI; k++) {
                        const int f = FPI * fq + k;
                        if (k > 0 && f >= nf)
                            break;
                        T u[5];
                        const float *rb = raw + f * plane + (j + NG) * RWX + (i + NG);
                        const int step = dy * RWX + dx;
#pragma unroll
                        for (int m = -2; m <= 2; m++)
                            u[m + 2] = (T)rb[so[dz > 0 ? m + 2 : (dz < 0 ? 2 - m : 2)] + m * step];
                        T vm, vp;
                        sawc |= ppm5(u[0], u[1], u[2], u[3], u[4], vm, vp);
                        temp[((2 * L) * nf + f) * NC + ci] = vm;
                        temp[((2 * L + 1) * nf + f) * NC + ci] = vp;
                    }
                }
            });
        }
        return sawc;
    }
}

// PRIM: the state array holds the primitive variables w of every cell
// (rho, v, p, tau, X_i) and PPM reconstructs them; each point is turned back
// into conserved fields (s = rho v, E = p/(gamma-1) + rho |v|^2/2,
// rho_i = rho X_i) with its reconstructed v and p kept for the flux.
// NT: threads per CTA (256, or 512 for one CTA per SM over 8x8 tiles).
template <class T, bool STAGED, int TXM, int TYM, int MINB, bool PRIM, int NT>
__global__ void __launch_bounds__(NT, MINB) rhs_kernel(RhsArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // FP64: primitives once per point, shared through shared memory (FP64
    // arithmetic is scarce); FP32: recomputed at each face point (cheap), which
    // saves a phase and its barrier per line group
    constexpr bool SHARED_PRIMS = sizeof(T) == 8;
    // scale of the face sums: 1 in FP64, 1/36 in FP32 (exact Simpson weights)
    constexpr double FSC = sizeof(T) == 8 ? 1.0 : 1.0 / 36.0;
    constexpr double HWS = sizeof(T) == 8 ? 1.0 / 36.0 : 1.0;  // Simpson weight scale
    const int nf = A.nf;
    const SmemPlan P = smem_plan(nf, sizeof(T), STAGED, TXM, TYM);
    constexpr int NC = TXM * TYM + 2 * TXM + 2 * TYM;
    constexpr int C64 = TXM * TYM;                 // interior cells of a full tile
    constexpr int FXS = (TXM + 1) * TYM;           // x faces of a full tile
    constexpr int FYS = TXM * (TYM + 1);           // y faces
    constexpr int XW = (FXS + 31) / 32 * 32, YW = (FYS + 31) / 32 * 32, ZW = (C64 + 31) / 32 * 32;
    static_assert(XW + YW + ZW <= NT, "face threads exceed the block");
    T *temp = reinterpret_cast<T *>(smem + P.temp);    // [8 slots][nf][NC] point values of the group
    T *saved = reinterpret_cast<T *>(smem + P.saved);  // [9][nf][64] +z ends of the previous plane
    T *pr = reinterpret_cast<T *>(smem + P.pr);        // [8 slots][5][NC] vx, vy, vz, p, c of the group
    T *prs = reinterpret_cast<T *>(smem + P.prs);      // [9][5][64] the same for the saved +z ends
    T *cpr = reinterpret_cast<T *>(smem + P.cpr);      // [5][NC] the same of the plane's cells (c < 0: none)
    T *faccx = reinterpret_cast<T *>(smem + P.faccx);  // [nf][72]
    T *faccy = reinterpret_cast<T *>(smem + P.faccy);  // [nf][72]
    T *zacc = reinterpret_cast<T *>(smem + P.zacc);    // [2][nf][64]
    double *dxy = reinterpret_cast<double *>(smem + P.dxy);  // [nf][64]
    float *raw = reinterpret_cast<float *>(smem + P.raw);    // [5][nf][14][14]
    double *red = reinterpret_cast<double *>(smem + P.red);
    int *lists = reinterpret_cast<int *>(smem + P.lists);    // [4][96] packed cells
    const int tid = threadIdx.x;
    const T gamma = Num<T>::from_d(A.gamma);
    const T gm1 = Num<T>::from_d(A.gamma - 1.0);
    const T ggm1 = Num<T>::from_d(A.gamma * (A.gamma - 1.0));
    const T eps1 = Num<T>::from_d(A.eps1);
    const T inv_gm1 = Num<T>::from_d(A.inv_gm1);
    constexpr int RWX = TXM + 2 * NG, RWY = TYM + 2 * NG;  // staged plane shape
    // the first line group with faces of each axis writes its face sums, the
    // later ones add to them: no zeroing of the face accumulators is needed
    int first_g[3] = {-1, -1, -1};
    for (int g = NGROUPS - 1; g >= 0; g--)
        for (int a = 0; a < 3; a++)
            if (c_groups[g].has[a])
                first_g[a] = g;
    bool bad = false;

    // work items: the first by block index, the rest from the ticket counter
    // in execution order (largest first), so that CTAs which finish early take
    // the remaining items; without a ticket, a static round robin
    __shared__ int s_next[2];  // by parity: an item that is skipped has no barrier of its own
    int par = 0;
    // whether phase A of a line group met a stencil of one value (uniform
    // data), by group parity: set in phase A, read after its barrier, cleared
    // for the group after next during phase B2.  Only then do phases B1 and
    // B2 look for uniform points and faces, so that data without uniform
    // regions pays nothing for those tests
    __shared__ int s_const[2];
    if (tid < 2)
        s_const[tid] = 0;
    // FP64, conserved reconstruction: the fields of the item that phase A
    // reconstructs (those not one value over the subgrid's ghosted block).
    // Not in the FP32 form: it is issue-bound, and looking the fields up in
    // the staging and the PPM items cost more there than the fields skipped
    // save (mixed RHS 0.76 -> 0.84 ms on the box, 2.92 -> 2.97 ms on the
    // 256^3 binary star)
    constexpr bool FSKIP = sizeof(T) == 8 && !STAGED && !PRIM;
    __shared__ unsigned char s_fmap[MAXNF];
    if (tid < MAXNF)
        s_fmap[tid] = (unsigned char)tid;
    unsigned cur_funi = 0u;  // the fields s_fmap leaves out
    __syncthreads();
    const int n_items = A.n_live != nullptr ? A.n_live[0] : A.n_items;
    for (int k = blockIdx.x; k < n_items;) {
        const int it = A.n_live != nullptr ? k : (A.order != nullptr ? A.order[k] : k);
        const WorkItem W = A.n_live != nullptr ? A.live_items[k] : A.items[it];
        const int s = W.s, x0 = W.x0, y0 = W.y0, tx = W.txty & 0xFF, ty = (W.txty >> 8) & 0xFF;
        if (A.sub_uniform != nullptr && A.sub_uniform[s] != 0) {
            // the subgrid's whole ghosted block holds one value per field: its
            // RHS and a_max were written by uniform_subgrid_kernel
            if (tid == 0)
                s_next[par] = A.ticket != nullptr ? (int)gridDim.x + atomicAdd(A.ticket, 1) : k + (int)gridDim.x;
            __syncthreads();
            k = s_next[par];
            par ^= 1;
            continue;
        }
        const int E = A.edge[s], B = E + 2 * NG;
        const long long FS = (long long)B * B * B;
        const double *Ub = A.U + A.off[s];
        double *dUb = A.dUdt + A.doff[s];
        const double rdx = (1.0 / A.dx[s]) * FSC;  // FP32 face sums carry a factor 36
        const unsigned m_tx = rcp_div(tx), m_tx1 = rcp_div(tx + 1), m_ty = rcp_div(ty);
        const int rows_s = ty + 2 * NG, cols_s = tx + 2 * NG;  // staged plane of this item
        const unsigned m_rc = rcp_div(rows_s * cols_s), m_cols = rcp_div(cols_s);
        const int ncin = tx * ty;
        double amax = 0.0;
        unsigned funi = 0u;  // fields whose whole ghosted block holds one value
        if constexpr (FSKIP) {
            if (A.field_uni != nullptr)
                funi = A.field_uni[s] & ((1u << nf) - 1u);
            if (funi != cur_funi) {  // the same for the whole CTA
                if (tid == 0) {
                    int k = 0;
                    for (int f = 0; f < nf; f++)
                        if (!((funi >> f) & 1u))
                            s_fmap[k++] = (unsigned char)f;
                }
                __syncthreads();
                cur_funi = funi;
            }
        }
        const int nfa = nf - __popc(funi);  // fields phase A takes: s_fmap[0 .. nfa)
        // this subgrid's boundary face fluxes, if wanted (looked up where used:
        // a pointer kept live across the plane loop costs registers)
        auto face_block = [&]() -> double * {
            const int sl = A.face_slot[s];
            return sl >= 0 ? A.faces + (long long)sl * 6 * nf * E * E : nullptr;
        };

        auto stage_plane = [&](int kz) {
            if constexpr (STAGED) {
                int slot = (kz + 3) % 5;
                int n = nf * rows_s * cols_s;
                for (int q = tid; q < n; q += NT) {
                    int f = div_by(q, m_rc), r = q - f * (rows_s * cols_s);
                    int jj = div_by(r, m_cols), ii = r - jj * cols_s;
                    double v = __ldg(Ub + f * FS + (long long)(kz + NG) * B * B + (long long)(y0 + jj) * B + (x0 + ii));
                    raw[((slot * nf + f) * RWY + jj) * RWX + ii] = __double2float_rn(v);
                }
            }
        };
        // cell lists of a plane: 0 interior, 1 + x ring, 2 + y ring, 3 both;
        // entry = (i + 1) | (j + 1) << 8 | compact index << 16
        int nlist[4];
        nlist[0] = ncin;
        nlist[1] = ncin + 2 * ty;
        nlist[2] = ncin + 2 * tx;
        nlist[3] = ncin + 2 * tx + 2 * ty;
        for (int q = tid; q < 4 * NC; q += NT) {
            int t = q / NC, c = q % NC;
            if (c >= nlist[t])
                continue;
            int i, j;
            if (c < ncin) {
                j = div_by(c, m_tx);
                i = c - j * tx;
            } else {
                int r = c - ncin;
                if ((t & 1) && r < 2 * ty) {
                    i = (r < ty) ? -1 : tx;
                    j = r - div_by(r, m_ty) * ty;
                } else {
                    if (t & 1)
                        r -= 2 * ty;
                    j = (r < tx) ? -1 : ty;
                    i = r - div_by(r, m_tx) * tx;
                }
            }
            lists[q] = (i + 1) | ((j + 1) << 8) | (cidx(i, j, tx, ty) << 16);
        }
        unsigned magic[4];
#pragma unroll
        for (int t = 0; t < 4; t++)
            magic[t] = rcp_div(nlist[t]);

        // ---- uniform column: when every value the item reads -- the tile
        // and its 3-cell halo over the planes -3 .. E+2, every field -- is one
        // value per field, every face flux of the column is the same, so each
        // cell's RHS is -(0 + 0) / dx = -0.0 exactly as the full path writes
        // it, and a_max is max_k |v_k| + c of that state (the same primitive
        // function as at the face points).  Both are written directly.  The
        // test reads the column in rounds of NT values and leaves at the
        // first round that finds a difference.  (Not with primitive
        // reconstruction, or when boundary face fluxes are wanted.) ----
        bool ucol = false;
        if constexpr (!PRIM) {
            if (A.faces == nullptr) {
                const int cols = tx + 2 * NG, rows = ty + 2 * NG, planes = E + 2 * NG;
                const double *ub0 = Ub + (long long)y0 * B + x0;  // ghosted (x0, y0, 0)
                constexpr int VPT = 4;  // loads in flight per thread per round
                int diff = 0;
                if (cols == B) {
                    // full-width tiles: each (field, plane) is one run of rows * B doubles,
                    // 16-byte aligned (blocks start on 32 bytes; B = 14, 18 or 22 is even
                    // and so is every row offset), read as double2
                    const int run = rows * B / 2, n = nf * planes * run;
                    const unsigned m_run = rcp_div(run), m_pl = rcp_div(planes);
                    for (int r0 = 0; r0 < n && !diff; r0 += VPT * NT) {
#pragma unroll
                        for (int u = 0; u < VPT; u++) {
                            const int q = r0 + u * NT + tid;
                            if (q < n) {
                                const int fz = div_by(q, m_run), v = q - fz * run;
                                const int f = div_by(fz, m_pl), z = fz - f * planes;
                                const double *fb = ub0 + f * FS;
                                const double2 w =
                                    __ldg(reinterpret_cast<const double2 *>(fb + (long long)z * B * B) + v);
                                const double ref = __ldg(fb);
                                diff |= (bit_diff(w.x, ref) | bit_diff(w.y, ref)) != 0u;
                            }
                        }
                        diff = __syncthreads_or(diff);
                    }
                } else {
                    const int per_f = planes * rows * cols, n = nf * per_f;
                    const unsigned m_pf = rcp_div(per_f), m_rcs = rcp_div(rows * cols), m_cols = rcp_div(cols);
                    for (int r0 = 0; r0 < n && !diff; r0 += VPT * NT) {
#pragma unroll
                        for (int u = 0; u < VPT; u++) {
                            const int q = r0 + u * NT + tid;
                            if (q < n) {
                                const int f = div_by(q, m_pf), r = q - f * per_f;
                                const int z = div_by(r, m_rcs), r2 = r - z * rows * cols;
                                const int y = div_by(r2, m_cols), x = r2 - y * cols;
                                const double v =
                                    __ldg(ub0 + f * FS + (long long)z * B * B + (long long)y * B + x);
                                diff |= bit_diff(v, __ldg(ub0 + f * FS)) != 0u;
                            }
                        }
                        diff = __syncthreads_or(diff);
                    }
                }
                ucol = !diff;
                if (ucol) {
                    T qh[6], v[3], p, c;
#pragma unroll
                    for (int f = 0; f < 6; f++)
                        qh[f] = Num<T>::from_d(__ldg(ub0 + f * FS));
                    prim_point(qh, gamma, gm1, ggm1, eps1, v, p, c, bad);
                    const T a = max_nonneg(max_nonneg(fabs(v[0]) + c, fabs(v[1]) + c), fabs(v[2]) + c);
                    amax = Num<T>::to_d(a);
                    const int per = E * ty * tx;
                    const unsigned m_per = rcp_div(per), m_tyx = rcp_div(ty * tx);
                    for (int q = tid; q < nf * per; q += NT) {
                        const int f = div_by(q, m_per), r = q - f * per;
                        const int z = div_by(r, m_tyx), r2 = r - z * ty * tx;
                        const int j = div_by(r2, m_tx), i = r2 - j * tx;
                        dUb[(long long)f * E * E * E + (long long)z * E * E + (long long)(y0 + j) * E + (x0 + i)] = -0.0;
                    }
                }
            }
        }
        if (!ucol) {
        if (funi != 0u) {
            // every stencil of such a field is constant, and PPM returns a
            // constant stencil's value unchanged: its point values are its one
            // value, in every group slot for the whole item (phase A writes only
            // the other fields' slots)
            for (int q = tid; q < 8 * nf * NC; q += NT) {
                const int sf = q / NC, f = sf - (sf / nf) * nf;
                if ((funi >> f) & 1u)
                    temp[q] = Num<T>::from_d(__ldg(Ub + f * FS));
            }
        }
        for (int kz = -3; kz <= 1; kz++)
            stage_plane(kz);
        __syncthreads();

        // the plane's cell primitives (FP64) are computed when the previous
        // plane met uniform data (and for the first plane of an item)
        bool cell_prev = true;
        for (int kz = -1; kz <= E; kz++) {
            const bool inplane = (kz >= 0 && kz < E);
            const bool cells_ready = cell_prev;
            bool plane_const = false;
            int so[5];  // staged-ring offsets of planes kz-2 .. kz+2
#pragma unroll
            for (int m = 0; m < 5; m++)
                so[m] = ((kz + m + 1) % 5) * nf * RWY * RWX;
            for (int g = 0; g < NGROUPS; g++) {
                const GroupTab &G = c_groups[g];
                if (!inplane && !G.has[2])
                    continue;
                const int nl = G.nl;
                // cells of each line's list: the x / y ring only for lines with
                // a nonzero x / y step, and only in planes that own x / y faces
                auto ltype = [&](int l) -> int {
                    return inplane ? ((G.line[l][0] != 0) | ((G.line[l][1] != 0) << 1)) : 0;
                };
                const int t0 = ltype(0), t1 = nl > 1 ? ltype(1) : 0, t2 = nl > 2 ? ltype(2) : 0,
                          t3 = nl > 3 ? ltype(3) : 0;
                const int n0 = nlist[t0], n1 = nl > 1 ? nlist[t1] : 0, n2 = nl > 2 ? nlist[t2] : 0,
                          n3 = nl > 3 ? nlist[t3] : 0;
                // ---- phase A: 1-D PPM for every (line, field, cell) of the group ----
                bool sawc = false;
                switch (g) {
#define OCT_PHASE_A(GG)                                                                                              \
    case GG:                                                                                                         \
        sawc = phase_a<T, STAGED, GG, NT>(temp, raw, Ub, FS, B, x0, y0, kz, inplane, nf, NC, RWX, RWY * RWX, lists,     \
                                          nlist, magic, so, tid, s_fmap, nfa);                                       \
        break;
                    OCT_PHASE_A(0)
                    OCT_PHASE_A(1)
                    OCT_PHASE_A(2)
                    OCT_PHASE_A(3)
#undef OCT_PHASE_A
                }
                if constexpr (SHARED_PRIMS && !PRIM) {
                    // primitives of the plane's cells themselves (interior and both
                    // rings), once per plane: a point that carries its cell's values
                    // takes them in phase B1 instead of computing its own.  A cell
                    // whose primitives are not physical gets c = -1 (no point takes
                    // them; its points are computed, and flagged, as usual)
                    if (g == 0 && cells_ready) {
                        const int t = inplane ? 3 : 0;
                        for (int q = tid; q < nlist[t]; q += NT) {
                            const int info = lists[t * NC + q];
                            const int i = (info & 0xFF) - 1, j = ((info >> 8) & 0xFF) - 1, ci = info >> 16;
                            const double *ub =
                                Ub + (long long)(kz + NG) * B * B + (long long)(y0 + j + NG) * B + (x0 + i + NG);
                            T qh[6], v[3], p, cs;
#pragma unroll
                            for (int f = 0; f < 6; f++)
                                qh[f] = __ldg(ub + f * FS);
                            bool cbad = false;
                            prim_point(qh, gamma, gm1, ggm1, eps1, v, p, cs, cbad);
                            cpr[ci] = v[0];
                            cpr[NC + ci] = v[1];
                            cpr[2 * NC + ci] = v[2];
                            cpr[3 * NC + ci] = p;
                            cpr[4 * NC + ci] = cbad ? T(-1) : cs;
                        }
                    }
                }
                if (sawc || funi != 0u)
                    s_const[g & 1] = 1;
                __syncthreads();
                const bool gconst = s_const[g & 1] != 0;
                plane_const = plane_const || gconst;
                if constexpr (SHARED_PRIMS) {
                // ---- phase B1: primitives of every needed point of the group:
                // both ends of interior cells (one end in the boundary planes),
                // the inward end of ring cells ----
                {
                    const int per_in = inplane ? 2 * ncin : ncin;
                    // points of each line; in the boundary planes only lines with a z step
                    auto mline = [&](int l, int nl_) -> int {
                        return (!inplane && G.line[l][2] == 0) ? 0 : per_in + (nl_ - ncin);
                    };
                    const int m0 = mline(0, n0), m1 = nl > 1 ? mline(1, n1) : 0, m2 = nl > 2 ? mline(2, n2) : 0,
                              m3 = nl > 3 ? mline(3, n3) : 0;
                    const int tot = m0 + m1 + m2 + m3;
                    for (int q = tid; q < tot; q += NT) {
                        int l = 0, r = q, t = t0;
                        if (r >= m0) {
                            r -= m0;
                            l = 1, t = t1;
                            if (r >= m1) {
                                r -= m1;
                                l = 2, t = t2;
                                if (r >= m2) {
                                    r -= m2;
                                    l = 3, t = t3;
                                }
                            }
                        }
                        const int lx = G.line[l][0], ly = G.line[l][1], lz = G.line[l][2];
                        int c, e;
                        if (r < per_in) {
                            if (inplane) {
                                c = r >> 1;
                                e = r & 1;
                            } else {
                                c = r;
                                // boundary planes: the end facing the interior (+z below, -z above)
                                e = ((kz < 0) == (lz > 0)) ? 1 : 0;
                            }
                        } else {
                            c = ncin + (r - per_in);
                        }
                        const int info = lists[t * NC + c];
                        const int i = (info & 0xFF) - 1, j = ((info >> 8) & 0xFF) - 1, ci = info >> 16;
                        if (r >= per_in) {
                            // ring cell: the end pointing into the tile
                            if (i < 0)
                                e = lx > 0 ? 1 : 0;
                            else if (i >= tx)
                                e = lx > 0 ? 0 : 1;
                            else if (j < 0)
                                e = ly > 0 ? 1 : 0;
                            else
                                e = ly > 0 ? 0 : 1;
                        }
                        const int slot = 2 * l + e;
                        T v[3], p, cs;
                        if constexpr (PRIM) {
                            // w -> conserved fields in place, v and p as reconstructed
                            T *q = temp + slot * nf * NC + ci;
                            const T rho = q[0];
                            v[0] = q[NC];
                            v[1] = q[2 * NC];
                            v[2] = q[3 * NC];
                            p = q[4 * NC];
                            cs = sound_from_w(rho, p, gamma, bad);
                            q[NC] = rho * v[0];
                            q[2 * NC] = rho * v[1];
                            q[3 * NC] = rho * v[2];
                            q[4 * NC] = fma(T(0.5) * rho, fma(v[2], v[2], fma(v[1], v[1], v[0] * v[0])), p * inv_gm1);
                            for (int f = F_SPC; f < nf; f++)
                                q[f * NC] = rho * q[f * NC];
                        } else {
                            T qh[6];
#pragma unroll
                            for (int f = 0; f < 6; f++)
                                qh[f] = temp[(slot * nf + f) * NC + ci];
                            // both ends of the line bitwise equal in every hydro field:
                            // then both carry the cell's own values (PPM leaves a value
                            // unchanged only by returning the cell value), and the
                            // point's primitives are the cell's
                            unsigned d = 1u;
                            if (gconst && cells_ready) {
                                d = 0u;
#pragma unroll
                                for (int f = 0; f < 6; f++)
                                    d |= bit_diff(qh[f], temp[((slot ^ 1) * nf + f) * NC + ci]);
                            }
                            if (d == 0u && __double2hiint(cpr[4 * NC + ci]) >= 0) {
                                v[0] = cpr[ci];
                                v[1] = cpr[NC + ci];
                                v[2] = cpr[2 * NC + ci];
                                p = cpr[3 * NC + ci];
                                cs = cpr[4 * NC + ci];
                            } else {
                                prim_point(qh, gamma, gm1, ggm1, eps1, v, p, cs, bad);
                            }
                        }
                        T *o = pr + slot * 5 * NC + ci;
                        o[0] = v[0];
                        o[NC] = v[1];
                        o[2 * NC] = v[2];
                        o[3 * NC] = p;
                        o[4 * NC] = cs;
                    }
                }
                __syncthreads();
                }
                // ---- phase B2: KT flux at the group's points, one thread per face;
                // the faces of the group's axes packed densely, each looping over
                // its axis's points of the group ----
                if (tid == 0)
                    s_const[(g + 1) & 1] = 0;  // for the next group (read before two barriers ago)
                {
                    const int nfx = (inplane && G.has[0]) ? (tx + 1) * ty : 0;
                    const int nfy = (inplane && G.has[1]) ? tx * (ty + 1) : 0;
                    const int nfz = G.has[2] ? ncin : 0;
                    int axis = 2, cl = 0, cr = 0, fslot = 0;
                    const bool act = tid < nfx + nfy + nfz;
                    if (tid < nfx) {
                        axis = 0;
                        int j = div_by(tid, m_tx1), p = tid - j * (tx + 1);
                        cl = cidx(p - 1, j, tx, ty);
                        cr = cidx(p, j, tx, ty);
                        fslot = tid;
                    } else if (tid < nfx + nfy) {
                        axis = 1;
                        int r = tid - nfx;
                        int p = div_by(r, m_tx), i = r - p * tx;
                        cl = cidx(i, p - 1, tx, ty);
                        cr = cidx(i, p, tx, ty);
                        fslot = r;
                    } else if (act) {
                        cl = cr = fslot = tid - nfx - nfy;
                    }
                    if (act && (axis < 2 || kz >= 0)) {
                        T acc[MAXNF];
#pragma unroll
                        for (int f = 0; f < MAXNF; f++)
                            acc[f] = T(0);
                        T pacc = T(0);
                        const int npa = axis == 0 ? G.nax[0] : (axis == 1 ? G.nax[1] : G.nax[2]);
                        for (int k = 0; k < npa; k++) {
                            const int pt = G.apt[axis][k];
                            // half the Simpson weight (16, 4 or 1)/36
                            // FP64: half the Simpson weight (16, 4 or 1)/36; FP32: 36 times
                            // that (8, 2 or 1/2, exact), the factor 1/36 applied in FP64
                            // after the face sum is promoted
                            const T hw = G.wcls[pt] == 0 ? T(8.0 * HWS) : (G.wcls[pt] == 1 ? T(2.0 * HWS) : T(0.5 * HWS));
                            const int ls = G.lslot[pt], rs = G.rslot[pt];
                            const T *qL, *pL_;
                            int sL;
                            if (ls >= 16) {
                                qL = saved + (ls - 16) * nf * C64 + cl;
                                pL_ = prs + (ls - 16) * 5 * C64 + cl;
                                sL = C64;
                            } else {
                                qL = temp + ls * nf * NC + cl;
                                pL_ = pr + ls * 5 * NC + cl;
                                sL = NC;
                            }
                            const T *qR = temp + rs * nf * NC + cr;
                            T vkL, pLv, cL, vkR, pRv, cR;
                            if constexpr (SHARED_PRIMS) {
                                const T *pR_ = pr + rs * 5 * NC + cr;
                                vkL = pL_[axis * sL], pLv = pL_[3 * sL], cL = pL_[4 * sL];
                                vkR = pR_[axis * NC], pRv = pR_[3 * NC], cR = pR_[4 * NC];
                            } else if constexpr (PRIM) {
                                // w on both sides: v and p as reconstructed
                                vkL = qL[(1 + axis) * sL];
                                pLv = qL[4 * sL];
                                cL = sound_from_w(qL[0], pLv, gamma, bad);
                                vkR = qR[(1 + axis) * NC];
                                pRv = qR[4 * NC];
                                cR = sound_from_w(qR[0], pRv, gamma, bad);
                            } else {
                                // primitives of both sides on the spot (cheap in FP32)
                                T qh[6], v[3];
#pragma unroll
                                for (int f = 0; f < 6; f++)
                                    qh[f] = qL[f * sL];
                                prim_point(qh, gamma, gm1, ggm1, eps1, v, pLv, cL, bad);
                                vkL = axis == 0 ? v[0] : (axis == 1 ? v[1] : v[2]);
#pragma unroll
                                for (int f = 0; f < 6; f++)
                                    qh[f] = qR[f * NC];
                                prim_point(qh, gamma, gm1, ggm1, eps1, v, pRv, cR, bad);
                                vkR = axis == 0 ? v[0] : (axis == 1 ? v[1] : v[2]);
                            }
                            const T a = max_nonneg(fabs(vkL) + cL, fabs(vkR) + cR);
                            amax = max_nonneg(amax, Num<T>::to_d(a));
                            // F_f = (F_f(L) + F_f(R))/2 - a (u_R - u_L)/2, plus the pressure
                            // terms of the normal momentum and the energy.  FP64: written per
                            // side, alpha u_L + beta u_R with alpha = (v_L + a)/2, beta =
                            // (v_R - a)/2 (two FMAs a field).  FP32: as alpha (u_L - u_R) +
                            // (alpha + beta) u_R, alpha + beta = (v_L + v_R)/2, whose rounding
                            // scales with the flux v u and the jump a (u_L - u_R) rather than
                            // with a u (a > |v| in subsonic flow, where the two per-side terms
                            // nearly cancel)
                            const T al = (vkL + a) * hw;
                            const T be = (vkR - a) * hw;
                            const T ab = (vkL + vkR) * hw;  // alpha + beta
                            auto kt = [&](T uL, T uR, T accf) -> T {
                                if constexpr (sizeof(T) == 8)
                                    return fma(al, uL, fma(be, uR, accf));
                                else
                                    return fma(al, uL - uR, fma(ab, uR, accf));
                            };
                            if constexpr (PRIM && !SHARED_PRIMS) {
                                // conserved fields of both sides from w, field by field
                                const T rL = qL[0], rR = qR[0];
                                const T vxL = qL[sL], vyL = qL[2 * sL], vzL = qL[3 * sL];
                                const T vxR = qR[NC], vyR = qR[2 * NC], vzR = qR[3 * NC];
#pragma unroll
                                for (int f = 0; f < MAXNF; f++)
                                    if (f < nf) {
                                        T uL, uR;
                                        if (f == F_RHO) {
                                            uL = rL, uR = rR;
                                        } else if (f == F_EGAS) {
                                            uL = fma(T(0.5) * rL, fma(vzL, vzL, fma(vyL, vyL, vxL * vxL)), pLv * inv_gm1);
                                            uR = fma(T(0.5) * rR, fma(vzR, vzR, fma(vyR, vyR, vxR * vxR)), pRv * inv_gm1);
                                        } else if (f == F_TAU) {
                                            uL = qL[f * sL], uR = qR[f * NC];
                                        } else {  // momenta and species: rho times v or X
                                            uL = rL * qL[f * sL], uR = rR * qR[f * NC];
                                        }
                                        acc[f] = kt(uL, uR, acc[f]);
                                    }
                            } else {
#pragma unroll
                                for (int f = 0; f < MAXNF; f++)
                                    if (f < nf)
                                        acc[f] = kt(qL[f * sL], qR[f * NC], acc[f]);
                            }
                            // pressure terms: the normal momentum's once per face (below),
                            // the energy's p v_k per point
                            if constexpr (sizeof(T) == 8)
                                pacc = fma(pLv + pRv, hw, pacc);
                            else
                                pacc = fma(pLv, hw, fma(pRv, hw, pacc));  // exact products (hw = 2^k)
                            acc[F_EGAS] = fma(fma(pLv, vkL, pRv * vkR), hw, acc[F_EGAS]);
                        }
#pragma unroll
                        for (int k = 0; k < 3; k++)
                            if (k == axis)
                                acc[F_SX + k] += pacc;
                        T *dst = axis == 0 ? faccx : (axis == 1 ? faccy : zacc + (kz & 1) * nf * C64);
                        const int stride = axis == 2 ? C64 : (axis == 0 ? FXS : FYS);
                        const bool first = g == (axis == 0 ? first_g[0] : (axis == 1 ? first_g[1] : first_g[2]));
#pragma unroll
                        for (int f = 0; f < MAXNF; f++)
                            if (f < nf) {
                                T *o = dst + f * stride + fslot;
                                *o = first ? acc[f] : *o + acc[f];
                            }
                    }
                    if (axis == 2 && act && kz < E) {
                        // leave this plane's +z ends (values and primitives) for the next plane
                        for (int z = 0; z < G.nzp; z++) {
                            const int src = G.zp_src[z], dsts = G.zp_dst[z];
                            for (int f = 0; f < nf; f++)
                                saved[(dsts * nf + f) * C64 + cl] = temp[(src * nf + f) * NC + cl];
                            if constexpr (SHARED_PRIMS) {
#pragma unroll
                                for (int v = 0; v < 5; v++)
                                    prs[(dsts * 5 + v) * C64 + cl] = pr[(src * 5 + v) * NC + cl];
                            }
                        }
                    }
                }
                if constexpr (STAGED) {
                    // phase A of the last line group (every group has lines with a z
                    // step, so it runs in every plane) was the last reader of plane
                    // kz-2 in the FP32 ring: plane kz+3 is staged into its slot now,
                    // while phase B2 occupies fewer than half the threads, and this
                    // barrier completes it before the next plane's phase A
                    if (g == NGROUPS - 1 && kz + 3 <= E + 2)
                        stage_plane(kz + 3);
                }
                __syncthreads();
            }
            // ---- plane end, one pass: the divergence of plane kz-1 (its upper z
            // face is done) and the in-plane part of plane kz's, by the same
            // thread for each (field, cell), so dxy is read before it is
            // rewritten ----
            for (int q = tid; q < nf * ncin; q += NT) {
                int f = div_by(q, magic[0]), c = q - f * ncin;
                int j = div_by(c, m_tx), i = c - j * tx;
                if (kz >= 1) {
                    const T *zp = zacc + (kz & 1) * nf * C64;
                    const T *zm = zacc + ((kz - 1) & 1) * nf * C64;
                    double dz = Num<T>::to_d(zp[f * C64 + c]) - Num<T>::to_d(zm[f * C64 + c]);
                    double d = -(dxy[f * C64 + c] + dz) * rdx;
                    dUb[(long long)f * E * E * E + (long long)(kz - 1) * E * E + (long long)(y0 + j) * E + (x0 + i)] = d;
                }
                if (inplane) {
                    const T *fx = faccx + f * FXS;
                    const T *fy = faccy + f * FYS;
                    double dX = Num<T>::to_d(fx[j * (tx + 1) + i + 1]) - Num<T>::to_d(fx[j * (tx + 1) + i]);
                    double dY = Num<T>::to_d(fy[(j + 1) * tx + i]) - Num<T>::to_d(fy[j * tx + i]);
                    dxy[f * C64 + c] = dX + dY;
                }
            }
            {
                double *fb;
                if (kz >= 1 && A.faces != nullptr && (kz == 1 || kz == E) && (fb = face_block()) != nullptr) {
                    // the subgrid's -z (below plane 0) or +z (above plane E-1) face
                    const T *zs = zacc + ((kz == 1 ? kz - 1 : kz) & 1) * nf * C64;
                    double *o = fb + (long long)(kz == 1 ? 4 : 5) * nf * E * E;
                    for (int q = tid; q < nf * ncin; q += NT) {
                        int f = div_by(q, magic[0]), c = q - f * ncin;
                        int j = div_by(c, m_tx), i = c - j * tx;
                        o[(long long)f * E * E + (y0 + j) * E + (x0 + i)] = Num<T>::to_d(zs[f * C64 + c]) * FSC;
                    }
                }
                if (inplane && A.faces != nullptr && (x0 == 0 || y0 == 0 || x0 + tx == E || y0 + ty == E) &&
                    (fb = face_block()) != nullptr) {
                    // x and y faces of plane kz on the subgrid's boundary
                    const long long EE = (long long)E * E;
                    if (x0 == 0 || x0 + tx == E)
                        for (int q = tid; q < nf * ty; q += NT) {
                            int f = div_by(q, m_ty), j = q - f * ty;
                            const T *fx = faccx + f * FXS + j * (tx + 1);
                            const long long o = f * EE + (long long)kz * E + (y0 + j);
                            if (x0 == 0)
                                fb[o] = Num<T>::to_d(fx[0]) * FSC;
                            if (x0 + tx == E)
                                fb[nf * EE + o] = Num<T>::to_d(fx[tx]) * FSC;
                        }
                    if (y0 == 0 || y0 + ty == E)
                        for (int q = tid; q < nf * tx; q += NT) {
                            int f = div_by(q, m_tx), i = q - f * tx;
                            const T *fy = faccy + f * FYS;
                            const long long o = f * EE + (long long)kz * E + (x0 + i);
                            if (y0 == 0)
                                fb[2 * nf * EE + o] = Num<T>::to_d(fy[i]) * FSC;
                            if (y0 + ty == E)
                                fb[3 * nf * EE + o] = Num<T>::to_d(fy[ty * tx + i]) * FSC;
                        }
                }
            }
            // nothing here is read by the next plane's phase A or phase B1, and
            // its phase B2 (which rewrites the face sums and the z-face slot read
            // above) comes after two more barriers
            cell_prev = plane_const;
        }
        }  // !ucol
        // ---- max signal speed of this item ----
        for (int o = 16; o > 0; o >>= 1)
            amax = fmax(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
        if ((tid & 31) == 0)
            red[tid >> 5] = amax;
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            for (int w = 0; w < NT / 32; w++)
                m = fmax(m, red[w]);
            const int slot = A.n_live != nullptr ? A.live_slot[k] : it;
            if (slot >= 0)
                A.amax_tile[slot] = m;
            else  // half of a static item: non-negative doubles order as their bits
                atomicMax(reinterpret_cast<unsigned long long *>(A.amax_tile + ~slot),
                          (unsigned long long)__double_as_longlong(m));
            s_next[par] = A.ticket != nullptr ? (int)gridDim.x + atomicAdd(A.ticket, 1) : k + (int)gridDim.x;
        }
        __syncthreads();
        k = s_next[par];
        par ^= 1;
    }
    if (A.ticket != nullptr && tid == 0) {
        // every CTA has drawn its last ticket before it counts itself done: the
        // last one to finish returns both counters to zero for the next launch
        __threadfence();
        if (atomicAdd(A.ticket + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(A.ticket, 0);
            atomicExch(A.ticket + 1, 0);
        }
    }
    if (bad)
        atomicOr(A.flags, 1u);
}

// Whole-subgrid uniform test ahead of the RHS kernel (conserved
// reconstruction, no boundary face fluxes wanted): when the ghosted block of
// subgrid s holds one value per field (bitwise), every work item of s would
// take the uniform-column path of rhs_kernel, so this kernel writes what that
// path writes -- RHS -0.0 for every cell, and a_max = max_k |v_k| + c of the
// state, from the same primitive function in the form's precision, for each
// of the subgrid's items -- and sets sub_uniform[s], which makes rhs_kernel
// skip those items.  One CTA per subgrid streams the block field by field
// (each field one contiguous run of B^3 doubles, read as double2), many CTAs
// per SM, leaving at the first field that differs.
constexpr int UNI_THREADS = 256;
// write_rhs = 0 (inside an RK3 step, whose combines take such subgrids
// whole and never read their RHS): a_max only.  only_unknown: the subgrids
// already marked uniform (by the test from a record) are left as they are.
template <class T>
__global__ void __launch_bounds__(UNI_THREADS) uniform_subgrid_kernel(RhsArgs A, const int *item_begin,
                                                                      int *sub_uniform, int write_rhs,
                                                                      int only_unknown)
{
    const int s = blockIdx.x, tid = threadIdx.x;
    if (only_unknown && sub_uniform[s] == 1)
        return;
    const int E = A.edge[s], B = E + 2 * NG;
    const int n2 = B * B * B / 2;  // B is even: whole double2 per field
    const double *Ub = A.U + A.off[s];
    const int nf = A.nf;
    // fields found to differ; with a per-field record wanted every field is
    // tested, else the test leaves at the first field that differs
    unsigned fdiff = 0u;
    for (int f = 0; f < nf && (fdiff == 0u || A.field_uni != nullptr); f++) {
        const double *fb = Ub + (long long)f * 2 * n2;
        const double2 *f2 = reinterpret_cast<const double2 *>(fb);
        const double ref = __ldg(fb);
        int diff = 0;
#pragma unroll 4
        for (int v = tid; v < n2; v += UNI_THREADS) {
            const double2 w = __ldg(f2 + v);
            diff |= (bit_diff(w.x, ref) | bit_diff(w.y, ref)) != 0u;
        }
        if (__syncthreads_or(diff))
            fdiff |= 1u << f;
    }
    if (fdiff != 0u) {
        if (tid == 0) {
            sub_uniform[s] = 0;
            if (A.field_uni != nullptr)
                A.field_uni[s] = ~fdiff & ((1u << nf) - 1u);
        }
        return;
    }
    const T gamma = Num<T>::from_d(A.gamma);
    const T gm1 = Num<T>::from_d(A.gamma - 1.0);
    const T ggm1 = Num<T>::from_d(A.gamma * (A.gamma - 1.0));
    const T eps1 = Num<T>::from_d(A.eps1);
    T qh[6], v[3], p, c;
#pragma unroll
    for (int f = 0; f < 6; f++)
        qh[f] = Num<T>::from_d(__ldg(Ub + (long long)f * 2 * n2));
    bool bad = false;
    prim_point(qh, gamma, gm1, ggm1, eps1, v, p, c, bad);
    const T a = max_nonneg(max_nonneg(fabs(v[0]) + c, fabs(v[1]) + c), fabs(v[2]) + c);
    const double amax = Num<T>::to_d(a);
    // the subgrid's RHS: nf E^3 doubles from doff[s] (an even count and offset)
    double2 *d2 = reinterpret_cast<double2 *>(A.dUdt + A.doff[s]);
    const int m2 = nf * E * E * E / 2;
    if (write_rhs)
        for (int q = tid; q < m2; q += UNI_THREADS)
            d2[q] = make_double2(-0.0, -0.0);
    for (int t = item_begin[s] + tid; t < item_begin[s + 1]; t += UNI_THREADS)
        A.amax_tile[t] = amax;
    if (tid == 0) {
        sub_uniform[s] = 1;
        if (bad)
            atomicOr(A.flags, 1u);
    }
}

// The work list of an RHS launch after the uniform test, on a batch of one
// edge: the static items of the subgrids not found uniform, in subgrid
// order, and -- as the static list does for its own last round -- when the
// last round of the persistent grid (G CTAs) would be at most half full,
// its r items cut in half along y (split: the static items are whole tiles
// of an even height of at least 4, so the halves are at least 2 high).  One CTA of LIVE_THREADS threads: each scans a contiguous run of
// subgrids, a block scan gives the positions.  Also zeroes the a_max slots
// that halves report to by atomic max.
constexpr int LIVE_THREADS = 1024;
static __global__ void __launch_bounds__(LIVE_THREADS)
    live_items_kernel(int n_sub, const int *sub_uniform, const int *item_begin, const WorkItem *items, int G,
                      int split, WorkItem *live, int *live_slot, int *n_live, double *amax_tile)
{
    __shared__ int wsum[LIVE_THREADS / 32];
    __shared__ int s_total;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int per = (n_sub + LIVE_THREADS - 1) / LIVE_THREADS;
    const int s0 = min(n_sub, tid * per), s1 = min(n_sub, s0 + per);
    int cnt = 0;
    for (int s = s0; s < s1; s++)
        if (!sub_uniform[s])
            cnt += item_begin[s + 1] - item_begin[s];
    // exclusive scan of cnt over the block
    int x = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o)
                v += y;
        }
        wsum[lane] = v;  // inclusive over warps
        if (lane == 31)
            s_total = v;
    }
    __syncthreads();
    int j = x - cnt + (w > 0 ? wsum[w - 1] : 0);  // first live item of this thread
    const int N = s_total;
    const int r = N % G;
    const int cut_from = (split && r > 0 && 2 * r <= G) ? N - r : N;
    for (int s = s0; s < s1; s++) {
        if (sub_uniform[s])
            continue;
        for (int i = item_begin[s]; i < item_begin[s + 1]; i++, j++) {
            const WorkItem it = items[i];
            if (j < cut_from) {
                live[j] = it;
                live_slot[j] = i;
            } else {
                const int ty = (it.txty >> 8) & 0xFF, tx = it.txty & 0xFF, h2 = ty / 2;
                const int p = cut_from + 2 * (j - cut_from);
                WorkItem a = it, b = it;
                a.txty = tx | (h2 << 8);
                b.y0 = it.y0 + h2;
                b.txty = tx | ((ty - h2) << 8);
                live[p] = a;
                live[p + 1] = b;
                live_slot[p] = ~i;
                live_slot[p + 1] = ~i;
                amax_tile[i] = 0.0;
            }
        }
    }
    if (tid == 0)
        n_live[0] = cut_from + 2 * (N - cut_from);
}

// Interior test of a state whose ghost cells are valid copies of interior
// cells (the state an RK3 step starts from, by the ABI's contract): per
// subgrid whether its interior holds one value per field (bitwise), and
// that value ([s * MAXNF + f]).  One warp per subgrid, no block barrier:
// each lane loads all fields of two cells at a time (22 loads in flight for
// 11 fields), the warp votes after each pair of cells.
constexpr int REC_THREADS = 256;
static __global__ void __launch_bounds__(REC_THREADS)
    interior_record_kernel(const double *U, const int *edge, const long long *off, int nf, int n_sub, int *rec_uni,
                           double *rec_val)
{
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (REC_THREADS / 32) + (threadIdx.x >> 5);
    if (s >= n_sub)
        return;
    const int E = edge[s], B = E + 2 * NG, E3 = E * E * E;
    const long long FS = (long long)B * B * B;
    const double *U0 = U + off[s] + ((long long)NG * B + NG) * B + NG;  // first interior cell
    const unsigned mE = rcp_div(E);
    double ref[MAXNF];
#pragma unroll
    for (int f = 0; f < MAXNF; f++)
        ref[f] = f < nf ? __ldg(U0 + f * FS) : 0.0;
    bool diff = false;
    for (int c0 = 0; c0 < E3 && !diff; c0 += 64) {
        unsigned d = 0;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int c = c0 + 32 * h + lane;
            if (c < E3) {
                const int zy = div_by(c, mE), z = div_by(zy, mE);
                const long long o = ((long long)z * B + (zy - z * E)) * B + (c - zy * E);
#pragma unroll
                for (int f = 0; f < MAXNF; f++)
                    if (f < nf)
                        d |= bit_diff(__ldg(U0 + f * FS + o), ref[f]);
            }
        }
        diff = __any_sync(0xFFFFFFFFu, d != 0u);
    }
    if (lane == 0)
        rec_uni[s] = !diff;
    if (!diff && lane < nf)
        rec_val[(long long)s * MAXNF + lane] = ref[lane];
}

// The whole-subgrid uniform test from a per-subgrid record of interiors (the
// interior test above, or the record the combines keep of the stage state),
// on a uniform level whose ghost cells are valid copies and all have a
// source: the ghosts of subgrid s copy cells of s itself or of its
// neighbours, so its ghosted block holds one value per field when s and
// every neighbour it has hold the same value (bitwise); a "no" is only
// conservative.  With item_begin (the first stage of a step, whose dt needs
// them), a_max of each uniform subgrid's items as the RHS kernel's uniform
// path would give it, in the form's precision.  One thread per subgrid.
template <class T>
__global__ void uniform_from_record_kernel(RhsArgs A, int n_sub, const int *nbr, const int *rec_uni,
                                           const double *rec_val, int *sub_uniform, const int *item_begin)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sub)
        return;
    const int nf = A.nf;
    int uni = rec_uni[s];
    for (int k = 0; k < 26 && uni; k++) {
        const int t = nbr[26 * (long long)s + k];
        if (t < 0)
            continue;
        uni = rec_uni[t];
        for (int f = 0; f < nf && uni; f++)
            uni = __double_as_longlong(rec_val[(long long)t * MAXNF + f]) ==
                  __double_as_longlong(rec_val[(long long)s * MAXNF + f]);
    }
    sub_uniform[s] = uni;
    if (!uni || item_begin == nullptr)
        return;
    const T gamma = Num<T>::from_d(A.gamma);
    const T gm1 = Num<T>::from_d(A.gamma - 1.0);
    const T ggm1 = Num<T>::from_d(A.gamma * (A.gamma - 1.0));
    const T eps1 = Num<T>::from_d(A.eps1);
    T qh[6], v[3], p, c;
#pragma unroll
    for (int f = 0; f < 6; f++)
        qh[f] = Num<T>::from_d(rec_val[(long long)s * MAXNF + f]);
    bool bad = false;
    prim_point(qh, gamma, gm1, ggm1, eps1, v, p, c, bad);
    const T a = max_nonneg(max_nonneg(fabs(v[0]) + c, fabs(v[1]) + c), fabs(v[2]) + c);
    const double amax = Num<T>::to_d(a);
    for (int t = item_begin[s]; t < item_begin[s + 1]; t++)
        A.amax_tile[t] = amax;
    if (bad)
        atomicOr(A.flags, 1u);
}

}  // namespace octh
