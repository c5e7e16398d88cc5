// rhs_kernel.cuh -- fused hydro right-hand side on sm_103a (one template,
// instantiated for FP64 and for the mixed form).
//
// Method (Octo-Tiger hydro solver, arXiv 2210.06439 Sec. II "Solvers"):
// PPM reconstruction of every conserved field to the 26 points of each cell
// (6 face centres, 12 edge midpoints, 8 corners; the value at x + d/2 comes
// from 1-D PPM along the cells x + m d), the Kurganov-Tadmor flux at the 9
// Newton-Cotes (tensor Simpson) points of every face with a local speed per
// point, the face average, and the finite-volume divergence.
//
// GPU organisation.  A CTA owns one work item: a tx * ty column of a subgrid
// (tx, ty <= 8) and streams through its z planes kz = -1 .. E.  For each plane
// the 13 lines are processed in 7 groups (x, y, z, xy, xz, yz, body
// diagonals); within a group both sides of each face quadrature point are
// available, so the flux of that point is formed as soon as the group's point
// values exist and no plane ever holds all 26 points of all fields:
//   phase A  every (line, cell, field) of the group: 1-D PPM -> both ends
//            into the group buffer (shared memory);
//   phase B  one thread per face: the group's quadrature points of that face,
//            primitives on both sides, KT flux, Simpson-weighted sum into the
//            face accumulator; the z faces below the plane take their L side
//            from the +z ends the previous plane left in the saved buffer, and
//            the same thread then replaces those with this plane's +z ends.
// After the 7 groups the in-plane (x, y) face fluxes are complete; the
// divergence of a plane is finished one plane later, once its upper z face
// is known.  The signal speed max over all face points is reduced per item.
#pragma once
#include "oct_common.cuh"

namespace octh {

// line-group tables, filled by the host at handle creation
__constant__ GroupTab c_groups[NGROUPS];

template <class T> struct Num;
template <> struct Num<double> {
    __device__ static __forceinline__ double from_d(double x) { return x; }
    __device__ static __forceinline__ double to_d(double x) { return x; }
    __device__ static __forceinline__ double sqrt_(double x) { return sqrt(x); }
    __device__ static __forceinline__ double pow_(double x, double y) { return pow(x, y); }
};
template <> struct Num<float> {
    __device__ static __forceinline__ float from_d(double x) { return d2f_rn(x); }
    __device__ static __forceinline__ double to_d(float x) { return f2d(x); }
    __device__ static __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    __device__ static __forceinline__ float pow_(float x, float y) { return powf(x, y); }
};

// Monotonised-central slope: minmod of the centred and twice the one-sided
// differences, zero unless all three share a strict sign.
template <class T>
__device__ __forceinline__ T mc_slope(T um, T u0, T up)
{
    T c = T(0.5) * (up - um);
    T l = T(2) * (u0 - um);
    T r = T(2) * (up - u0);
    T mag = fmin(fabs(c), fmin(fabs(l), fabs(r)));
    bool pos = (c > T(0)) && (l > T(0)) && (r > T(0));
    bool neg = (c < T(0)) && (l < T(0)) && (r < T(0));
    return pos ? mag : (neg ? -mag : T(0));
}

// CW84 PPM on u_{-2..2}: limited values at the cell's two ends.
template <class T>
__device__ __forceinline__ void ppm5(T um2, T um1, T u0, T up1, T up2, T &vm, T &vp)
{
    T dm = mc_slope(um2, um1, u0);
    T d0 = mc_slope(um1, u0, up1);
    T dp = mc_slope(u0, up1, up2);
    T up = T(0.5) * (u0 + up1) - (dp - d0) * T(1.0 / 6.0);
    T um = T(0.5) * (um1 + u0) - (d0 - dm) * T(1.0 / 6.0);
    T a = up - u0, b = u0 - um;
    if (a * b <= T(0)) {
        um = u0;
        up = u0;
    } else {
        T du = up - um;
        T m6 = du * (u0 - T(0.5) * (up + um));
        T dd = du * du * T(1.0 / 6.0);
        if (m6 > dd)
            um = T(3) * u0 - T(2) * up;
        else if (-dd > m6)
            up = T(3) * u0 - T(2) * um;
    }
    vm = um;
    vp = up;
}

// Shared-memory plan of one CTA (dynamic shared memory), sizes for the
// largest tile (8 x 8) and nf fields.
struct SmemPlan {
    int nc;          // cells per plane buffer row: 64 interior + 32 ring
    size_t temp, saved, faccx, faccy, zacc, dxy, raw, red, total;
};

__host__ __device__ inline SmemPlan smem_plan(int nf, int elem, bool staged)
{
    SmemPlan p;
    p.nc = MAXT * MAXT + 4 * MAXT;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o += (bytes + 15) / 16 * 16; return at; };
    p.temp = take((size_t)8 * nf * p.nc * elem);
    p.saved = take((size_t)9 * nf * MAXT * MAXT * elem);
    p.faccx = take((size_t)nf * (MAXT + 1) * MAXT * elem);
    p.faccy = take((size_t)nf * (MAXT + 1) * MAXT * elem);
    p.zacc = take((size_t)2 * nf * MAXT * MAXT * elem);
    p.dxy = take((size_t)nf * MAXT * MAXT * sizeof(double));
    p.raw = staged ? take((size_t)5 * nf * (MAXT + 2 * NG) * (MAXT + 2 * NG) * sizeof(float)) : 0;
    p.red = take(64 * sizeof(double));
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

// Point primitives and flux at one quadrature point.  qL, qR: point values of
// the nf fields on both sides; k: face normal; w: Simpson weight.  Adds
// w * F_KT to acc and returns the local signal speed a.
template <class T>
__device__ __forceinline__ T kt_point(int k, int nf, const T *qL, const T *qR, T w, T gamma, T eps1, T *acc,
                                      bool &bad)
{
    T vL[3], vR[3], pL, pR, cL, cR;
    {
        T rho = qL[F_RHO], ir = T(1) / rho;
        vL[0] = qL[F_SX] * ir;
        vL[1] = qL[F_SY] * ir;
        vL[2] = qL[F_SZ] * ir;
        T ek = T(0.5) * (qL[F_SX] * vL[0] + qL[F_SY] * vL[1] + qL[F_SZ] * vL[2]);
        T ei = qL[F_EGAS] - ek;
        if (ei < eps1 * qL[F_EGAS])
            ei = Num<T>::pow_(qL[F_TAU], gamma);
        pL = (gamma - T(1)) * ei;
        cL = Num<T>::sqrt_(gamma * pL * ir);
        bad |= !(rho > T(0)) || !(cL == cL);
    }
    {
        T rho = qR[F_RHO], ir = T(1) / rho;
        vR[0] = qR[F_SX] * ir;
        vR[1] = qR[F_SY] * ir;
        vR[2] = qR[F_SZ] * ir;
        T ek = T(0.5) * (qR[F_SX] * vR[0] + qR[F_SY] * vR[1] + qR[F_SZ] * vR[2]);
        T ei = qR[F_EGAS] - ek;
        if (ei < eps1 * qR[F_EGAS])
            ei = Num<T>::pow_(qR[F_TAU], gamma);
        pR = (gamma - T(1)) * ei;
        cR = Num<T>::sqrt_(gamma * pR * ir);
        bad |= !(rho > T(0)) || !(cR == cR);
    }
    const T vkL = k == 0 ? vL[0] : (k == 1 ? vL[1] : vL[2]);
    const T vkR = k == 0 ? vR[0] : (k == 1 ? vR[1] : vR[2]);
    T a = fmax(fabs(vkL) + cL, fabs(vkR) + cR);
    // F_f = (F_f(L) + F_f(R))/2 - a (u_R - u_L)/2, written per side:
    // alpha u_L + beta u_R with alpha = (v_L + a)/2, beta = (v_R - a)/2,
    // plus the pressure terms of the normal momentum and the energy.
    T al = T(0.5) * (vkL + a) * w;
    T be = T(0.5) * (vkR - a) * w;
    const T pm = T(0.5) * w * (pL + pR);
    const T pe = T(0.5) * w * (pL * vkL + pR * vkR);
#pragma unroll
    for (int f = 0; f < MAXNF; f++)
        if (f < nf) {
            T add = al * qL[f] + be * qR[f];
            if (f == F_SX + k)
                add += pm;
            if (f == F_EGAS)
                add += pe;
            acc[f] += add;
        }
    return a;
}

template <class T, bool STAGED>
__global__ void __launch_bounds__(NTHREADS, 1) rhs_kernel(RhsArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nf = A.nf;
    const SmemPlan P = smem_plan(nf, sizeof(T), STAGED);
    const int NC = P.nc;
    T *temp = reinterpret_cast<T *>(smem + P.temp);    // [8 slots][nf][NC]
    T *saved = reinterpret_cast<T *>(smem + P.saved);  // [9][nf][64]
    T *faccx = reinterpret_cast<T *>(smem + P.faccx);  // [nf][72]
    T *faccy = reinterpret_cast<T *>(smem + P.faccy);  // [nf][72]
    T *zacc = reinterpret_cast<T *>(smem + P.zacc);    // [2][nf][64]
    double *dxy = reinterpret_cast<double *>(smem + P.dxy);  // [nf][64]
    float *raw = reinterpret_cast<float *>(smem + P.raw);    // [5][nf][14][14]
    double *red = reinterpret_cast<double *>(smem + P.red);
    const int tid = threadIdx.x;
    const T gamma = Num<T>::from_d(A.gamma);
    const T eps1 = Num<T>::from_d(A.eps1);
    const int RW = MAXT + 2 * NG;  // staged row width
    bool bad = false;

    for (int it = blockIdx.x; it < A.n_items; it += gridDim.x) {
        const WorkItem W = A.items[it];
        const int s = W.s, x0 = W.x0, y0 = W.y0, tx = W.txty & 0xFF, ty = (W.txty >> 8) & 0xFF;
        const int E = A.edge[s], B = E + 2 * NG;
        const long long FS = (long long)B * B * B;
        const double *Ub = A.U + A.off[s];
        double *dUb = A.dUdt + A.doff[s];
        const double rdx = 1.0 / A.dx[s];
        const int ncin = tx * ty;
        double amax = 0.0;

        // raw field value at tile-relative (i, j) of plane kz (interior coords)
        auto rawv = [&](int f, int kz, int j, int i) -> T {
            if constexpr (STAGED) {
                int slot = (kz + 3 + 10) % 5;
                return (T)raw[((slot * nf + f) * RW + (j + NG)) * RW + (i + NG)];
            } else {
                return Num<T>::from_d(__ldg(Ub + f * FS + (long long)(kz + NG) * B * B + (long long)(y0 + j + NG) * B +
                                            (x0 + i + NG)));
            }
        };
        auto stage_plane = [&](int kz) {
            if constexpr (STAGED) {
                int slot = (kz + 3 + 10) % 5;
                int rows = ty + 2 * NG, cols = tx + 2 * NG;
                int n = nf * rows * cols;
                for (int q = tid; q < n; q += NTHREADS) {
                    int f = q / (rows * cols), r = q % (rows * cols);
                    int jj = r / cols, ii = r % cols;
                    double v = __ldg(Ub + f * FS + (long long)(kz + NG) * B * B + (long long)(y0 + jj) * B + (x0 + ii));
                    raw[((slot * nf + f) * RW + jj) * RW + ii] = d2f_rn(v);
                }
            }
        };

        // zero accumulators
        for (int q = tid; q < nf * (MAXT + 1) * MAXT; q += NTHREADS) {
            faccx[q] = T(0);
            faccy[q] = T(0);
        }
        for (int q = tid; q < 2 * nf * MAXT * MAXT; q += NTHREADS)
            zacc[q] = T(0);
        for (int kz = -3; kz <= 1; kz++)
            stage_plane(kz);
        __syncthreads();

        for (int kz = -1; kz <= E; kz++) {
            const bool inplane = (kz >= 0 && kz < E);
            for (int g = 0; g < NGROUPS; g++) {
                const GroupTab &G = c_groups[g];
                if (!inplane && !G.has[2])
                    continue;
                // ---- phase A: 1-D PPM for every (line, field, cell) ----
                int ncl[4], tot = 0;
                for (int l = 0; l < G.nl; l++) {
                    int n = ncin;
                    if (inplane) {
                        if (G.line[l][0]) n += 2 * ty;
                        if (G.line[l][1]) n += 2 * tx;
                    }
                    ncl[l] = n;
                    tot += nf * n;
                }
                for (int q = tid; q < tot; q += NTHREADS) {
                    int r = q, l = 0;
                    while (r >= nf * ncl[l]) {
                        r -= nf * ncl[l];
                        l++;
                    }
                    int f = r / ncl[l], c = r % ncl[l];
                    const int ddx = G.line[l][0], ddy = G.line[l][1], ddz = G.line[l][2];
                    int i, j;
                    if (c < ncin) {
                        i = c % tx;
                        j = c / tx;
                    } else {
                        c -= ncin;
                        if (ddx && c < 2 * ty) {
                            i = (c < ty) ? -1 : tx;
                            j = c % ty;
                        } else {
                            if (ddx) c -= 2 * ty;
                            j = (c < tx) ? -1 : ty;
                            i = c % tx;
                        }
                    }
                    T u[5];
#pragma unroll
                    for (int m = -2; m <= 2; m++)
                        u[m + 2] = rawv(f, kz + m * ddz, j + m * ddy, i + m * ddx);
                    T vm, vp;
                    ppm5(u[0], u[1], u[2], u[3], u[4], vm, vp);
                    int ci = cidx(i, j, tx, ty);
                    temp[((2 * l + 0) * nf + f) * NC + ci] = vm;
                    temp[((2 * l + 1) * nf + f) * NC + ci] = vp;
                }
                __syncthreads();
                // ---- phase B: one thread per face ----
                const int nfx = (inplane && G.has[0]) ? (tx + 1) * ty : 0;
                const int nfy = (inplane && G.has[1]) ? tx * (ty + 1) : 0;
                const int nfz = G.has[2] ? ncin : 0;
                for (int q = tid; q < nfx + nfy + nfz; q += NTHREADS) {
                    T acc[MAXNF];
#pragma unroll
                    for (int f = 0; f < MAXNF; f++)
                        acc[f] = T(0);
                    T qL[MAXNF], qR[MAXNF];
                    int axis, cl, cr, fslot;
                    if (q < nfx) {
                        axis = 0;
                        int p = q % (tx + 1), j = q / (tx + 1);
                        cl = cidx(p - 1, j, tx, ty);
                        cr = cidx(p, j, tx, ty);
                        fslot = q;
                    } else if (q < nfx + nfy) {
                        axis = 1;
                        int r = q - nfx;
                        int i = r % tx, p = r / tx;
                        cl = cidx(i, p - 1, tx, ty);
                        cr = cidx(i, p, tx, ty);
                        fslot = r;
                    } else {
                        axis = 2;
                        cl = cr = fslot = q - nfx - nfy;
                    }
                    if (axis < 2 || kz >= 0) {
                        for (int pt = 0; pt < G.npt; pt++) {
                            if (G.axis[pt] != axis)
                                continue;
                            const T w = G.wcls[pt] == 0 ? T(16.0 / 36.0) : (G.wcls[pt] == 1 ? T(4.0 / 36.0) : T(1.0 / 36.0));
                            int ls = G.lslot[pt], rs = G.rslot[pt];
#pragma unroll
                            for (int f = 0; f < MAXNF; f++) {
                                if (f < nf) {
                                    qL[f] = (ls >= 16) ? saved[((ls - 16) * nf + f) * (MAXT * MAXT) + cl]
                                                       : temp[(ls * nf + f) * NC + cl];
                                    qR[f] = temp[(rs * nf + f) * NC + cr];
                                }
                            }
                            T a = kt_point<T>(axis, nf, qL, qR, w, gamma, eps1, acc, bad);
                            amax = fmax(amax, (double)Num<T>::to_d(a));
                        }
                        T *dst = axis == 0 ? faccx : (axis == 1 ? faccy : zacc + (kz & 1) * nf * MAXT * MAXT);
                        const int stride = axis == 2 ? MAXT * MAXT : (MAXT + 1) * MAXT;
#pragma unroll
                        for (int f = 0; f < MAXNF; f++)
                            if (f < nf)
                                dst[f * stride + fslot] += acc[f];
                    }
                    if (axis == 2 && kz < E) {
                        // leave this plane's +z ends for the z faces of the next plane
                        for (int z = 0; z < G.nzp; z++)
                            for (int f = 0; f < nf; f++)
                                saved[(G.zp_dst[z] * nf + f) * (MAXT * MAXT) + cl] =
                                    temp[(G.zp_src[z] * nf + f) * NC + cl];
                    }
                }
                __syncthreads();
            }
            // ---- finish the divergence of plane kz-1 (its upper z face is done) ----
            if (kz >= 1) {
                const T *zp = zacc + (kz & 1) * nf * MAXT * MAXT;
                const T *zm = zacc + ((kz - 1) & 1) * nf * MAXT * MAXT;
                for (int q = tid; q < nf * ncin; q += NTHREADS) {
                    int f = q / ncin, c = q % ncin;
                    int i = c % tx, j = c / tx;
                    double dz = Num<T>::to_d(zp[f * MAXT * MAXT + c]) - Num<T>::to_d(zm[f * MAXT * MAXT + c]);
                    double d = -(dxy[f * MAXT * MAXT + c] + dz) * rdx;
                    dUb[(long long)f * E * E * E + (long long)(kz - 1) * E * E + (long long)(y0 + j) * E + (x0 + i)] = d;
                }
            }
            __syncthreads();
            if (kz >= 1) {
                T *zm = zacc + ((kz - 1) & 1) * nf * MAXT * MAXT;
                for (int q = tid; q < nf * MAXT * MAXT; q += NTHREADS)
                    zm[q] = T(0);
            }
            if (inplane) {
                for (int q = tid; q < nf * ncin; q += NTHREADS) {
                    int f = q / ncin, c = q % ncin;
                    int i = c % tx, j = c / tx;
                    const T *fx = faccx + f * (MAXT + 1) * MAXT;
                    const T *fy = faccy + f * (MAXT + 1) * MAXT;
                    double dX = Num<T>::to_d(fx[j * (tx + 1) + i + 1]) - Num<T>::to_d(fx[j * (tx + 1) + i]);
                    double dY = Num<T>::to_d(fy[(j + 1) * tx + i]) - Num<T>::to_d(fy[j * tx + i]);
                    dxy[f * MAXT * MAXT + c] = dX + dY;
                }
            }
            __syncthreads();
            if (inplane)
                for (int q = tid; q < nf * (MAXT + 1) * MAXT; q += NTHREADS) {
                    faccx[q] = T(0);
                    faccy[q] = T(0);
                }
            if (kz + 3 <= E + 2)
                stage_plane(kz + 3);
            __syncthreads();
        }
        // ---- max signal speed of this item ----
        for (int o = 16; o > 0; o >>= 1)
            amax = fmax(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
        if ((tid & 31) == 0)
            red[tid >> 5] = amax;
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            for (int w = 0; w < NTHREADS / 32; w++)
                m = fmax(m, red[w]);
            A.amax_tile[it] = m;
        }
        __syncthreads();
    }
    if (bad)
        atomicOr(A.flags, 1u);
}

}  // namespace octh
