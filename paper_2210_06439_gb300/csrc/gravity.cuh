// gravity.cuh -- same-level monopole interactions of the gravity solver
// (Sec. II "Solvers": the FMM's most compute-intensive step is the
// same-level interaction between close-by cells; for non-refined cells it is
// the monopole kernel).  Every interior cell i of a subgrid receives, from
// each cell j of its level within r_s cell widths (0 < |d| <= r_s, d = j - i
// in cells), the potential and acceleration of a point mass
// m_j = rho_j dx^3 at the cell centre:
//     phi_i = -(G / dx)   sum_j m_j / |d|,
//     g_i   =  (G / dx^2) sum_j m_j d / |d|^3.
// A direct sum over a fixed stencil: the same offsets, 1/|d| and d/|d|^3 for
// every cell, built once on the host (z outermost, then y, then x, each
// ascending).
//
// GPU organisation: one CTA per subgrid.  The masses of the subgrid and of
// the R = floor(r_s) cells around it (from the neighbour subgrids' interiors,
// zero where a neighbour is missing) are staged into shared memory, S^3
// doubles with S = E + 2R, together with the stencil; each thread then sums
// the stencil for two target cells (eight independent FMA chains), the
// stencil entry warp-uniform (a broadcast) and the masses of neighbouring
// targets in consecutive shared-memory words.  Four FP64 FMAs per pair: the
// kernel is bound by the FP64 pipe.
#pragma once
#include "oct_common.cuh"

namespace octh {

// One stencil entry: the offset in the staged block (dz S^2 + dy S + dx) and
// 1/|d|, d_x/|d|^3, d_y/|d|^3, d_z/|d|^3.
struct GravEntry {
    double k0, kx, ky, kz;
};

__host__ __device__ inline size_t monopole_smem(int S, int n_st)
{
    return ((size_t)S * S * S * sizeof(double) + 31) / 32 * 32 + (size_t)n_st * sizeof(GravEntry) +
           (size_t)n_st * sizeof(int);
}

constexpr int MONO_THREADS = 256;

__global__ void __launch_bounds__(MONO_THREADS, 2)
    monopole_kernel(const double *U, const long long *off, int E, const int *nbr, int R, int n_st,
                    const int *st_off, const GravEntry *st_k, double dx3, double phi_scale, double g_scale,
                    double *phi, double *g)
{
    extern __shared__ __align__(16) unsigned char smem_g[];
    const int S = E + 2 * R;
    const int S3 = S * S * S;
    double *mass = reinterpret_cast<double *>(smem_g);
    GravEntry *K = reinterpret_cast<GravEntry *>(smem_g + ((size_t)S3 * sizeof(double) + 31) / 32 * 32);
    int *O = reinterpret_cast<int *>(K + n_st);
    const int s = blockIdx.x;
    const int B = E + 2 * NG;
    const unsigned m_S = rcp_div(S);
    // masses of the subgrid and its halo of R cells
    for (int q = threadIdx.x; q < S3; q += blockDim.x) {
        const int zy = div_by(q, m_S), z = div_by(zy, m_S);
        int c[3] = {q - zy * S - R, zy - z * S - R, z - R};
        int o[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            o[a] = c[a] < 0 ? -1 : (c[a] >= E ? 1 : 0);
            c[a] -= o[a] * E;
        }
        int src = s;
        if (o[0] | o[1] | o[2]) {
            int n = (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1);
            src = nbr[26 * (long long)s + (n > 13 ? n - 1 : n)];
        }
        double m = 0.0;
        if (src >= 0)
            m = __ldg(U + off[src] + ((long long)(c[2] + NG) * B + (c[1] + NG)) * B + (c[0] + NG)) * dx3;
        mass[q] = m;
    }
    for (int q = threadIdx.x; q < n_st; q += blockDim.x) {
        K[q] = st_k[q];
        O[q] = st_off[q];
    }
    __syncthreads();
    const int E3 = E * E * E;
    const unsigned m_E = rcp_div(E);
    // two targets per thread per pass: t and t + blockDim.x
    for (int t0 = threadIdx.x; t0 < E3; t0 += 2 * blockDim.x) {
        const int t1 = t0 + blockDim.x;
        const bool has1 = t1 < E3;
        auto base = [&](int t) {
            const int zy = div_by(t, m_E), z = div_by(zy, m_E);
            return ((z + R) * S + (zy - z * E + R)) * S + (t - zy * E + R);
        };
        const int b0 = base(t0), b1 = has1 ? base(t1) : b0;
        double p0 = 0.0, x0 = 0.0, y0 = 0.0, z0 = 0.0, p1 = 0.0, x1 = 0.0, y1 = 0.0, z1 = 0.0;
#pragma unroll 4
        for (int e = 0; e < n_st; e++) {
            const int o = O[e];
            const GravEntry k = K[e];
            const double m0 = mass[b0 + o], m1 = mass[b1 + o];
            p0 = fma(m0, k.k0, p0);
            x0 = fma(m0, k.kx, x0);
            y0 = fma(m0, k.ky, y0);
            z0 = fma(m0, k.kz, z0);
            p1 = fma(m1, k.k0, p1);
            x1 = fma(m1, k.kx, x1);
            y1 = fma(m1, k.ky, y1);
            z1 = fma(m1, k.kz, z1);
        }
        const long long o0 = (long long)s * E3;
        phi[o0 + t0] = phi_scale * p0;
        g[3 * o0 + t0] = g_scale * x0;
        g[3 * o0 + E3 + t0] = g_scale * y0;
        g[3 * o0 + 2 * E3 + t0] = g_scale * z0;
        if (has1) {
            phi[o0 + t1] = phi_scale * p1;
            g[3 * o0 + t1] = g_scale * x1;
            g[3 * o0 + E3 + t1] = g_scale * y1;
            g[3 * o0 + 2 * E3 + t1] = g_scale * z1;
        }
    }
}

}  // namespace octh
