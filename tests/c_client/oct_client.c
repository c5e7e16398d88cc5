/* A plain C client of the C ABI (no Python, no PyTorch): a uniform moving
 * state on a periodic 2x2x2 tiling gives an exactly zero RHS and the
 * closed-form CFL step dt = cfl * dx / (max |v| + c), and an RK3 step keeps it.
 * Exit status 0 on success; prints the failing check otherwise. */
#include <cuda_runtime_api.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "oct_hydro.h"

#define CHECK(cond, what)                                      \
    do {                                                       \
        if (!(cond)) {                                         \
            fprintf(stderr, "FAILED: %s (%s)\n", what, oct_hydro_last_error()); \
            return 1;                                          \
        }                                                      \
    } while (0)

int main(void)
{
    const int E = 8, B = E + 6, NS = 2, NF = 6 + NS, N = 8;
    const double gamma = 5.0 / 3.0, rho = 1.3, p = 0.9, vx = 0.7, vy = -0.4, vz = 0.25;
    oct_hydro_t h = NULL;
    CHECK(oct_hydro_create(N, E, 3, NS, gamma, &h) == OCT_OK, "create");
    /* periodic 2x2x2 tiling: neighbour (dx,dy,dz) of subgrid (sx,sy,sz) */
    int32_t nbr[26 * 8];
    for (int s = 0; s < N; s++) {
        int sx = s % 2, sy = (s / 2) % 2, sz = s / 4, k = 0;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    if (!dx && !dy && !dz)
                        continue;
                    int tx = (sx + dx + 2) % 2, ty = (sy + dy + 2) % 2, tz = (sz + dz + 2) % 2;
                    nbr[26 * s + k++] = (tz * 2 + ty) * 2 + tx;
                }
    }
    double dx[8];
    for (int s = 0; s < N; s++)
        dx[s] = 1.0 / 16.0;
    CHECK(oct_hydro_set_layout(h, NULL, NULL, dx, NULL, nbr, OCT_BC_PERIODIC) == OCT_OK, "set_layout");
    CHECK(oct_hydro_set_params(h, OCT_FP64, 0.4, 1e-12, 1e-3, 0.1) == OCT_OK, "set_params");
    const int64_t n = oct_hydro_state_len(h), nr = oct_hydro_rhs_len(h);
    CHECK(n >= (int64_t)N * NF * B * B * B && nr == (int64_t)N * NF * E * E * E, "lengths");
    /* the uniform state, ghosts included, in the packed layout */
    const double e = p / (gamma - 1.0);
    const double q[8] = {rho, rho * vx, rho * vy, rho * vz, e + 0.5 * rho * (vx * vx + vy * vy + vz * vz),
                         pow(e, 1.0 / gamma), 0.5 * rho, 0.5 * rho};
    double *U = (double *)calloc((size_t)n, sizeof(double));
    const int64_t blk = ((int64_t)NF * B * B * B + 3) / 4 * 4;
    for (int s = 0; s < N; s++)
        for (int f = 0; f < NF; f++)
            for (int c = 0; c < B * B * B; c++)
                U[s * blk + (int64_t)f * B * B * B + c] = q[f];
    double *dU = NULL, *dR = NULL;
    CHECK(cudaMalloc((void **)&dU, sizeof(double) * n) == cudaSuccess, "cudaMalloc U");
    CHECK(cudaMalloc((void **)&dR, sizeof(double) * nr) == cudaSuccess, "cudaMalloc dUdt");
    CHECK(cudaMemcpy(dU, U, sizeof(double) * n, cudaMemcpyHostToDevice) == cudaSuccess, "copy in");
    CHECK(oct_hydro_rhs(h, dU, dR, NULL, NULL) == OCT_OK, "rhs");
    double *R = (double *)malloc(sizeof(double) * nr);
    CHECK(cudaMemcpy(R, dR, sizeof(double) * nr, cudaMemcpyDeviceToHost) == cudaSuccess, "copy out");
    for (int64_t i = 0; i < nr; i++)
        CHECK(R[i] == 0.0, "uniform state gives an exactly zero RHS");
    double dt = 0.0;
    CHECK(oct_hydro_max_dt(h, dU, &dt, NULL) == OCT_OK, "max_dt");
    const double c = sqrt(gamma * p / rho), want = 0.4 * (1.0 / 16.0) / (fabs(vx) + c);
    CHECK(fabs(dt - want) <= 1e-14 * want, "closed-form dt");
    double dt_step = 0.0;
    CHECK(oct_hydro_rk_step(h, dU, &dt_step, NULL) == OCT_OK, "rk_step");
    CHECK(dt_step == dt, "step uses the CFL dt");
    uint32_t flags = 1;
    CHECK(oct_hydro_get_error_flags(h, &flags) == OCT_OK && flags == 0, "no device flags");
    /* a bad call is a status, not a crash */
    CHECK(oct_hydro_rhs(h, dU, dU, NULL, NULL) == OCT_E_ARG, "overlap rejected");
    oct_hydro_destroy(h);
    cudaFree(dU);
    cudaFree(dR);
    free(U);
    free(R);
    printf("c client ok: dt = %.17g\n", dt);
    return 0;
}
