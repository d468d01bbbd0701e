/* A lattice driven through the C ABI alone (no Python): a 64 x 48 clustered
 * lid-driven cavity, 500 steps, then the moments and the FP64 mass.  Prints
 * "sum_u1 sum_u2 mass max_rho" with 17 significant digits; exit status 0 on
 * success, 1 with the library's message on any error. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "goc.h"

#define CHECK(call)                                                              \
    do {                                                                         \
        goc_status s_ = (call);                                                  \
        if (s_ != GOC_OK) {                                                      \
            fprintf(stderr, "%s: status %d: %s\n", #call, (int)s_, goc_last_error()); \
            return 1;                                                            \
        }                                                                        \
    } while (0)

int main(void) {
    goc_grid g;
    memset(&g, 0, sizeof g);
    g.nx = 64;
    g.ny = 48;
    for (int s = 0; s < 4; s++) g.bc[s] = GOC_BC_WALL;
    g.wall_u[3] = 0.01;   /* the N lid, along xi1 */
    goc_map m;
    memset(&m, 0, sizeof m);
    m.kind[0] = m.kind[1] = GOC_MAP_TANH2;
    m.beta[0] = 1.2;
    m.beta[1] = 1.4;
    goc_flow f;
    memset(&f, 0, sizeof f);
    f.rho0 = 1.0;
    f.nu = 0.02;
    f.gi_correction = 1;
    goc_lattice *lat = NULL;
    CHECK(goc_create(&g, &m, &f, NULL, NULL, &lat));
    CHECK(goc_step(lat, 500));
    CHECK(goc_sync(lat));
    const size_t n = (size_t)g.nx * g.ny;
    double *rho = malloc(n * sizeof *rho), *u1 = malloc(n * sizeof *u1), *u2 = malloc(n * sizeof *u2);
    if (!rho || !u1 || !u2) return 1;
    CHECK(goc_moments(lat, 0, rho, u1, u2, NULL, NULL));
    double mass = 0.0, su = 0.0, sv = 0.0, rmax = 0.0;
    CHECK(goc_diagnostics(lat, &mass, NULL, NULL));
    for (size_t k = 0; k < n; k++) {
        su += u1[k];
        sv += u2[k];
        if (rho[k] > rmax) rmax = rho[k];
    }
    printf("%.17g %.17g %.17g %.17g\n", su, sv, mass, rmax);
    free(rho);
    free(u1);
    free(u2);
    goc_destroy(lat);
    return 0;
}
