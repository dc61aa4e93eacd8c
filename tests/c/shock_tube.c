/*
 * A shock tube through the C ABI alone (include/rlb.h), with no Python:
 * the weakly relativistic tube of Sec. III (800 cells, open ends, pressure
 * ratio 5.43/2.22 at T_left = 2, eta/s 0.1, dt/dx 0.25, 1600 steps).
 *
 * Without a CUDA device the host-side check passes and rlb_create reports
 * RLB_E_CUDA; the program then prints that status and exits 0.  With a
 * device it runs the steps and prints the plateau velocity and the
 * conserved totals.  Exit code 1 means a call failed in some other way.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "rlb.h"

#define NX 800

int main(void)
{
    const double pi = 3.14159265358979323846;
    const double n_right = 16.0 / (pi * pi);                 /* n_eq(T = 1) */
    const double p_left = 5.43 / 2.22 * n_right;             /* P = n T */
    rlb_grid grid = {NX, 1, 1, {RLB_BC_OUTFLOW, 0, 0}, {RLB_BC_OUTFLOW, 0, 0}, 1.0, 1.0, {0, 0, 0}};
    rlb_options opts;
    rlb_ctx *ctx = NULL;
    rlb_status st;
    static double n[NX], T[NX], ux[NX], uy[NX], uz[NX], out[6 * NX];
    double totals[5];
    int x;

    rlb_default_options(&opts);
    opts.dt_over_dx = 0.25;
    st = rlb_check_config(&grid, 19, 0.1, 0.0, RLB_LIMITER_MINMOD, &opts);
    if (st != RLB_OK) {
        fprintf(stderr, "check_config: %s\n", rlb_status_string(st));
        return 1;
    }
    st = rlb_create(&grid, 19, 0.1, 0.0, RLB_LIMITER_MINMOD, &opts, &ctx);
    if (st == RLB_E_CUDA) {
        printf("no CUDA device: %s\n", rlb_status_string(st));
        return 0;
    }
    if (st != RLB_OK) {
        fprintf(stderr, "create: %s\n", rlb_status_string(st));
        return 1;
    }
    for (x = 0; x < NX; ++x) {
        T[x] = x < NX / 2 ? 2.0 : 1.0;
        n[x] = x < NX / 2 ? p_left / 2.0 : n_right;
        ux[x] = uy[x] = uz[x] = 0.0;
    }
    if ((st = rlb_init(ctx, n, T, ux, uy, uz, 0)) != RLB_OK ||
        (st = rlb_step(ctx, 1600)) != RLB_OK ||
        (st = rlb_macroscopic(ctx, out, 0)) != RLB_OK ||
        (st = rlb_conserved_totals(ctx, totals)) != RLB_OK) {
        fprintf(stderr, "%s: %s\n", rlb_status_string(st), rlb_last_error(ctx));
        rlb_destroy(ctx);
        return 1;
    }
    printf("u_x at the membrane: %.4f\n", out[2 * NX + NX / 2]);
    printf("totals: %.9e %.9e %.9e\n", totals[0], totals[1], totals[4]);
    rlb_destroy(ctx);
    return 0;
}
