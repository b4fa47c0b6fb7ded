/* A plain C client of the library: a colloid between two homeotropic walls,
 * random start, FIRE to a force tolerance, energy and order parameter out.
 * Built and run by the tests (it uses nothing but include/lqmin.h). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lqmin.h"

#define CHECK(call)                                                              \
    do {                                                                         \
        lq_status st_ = (call);                                                  \
        if (st_ != LQ_OK && st_ != LQ_ENOTCONVERGED) {                           \
            fprintf(stderr, "%s failed (%d): %s\n", #call, (int)st_,             \
                    s ? lq_last_error(s) : lq_create_error());                  \
            return 1;                                                            \
        }                                                                        \
    } while (0)

int main(void) {
    lq_solver *s = NULL;
    lq_lattice lat = {32, 32, 24, 1.0, {1, 1, 1}};
    lq_material mat = {0};
    mat.A = -0.172; mat.B = -2.12; mat.C = 1.73;
    mat.L1 = 2.32; mat.L2 = 0.5; mat.L3 = 0.3;
    mat.n_constants = 3;
    CHECK(lq_create(&lat, &mat, LQ_FP64, NULL, &s));
    lq_anchoring hom = {LQ_ANCHOR_ND_HOMEOTROPIC, 5.3, {0.0, 0.0, 1.0}};
    const double c[3] = {16.0, 16.0, 12.0};
    CHECK(lq_add_wall(s, 2, 0, &hom));
    CHECK(lq_add_wall(s, 2, 23, &hom));
    CHECK(lq_add_sphere(s, c, 5.0, &hom));
    CHECK(lq_init_random_uniaxial(s, 7, 0.0));
    lq_fire_params p = {0};
    p.dt0 = 1e-3; p.dt_max = 1e-2; p.alpha0 = 0.99; p.f_alpha = 0.99;
    p.f_inc = 1.1; p.f_dec = 0.5; p.n_min = 5; p.max_iter = 200000; p.force_tol = 1e-6;
    lq_result r;
    CHECK(lq_minimize(s, &p, &r));
    double total, parts[3];
    CHECK(lq_energy(s, &total, parts));
    int64_t nsim = 0, nrec = 0;
    CHECK(lq_geometry_info(s, &nsim, &nrec));
    size_t n = (size_t)lat.nx * lat.ny * lat.nz;
    double *S = (double *)malloc(n * sizeof(double));
    if (!S) return 1;
    CHECK(lq_order_field(s, S));
    double smin = 1.0;
    for (size_t i = 0; i < n; ++i)
        if (S[i] > 0.0 && S[i] < smin) smin = S[i];
    printf("status %d iterations %lld max_force %.3e energy %.17g parts %.6e %.6e %.6e "
           "simulated %lld anchored %lld minS %.4f\n",
           r.fire_status, (long long)r.iterations, r.max_force, total, parts[0], parts[1],
           parts[2], (long long)nsim, (long long)nrec, smin);
    free(S);
    lq_destroy(s);
    return r.fire_status == LQ_FIRE_CONVERGED && fabs(total - r.energy) <= 1e-9 * fabs(total) ? 0 : 2;
}
