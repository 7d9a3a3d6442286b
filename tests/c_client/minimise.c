/* A plain C client of the library (no Python): a 16 nm cube of Nd2Fe14B with
 * two instances (different applied fields) minimised in mixed precision, then
 * the energies read back.  Build: gcc -std=c99 -I include minimise.c -llbm.
 * Run it on a GPU; it prints one line per instance and returns 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm.h"

#define CHECK(call)                                                        \
    do {                                                                   \
        int rc_ = (call);                                                  \
        if (rc_ != LBM_OK) {                                               \
            fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, lbm_last_error()); \
            return 1;                                                      \
        }                                                                  \
    } while (0)

int main(void) {
    const int n = 8, batch = 2;
    lbm_ctx* ctx = NULL;
    CHECK(lbm_create(&ctx, 0, NULL));
    lbm_mesh mesh;
    CHECK(lbm_mesh_cube(ctx, 2e-9, n, &mesh));
    int64_t info[8];
    CHECK(lbm_mesh_info(ctx, mesh, info));
    const int64_t N = info[0];
    lbm_inst inst;
    CHECK(lbm_instance_create(ctx, mesh, batch, LBM_MIXED, &inst));
    lbm_material mats[2];
    for (int b = 0; b < batch; ++b) {
        mats[b].Js = 1.61;
        mats[b].A = 7.7e-12;
        mats[b].K1 = 4.3e6;
        mats[b].axis[0] = sin(0.02 * (b + 1));
        mats[b].axis[1] = 0.0;
        mats[b].axis[2] = cos(0.02 * (b + 1));
    }
    CHECK(lbm_set_material(ctx, inst, mats));
    const double h[6] = {0.0, 0.0, -1.0, 0.0, 0.0, -4.0};   /* tesla */
    CHECK(lbm_set_field(ctx, inst, h));
    double* m = (double*)malloc(sizeof(double) * batch * N * 3);
    if (!m) return 1;
    for (int64_t i = 0; i < batch * N; ++i) {
        m[3 * i] = 0.01;
        m[3 * i + 1] = 0.0;
        m[3 * i + 2] = 0.99995;
    }
    CHECK(lbm_set_m(ctx, inst, m));
    lbm_solve_opts opt;
    lbm_default_opts(&opt, LBM_MIXED);
    lbm_result res[2];
    CHECK(lbm_minimise(ctx, inst, &opt, res));
    double e[10];
    CHECK(lbm_energy(ctx, inst, e));
    int ok = 1;
    for (int b = 0; b < batch; ++b) {
        printf("instance %d: status %d, %d iterations, torque %.3e, energy %.6e J (lbm_energy %.6e J)\n", b,
               res[b].status, res[b].iterations, res[b].torque, res[b].energy[4], e[5 * b + 4]);
        ok &= res[b].status == LBM_OK && res[b].torque < opt.tol;
    }
    free(m);
    CHECK(lbm_instance_destroy(ctx, inst));
    CHECK(lbm_mesh_destroy(ctx, mesh));
    CHECK(lbm_destroy(ctx));
    return ok ? 0 : 2;
}
