/* A plain-C client of the library: the header compiles as C99 and the entry
 * points link from C. With a GPU it runs a small lattice through the C ABI and
 * prints the time, the total mass and momentum and the first entries of the
 * correlations, for comparison with the same run through the Python binding. */
#include <stdio.h>
#include <stdlib.h>

#include "flb.h"

static int check(int rc, const char* what) {
    if (rc != FLB_OK) {
        fprintf(stderr, "%s: %s (%d)\n", what, flb_error_string(rc), rc);
        exit(1);
    }
    return rc;
}

int main(void) {
    flb_params p = {0};
    p.Lx = 96;
    p.Ly = 40;
    p.rho0 = 1.0;
    p.ux0 = 0.1;
    p.uy0 = 0.0;
    p.kT = 1e-4;
    for (int a = 3; a < 9; ++a) p.omega[a] = a < 5 ? 1.1 : (a == 5 ? 0.8 : 1.3);
    p.basis = FLB_BASIS_LOCAL;
    p.precision = FLB_FP32;
    p.seed = 2024;
    p.replica = 0;

    flb_lattice h = NULL;
    check(flb_create(&p, NULL, 0, NULL, &h), "flb_create");
    check(flb_set_sampling(h, 10, 1), "flb_set_sampling");
    check(flb_step(h, 50), "flb_step");
    check(flb_sync(h), "flb_sync");
    int64_t t = 0, n = 0;
    double sums[3], Cff[81], CMM[81], mean[9];
    check(flb_time(h, &t), "flb_time");
    check(flb_conservation(h, sums), "flb_conservation");
    check(flb_correlations(h, FLB_BASIS_LOCAL, Cff, CMM, mean, &n), "flb_correlations");
    printf("%lld %lld %.17g %.17g %.17g %.17g %.17g\n", (long long)t, (long long)n, sums[0], sums[1],
           sums[2], Cff[0], CMM[3 * 9 + 3]);
    check(flb_destroy(h), "flb_destroy");
    return 0;
}
