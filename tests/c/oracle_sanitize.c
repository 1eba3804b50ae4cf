/* Drives the oracle's C entry points on small random grids (odd sizes,
 * periodic, zero-gradient and tiny axes) for the sanitizer test
 * (tests/test_oracle_sanitize.py): built with -fsanitize=address,undefined
 * together with oracle/vof_oracle.c, it must run without a report. */
#include <stdio.h>
#include <stdlib.h>

void orc_step_scheme(const int dims[3], const int bc[3], const double par[5], double *c, double *e,
                     const double *u, const double *v, const double *w, double dt, long step_index,
                     const double *dd, double dd_uniform, double *sums, int scheme);
void orc_mass_transfer(const int dims[3], const int bc[3], const double par[5], const double *c, const double *e,
                       const double mpar[3], double *mdot, double *d_gamma, double *grad_n);
void orc_reconstruct(const int dims[3], const int bc[3], const double par[5], const double *c, double *m_soa,
                     double *alpha, unsigned char *mixed);

static double rnd(unsigned long long *s) {
    *s = *s * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(*s >> 11) / 9007199254740992.0;
}

int main(void) {
    const int shapes[][3] = {{7, 5, 3}, {1, 4, 6}, {2, 2, 2}, {9, 1, 1}};
    const int bcs[][3] = {{0, 0, 0}, {1, 1, 1}, {0, 1, 0}, {1, 0, 1}};
    unsigned long long seed = 12345;
    for (int si = 0; si < 4; ++si)
        for (int bi = 0; bi < 4; ++bi) {
            const int *dims = shapes[si], *bc = bcs[bi];
            long N = (long)dims[0] * dims[1] * dims[2];
            double par[5] = {0.1, 3.0, 1.0, 1.0, 1e-12};
            double *c = malloc(sizeof(double) * N), *e = malloc(sizeof(double) * N);
            double *dd = malloc(sizeof(double) * N);
            double *u = malloc(sizeof(double) * dims[2] * dims[1] * (dims[0] + 1));
            double *v = malloc(sizeof(double) * dims[2] * (dims[1] + 1) * dims[0]);
            double *w = malloc(sizeof(double) * (dims[2] + 1) * dims[1] * dims[0]);
            for (long i = 0; i < N; ++i) {
                double r = rnd(&seed);
                c[i] = r < 0.3 ? 0.0 : (r > 0.7 ? 1.0 : rnd(&seed));
                e[i] = (3.0 * c[i] + (1.0 - c[i])) * (1.0 + rnd(&seed));
                dd[i] = 0.02 * (rnd(&seed) - 0.5);
            }
            for (long i = 0; i < (long)dims[2] * dims[1] * (dims[0] + 1); ++i) u[i] = 0.4 * (rnd(&seed) - 0.5);
            for (long i = 0; i < (long)dims[2] * (dims[1] + 1) * dims[0]; ++i) v[i] = 0.4 * (rnd(&seed) - 0.5);
            for (long i = 0; i < (long)(dims[2] + 1) * dims[1] * dims[0]; ++i) w[i] = 0.4 * (rnd(&seed) - 0.5);
            double sums[6];
            for (int scheme = 0; scheme < 2; ++scheme)
                for (long s = 0; s < 2; ++s)
                    orc_step_scheme(dims, bc, par, c, e, u, v, w, 0.1, s, s ? dd : NULL, -0.01, sums, scheme);
            double mpar[3] = {0.5, 0.05, 10.0};
            double *mdot = malloc(sizeof(double) * N), *dg = malloc(sizeof(double) * N);
            double *gn = malloc(sizeof(double) * N), *m = malloc(sizeof(double) * 3 * N), *al = malloc(sizeof(double) * N);
            unsigned char *mx = malloc(N);
            orc_mass_transfer(dims, bc, par, c, e, mpar, mdot, dg, gn);
            orc_reconstruct(dims, bc, par, c, m, al, mx);
            free(c); free(e); free(dd); free(u); free(v); free(w);
            free(mdot); free(dg); free(gn); free(m); free(al); free(mx);
        }
    printf("sanitize driver ok\n");
    return 0;
}
