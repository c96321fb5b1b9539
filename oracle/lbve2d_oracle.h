/*
 * lbve2d_oracle.h -- plain FP64 CPU reference of the two-dimensional form of the coupled
 * LB + Oldroyd-B step (D2Q9 lattice Boltzmann solvent, D2Q5 finite-volume stress) of
 * Kuron et al., arXiv:2009.12279, used by the paper for its lid-driven cavity and
 * four-roll mill.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests to check the CUDA library; never by the
 * product path, and it shares no code with it.
 */
#ifndef LBVE2D_ORACLE_H
#define LBVE2D_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC2_FV_FLUX 1
#define ORC2_FV_SOURCE 2

typedef struct {
    int nx, ny;
    int periodic[2];
    double eta, beta, lambda_p, rho0;
    double g[2];     /* uniform body-force density */
    double magic;    /* TRT magic parameter (3/16) */
    int fv_terms;    /* ORC2_FV_* bits */
} orc2_params;

typedef struct orc2_state orc2_state;

orc2_state *orc2_create(const orc2_params *p);
void orc2_destroy(orc2_state *s);
/* flags: 0 fluid, any other value solid; ub (2n, may be NULL) the velocity of each solid
 * cell for Eq. (ubb) (x fastest; components interleaved per field: ub[a * n + r]). */
int orc2_set_flags(orc2_state *s, const uint8_t *flags, const double *ub);
/* Per-cell body-force density added to g (2n, NULL clears it). */
void orc2_set_force(orc2_state *s, const double *F);
int orc2_init_fields(orc2_state *s, const double *rho, const double *u, const double *tau);
void orc2_step(orc2_state *s, int nsteps);
long orc2_time(const orc2_state *s);
/* rho (n), u (2n, the physical (j + F/2)/rho), tau (3n: xx, yy, xy); 0 in solid cells. */
void orc2_read_fields(orc2_state *s, double *rho, double *u, double *tau);
void orc2_read_pdfs(const orc2_state *s, double *f);
void orc2_write_pdfs(orc2_state *s, const double *f);
void orc2_write_tau(orc2_state *s, const double *tau);
void orc2_lattice(int c[9][2], double w[9], int opp[9]);
/* One finite-volume update of the stress from the given velocity field (pins). */
void orc2_fv_update_field(orc2_state *s, const double *u, double *tau_out);

#ifdef __cplusplus
}
#endif
#endif
