/*
 * lbve_oracle.h -- plain FP64 CPU reference of one time step of the coupled
 * lattice Boltzmann (LB) + Oldroyd-B method of Kuron, Stewart, de Graaf and
 * Holm, "An extensible lattice Boltzmann method for viscoelastic flows:
 * complex and moving boundaries in Oldroyd-B fluids" (arXiv:2009.12279).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library
 * against the paper.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Conventions (identical to the CUDA library's public interface, which is a
 * separate header; the two are kept in step by the parity tests):
 *   - grid nx*ny*nz, cell index x + nx*(y + ny*z), x fastest;
 *   - PDFs as 19 arrays of n cells, D3Q19 direction order
 *       0:(0,0,0) 1:(+x) 2:(-x) 3:(+y) 4:(-y) 5:(+z) 6:(-z)
 *       7:(+x+y) 8:(-x-y) 9:(+x-y) 10:(-x+y) 11:(+x+z) 12:(-x-z)
 *       13:(+x-z) 14:(-x+z) 15:(+y+z) 16:(-y-z) 17:(+y-z) 18:(-y+z);
 *   - stress as 6 arrays of n cells: xx, yy, zz, xy, xz, yz;
 *   - flags: 0 fluid, 1 no-slip wall, 2+k moving-wall class k (k < 16),
 *     64+p cells covered by particle p (p < 64).
 */
#ifndef LBVE_ORACLE_H
#define LBVE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_Q 19
#define ORC_FLUID 0
#define ORC_NOSLIP 1
#define ORC_WALL0 2
#define ORC_MAX_WALL 16
#define ORC_PART0 64
#define ORC_MAX_PART 64

/* fv_terms bits: which parts of the finite-volume stress update run. */
#define ORC_FV_FLUX 1   /* upwind advective flux (Stability improvements) */
#define ORC_FV_SOURCE 2 /* Eq. (source) */
#define ORC_FV_CTU 4    /* face fluxes scaled by the corner-transport-upwind transverse
                           overlap (1 - |u_a|)(1 - |u_b|) of the donor cell */
#define ORC_FV_DIVU 8   /* the tau_ij div(u) term of Eq. (source), which the paper sets to 0 */

typedef struct {
    int nx, ny, nz;
    int periodic[3];
    double eta;      /* total viscosity eta = eta_n + eta_p */
    double beta;     /* polymer fraction eta_p / eta */
    double lambda_p; /* polymer relaxation time (steps) */
    double rho0;     /* reference density */
    double g[3];     /* body-force density applied to every fluid cell */
    double magic;    /* TRT magic parameter, 3/16 in the paper */
    int n_wall;      /* number of moving-wall classes */
    double wall_vel[ORC_MAX_WALL][3];
    int fv_terms;    /* ORC_FV_* bits; ORC_FV_FLUX | ORC_FV_SOURCE for the method */
    double giesekus_alpha; /* Giesekus mobility in [0, 1/2]; 0 is Oldroyd-B (the method) */
    double fene_L2;  /* FENE-P maximum extensibility L^2 (> 3); 0 is Oldroyd-B (the method).
                        In FENE-P mode the stored tensor is the conformation A (see the
                        oracle's header); fields are read and written as stress tau */
} orc_params;

typedef struct orc_state orc_state;

/* Lifetime and state. Return 0 on success, negative on invalid input. */
orc_state *orc_create(const orc_params *p);
void orc_destroy(orc_state *s);
int orc_set_flags(orc_state *s, const uint8_t *flags);
int orc_init_fields(orc_state *s, const double *rho, const double *u, const double *tau);
int orc_add_particle(orc_state *s, const double X[3], double R, double rho_p, const double v[3],
                     const double w[3], const double Fext[3], const double Text[3]);
int orc_set_particle(orc_state *s, int id, const double X[3], const double v[3], const double w[3]);
void orc_step(orc_state *s, int nsteps);
long orc_time(const orc_state *s);

/* Read-back. u is the physical velocity (j + F/2)/rho with F = g + F^p(tau). */
void orc_read_fields(orc_state *s, double *rho, double *u, double *tau, uint8_t *flags);
void orc_read_pdfs(const orc_state *s, double *f);
void orc_write_pdfs(orc_state *s, const double *f);
void orc_write_tau(orc_state *s, const double *tau);
/* out[0..2] X, [3..5] v, [6..8] omega, [9..11] F, [12..14] T (momentum exchange of the
 * last step), [15..17] fill/drain impulse dP, [18..20] dL, [21] m, [22] I, [23] R. */
int orc_read_particle(const orc_state *s, int id, double out[24]);
/* Momentum-exchange force per flag value (256 x 3) from the last step. */
void orc_read_body_forces(const orc_state *s, double *out);
/* [0..5] stress dropped by fill/drain with no fluid neighbour, [6] cells destroyed,
 * [7] cells created (totals since creation). */
void orc_read_diag(const orc_state *s, double out[8]);
void orc_rates(const orc_state *s, double out[5]); /* omega+, omega-, eta_p, eta_p/lambda, 1/lambda */

/* Sub-steps, exposed so that tests can pin each against closed forms. */
void orc_lattice(int c[19][3], double w[19], int opp[19]);
void orc_equilibrium(double rho, const double u[3], double feq[19]);
void orc_forcing(const double u[3], const double F[3], double omega_p, double omega_m, double D[19]);
void orc_collide(const double f[19], const double F[3], double omega_p, double omega_m, double fs[19]);
void orc_source(const double tau[6], const double G[9], double ep_l, double inv_l, double S[6]);
/* FENE-P: stress of a conformation tensor, and the conformation of a stress. */
void orc_fene_stress(const double A[6], double eta_p, double lambda_p, double L2, double tau[6]);
void orc_fene_conformation(const double tau[6], double eta_p, double lambda_p, double L2, double A[6]);
void orc_polymer_force_field(orc_state *s, double *Fp);
void orc_velocity_field(orc_state *s, double *u);
void orc_fv_update_field(orc_state *s, const double *u, double *tau_out);
void orc_fill_drain(orc_state *s);

#ifdef __cplusplus
}
#endif
#endif
