/*
 * lbve2d.h -- C ABI of the two-dimensional form of the coupled lattice Boltzmann +
 * Oldroyd-B step (Kuron et al., arXiv:2009.12279), the lattices the paper uses for its
 * lid-driven cavity (Sec. "Lid-driven cavity") and four-roll mill (Sec. "Four-roll
 * mill"): a D2Q9 two-relaxation-time solvent with Guo forcing (Eqs. (lb),
 * (lb-equilibrium), (guo)) coupled through the polymer force (Eq. (force)) to a D2Q5
 * finite-volume update of the three-component stress xx, yy, xy (Eqs.
 * (continuity)-(source), Sec. "Stability improvements"), with link bounce-back from
 * walls moving at a prescribed per-cell velocity (Eq. (ubb)) and a per-cell body-force
 * field.  The readings of garbled passages are those of the three-dimensional library
 * (include/lbve.h).
 *
 * Layout: cell index x + nx * y (x fastest); vector fields are component-major (u[a * n
 * + r]), stress xx, yy, xy likewise.  Host buffers are caller-owned and copied on the
 * call.  Every call returns a status and never aborts.
 */
#ifndef LBVE2D_H
#define LBVE2D_H

#include "lbve.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbve2d_ctx lbve2d_ctx;

typedef struct {
    int nx, ny;
    int periodic[2];       /* non-periodic directions need solid first and last layers */
    double eta, beta;      /* total viscosity, polymer fraction eta_p / eta */
    double lambda_p, rho0; /* polymer relaxation time (steps), reference density */
    double body_force[2];  /* uniform force density, added to the per-cell field */
    double magic;          /* TRT magic product (3/16) */
    int pdf_prec;          /* LBVE_F64 (parity) or LBVE_F32 (shifted deviations f_i - w_i rho0) */
    int fv_terms;          /* LBVE_FV_FLUX | LBVE_FV_SOURCE bits; none set selects both */
} lbve2d_params;

/* Defaults: 32 x 32 periodic, eta 1/6, beta 0.5, lambda 1000, rho0 1, FP32. */
void lbve2d_default_params(lbve2d_params *p);

/* Create a solve on the current device, at rest with zero stress; stream may be NULL.
 * Errors: EINVAL (parameters), ENOMEM, ECUDA. */
lbve_status lbve2d_create(const lbve2d_params *p, void *cuda_stream, lbve2d_ctx **out);
lbve_status lbve2d_destroy(lbve2d_ctx *ctx);

/* Flag field (host, n bytes): 0 fluid, anything else solid.  ub (host, 2n doubles, NULL:
 * all zero) is the velocity u_b of each solid cell used in Eq. (ubb) for the links into
 * it and as the face value of the velocity gradient; a regularised lid is a row of solid
 * cells with ub_x = 16 u0 xi^2 (1 - xi)^2.  Errors: EINVAL (fluid cell in the outer
 * layer of a non-periodic direction). */
lbve_status lbve2d_set_geometry(lbve2d_ctx *ctx, const uint8_t *flags, const double *ub);

/* Per-cell body-force density (host, 2n doubles, e.g. the four-roll-mill forcing in the
 * lattice's components), added to params.body_force; NULL removes it. */
lbve_status lbve2d_set_force_field(lbve2d_ctx *ctx, const double *F);

/* Initial state: f = f^eq(rho, u) of Eq. (lb-equilibrium) (rho NULL: rho0; u NULL: 0),
 * stress tau (3n, NULL: 0).  Resets the step counter. */
lbve_status lbve2d_init_fields(lbve2d_ctx *ctx, const double *rho, const double *u, const double *tau);

/* Advance nsteps steps: polymer force and moments, finite-volume stress update, TRT
 * collision with forcing, push streaming with bounce-back.  Asynchronous. */
lbve_status lbve2d_step(lbve2d_ctx *ctx, int nsteps);

/* rho (n), the physical velocity (j + F/2)/rho (2n), tau (3n); 0 in solid cells (each may
 * be NULL).  Synchronises. */
lbve_status lbve2d_read_fields(lbve2d_ctx *ctx, double *rho, double *u, double *tau);

/* The 9 PDFs f_i (9n, direction-major; directions rest, +x, -x, +y, -y, (+,+), (-,-),
 * (+,-), (-,+)) as full populations.  Synchronises. */
lbve_status lbve2d_read_pdfs(lbve2d_ctx *ctx, double *f);

long long lbve2d_time(const lbve2d_ctx *ctx);
const char *lbve2d_last_error(const lbve2d_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
