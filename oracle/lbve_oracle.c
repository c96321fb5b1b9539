/*
 * lbve_oracle.c -- plain FP64 CPU reference of the coupled LB + Oldroyd-B step of
 * Kuron et al., arXiv:2009.12279.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the package smoke check and the
 * benchmark's CPU baseline; never by the CUDA product path, and it shares no code
 * with it.  Slow on purpose: two PDF arrays with push streaming, one loop per
 * sub-step, every formula written as the paper states it (or, where the paper is
 * garbled or silent, as the reading recorded beside the formula).
 *
 * One time step t -> t+1, in this order:
 *   1. polymer force F^p from tau^t                      Eq. (force), Eq. (extrapolation)
 *   2. rho, u = (j + F/2)/rho with F = g + F^p           Eq. (macroscopic-velocity)
 *   3. finite-volume stress update tau^t -> tau^{t+1}     Eqs. (continuity)-(source),
 *      with donor-cell (upwind) face fluxes and zero      Sec. "Stability improvements",
 *      flux across solid links                            Sec. "Discretization"
 *   4. TRT collision with Guo forcing                     Eq. (lb), Eq. (guo)
 *   5. push streaming with link bounce-back (moving       Eq. (lb), Eq. (ubb)
 *      walls and particles) and momentum exchange         Sec. "Moving boundaries"
 *   6. particle update, symplectic Euler                  Sec. "Moving boundaries"
 *   7. re-voxelisation and fill/drain with stress         Sec. "Moving boundaries"
 *      redistribution
 *
 * Readings of passages that are garbled or silent (all also listed in the design
 * notes of the repository):
 *   - Eq. (lb-equilibrium) prints 1/6 for the quadratic coefficients; the standard
 *     second-order form w rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2) is used (it is the
 *     only one with the moments the LB viscosity relation assumes).
 *   - lambda_+ / lambda_- in Eq. (lb) are rates; omega+ = 1/(3 nu_n + 1/2) and the
 *     magic relation (1/omega+ - 1/2)(1/omega- - 1/2) = 3/16.
 *   - Eq. (guo) is taken as Guo forcing split for TRT, F a force density:
 *     D_i = w_i [3 (1 - omega-/2) c.F + 9/2 (1 - omega+/2) (uF + Fu):(cc - I/3)].
 *   - Upwind flux: donor cell on the D3Q7 faces, max(+-u_k,0) tau of the upwind cell,
 *     no transverse overlap factors (they are O(u^2) like the dropped edge fluxes).
 *     Variant ORC_FV_CTU keeps them: the donor cell displaced by its velocity overlaps
 *     the face neighbour along k by |u_k| (1 - |u_a|)(1 - |u_b|) (a, b the other two
 *     axes), the corner-transport-upwind overlap restricted to the D3Q7 faces; the edge
 *     and corner overlaps stay in the donor cell.
 *   - The tau div(u) source term is dropped, as the paper marks it zero (variant
 *     ORC_FV_DIVU adds it, with div(u) the trace of the central-point gradient).
 *   - Giesekus (named among the constitutive laws of Sec. "Oldroyd-B fluids", no
 *     equation printed): the textbook law tau + lambda tau_(1) + (alpha lambda / eta_p)
 *     tau.tau = eta_p (grad u + grad u^T) adds -(alpha / eta_p) tau.tau to the source of
 *     Eq. (source); alpha = 0 is Oldroyd-B.
 *   - FENE-P (named beside Giesekus among the laws of Sec. "Oldroyd-B fluids" and Sec.
 *     "Implementation and extensibility", no equation printed): the textbook Peterlin
 *     closure written for the conformation tensor A, which is what the finite-volume
 *     update then transports (the paper's scheme carries "stress or conformation"):
 *         A_(1) = -(1/lambda) (f A - I),   tau = (eta_p / lambda) (f A - I),
 *         f = 1 / (1 - tr A / L^2),
 *     so the source of Eq. (source) becomes A.grad u + (A.grad u)^T - (f A - I)/lambda
 *     (no eta_p/lambda (grad u + grad u^T) term), the flux moves A, and the polymer force
 *     of Eq. (force) takes the stress of each cell's A.  L^2 -> infinity recovers
 *     Oldroyd-B with tau = (eta_p/lambda)(A - I).  Stress given or read at the boundary
 *     of the solver converts by A = (I + lambda tau / eta_p) / f, f = 1 + (3 + lambda
 *     tr tau / eta_p) / L^2 (the closed-form inverse).  Moving particles are not
 *     combined with FENE-P.
 *   - grad u next to a solid cell uses the boundary velocity as the face value.
 *   - Stress extrapolation is per link: the face value towards a solid cell is tau(r).
 *   - Momentum exchange on a link r -> r+c_i (solid): c_i (2 f*_i - 6 w_i rho c_i.u_b),
 *     lever arm r_b - X with r_b the solid cell centre.
 *   - Fill/drain: N_f counts D3Q7 neighbours that are fluid before and after the
 *     re-voxelisation; all stress moves are computed from the pre-fill/drain stress;
 *     a created cell gets rho = mean density of such D3Q19 neighbours (rho0 if none);
 *     the impulse on the particle is the momentum of the deleted / created PDFs,
 *     applied at the converted cell centre (force and its torque).
 */
#include "lbve_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* D3Q19 velocity set and weights, Sec. "Lattice Boltzmann".                  */
/* ------------------------------------------------------------------------- */
static const int C[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const int OPP[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
static const double W0 = 1.0 / 3.0, W1 = 1.0 / 18.0, W2 = 1.0 / 36.0;
static double W[19];

/* D3Q7 finite-volume neighbour set (faces +x,-x,+y,-y,+z,-z), Sec. "Discretization". */
static const int FACE_AXIS[6] = {0, 0, 1, 1, 2, 2};
static const double FACE_SIGN[6] = {1.0, -1.0, 1.0, -1.0, 1.0, -1.0};

/* symmetric-tensor component layout xx,yy,zz,xy,xz,yz */
static const int COMP[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
static const int CI[6] = {0, 1, 2, 0, 0, 1};
static const int CJ[6] = {0, 1, 2, 1, 2, 2};

static void init_weights(void) {
    W[0] = W0;
    for (int i = 1; i < 7; ++i) W[i] = W1;
    for (int i = 7; i < 19; ++i) W[i] = W2;
}

typedef struct {
    double X[3], v[3], w[3];
    double R, rho_p, m, I;
    double Fext[3], Text[3];
    double Fme[3], Tme[3];
    double dP[3], dL[3];
} orc_particle;

struct orc_state {
    orc_params p;
    long n;
    double omega_p, omega_m, eta_p, ep_l, inv_l;
    double gk; /* alpha / eta_p of the Giesekus term (0: Oldroyd-B) */
    int fene;  /* FENE-P: the stored tensor is the conformation A */
    double *f, *fn;     /* [19][n] */
    double *tau, *taun; /* [6][n] */
    double *rho, *u, *F; /* per-step scratch: [n], [3][n], [3][n] */
    uint8_t *flag;
    int np;
    orc_particle part[ORC_MAX_PART];
    double body_F[256][3];
    double dropped[6];
    long n_destroyed, n_created;
    long t;
};

/* ------------------------------------------------------------------------- */
/* geometry helpers                                                          */
/* ------------------------------------------------------------------------- */
static long cell_index(const orc_state *s, int x, int y, int z) {
    return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * (long)z);
}

static void cell_coords(const orc_state *s, long r, int *x, int *y, int *z) {
    *x = (int)(r % s->p.nx);
    *y = (int)((r / s->p.nx) % s->p.ny);
    *z = (int)(r / ((long)s->p.nx * s->p.ny));
}

/* Neighbour r + d with periodic wrap; -1 if it leaves a non-periodic side. */
static long neighbour(const orc_state *s, long r, int dx, int dy, int dz) {
    int x, y, z;
    cell_coords(s, r, &x, &y, &z);
    int q[3] = {x + dx, y + dy, z + dz};
    int nn[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int a = 0; a < 3; ++a) {
        if (q[a] < 0 || q[a] >= nn[a]) {
            if (!s->p.periodic[a]) return -1;
            q[a] = (q[a] + nn[a]) % nn[a];
        }
    }
    return cell_index(s, q[0], q[1], q[2]);
}

static int is_fluid(const orc_state *s, long r) { return r >= 0 && s->flag[r] == ORC_FLUID; }

static int is_particle_flag(uint8_t fl) { return fl >= ORC_PART0 && fl < ORC_PART0 + ORC_MAX_PART; }

/* minimum-image displacement of cell r from point X */
static void displacement(const orc_state *s, long r, const double X[3], double d[3]) {
    int x, y, z;
    cell_coords(s, r, &x, &y, &z);
    double q[3] = {(double)x, (double)y, (double)z};
    int nn[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int a = 0; a < 3; ++a) {
        d[a] = q[a] - X[a];
        if (s->p.periodic[a]) d[a] -= nn[a] * floor(d[a] / nn[a] + 0.5);
    }
}

/* Boundary velocity of solid cell r: Eq. (ubb) wall velocity or Eq. (surface-velocity). */
static void boundary_velocity(const orc_state *s, long r, double ub[3]) {
    ub[0] = ub[1] = ub[2] = 0.0;
    if (r < 0) return;
    uint8_t fl = s->flag[r];
    if (fl >= ORC_WALL0 && fl < ORC_WALL0 + ORC_MAX_WALL) {
        int k = fl - ORC_WALL0;
        if (k < s->p.n_wall) {
            ub[0] = s->p.wall_vel[k][0];
            ub[1] = s->p.wall_vel[k][1];
            ub[2] = s->p.wall_vel[k][2];
        }
    } else if (is_particle_flag(fl)) {
        const orc_particle *P = &s->part[fl - ORC_PART0];
        double d[3];
        displacement(s, r, P->X, d);
        ub[0] = P->v[0] + (P->w[1] * d[2] - P->w[2] * d[1]);
        ub[1] = P->v[1] + (P->w[2] * d[0] - P->w[0] * d[2]);
        ub[2] = P->v[2] + (P->w[0] * d[1] - P->w[1] * d[0]);
    }
}

/* ------------------------------------------------------------------------- */
/* per-cell formulas                                                          */
/* ------------------------------------------------------------------------- */
void orc_lattice(int c[19][3], double w[19], int opp[19]) {
    init_weights();
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[i][a] = C[i][a];
        w[i] = W[i];
        opp[i] = OPP[i];
    }
}

/* Eq. (lb-equilibrium), second-order form (reading of the garbled coefficients). */
void orc_equilibrium(double rho, const double u[3], double feq[19]) {
    init_weights();
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        feq[i] = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Eq. (guo) with G = (1 - omega+/2)(uF + Fu), first-order term weighted (1 - omega-/2). */
void orc_forcing(const double u[3], const double F[3], double omega_p, double omega_m, double D[19]) {
    init_weights();
    double A = 3.0 * (1.0 - 0.5 * omega_m);
    double B = 1.0 - 0.5 * omega_p;
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    for (int i = 0; i < 19; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        double cF = C[i][0] * F[0] + C[i][1] * F[1] + C[i][2] * F[2];
        D[i] = W[i] * (A * cF + B * (9.0 * cu * cF - 3.0 * uF));
    }
}

/* Eq. (macroscopic-velocity): rho = sum f, u = (j + F/2)/rho. */
static void moments(const double f[19], const double F[3], double *rho, double u[3]) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) r += f[i];
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 19; ++i) j[a] += f[i] * C[i][a];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / r;
    *rho = r;
}

/* Eq. (lb) TRT collision with forcing, for one cell with given rho, u. */
static void collide_cell(const double f[19], double rho, const double u[3], const double F[3],
                         double omega_p, double omega_m, double fs[19]) {
    double feq[19], D[19];
    orc_equilibrium(rho, u, feq);
    orc_forcing(u, F, omega_p, omega_m, D);
    for (int i = 0; i < 19; ++i) {
        int ip = OPP[i];
        double fp = 0.5 * (f[i] + f[ip]);
        double fm = 0.5 * (f[i] - f[ip]);
        double ep = 0.5 * (feq[i] + feq[ip]);
        double em = 0.5 * (feq[i] - feq[ip]);
        fs[i] = f[i] - omega_p * (fp - ep) - omega_m * (fm - em) + D[i];
    }
}

void orc_collide(const double f[19], const double F[3], double omega_p, double omega_m, double fs[19]) {
    double rho, u[3];
    moments(f, F, &rho, u);
    collide_cell(f, rho, u, F, omega_p, omega_m, fs);
}

/* Eq. (source) without the tau div(u) term.  G[k*3+j] = d_k u_j. */
void orc_source(const double tau[6], const double G[9], double ep_l, double inv_l, double S[6]) {
    double T[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T[a][b] = tau[COMP[a][b]];
    for (int c = 0; c < 6; ++c) {
        int i = CI[c], j = CJ[c];
        double a = 0.0, b = 0.0;
        for (int k = 0; k < 3; ++k) a += T[i][k] * G[k * 3 + j];
        for (int k = 0; k < 3; ++k) b += T[k][j] * G[k * 3 + i];
        S[c] = a + b + ep_l * (G[i * 3 + j] + G[j * 3 + i]) - inv_l * T[i][j];
    }
}

/* FENE-P stress of a conformation tensor: tau = (eta_p/lambda)(f A - I),
 * f = 1 / (1 - tr A / L^2). */
void orc_fene_stress(const double A[6], double eta_p, double lambda_p, double L2, double tau[6]) {
    double f = 1.0 / (1.0 - (A[0] + A[1] + A[2]) / L2);
    for (int c = 0; c < 6; ++c) tau[c] = (eta_p / lambda_p) * (f * A[c] - (c < 3 ? 1.0 : 0.0));
}

/* Its inverse: f A = I + lambda tau / eta_p, and taking the trace with
 * 1/f = 1 - tr A / L^2 gives f = 1 + (3 + lambda tr tau / eta_p) / L^2. */
void orc_fene_conformation(const double tau[6], double eta_p, double lambda_p, double L2, double A[6]) {
    double s = 3.0 + lambda_p * (tau[0] + tau[1] + tau[2]) / eta_p;
    double f = 1.0 + s / L2;
    for (int c = 0; c < 6; ++c) A[c] = ((c < 3 ? 1.0 : 0.0) + lambda_p * tau[c] / eta_p) / f;
}

/* ------------------------------------------------------------------------- */
/* fields                                                                    */
/* ------------------------------------------------------------------------- */
static void gather_f(const orc_state *s, const double *f, long r, double out[19]) {
    for (int i = 0; i < 19; ++i) out[i] = f[(long)i * s->n + r];
}

/* Eq. (force) on the D3Q7 faces (A_0 = 1, |c| = 1), faces by Eq. (interpolation),
 * a solid neighbour's stress replaced by tau(r) per Eq. (extrapolation). */
/* Stress of cell r from the stored tensor: tau itself, or in FENE-P mode the stress of
 * the conformation tensor A. */
static void cell_stress(const orc_state *s, const double *stored, long r, double t[6]) {
    double a[6];
    for (int c = 0; c < 6; ++c) a[c] = stored[(long)c * s->n + r];
    if (s->fene)
        orc_fene_stress(a, s->eta_p, s->p.lambda_p, s->p.fene_L2, t);
    else
        for (int c = 0; c < 6; ++c) t[c] = a[c];
}

static void polymer_force_cell(const orc_state *s, const double *tau, long r, double Fp[3]) {
    Fp[0] = Fp[1] = Fp[2] = 0.0;
    double tr6[6], tn6[6];
    cell_stress(s, tau, r, tr6);
    for (int l = 0; l < 6; ++l) {
        int k = FACE_AXIS[l];
        double sg = FACE_SIGN[l];
        int d[3] = {0, 0, 0};
        d[k] = (int)sg;
        long nb = neighbour(s, r, d[0], d[1], d[2]);
        int fl = is_fluid(s, nb);
        if (fl) cell_stress(s, tau, nb, tn6);
        for (int j = 0; j < 3; ++j) {
            int c = COMP[k][j];
            double tr = tr6[c];
            double tf = fl ? 0.5 * (tr + tn6[c]) : tr;
            Fp[j] += sg * tf;
        }
    }
}

void orc_polymer_force_field(orc_state *s, double *Fp) {
    for (long r = 0; r < s->n; ++r) {
        double F3[3] = {0.0, 0.0, 0.0};
        if (is_fluid(s, r)) polymer_force_cell(s, s->tau, r, F3);
        for (int a = 0; a < 3; ++a) Fp[(long)a * s->n + r] = F3[a];
    }
}

/* Steps 1-2: F = g + F^p and u = (j + F/2)/rho for every fluid cell. */
static void macroscopic(orc_state *s) {
    long n = s->n;
#pragma omp parallel for schedule(static) if (n >= 32768)
    for (long r = 0; r < n; ++r) {
        if (!is_fluid(s, r)) {
            s->rho[r] = 0.0;
            for (int a = 0; a < 3; ++a) {
                s->u[(long)a * n + r] = 0.0;
                s->F[(long)a * n + r] = 0.0;
            }
            continue;
        }
        double Fp[3], F[3], f[19], rho, u[3];
        polymer_force_cell(s, s->tau, r, Fp);
        for (int a = 0; a < 3; ++a) F[a] = s->p.g[a] + Fp[a];
        gather_f(s, s->f, r, f);
        moments(f, F, &rho, u);
        s->rho[r] = rho;
        for (int a = 0; a < 3; ++a) {
            s->u[(long)a * n + r] = u[a];
            s->F[(long)a * n + r] = F[a];
        }
    }
}

void orc_velocity_field(orc_state *s, double *u) {
    macroscopic(s);
    memcpy(u, s->u, sizeof(double) * 3 * (size_t)s->n);
}

/* Step 3: Eqs. (continuity)-(source) on cell averages, explicit Euler, D3Q7 faces. */
static void fv_update(orc_state *s, const double *u, const double *tau, double *taun) {
    long n = s->n;
    int flux_on = (s->p.fv_terms & ORC_FV_FLUX) != 0;
    int src_on = (s->p.fv_terms & ORC_FV_SOURCE) != 0;
    int ctu_on = (s->p.fv_terms & ORC_FV_CTU) != 0;
    int divu_on = (s->p.fv_terms & ORC_FV_DIVU) != 0;
#pragma omp parallel for schedule(static) if (n >= 32768)
    for (long r = 0; r < n; ++r) {
        if (!is_fluid(s, r)) {
            for (int c = 0; c < 6; ++c) taun[(long)c * n + r] = 0.0;
            continue;
        }
        double G[9], net[6] = {0, 0, 0, 0, 0, 0}, tr[6];
        for (int c = 0; c < 6; ++c) tr[c] = tau[(long)c * n + r];
        /* velocity gradient d_k u_j = u_j(face +k) - u_j(face -k) (central point rule);
         * a face towards a solid cell takes the boundary velocity. */
        for (int k = 0; k < 3; ++k) {
            int d[3] = {0, 0, 0};
            d[k] = 1;
            long np_ = neighbour(s, r, d[0], d[1], d[2]);
            long nm_ = neighbour(s, r, -d[0], -d[1], -d[2]);
            double ubp[3], ubm[3];
            boundary_velocity(s, np_, ubp);
            boundary_velocity(s, nm_, ubm);
            for (int j = 0; j < 3; ++j) {
                double ur = u[(long)j * n + r];
                double up = is_fluid(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ubp[j];
                double um = is_fluid(s, nm_) ? 0.5 * (ur + u[(long)j * n + nm_]) : ubm[j];
                G[k * 3 + j] = up - um;
            }
        }
        /* donor-cell advective flux through each fluid-fluid face, zero across solid links */
        if (flux_on) {
            for (int l = 0; l < 6; ++l) {
                int k = FACE_AXIS[l];
                double sg = FACE_SIGN[l];
                int d[3] = {0, 0, 0};
                d[k] = (int)sg;
                long nb = neighbour(s, r, d[0], d[1], d[2]);
                if (!is_fluid(s, nb)) continue;
                double vout = sg * u[(long)k * n + r];
                double vin = -sg * u[(long)k * n + nb];
                /* transverse overlap of the displaced donor cell with the face neighbour */
                double tout = 1.0, tin = 1.0;
                if (ctu_on) {
                    int a = (k + 1) % 3, b = (k + 2) % 3;
                    tout = (1.0 - fabs(u[(long)a * n + r])) * (1.0 - fabs(u[(long)b * n + r]));
                    tin = (1.0 - fabs(u[(long)a * n + nb])) * (1.0 - fabs(u[(long)b * n + nb]));
                }
                for (int c = 0; c < 6; ++c) {
                    double Jo = vout > 0.0 ? (vout * tout) * tr[c] : 0.0;
                    double Ji = vin > 0.0 ? (vin * tin) * tau[(long)c * n + nb] : 0.0;
                    double J = Jo - Ji;
                    net[c] += J;
                }
            }
        }
        double S[6] = {0, 0, 0, 0, 0, 0};
        if (src_on && !s->fene) orc_source(tr, G, s->ep_l, s->inv_l, S);
        if (src_on && s->fene) {
            /* A.grad u + (A.grad u)^T - (f A - I) / lambda, f = 1 / (1 - tr A / L^2) */
            double fA = 1.0 / (1.0 - (tr[0] + tr[1] + tr[2]) / s->p.fene_L2);
            for (int c = 0; c < 6; ++c) {
                int i = CI[c], j = CJ[c];
                double a = 0.0, b = 0.0;
                for (int k = 0; k < 3; ++k) a += tr[COMP[i][k]] * G[k * 3 + j];
                for (int k = 0; k < 3; ++k) b += tr[COMP[k][j]] * G[k * 3 + i];
                S[c] = a + b - s->inv_l * (fA * tr[c] - (i == j ? 1.0 : 0.0));
            }
        }
        if (divu_on) {
            double divu = (G[0] + G[4]) + G[8];
            for (int c = 0; c < 6; ++c) S[c] = S[c] + tr[c] * divu;
        }
        /* Giesekus: -(alpha / eta_p) (tau . tau)_ij */
        if (src_on && s->gk != 0.0) {
            for (int c = 0; c < 6; ++c) {
                int i = CI[c], j = CJ[c];
                double q = 0.0;
                for (int k = 0; k < 3; ++k) q += tr[COMP[i][k]] * tr[COMP[k][j]];
                S[c] = S[c] - s->gk * q;
            }
        }
        for (int c = 0; c < 6; ++c) taun[(long)c * n + r] = tr[c] - net[c] + S[c];
    }
}

void orc_fv_update_field(orc_state *s, const double *u, double *tau_out) { fv_update(s, u, s->tau, tau_out); }

/* ------------------------------------------------------------------------- */
/* particles: Sec. "Moving boundaries"                                        */
/* ------------------------------------------------------------------------- */
static int inside_particle(const orc_state *s, const orc_particle *P, long r) {
    double d[3];
    displacement(s, r, P->X, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= P->R * P->R;
}

static void cross(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Re-voxelise all particles at their current positions and convert cells. */
void orc_fill_drain(orc_state *s) {
    long n = s->n;
    uint8_t *nf = (uint8_t *)malloc((size_t)n);
    memcpy(nf, s->flag, (size_t)n);
    for (long r = 0; r < n; ++r) {
        uint8_t fl = s->flag[r];
        if (fl != ORC_FLUID && !is_particle_flag(fl)) continue;
        int owner = -1;
        for (int q = 0; q < s->np; ++q)
            if (inside_particle(s, &s->part[q], r)) {
                owner = q;
                break;
            }
        nf[r] = owner >= 0 ? (uint8_t)(ORC_PART0 + owner) : (uint8_t)ORC_FLUID;
    }
    for (int q = 0; q < s->np; ++q)
        for (int a = 0; a < 3; ++a) s->part[q].dP[a] = s->part[q].dL[a] = 0.0;

    /* 0 stable solid/other, 1 stable fluid, 2 destroyed (fluid->particle), 3 created */
    uint8_t *kind = (uint8_t *)calloc((size_t)n, 1);
    for (long r = 0; r < n; ++r) {
        int was = s->flag[r] == ORC_FLUID, now = nf[r] == ORC_FLUID;
        kind[r] = (uint8_t)(was && now ? 1 : (was && !now ? 2 : (!was && now ? 3 : 0)));
    }
    /* N_f and the new stress of created cells, from the pre-conversion stress */
    int *Nf = (int *)calloc((size_t)n, sizeof(int));
    double *tnew = (double *)calloc((size_t)6 * n, sizeof(double));
    for (long r = 0; r < n; ++r) {
        if (kind[r] != 2 && kind[r] != 3) continue;
        double sum[6] = {0, 0, 0, 0, 0, 0};
        for (int l = 0; l < 6; ++l) {
            int d[3] = {0, 0, 0};
            d[FACE_AXIS[l]] = (int)FACE_SIGN[l];
            long nb = neighbour(s, r, d[0], d[1], d[2]);
            if (nb < 0 || kind[nb] != 1) continue;
            Nf[r]++;
            for (int c = 0; c < 6; ++c) sum[c] += s->tau[(long)c * n + nb];
        }
        if (kind[r] == 3)
            for (int c = 0; c < 6; ++c) tnew[(long)c * n + r] = sum[c] / (double)(Nf[r] + 1);
    }
    /* destroyed cells: momentum of the deleted PDFs goes to the particle */
    for (long r = 0; r < n; ++r) {
        if (kind[r] != 2) continue;
        orc_particle *P = &s->part[nf[r] - ORC_PART0];
        double Pm[3] = {0, 0, 0}, d[3], L[3];
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < 19; ++i) Pm[a] += s->f[(long)i * n + r] * C[i][a];
        displacement(s, r, P->X, d);
        cross(d, Pm, L);
        for (int a = 0; a < 3; ++a) {
            P->dP[a] += Pm[a];
            P->dL[a] += L[a];
        }
        if (Nf[r] == 0)
            for (int c = 0; c < 6; ++c) s->dropped[c] += s->tau[(long)c * n + r];
        s->n_destroyed++;
    }
    /* created cells: f = f^eq(rho_bar, u_b), momentum taken from the particle */
    for (long r = 0; r < n; ++r) {
        if (kind[r] != 3) continue;
        orc_particle *P = &s->part[s->flag[r] - ORC_PART0];
        double rsum = 0.0;
        int cnt = 0;
        for (int i = 1; i < 19; ++i) {
            long nb = neighbour(s, r, C[i][0], C[i][1], C[i][2]);
            if (nb < 0 || kind[nb] != 1) continue;
            double rn = 0.0;
            for (int k = 0; k < 19; ++k) rn += s->f[(long)k * n + nb];
            rsum += rn;
            cnt++;
        }
        double rho_bar = cnt > 0 ? rsum / (double)cnt : s->p.rho0;
        double d[3], ub[3], wx[3], feq[19], Pm[3] = {0, 0, 0}, L[3];
        displacement(s, r, P->X, d);
        cross(P->w, d, wx);
        for (int a = 0; a < 3; ++a) ub[a] = P->v[a] + wx[a];
        orc_equilibrium(rho_bar, ub, feq);
        for (int i = 0; i < 19; ++i) s->fn[(long)i * n + r] = feq[i];
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < 19; ++i) Pm[a] += feq[i] * C[i][a];
        cross(d, Pm, L);
        for (int a = 0; a < 3; ++a) {
            P->dP[a] -= Pm[a];
            P->dL[a] -= L[a];
        }
        s->n_created++;
    }
    for (long r = 0; r < n; ++r)
        if (kind[r] == 3)
            for (int i = 0; i < 19; ++i) s->f[(long)i * n + r] = s->fn[(long)i * n + r];
    /* stress redistribution, gathered per stable fluid cell in D3Q7 face order */
    for (long r = 0; r < n; ++r) {
        if (kind[r] != 1) continue;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        int touched = 0;
        for (int l = 0; l < 6; ++l) {
            int d[3] = {0, 0, 0};
            d[FACE_AXIS[l]] = (int)FACE_SIGN[l];
            long nb = neighbour(s, r, d[0], d[1], d[2]);
            if (nb < 0) continue;
            if (kind[nb] == 2) {
                for (int c = 0; c < 6; ++c) acc[c] += s->tau[(long)c * n + nb] / (double)Nf[nb];
                touched = 1;
            } else if (kind[nb] == 3) {
                for (int c = 0; c < 6; ++c) acc[c] -= tnew[(long)c * n + nb] / (double)Nf[nb];
                touched = 1;
            }
        }
        if (touched)
            for (int c = 0; c < 6; ++c) s->taun[(long)c * n + r] = s->tau[(long)c * n + r] + acc[c];
        else
            for (int c = 0; c < 6; ++c) s->taun[(long)c * n + r] = s->tau[(long)c * n + r];
    }
    for (long r = 0; r < n; ++r) {
        if (kind[r] == 1) {
            for (int c = 0; c < 6; ++c) s->tau[(long)c * n + r] = s->taun[(long)c * n + r];
        } else if (kind[r] == 3) {
            for (int c = 0; c < 6; ++c) s->tau[(long)c * n + r] = tnew[(long)c * n + r];
        } else if (kind[r] == 2) {
            for (int c = 0; c < 6; ++c) s->tau[(long)c * n + r] = 0.0;
        }
    }
    memcpy(s->flag, nf, (size_t)n);
    for (int q = 0; q < s->np; ++q) {
        orc_particle *P = &s->part[q];
        for (int a = 0; a < 3; ++a) {
            P->v[a] += P->dP[a] / P->m;
            P->w[a] += P->dL[a] / P->I;
        }
    }
    free(tnew);
    free(Nf);
    free(kind);
    free(nf);
}

/* ------------------------------------------------------------------------- */
/* one time step                                                             */
/* ------------------------------------------------------------------------- */
static void one_step(orc_state *s) {
    long n = s->n;
    /* 1-2: F^p(tau^t), rho^t, u^t */
    macroscopic(s);
    /* 3: tau^{t+1} from tau^t and u^t */
    fv_update(s, s->u, s->tau, s->taun);
    /* 4: collision (in place: f becomes the post-collision f*) */
#pragma omp parallel for schedule(static) if (n >= 32768)
    for (long r = 0; r < n; ++r) {
        if (!is_fluid(s, r)) continue;
        double f[19], fs[19], u[3], F[3];
        gather_f(s, s->f, r, f);
        for (int a = 0; a < 3; ++a) {
            u[a] = s->u[(long)a * n + r];
            F[a] = s->F[(long)a * n + r];
        }
        collide_cell(f, s->rho[r], u, F, s->omega_p, s->omega_m, fs);
        for (int i = 0; i < 19; ++i) s->f[(long)i * n + r] = fs[i];
    }
    /* 5: push streaming; a link into a solid cell bounces back with Eq. (ubb) */
#pragma omp parallel for schedule(static) if (n >= 32768)
    for (long r = 0; r < n; ++r) {
        if (!is_fluid(s, r)) continue;
        for (int i = 0; i < 19; ++i) {
            long nb = neighbour(s, r, C[i][0], C[i][1], C[i][2]);
            double fsi = s->f[(long)i * n + r];
            if (is_fluid(s, nb)) {
                s->fn[(long)i * n + nb] = fsi;
            } else {
                double ub[3];
                boundary_velocity(s, nb, ub);
                double cub = C[i][0] * ub[0] + C[i][1] * ub[1] + C[i][2] * ub[2];
                double X = 6.0 * W[i] * s->rho[r] * cub;
                s->fn[(long)OPP[i] * n + r] = fsi - X;
            }
        }
    }
    /* momentum exchange on every link into a wall class or particle, cell order then
     * direction order */
    memset(s->body_F, 0, sizeof(s->body_F));
    for (int q = 0; q < s->np; ++q)
        for (int a = 0; a < 3; ++a) s->part[q].Fme[a] = s->part[q].Tme[a] = 0.0;
    int has_bodies = s->np > 0;
    for (long r = 0; r < n && !has_bodies; ++r) has_bodies = s->flag[r] >= ORC_WALL0;
    for (long r = 0; r < n && has_bodies; ++r) {
        if (!is_fluid(s, r)) continue;
        for (int i = 1; i < 19; ++i) {
            long nb = neighbour(s, r, C[i][0], C[i][1], C[i][2]);
            if (nb < 0) continue;
            uint8_t fl = s->flag[nb];
            if (fl < ORC_WALL0) continue;
            double ub[3];
            boundary_velocity(s, nb, ub);
            double cub = C[i][0] * ub[0] + C[i][1] * ub[1] + C[i][2] * ub[2];
            double X = 6.0 * W[i] * s->rho[r] * cub;
            double m = 2.0 * s->f[(long)i * n + r] - X;
            double Fl[3] = {C[i][0] * m, C[i][1] * m, C[i][2] * m};
            for (int a = 0; a < 3; ++a) s->body_F[fl][a] += Fl[a];
            if (is_particle_flag(fl)) {
                orc_particle *P = &s->part[fl - ORC_PART0];
                double d[3], T[3];
                displacement(s, nb, P->X, d);
                cross(d, Fl, T);
                for (int a = 0; a < 3; ++a) {
                    P->Fme[a] += Fl[a];
                    P->Tme[a] += T[a];
                }
            }
        }
    }
    double *tmp = s->f;
    s->f = s->fn;
    s->fn = tmp;
    tmp = s->tau;
    s->tau = s->taun;
    s->taun = tmp;
    /* 6: particle update, symplectic Euler (velocity first, then position) */
    for (int q = 0; q < s->np; ++q) {
        orc_particle *P = &s->part[q];
        for (int a = 0; a < 3; ++a) {
            P->v[a] += (P->Fme[a] + P->Fext[a]) / P->m;
            P->w[a] += (P->Tme[a] + P->Text[a]) / P->I;
            P->X[a] += P->v[a];
        }
    }
    /* 7: fill/drain */
    if (s->np > 0) orc_fill_drain(s);
    s->t++;
}

void orc_step(orc_state *s, int nsteps) {
    for (int k = 0; k < nsteps; ++k) one_step(s);
}

long orc_time(const orc_state *s) { return s->t; }

/* ------------------------------------------------------------------------- */
/* lifetime                                                                   */
/* ------------------------------------------------------------------------- */
orc_state *orc_create(const orc_params *p) {
    init_weights();
    if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (!(p->eta > 0.0) || !(p->beta >= 0.0 && p->beta < 1.0) || !(p->rho0 > 0.0)) return NULL;
    if (p->beta > 0.0 && !(p->lambda_p > 0.0)) return NULL;
    if (p->n_wall < 0 || p->n_wall > ORC_MAX_WALL) return NULL;
    if (!(p->giesekus_alpha >= 0.0 && p->giesekus_alpha <= 0.5)) return NULL;
    if (!(p->fene_L2 == 0.0 || p->fene_L2 > 3.0)) return NULL;
    if (p->fene_L2 > 0.0 && (!(p->beta > 0.0) || p->giesekus_alpha != 0.0)) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    s->p = *p;
    s->n = (long)p->nx * p->ny * p->nz;
    long n = s->n;
    s->f = (double *)calloc((size_t)19 * n, sizeof(double));
    s->fn = (double *)calloc((size_t)19 * n, sizeof(double));
    s->tau = (double *)calloc((size_t)6 * n, sizeof(double));
    s->taun = (double *)calloc((size_t)6 * n, sizeof(double));
    s->rho = (double *)calloc((size_t)n, sizeof(double));
    s->u = (double *)calloc((size_t)3 * n, sizeof(double));
    s->F = (double *)calloc((size_t)3 * n, sizeof(double));
    s->flag = (uint8_t *)calloc((size_t)n, 1);
    /* relaxation rates, Sec. "Lattice Boltzmann" (rates reading) */
    double eta_n = (1.0 - p->beta) * p->eta;
    double nu_n = eta_n / p->rho0;
    s->omega_p = 1.0 / (3.0 * nu_n + 0.5);
    double tp = 1.0 / s->omega_p - 0.5;
    s->omega_m = 1.0 / (p->magic / tp + 0.5);
    s->eta_p = p->beta * p->eta;
    s->ep_l = p->beta > 0.0 ? s->eta_p / p->lambda_p : 0.0;
    s->inv_l = p->lambda_p > 0.0 ? 1.0 / p->lambda_p : 0.0;
    s->gk = p->beta > 0.0 ? p->giesekus_alpha / s->eta_p : 0.0;
    s->fene = p->fene_L2 > 0.0;
    orc_init_fields(s, NULL, NULL, NULL);
    return s;
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free(s->f);
    free(s->fn);
    free(s->tau);
    free(s->taun);
    free(s->rho);
    free(s->u);
    free(s->F);
    free(s->flag);
    free(s);
}

int orc_set_flags(orc_state *s, const uint8_t *flags) {
    int nn[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (long r = 0; r < s->n; ++r) {
        uint8_t fl = flags[r];
        if (fl >= ORC_WALL0 + ORC_MAX_WALL) return -1;
        if (fl >= ORC_WALL0 && fl - ORC_WALL0 >= s->p.n_wall) return -1;
        int x, y, z;
        cell_coords(s, r, &x, &y, &z);
        int q[3] = {x, y, z};
        if (fl == ORC_FLUID)
            for (int a = 0; a < 3; ++a)
                if (!s->p.periodic[a] && (q[a] == 0 || q[a] == nn[a] - 1)) return -2;
    }
    memcpy(s->flag, flags, (size_t)s->n);
    return 0;
}

int orc_init_fields(orc_state *s, const double *rho, const double *u, const double *tau) {
    long n = s->n;
    for (long r = 0; r < n; ++r) {
        double rr = rho ? rho[r] : s->p.rho0;
        double uu[3] = {0, 0, 0}, feq[19];
        if (u)
            for (int a = 0; a < 3; ++a) uu[a] = u[(long)a * n + r];
        orc_equilibrium(rr, uu, feq);
        for (int i = 0; i < 19; ++i) s->f[(long)i * n + r] = feq[i];
        double t6[6], a6[6];
        for (int c = 0; c < 6; ++c) t6[c] = tau ? tau[(long)c * n + r] : 0.0;
        if (s->fene) orc_fene_conformation(t6, s->eta_p, s->p.lambda_p, s->p.fene_L2, a6);
        for (int c = 0; c < 6; ++c) s->tau[(long)c * n + r] = s->fene ? a6[c] : t6[c];
    }
    return 0;
}

int orc_add_particle(orc_state *s, const double X[3], double R, double rho_p, const double v[3],
                     const double w[3], const double Fext[3], const double Text[3]) {
    if (s->np >= ORC_MAX_PART || !(R > 0.0) || !(rho_p > 0.0) || s->fene) return -1;
    int id = s->np++;
    orc_particle *P = &s->part[id];
    memset(P, 0, sizeof(*P));
    for (int a = 0; a < 3; ++a) {
        P->X[a] = X[a];
        P->v[a] = v ? v[a] : 0.0;
        P->w[a] = w ? w[a] : 0.0;
        P->Fext[a] = Fext ? Fext[a] : 0.0;
        P->Text[a] = Text ? Text[a] : 0.0;
    }
    P->R = R;
    P->rho_p = rho_p;
    P->m = rho_p * (4.0 / 3.0) * M_PI * R * R * R;
    P->I = 0.4 * P->m * R * R;
    /* initial placement: covered fluid cells become particle cells, no impulse */
    for (long r = 0; r < s->n; ++r) {
        if (s->flag[r] != ORC_FLUID || !inside_particle(s, P, r)) continue;
        s->flag[r] = (uint8_t)(ORC_PART0 + id);
        for (int c = 0; c < 6; ++c) s->tau[(long)c * s->n + r] = 0.0;
    }
    return id;
}

int orc_set_particle(orc_state *s, int id, const double X[3], const double v[3], const double w[3]) {
    if (id < 0 || id >= s->np) return -1;
    for (int a = 0; a < 3; ++a) {
        if (X) s->part[id].X[a] = X[a];
        if (v) s->part[id].v[a] = v[a];
        if (w) s->part[id].w[a] = w[a];
    }
    return 0;
}

void orc_read_fields(orc_state *s, double *rho, double *u, double *tau, uint8_t *flags) {
    long n = s->n;
    macroscopic(s);
    if (rho) memcpy(rho, s->rho, sizeof(double) * (size_t)n);
    if (u) memcpy(u, s->u, sizeof(double) * 3 * (size_t)n);
    if (tau)
        for (long r = 0; r < n; ++r) {
            double t6[6] = {0, 0, 0, 0, 0, 0};
            if (is_fluid(s, r)) cell_stress(s, s->tau, r, t6);
            for (int c = 0; c < 6; ++c) tau[(long)c * n + r] = t6[c];
        }
    if (flags) memcpy(flags, s->flag, (size_t)n);
}

void orc_read_pdfs(const orc_state *s, double *f) { memcpy(f, s->f, sizeof(double) * 19 * (size_t)s->n); }
void orc_write_pdfs(orc_state *s, const double *f) { memcpy(s->f, f, sizeof(double) * 19 * (size_t)s->n); }
void orc_write_tau(orc_state *s, const double *tau) { memcpy(s->tau, tau, sizeof(double) * 6 * (size_t)s->n); }

int orc_read_particle(const orc_state *s, int id, double out[24]) {
    if (id < 0 || id >= s->np) return -1;
    const orc_particle *P = &s->part[id];
    for (int a = 0; a < 3; ++a) {
        out[a] = P->X[a];
        out[3 + a] = P->v[a];
        out[6 + a] = P->w[a];
        out[9 + a] = P->Fme[a];
        out[12 + a] = P->Tme[a];
        out[15 + a] = P->dP[a];
        out[18 + a] = P->dL[a];
    }
    out[21] = P->m;
    out[22] = P->I;
    out[23] = P->R;
    return 0;
}

void orc_read_body_forces(const orc_state *s, double *out) { memcpy(out, s->body_F, sizeof(s->body_F)); }

void orc_read_diag(const orc_state *s, double out[8]) {
    for (int c = 0; c < 6; ++c) out[c] = s->dropped[c];
    out[6] = (double)s->n_destroyed;
    out[7] = (double)s->n_created;
}

void orc_rates(const orc_state *s, double out[5]) {
    out[0] = s->omega_p;
    out[1] = s->omega_m;
    out[2] = s->eta_p;
    out[3] = s->ep_l;
    out[4] = s->inv_l;
}
