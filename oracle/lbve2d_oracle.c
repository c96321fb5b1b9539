/*
 * lbve2d_oracle.c -- plain FP64 CPU reference of the two-dimensional coupled step:
 * D2Q9 two-relaxation-time lattice Boltzmann with Guo forcing, coupled through the
 * polymer force to a D2Q5 finite-volume update of the three-component Oldroyd-B stress
 * (xx, yy, xy), as the paper uses for its lid-driven cavity and four-roll mill (Sec.
 * "Lid-driven cavity", Sec. "Four-roll mill"; the 2-D lattices are named in Sec.
 * "Implementation and extensibility").
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests to check the CUDA library; never by the
 * product path, and it shares no code with it.  Slow on purpose: two PDF arrays with
 * push streaming, one loop per sub-step, every formula as the paper states it.
 *
 * One step t -> t+1, in the order of the three-dimensional oracle:
 *   1. F = g + F_field(r) + F^p(tau^t), F^p by Eq. (force) on the D2Q5 faces with
 *      Eq. (interpolation) and the per-link extrapolation of Eq. (extrapolation)
 *   2. rho, u = (j + F/2)/rho                                Eq. (macroscopic-velocity)
 *   3. tau^{t+1} by Eqs. (continuity)-(source): donor-cell face fluxes, zero flux across
 *      solid links, central-point gradient with the boundary velocity as the face value
 *      at solid faces, explicit Euler
 *   4. TRT collision with Guo forcing                         Eqs. (lb), (lb-equilibrium),
 *                                                             (guo)
 *   5. push streaming; a link into a solid cell bounces back with -6 w_i rho c_i.u_b,
 *      u_b the solid cell's prescribed velocity               Eq. (ubb)
 * The readings of garbled passages are those of the three-dimensional oracle
 * (equilibrium coefficients, TRT rates from the magic product, Guo forcing split for
 * TRT, the tau div u term dropped).  The per-cell boundary velocity carries the
 * regularised lid of Sec. "Lid-driven cavity", and the per-cell force field the
 * four-roll mill forcing of Sec. "Four-roll mill" (both evaluated by the caller).
 */
#include "lbve2d_oracle.h"

#include <stdlib.h>
#include <string.h>

/* D2Q9 velocities (rest, 4 axis directions, 4 diagonals; each odd i paired with the
 * opposite direction i + 1) and weights 4/9, 1/9, 1/36 (Sec. "Lattice Boltzmann"). */
static const int C2[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
static const int OPP2[9] = {0, 2, 1, 4, 3, 6, 5, 8, 7};
static double W2[9];

/* D2Q5 faces +x, -x, +y, -y */
static const int FAX[4] = {0, 0, 1, 1};
static const double FSG[4] = {1.0, -1.0, 1.0, -1.0};
/* symmetric 2x2 tensor layout xx, yy, xy */
static const int CMP[2][2] = {{0, 2}, {2, 1}};
static const int CI2[3] = {0, 1, 0};
static const int CJ2[3] = {0, 1, 1};

static void weights(void) {
    W2[0] = 4.0 / 9.0;
    for (int i = 1; i < 5; ++i) W2[i] = 1.0 / 9.0;
    for (int i = 5; i < 9; ++i) W2[i] = 1.0 / 36.0;
}

struct orc2_state {
    orc2_params p;
    long n;
    double omega_p, omega_m, eta_p, ep_l, inv_l;
    double *f, *fn, *tau, *taun, *rho, *u, *F, *ub, *Ff;
    uint8_t *flag;
    long t;
};

static long nb2(const orc2_state *s, long r, int dx, int dy) {
    int x = (int)(r % s->p.nx), y = (int)(r / s->p.nx);
    int q[2] = {x + dx, y + dy}, nn[2] = {s->p.nx, s->p.ny};
    for (int a = 0; a < 2; ++a)
        if (q[a] < 0 || q[a] >= nn[a]) {
            if (!s->p.periodic[a]) return -1;
            q[a] = (q[a] + nn[a]) % nn[a];
        }
    return (long)q[0] + (long)s->p.nx * q[1];
}

static int fluid2(const orc2_state *s, long r) { return r >= 0 && s->flag[r] == 0; }

static void ub_of(const orc2_state *s, long r, double ub[2]) {
    ub[0] = ub[1] = 0.0;
    if (r >= 0) {
        ub[0] = s->ub[r];
        ub[1] = s->ub[s->n + r];
    }
}

void orc2_lattice(int c[9][2], double w[9], int opp[9]) {
    weights();
    for (int i = 0; i < 9; ++i) {
        c[i][0] = C2[i][0];
        c[i][1] = C2[i][1];
        w[i] = W2[i];
        opp[i] = OPP2[i];
    }
}

/* Eq. (lb-equilibrium), second-order form. */
static void equilibrium2(double rho, const double u[2], double feq[9]) {
    double usq = u[0] * u[0] + u[1] * u[1];
    for (int i = 0; i < 9; ++i) {
        double cu = C2[i][0] * u[0] + C2[i][1] * u[1];
        feq[i] = W2[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Polymer force of Eq. (force) on the D2Q5 faces. */
static void polymer_force2(const orc2_state *s, long r, double Fp[2]) {
    Fp[0] = Fp[1] = 0.0;
    for (int l = 0; l < 4; ++l) {
        int k = FAX[l];
        int d[2] = {0, 0};
        d[k] = (int)FSG[l];
        long nb = nb2(s, r, d[0], d[1]);
        int fl = fluid2(s, nb);
        for (int j = 0; j < 2; ++j) {
            int c = CMP[k][j];
            double tr = s->tau[(long)c * s->n + r];
            double tf = fl ? 0.5 * (tr + s->tau[(long)c * s->n + nb]) : tr;
            Fp[j] += FSG[l] * tf;
        }
    }
}

static void macroscopic2(orc2_state *s) {
    long n = s->n;
    for (long r = 0; r < n; ++r) {
        if (!fluid2(s, r)) {
            s->rho[r] = 0.0;
            for (int a = 0; a < 2; ++a) s->u[(long)a * n + r] = s->F[(long)a * n + r] = 0.0;
            continue;
        }
        double Fp[2], F[2], rho = 0.0, j[2] = {0.0, 0.0};
        polymer_force2(s, r, Fp);
        for (int a = 0; a < 2; ++a) F[a] = (s->p.g[a] + s->Ff[(long)a * n + r]) + Fp[a];
        for (int i = 0; i < 9; ++i) rho += s->f[(long)i * n + r];
        for (int a = 0; a < 2; ++a)
            for (int i = 0; i < 9; ++i) j[a] += s->f[(long)i * n + r] * C2[i][a];
        s->rho[r] = rho;
        for (int a = 0; a < 2; ++a) {
            s->u[(long)a * n + r] = (j[a] + 0.5 * F[a]) / rho;
            s->F[(long)a * n + r] = F[a];
        }
    }
}

/* Eqs. (continuity)-(source) on the D2Q5 faces, explicit Euler. */
static void fv2(orc2_state *s, const double *u, const double *tau, double *taun) {
    long n = s->n;
    int flux_on = (s->p.fv_terms & ORC2_FV_FLUX) != 0, src_on = (s->p.fv_terms & ORC2_FV_SOURCE) != 0;
    for (long r = 0; r < n; ++r) {
        if (!fluid2(s, r)) {
            for (int c = 0; c < 3; ++c) taun[(long)c * n + r] = 0.0;
            continue;
        }
        double G[4], net[3] = {0, 0, 0}, tr[3];
        for (int c = 0; c < 3; ++c) tr[c] = tau[(long)c * n + r];
        for (int k = 0; k < 2; ++k) {
            int d[2] = {0, 0};
            d[k] = 1;
            long np_ = nb2(s, r, d[0], d[1]), nm_ = nb2(s, r, -d[0], -d[1]);
            double ubp[2], ubm[2];
            ub_of(s, np_, ubp);
            ub_of(s, nm_, ubm);
            for (int j = 0; j < 2; ++j) {
                double ur = u[(long)j * n + r];
                double up = fluid2(s, np_) ? 0.5 * (ur + u[(long)j * n + np_]) : ubp[j];
                double um = fluid2(s, nm_) ? 0.5 * (ur + u[(long)j * n + nm_]) : ubm[j];
                G[k * 2 + j] = up - um;
            }
        }
        if (flux_on) {
            for (int l = 0; l < 4; ++l) {
                int k = FAX[l];
                double sg = FSG[l];
                int d[2] = {0, 0};
                d[k] = (int)sg;
                long nb = nb2(s, r, d[0], d[1]);
                if (!fluid2(s, nb)) continue;
                double vout = sg * u[(long)k * n + r];
                double vin = -sg * u[(long)k * n + nb];
                for (int c = 0; c < 3; ++c) {
                    double Jo = vout > 0.0 ? vout * tr[c] : 0.0;
                    double Ji = vin > 0.0 ? vin * tau[(long)c * n + nb] : 0.0;
                    net[c] += Jo - Ji;
                }
            }
        }
        for (int c = 0; c < 3; ++c) {
            double S = 0.0;
            if (src_on) {
                int i = CI2[c], j = CJ2[c];
                double a = 0.0, b = 0.0;
                for (int k = 0; k < 2; ++k) a += tr[CMP[i][k]] * G[k * 2 + j];
                for (int k = 0; k < 2; ++k) b += tr[CMP[k][j]] * G[k * 2 + i];
                S = a + b + s->ep_l * (G[i * 2 + j] + G[j * 2 + i]) - s->inv_l * tr[c];
            }
            taun[(long)c * n + r] = tr[c] - net[c] + S;
        }
    }
}

void orc2_fv_update_field(orc2_state *s, const double *u, double *tau_out) { fv2(s, u, s->tau, tau_out); }

static void step2(orc2_state *s) {
    long n = s->n;
    macroscopic2(s);
    fv2(s, s->u, s->tau, s->taun);
    double A = 3.0 * (1.0 - 0.5 * s->omega_m), B = 1.0 - 0.5 * s->omega_p;
    for (long r = 0; r < n; ++r) {
        if (!fluid2(s, r)) continue;
        double f[9], feq[9], D[9], u[2], F[2];
        for (int i = 0; i < 9; ++i) f[i] = s->f[(long)i * n + r];
        for (int a = 0; a < 2; ++a) {
            u[a] = s->u[(long)a * n + r];
            F[a] = s->F[(long)a * n + r];
        }
        equilibrium2(s->rho[r], u, feq);
        double uF = u[0] * F[0] + u[1] * F[1];
        for (int i = 0; i < 9; ++i) {
            double cu = C2[i][0] * u[0] + C2[i][1] * u[1];
            double cF = C2[i][0] * F[0] + C2[i][1] * F[1];
            D[i] = W2[i] * (A * cF + B * (9.0 * cu * cF - 3.0 * uF));
        }
        for (int i = 0; i < 9; ++i) {
            int ip = OPP2[i];
            double fp = 0.5 * (f[i] + f[ip]), fm = 0.5 * (f[i] - f[ip]);
            double ep = 0.5 * (feq[i] + feq[ip]), em = 0.5 * (feq[i] - feq[ip]);
            double fs = f[i] - s->omega_p * (fp - ep) - s->omega_m * (fm - em) + D[i];
            s->fn[(long)i * n + r] = fs; /* post-collision, streamed below */
        }
    }
    /* push streaming out of the post-collision values (held in fn), into f */
    for (long r = 0; r < n; ++r) {
        if (!fluid2(s, r)) continue;
        for (int i = 0; i < 9; ++i) {
            long nb = nb2(s, r, C2[i][0], C2[i][1]);
            double fsi = s->fn[(long)i * n + r];
            if (fluid2(s, nb)) {
                s->f[(long)i * n + nb] = fsi;
            } else {
                double ub[2];
                ub_of(s, nb, ub);
                double cub = C2[i][0] * ub[0] + C2[i][1] * ub[1];
                s->f[(long)OPP2[i] * n + r] = fsi - 6.0 * W2[i] * s->rho[r] * cub;
            }
        }
    }
    double *tmp = s->tau;
    s->tau = s->taun;
    s->taun = tmp;
    s->t++;
}

void orc2_step(orc2_state *s, int nsteps) {
    for (int k = 0; k < nsteps; ++k) step2(s);
}

long orc2_time(const orc2_state *s) { return s->t; }

orc2_state *orc2_create(const orc2_params *p) {
    weights();
    if (!p || p->nx < 1 || p->ny < 1 || !(p->eta > 0.0) || !(p->beta >= 0.0 && p->beta < 1.0) || !(p->rho0 > 0.0))
        return NULL;
    if (p->beta > 0.0 && !(p->lambda_p > 0.0)) return NULL;
    orc2_state *s = (orc2_state *)calloc(1, sizeof(orc2_state));
    s->p = *p;
    s->n = (long)p->nx * p->ny;
    long n = s->n;
    s->f = (double *)calloc((size_t)9 * n, sizeof(double));
    s->fn = (double *)calloc((size_t)9 * n, sizeof(double));
    s->tau = (double *)calloc((size_t)3 * n, sizeof(double));
    s->taun = (double *)calloc((size_t)3 * n, sizeof(double));
    s->rho = (double *)calloc((size_t)n, sizeof(double));
    s->u = (double *)calloc((size_t)2 * n, sizeof(double));
    s->F = (double *)calloc((size_t)2 * n, sizeof(double));
    s->ub = (double *)calloc((size_t)2 * n, sizeof(double));
    s->Ff = (double *)calloc((size_t)2 * n, sizeof(double));
    s->flag = (uint8_t *)calloc((size_t)n, 1);
    double nu_n = (1.0 - p->beta) * p->eta / p->rho0;
    s->omega_p = 1.0 / (3.0 * nu_n + 0.5);
    double tp = 1.0 / s->omega_p - 0.5;
    s->omega_m = 1.0 / (p->magic / tp + 0.5);
    s->eta_p = p->beta * p->eta;
    s->ep_l = p->beta > 0.0 ? s->eta_p / p->lambda_p : 0.0;
    s->inv_l = p->lambda_p > 0.0 ? 1.0 / p->lambda_p : 0.0;
    orc2_init_fields(s, NULL, NULL, NULL);
    return s;
}

void orc2_destroy(orc2_state *s) {
    if (!s) return;
    free(s->f);
    free(s->fn);
    free(s->tau);
    free(s->taun);
    free(s->rho);
    free(s->u);
    free(s->F);
    free(s->ub);
    free(s->Ff);
    free(s->flag);
    free(s);
}

int orc2_set_flags(orc2_state *s, const uint8_t *flags, const double *ub) {
    int nn[2] = {s->p.nx, s->p.ny};
    for (long r = 0; r < s->n; ++r) {
        int q[2] = {(int)(r % s->p.nx), (int)(r / s->p.nx)};
        if (flags[r] == 0)
            for (int a = 0; a < 2; ++a)
                if (!s->p.periodic[a] && (q[a] == 0 || q[a] == nn[a] - 1)) return -2;
    }
    memcpy(s->flag, flags, (size_t)s->n);
    for (long k = 0; k < 2 * s->n; ++k) s->ub[k] = ub ? ub[k] : 0.0;
    return 0;
}

void orc2_set_force(orc2_state *s, const double *F) {
    for (long k = 0; k < 2 * s->n; ++k) s->Ff[k] = F ? F[k] : 0.0;
}

int orc2_init_fields(orc2_state *s, const double *rho, const double *u, const double *tau) {
    long n = s->n;
    for (long r = 0; r < n; ++r) {
        double uu[2] = {u ? u[r] : 0.0, u ? u[n + r] : 0.0}, feq[9];
        equilibrium2(rho ? rho[r] : s->p.rho0, uu, feq);
        for (int i = 0; i < 9; ++i) s->f[(long)i * n + r] = feq[i];
        for (int c = 0; c < 3; ++c) s->tau[(long)c * n + r] = tau ? tau[(long)c * n + r] : 0.0;
    }
    s->t = 0;
    return 0;
}

void orc2_read_fields(orc2_state *s, double *rho, double *u, double *tau) {
    long n = s->n;
    macroscopic2(s);
    if (rho) memcpy(rho, s->rho, sizeof(double) * (size_t)n);
    if (u) memcpy(u, s->u, sizeof(double) * 2 * (size_t)n);
    if (tau)
        for (long r = 0; r < n; ++r)
            for (int c = 0; c < 3; ++c) tau[(long)c * n + r] = fluid2(s, r) ? s->tau[(long)c * n + r] : 0.0;
}

void orc2_read_pdfs(const orc2_state *s, double *f) { memcpy(f, s->f, sizeof(double) * 9 * (size_t)s->n); }
void orc2_write_pdfs(orc2_state *s, const double *f) { memcpy(s->f, f, sizeof(double) * 9 * (size_t)s->n); }
void orc2_write_tau(orc2_state *s, const double *tau) { memcpy(s->tau, tau, sizeof(double) * 3 * (size_t)s->n); }
