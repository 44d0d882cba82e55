/*
 * FP64 CPU oracle: the paper's lattice Boltzmann time step written out plainly.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Slow on purpose: one pass per
 * stage of the algorithm, per-cell loops, push streaming, FP64 throughout.
 * The per-node loops of a stage may run on several host threads (OpenMP, when
 * the build has it; orc_set_threads): every node writes only its own outputs
 * and the arithmetic of a node does not depend on the thread count, so results
 * are bit-identical to one thread.  Sums (orc_conserved) stay serial.  It
 * shares nothing with the CUDA library.
 *
 * Paper: B. Chen, C. Zhan, Z. Chai, B. Shi, "A phase-field-based lattice
 * Boltzmann method for two-phase flows with the interfacial mass/heat
 * transfer", arXiv 2402.15752.  Equation numbers follow the paper's sequential
 * numbering: Eq. (1) conservative Allen-Cahn, (2) tanh profile, (4)-(5)
 * chemical potential, (6) density, (7) linear viscosity, (17) two-scalar
 * model, (18) mixed diffusivity, (23)-(27) phase-field LB, (28)-(33) flow LB,
 * (34)-(38) two-scalar LB, (41) isotropic gradient, (42) Laplacian, (48)
 * concentration-dependent viscosity.
 *
 * Readings where the paper is silent (each one is shared with the GPU path
 * only through the written description, never through code):
 *  - d/dt(chi u) is the first-order backward difference (chi u)^n - (chi u)^{n-1};
 *    before the first step the "previous" macros are the initial ones with u = 0.
 *  - n = grad(phi) / (|grad(phi)| + 1e-4).  With a much smaller regulariser, rounding
 *    noise in grad(phi) where it vanishes by symmetry (droplet centres) flips n
 *    to an arbitrary unit vector and the result depends on summation order.
 *  - gradients/Laplacian use the D2Q9 isotropic stencils (Eqs. 41-42) for phi,
 *    c1 and c2 even when h1/h2 live on D2Q5.
 *  - at walls the stencils see mirror ghosts: chi(ghost) = chi(adjacent node).
 *  - the implicit c1, c2 of Eq. (37) are found by the exact 2x2 solve.
 *  - D_m = 0 where its denominator is <= 0.
 *  - body force G = (rho - g_rho_ref) g + (Fx, Fy).
 *  - viscosity model 2: mu = mu_lin(phi) * exp(-beta (c1 + c2)).
 *  - rho (Eq. 6) and the linear mu (Eq. 7) take phi clipped to [0, 1].
 *  - initial populations: f_i = w_i phi, g_i = 0 (p = 0, u = 0),
 *    h_k,i = w_i (c_k - S_k / 2) so that Eq. (37) returns the initial c_k.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattice (Sec. IV: D2Q9 in two dimensions; D2Q5 option for scalars) ---- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double W5[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
static const double CS2 = 1.0 / 3.0;
static const double DT = 1.0;
static const double NORMAL_EPS = 1e-4;

/* index of the velocity opposite to c_i, found by search */
static int opposite(int i) {
    for (int j = 0; j < 9; ++j)
        if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;
    return -1;
}

static const double* scalar_weights(int q) { return q == 5 ? W5 : W9; }

struct orc_sim {
    orc_params p;
    int N;
    double tau_f, tau_h1, tau_h2;
    double *f, *g, *h1, *h2;     /* populations at the current time            */
    double *fc, *gc, *h1c, *h2c; /* post-collision populations                */
    double *phi, *c1, *c2;       /* zeroth moments of the current populations  */
    double *prev;                /* 5*N: phi, ux, uy, c1, c2 of the last step  */
    double *cur;                 /* 5*N: the same macros of the step in flight */
};

/* ---- closed-form relations of the model ---- */

/* Eqs. (27), (38): coefficient = dt (tau - 1/2) cs^2, solved for tau. */
static double tau_from_coefficient(double coeff) { return coeff / (DT * CS2) + 0.5; }

/* material properties are evaluated at phi clipped to [0, 1] (the physical range
 * of the order parameter), so that small overshoots of phi cannot make rho or mu
 * leave [rho2, rho1] / [mu2, mu1] at large property ratios */
static double clip01(double phi) { return phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi); }

/* Eq. (6) */
static double density(const orc_params* p, double phi) {
    return clip01(phi) * (p->rho1 - p->rho2) + p->rho2;
}

/* Eqs. (4)-(5): mu_phi = 4 beta phi (phi - 1)(phi - 1/2) - k lap(phi) */
static double chemical_potential(const orc_params* p, double phi, double lap) {
    double beta = 12.0 * p->sigma / p->W;
    double k = 1.5 * p->sigma * p->W;
    return 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - k * lap;
}

/* Eq. (18); zero where the denominator is not positive */
static double mixed_diffusivity(const orc_params* p, double phi) {
    double den = p->Keq * p->D1 * (1.0 - phi) + p->D2 * phi;
    if (!(den > 0.0)) return 0.0;
    return p->D1 * p->D2 / den;
}

/* interfacial exchange term A D_m [K c2 phi - c1 (1 - phi)] of Eq. (17a) */
static double exchange_source(const orc_params* p, double phi, double c1, double c2) {
    return p->A * mixed_diffusivity(p, phi) * (p->Keq * c2 * phi - c1 * (1.0 - phi));
}

/* One-scalar model (Eq. 31 and the two relations after it), with phi clipped
 * to [0, 1]: K_eff = K phi + (1 - phi), D_eff = D1 K phi + D2 (1 - phi). */
static double k_eff(const orc_params* p, double phi) {
    const double ph = clip01(phi);
    return p->Keq * ph + (1.0 - ph);
}
static double d_eff(const orc_params* p, double phi) {
    const double ph = clip01(phi);
    return p->D1 * p->Keq * ph + p->D2 * (1.0 - ph);
}
/* c split between the phases at the Henry equilibrium c1/phi = K c2/(1 - phi)
 * (c1 = K phi c / K_eff, c2 = (1 - phi) c / K_eff): how the one-scalar model
 * reports c1 and c2 and feeds the viscosity relations. */
static void henry_split(const orc_params* p, double phi, double c, double* c1, double* c2) {
    const double ph = clip01(phi), ke = k_eff(p, phi);
    *c1 = p->Keq * ph * c / ke;
    *c2 = (1.0 - ph) * c / ke;
}

/* Eq. (7), Eq. (48), or the exponential scalar relation */
static double viscosity(const orc_params* p, double phi, double c1, double c2) {
    double mu_lin = clip01(phi) * (p->mu1 - p->mu2) + p->mu2;
    if (p->visc_model == 1) return exp(c1 * log(p->mu1) + c2 * log(p->mu2));
    if (p->visc_model == 2) return mu_lin * exp(-p->visc_beta * (c1 + c2));
    return mu_lin;
}

/* Eq. (37) written as a linear system in (c1, c2) and solved exactly:
 *   c1 = P1 + (dt/2) A D_m [K c2 phi - c1 (1 - phi)]
 *   c2 = P2 + (dt/2) A D_m [c1 (1 - phi) - K c2 phi]                       */
static void solve_scalars(const orc_params* p, double phi, double P1, double P2,
                          double* c1, double* c2) {
    double a = 0.5 * DT * p->A * mixed_diffusivity(p, phi);
    /* [1 + a(1-phi)   -a K phi    ] [c1]   [P1]
       [-a(1-phi)      1 + a K phi ] [c2] = [P2]                            */
    double m11 = 1.0 + a * (1.0 - phi), m12 = -a * p->Keq * phi;
    double m21 = -a * (1.0 - phi), m22 = 1.0 + a * p->Keq * phi;
    double det = m11 * m22 - m12 * m21;
    *c1 = (P1 * m22 - m12 * P2) / det;
    *c2 = (m11 * P2 - m21 * P1) / det;
}

/* ---- per-cell discrete functions: Eqs. (24), (25), (29)-(31), (35), (36) ---- */

typedef struct {
    double phi, ux, uy, p, c1, c2;
    double dphix, dphiy, lap;
    double dc1x, dc1y, dc2x, dc2y;
    double dtpux, dtpuy, dtc1ux, dtc1uy, dtc2ux, dtc2uy;
} cell_in;

typedef struct {
    double feq[9], F[9], geq[9], G[9];
    double h1eq[9], h2eq[9], H1[9], H2[9], Ht1[9], Ht2[9];
} cell_out;

static void body_force(const orc_params* p, double rho, double* Gx, double* Gy) {
    *Gx = (rho - p->g_rho_ref) * p->gx + p->Fx;
    *Gy = (rho - p->g_rho_ref) * p->gy + p->Fy;
}

static void discrete_functions(const orc_params* p, const cell_in* c, cell_out* o) {
    const double phi = c->phi, ux = c->ux, uy = c->uy;
    const double rho = density(p, phi);
    const double mu_phi = chemical_potential(p, phi, c->lap);
    double Gx, Gy;
    body_force(p, rho, &Gx, &Gy);
    /* total force mu_phi grad(phi) + G (Eq. 3b) */
    const double Ftx = mu_phi * c->dphix + Gx, Fty = mu_phi * c->dphiy + Gy;
    /* unit normal n = grad(phi)/|grad(phi)| (Eq. 1) */
    const double gnorm = sqrt(c->dphix * c->dphix + c->dphiy * c->dphiy);
    const double nx = c->dphix / (gnorm + NORMAL_EPS), ny = c->dphiy / (gnorm + NORMAL_EPS);
    const double Dm = mixed_diffusivity(p, phi);
    const double S1 = exchange_source(p, phi, c->c1, c->c2);
    /* grad(phi) . grad(c1 + K c2) */
    const double flux = c->dphix * (c->dc1x + p->Keq * c->dc2x) + c->dphiy * (c->dc1y + p->Keq * c->dc2y);
    const double uu = ux * ux + uy * uy;

    memset(o, 0, sizeof(*o));
    for (int i = 0; i < 9; ++i) {
        const double w = W9[i];
        const double cu = CX[i] * ux + CY[i] * uy;
        /* Eq. (24) */
        o->feq[i] = w * phi * (1.0 + cu / CS2);
        /* Eq. (25) */
        o->F[i] = w * ((CX[i] * c->dtpux + CY[i] * c->dtpuy) / CS2
                       + (CX[i] * nx + CY[i] * ny) * 4.0 * phi * (1.0 - phi) / p->W);
        /* Eqs. (29)-(30) */
        const double s = w * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
        o->geq[i] = (i == 0 ? c->p / CS2 * (w - 1.0) : c->p / CS2 * w) + rho * s;
        /* Eq. (31): u grad(phi) : c_i c_i = (c_i . u)(c_i . grad(phi)) */
        const double cg = CX[i] * c->dphix + CY[i] * c->dphiy;
        o->G[i] = w * ((CX[i] * Ftx + CY[i] * Fty) / CS2 + (p->rho1 - p->rho2) * cu * cg / CS2);
    }
    const double* ws = scalar_weights(p->scalar_q);
    for (int i = 0; i < p->scalar_q; ++i) {
        const double w = ws[i];
        const double cu = CX[i] * ux + CY[i] * uy;
        const double cn = CX[i] * nx + CY[i] * ny;
        /* Eq. (35) */
        o->h1eq[i] = w * c->c1 * (1.0 + cu / CS2);
        o->h2eq[i] = w * c->c2 * (1.0 + cu / CS2);
        /* Eq. (36a)-(36b) */
        o->H1[i] = w * ((CX[i] * c->dtc1ux + CY[i] * c->dtc1uy) / CS2
                        + cn * 4.0 * (1.0 - phi) * c->c1 / p->W + S1);
        o->H2[i] = w * ((CX[i] * c->dtc2ux + CY[i] * c->dtc2uy) / CS2
                        - cn * 4.0 * phi * c->c2 / p->W - S1);
        /* Eq. (36c)-(36d) */
        o->Ht1[i] = -w * Dm * flux;
        o->Ht2[i] = w * Dm * flux;
    }
}

/* ---- neighbours: periodic wrap, or mirror ghost at a wall ---- */
static int neighbour_coord(int v, int n, int wall) {
    if (wall) return v < 0 ? 0 : (v >= n ? n - 1 : v);
    return ((v % n) + n) % n;
}

static double field_at(const orc_sim* s, const double* fld, int x, int y) {
    int xx = neighbour_coord(x, s->p.nx, s->p.wall_x);
    int yy = neighbour_coord(y, s->p.ny, s->p.wall_y);
    return fld[yy * s->p.nx + xx];
}

/* Eq. (41): grad chi = sum_{i!=0} w_i c_i chi(x + c_i dt) / (cs^2 dt) */
static void gradient(const orc_sim* s, const double* fld, int x, int y, double* gx, double* gy) {
    double ax = 0.0, ay = 0.0;
    for (int i = 1; i < 9; ++i) {
        double v = field_at(s, fld, x + CX[i], y + CY[i]);
        ax += W9[i] * CX[i] * v;
        ay += W9[i] * CY[i] * v;
    }
    *gx = ax / (CS2 * DT);
    *gy = ay / (CS2 * DT);
}

/* Eq. (42): lap phi = sum_{i!=0} 2 w_i [phi(x + c_i dt) - phi(x)] / (cs^2 dt^2) */
static double laplacian(const orc_sim* s, const double* fld, int x, int y) {
    double c = field_at(s, fld, x, y), a = 0.0;
    for (int i = 1; i < 9; ++i) a += 2.0 * W9[i] * (field_at(s, fld, x + CX[i], y + CY[i]) - c);
    return a / (CS2 * DT * DT);
}

/* ---- stage 1: zeroth moments phi (Eq. 26) and c1, c2 (Eq. 37) ---- */
static void zeroth_moments(orc_sim* s) {
    const int N = s->N, qs = s->p.scalar_q;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < N; ++k) {
        double phi = 0.0, P1 = 0.0, P2 = 0.0;
        for (int i = 0; i < 9; ++i) phi += s->f[i * N + k];
        for (int i = 0; i < qs; ++i) {
            P1 += s->h1[i * N + k];
            P2 += s->h2[i * N + k];
        }
        s->phi[k] = phi;
        if (s->p.scalar_model == 1)
            henry_split(&s->p, phi, P1, &s->c1[k], &s->c2[k]);  /* c = sum_i h3_i */
        else
            solve_scalars(&s->p, phi, P1, P2, &s->c1[k], &s->c2[k]);
    }
}

/* ---- stage 2: stencils, force, velocity, pressure, viscosity of one cell ---- */
typedef struct {
    cell_in in;
    double rho, mu, tau_g;
} cell_macros;

/* Local grad phi (the scheme given after Eq. 39): with D = -tau_f cs^2 dt,
 * B = 4 M dt phi (1 - phi) / W and C = sum_i c_i f_i - phi u + dt/2 d_t(phi u),
 * |grad phi| = (-|C| - B) / D and grad phi = C / (D + B / |grad phi|), which
 * simplifies to grad phi = -C (|C| + B) / (tau_f cs^2 dt |C|) (0 where C = 0).
 * Reading: u is not known before grad phi (the surface force needs it), so C
 * uses the previous step's velocity: phi u - dt/2 d_t(phi u) becomes
 * (phi + phi_prev) u_prev / 2 with the backward difference of d_t. */
static void local_phi_gradient(const orc_sim* s, int k, double phi, double* gx, double* gy) {
    const orc_params* p = &s->p;
    const int N = s->N;
    double mx = 0.0, my = 0.0;
    for (int i = 0; i < 9; ++i) {
        mx += CX[i] * s->f[i * N + k];
        my += CY[i] * s->f[i * N + k];
    }
    const double php = s->prev[0 * N + k], uxp = s->prev[1 * N + k], uyp = s->prev[2 * N + k];
    const double Cx = mx - 0.5 * (phi + php) * uxp, Cy = my - 0.5 * (phi + php) * uyp;
    const double B = 4.0 * p->M * DT * phi * (1.0 - phi) / p->W;
    const double Cn = sqrt(Cx * Cx + Cy * Cy);
    if (!(Cn > 0.0)) { *gx = 0.0; *gy = 0.0; return; }
    const double a = -(Cn + B) / (s->tau_f * CS2 * DT * Cn);
    *gx = a * Cx;
    *gy = a * Cy;
}

/* Local grad c1, grad c2 (Eq. 39) from the first moments of h1, h2, once u and
 * the time derivatives are known; n = grad phi / (|grad phi| + eps) as in the
 * collision. */
static void local_scalar_gradients(const orc_sim* s, int k, cell_in* c) {
    const orc_params* p = &s->p;
    const int N = s->N, qs = p->scalar_q;
    double m1x = 0.0, m1y = 0.0, m2x = 0.0, m2y = 0.0;
    for (int i = 0; i < qs; ++i) {
        m1x += CX[i] * s->h1[i * N + k];
        m1y += CY[i] * s->h1[i * N + k];
        m2x += CX[i] * s->h2[i * N + k];
        m2y += CY[i] * s->h2[i * N + k];
    }
    const double gn = sqrt(c->dphix * c->dphix + c->dphiy * c->dphiy);
    const double nx = c->dphix / (gn + NORMAL_EPS), ny = c->dphiy / (gn + NORMAL_EPS);
    const double s1 = p->D1 * 4.0 * (1.0 - c->phi) * c->c1 / p->W;
    const double s2 = p->D2 * 4.0 * c->phi * c->c2 / p->W;
    const double d1 = s->tau_h1 * DT * CS2, d2 = s->tau_h2 * DT * CS2;
    c->dc1x = (-m1x + c->c1 * c->ux - 0.5 * DT * c->dtc1ux + s1 * nx) / d1;
    c->dc1y = (-m1y + c->c1 * c->uy - 0.5 * DT * c->dtc1uy + s1 * ny) / d1;
    c->dc2x = (-m2x + c->c2 * c->ux - 0.5 * DT * c->dtc2ux - s2 * nx) / d2;
    c->dc2y = (-m2y + c->c2 * c->uy - 0.5 * DT * c->dtc2uy - s2 * ny) / d2;
}

static void macros_of_cell(const orc_sim* s, int x, int y, cell_macros* m) {
    const orc_params* p = &s->p;
    const int N = s->N, k = y * p->nx + x;
    cell_in* c = &m->in;
    memset(m, 0, sizeof(*m));
    c->phi = s->phi[k];
    c->c1 = s->c1[k];
    c->c2 = s->c2[k];
    if (p->grad_scheme == 2)
        local_phi_gradient(s, k, c->phi, &c->dphix, &c->dphiy);
    else
        gradient(s, s->phi, x, y, &c->dphix, &c->dphiy);
    c->lap = laplacian(s, s->phi, x, y);
    gradient(s, s->c1, x, y, &c->dc1x, &c->dc1y);
    gradient(s, s->c2, x, y, &c->dc2x, &c->dc2y);

    m->rho = density(p, c->phi);
    const double mu_phi = chemical_potential(p, c->phi, c->lap);
    double Gx, Gy;
    body_force(p, m->rho, &Gx, &Gy);
    const double Ftx = mu_phi * c->dphix + Gx, Fty = mu_phi * c->dphiy + Gy;

    /* Eq. (32a): u = [sum_i c_i g_i + dt/2 (mu_phi grad phi + G)] / rho */
    double jx = 0.0, jy = 0.0, gsum = 0.0;
    for (int i = 0; i < 9; ++i) {
        jx += CX[i] * s->g[i * N + k];
        jy += CY[i] * s->g[i * N + k];
        if (i != 0) gsum += s->g[i * N + k];
    }
    c->ux = (jx + 0.5 * DT * Ftx) / m->rho;
    c->uy = (jy + 0.5 * DT * Fty) / m->rho;

    /* Eq. (32b): p = cs^2/(1-w0) [sum_{i!=0} g_i + dt/2 (rho1-rho2) u.grad phi + rho s_0(u)] */
    const double uu = c->ux * c->ux + c->uy * c->uy;
    const double s0 = W9[0] * (-uu / (2.0 * CS2));
    c->p = CS2 / (1.0 - W9[0])
           * (gsum + 0.5 * DT * (p->rho1 - p->rho2) * (c->ux * c->dphix + c->uy * c->dphiy) + m->rho * s0);

    /* Eq. (33) solved for tau_g with the cell's viscosity */
    m->mu = viscosity(p, c->phi, c->c1, c->c2);
    m->tau_g = tau_from_coefficient(m->mu / m->rho);
}

/* ---- stage 3 for the one-scalar model: f and g as in the two-scalar model,
 * one lattice h3 for c (Sec. III D):
 *   h3_0^eq = c + (w_0 - 1) c / K_eff,  h3_i^eq = w_i c / K_eff + w_i c_i.(c u) / cs^2,
 *   H3_i = w_i c_i . d_t(c u) / cs^2,  tau_h3 = D_eff / (cs^2 dt) + 1/2 (per cell).
 * The previous-step slot of c1 holds c, the slot of c2 holds 0. */
static void collide_cell_one_scalar(orc_sim* s, int k, cell_macros* m, double phip, double uxp,
                                    double uyp, double cp) {
    const orc_params* p = &s->p;
    const int N = s->N, qs = p->scalar_q;
    cell_in* c = &m->in;
    const double ct = c->c1 + c->c2;  /* c = sum_i h3_i */
    c->dtpux = (c->phi * c->ux - phip * uxp) / DT;
    c->dtpuy = (c->phi * c->uy - phip * uyp) / DT;
    const double dtcux = (ct * c->ux - cp * uxp) / DT, dtcuy = (ct * c->uy - cp * uyp) / DT;

    double* cu = s->cur;
    cu[0 * N + k] = c->phi;
    cu[1 * N + k] = c->ux;
    cu[2 * N + k] = c->uy;
    cu[3 * N + k] = ct;
    cu[4 * N + k] = 0.0;

    cell_out o;
    discrete_functions(p, c, &o);
    for (int i = 0; i < 9; ++i) {
        const double fi = s->f[i * N + k], gi = s->g[i * N + k];
        s->fc[i * N + k] = fi - (fi - o.feq[i]) / s->tau_f + DT * (1.0 - 0.5 / s->tau_f) * o.F[i];
        s->gc[i * N + k] = gi - (gi - o.geq[i]) / m->tau_g + DT * (1.0 - 0.5 / m->tau_g) * o.G[i];
    }
    const double* ws = scalar_weights(qs);
    const double ke = k_eff(p, c->phi), tau3 = tau_from_coefficient(d_eff(p, c->phi));
    for (int i = 0; i < qs; ++i) {
        const double cuv = CX[i] * c->ux + CY[i] * c->uy;
        const double eq = (i == 0 ? ct + (ws[0] - 1.0) * ct / ke : ws[i] * ct / ke) + ws[i] * cuv * ct / CS2;
        const double H3 = ws[i] * (CX[i] * dtcux + CY[i] * dtcuy) / CS2;
        const double a = s->h1[i * N + k];
        s->h1c[i * N + k] = a - (a - eq) / tau3 + DT * (1.0 - 0.5 / tau3) * H3;
        s->h2c[i * N + k] = 0.0;
    }
}

/* ---- stage 3: BGK collision (Eqs. 23, 28, 34) ---- */
static void collide_cell(orc_sim* s, int x, int y) {
    const orc_params* p = &s->p;
    const int N = s->N, k = y * p->nx + x, qs = p->scalar_q;
    cell_macros m;
    macros_of_cell(s, x, y, &m);
    cell_in* c = &m.in;

    /* backward time differences against the previous step's macros */
    const double* pv = s->prev;
    const double phip = pv[0 * N + k], uxp = pv[1 * N + k], uyp = pv[2 * N + k];
    const double c1p = pv[3 * N + k], c2p = pv[4 * N + k];
    if (p->scalar_model == 1) {
        collide_cell_one_scalar(s, k, &m, phip, uxp, uyp, c1p);
        return;
    }
    c->dtpux = (c->phi * c->ux - phip * uxp) / DT;
    c->dtpuy = (c->phi * c->uy - phip * uyp) / DT;
    c->dtc1ux = (c->c1 * c->ux - c1p * uxp) / DT;
    c->dtc1uy = (c->c1 * c->uy - c1p * uyp) / DT;
    c->dtc2ux = (c->c2 * c->ux - c2p * uxp) / DT;
    c->dtc2uy = (c->c2 * c->uy - c2p * uyp) / DT;
    if (p->grad_scheme >= 1) local_scalar_gradients(s, k, c);

    double* cu = s->cur;
    cu[0 * N + k] = c->phi;
    cu[1 * N + k] = c->ux;
    cu[2 * N + k] = c->uy;
    cu[3 * N + k] = c->c1;
    cu[4 * N + k] = c->c2;

    cell_out o;
    discrete_functions(p, c, &o);

    for (int i = 0; i < 9; ++i) {
        const double fi = s->f[i * N + k], gi = s->g[i * N + k];
        s->fc[i * N + k] = fi - (fi - o.feq[i]) / s->tau_f + DT * (1.0 - 0.5 / s->tau_f) * o.F[i];
        s->gc[i * N + k] = gi - (gi - o.geq[i]) / m.tau_g + DT * (1.0 - 0.5 / m.tau_g) * o.G[i];
    }
    for (int i = 0; i < qs; ++i) {
        const double a = s->h1[i * N + k], b = s->h2[i * N + k];
        s->h1c[i * N + k] = a - (a - o.h1eq[i]) / s->tau_h1 + DT * (1.0 - 0.5 / s->tau_h1) * o.H1[i]
                            + DT * o.Ht1[i];
        s->h2c[i * N + k] = b - (b - o.h2eq[i]) / s->tau_h2 + DT * (1.0 - 0.5 / s->tau_h2) * o.H2[i]
                            + DT * o.Ht2[i];
    }
}

/* ---- stage 4: push streaming with half-way bounce-back (Sec. IV) ---- */
static void stream_lattice(orc_sim* s, const double* post, double* dst, int q) {
    const orc_params* p = &s->p;
    const int N = s->N;
    /* every (direction, destination) entry is written by exactly one source node */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const int k = y * p->nx + x;
            for (int i = 0; i < q; ++i) {
                int tx = x + CX[i], ty = y + CY[i];
                int out_x = tx < 0 || tx >= p->nx, out_y = ty < 0 || ty >= p->ny;
                if ((out_x && p->wall_x) || (out_y && p->wall_y)) {
                    /* reflected back into the node it left, opposite direction */
                    dst[opposite(i) * N + k] = post[i * N + k];
                } else {
                    tx = neighbour_coord(tx, p->nx, 0);
                    ty = neighbour_coord(ty, p->ny, 0);
                    dst[i * N + ty * p->nx + tx] = post[i * N + k];
                }
            }
        }
}

/* ---- public API ---- */

orc_sim* orc_create(const orc_params* p) {
    if (!p || p->nx < 1 || p->ny < 1) return NULL;
    if (p->scalar_q != 5 && p->scalar_q != 9) return NULL;
    if (!(p->W > 0) || !(p->M > 0) || !(p->D1 > 0) || !(p->D2 > 0)) return NULL;
    if (!(p->rho1 > 0) || !(p->rho2 > 0) || !(p->mu1 > 0) || !(p->mu2 > 0)) return NULL;
    if (!(p->Keq > 0) || !(p->A >= 0) || !(p->sigma >= 0)) return NULL;
    if (p->visc_model < 0 || p->visc_model > 2) return NULL;
    if (p->scalar_model != 0 && p->scalar_model != 1) return NULL;
    if (p->grad_scheme < 0 || p->grad_scheme > 2) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    s->N = p->nx * p->ny;
    s->tau_f = tau_from_coefficient(p->M);
    s->tau_h1 = tau_from_coefficient(p->D1);
    s->tau_h2 = tau_from_coefficient(p->D2);
    const size_t N = (size_t)s->N;
    s->f = calloc(9 * N, sizeof(double));
    s->g = calloc(9 * N, sizeof(double));
    s->h1 = calloc(9 * N, sizeof(double));
    s->h2 = calloc(9 * N, sizeof(double));
    s->fc = calloc(9 * N, sizeof(double));
    s->gc = calloc(9 * N, sizeof(double));
    s->h1c = calloc(9 * N, sizeof(double));
    s->h2c = calloc(9 * N, sizeof(double));
    s->phi = calloc(N, sizeof(double));
    s->c1 = calloc(N, sizeof(double));
    s->c2 = calloc(N, sizeof(double));
    s->prev = calloc(5 * N, sizeof(double));
    s->cur = calloc(5 * N, sizeof(double));
    if (!s->cur || !s->f || !s->g || !s->h1 || !s->h2 || !s->fc || !s->gc || !s->h1c || !s->h2c || !s->phi
        || !s->c1 || !s->c2 || !s->prev) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f); free(s->g); free(s->h1); free(s->h2);
    free(s->fc); free(s->gc); free(s->h1c); free(s->h2c);
    free(s->phi); free(s->c1); free(s->c2); free(s->prev); free(s->cur);
    free(s);
}

void orc_init_fields(orc_sim* s, const double* phi, const double* c1, const double* c2) {
    const orc_params* p = &s->p;
    const int N = s->N, qs = p->scalar_q;
    const double* ws = scalar_weights(qs);
    memset(s->g, 0, 9 * (size_t)N * sizeof(double));
    memset(s->h1, 0, 9 * (size_t)N * sizeof(double));
    memset(s->h2, 0, 9 * (size_t)N * sizeof(double));
    for (int k = 0; k < N; ++k) {
        for (int i = 0; i < 9; ++i) s->f[i * N + k] = W9[i] * phi[k];
        s->prev[0 * N + k] = phi[k];
        s->prev[1 * N + k] = 0.0;
        s->prev[2 * N + k] = 0.0;
        if (p->scalar_model == 1) {
            /* h3 at its equilibrium for c = c1 + c2 (u = 0) */
            const double c = c1[k] + c2[k], ke = k_eff(p, phi[k]);
            for (int i = 0; i < qs; ++i) s->h1[i * N + k] = i == 0 ? c + (ws[0] - 1.0) * c / ke : ws[i] * c / ke;
            s->prev[3 * N + k] = c;
            s->prev[4 * N + k] = 0.0;
            continue;
        }
        /* S_1 at the initial state; h sums to c - dt S/2, so Eq. (37) returns c */
        const double S1 = exchange_source(p, phi[k], c1[k], c2[k]);
        for (int i = 0; i < qs; ++i) {
            s->h1[i * N + k] = ws[i] * (c1[k] - 0.5 * DT * S1);
            s->h2[i * N + k] = ws[i] * (c2[k] + 0.5 * DT * S1);
        }
        s->prev[3 * N + k] = c1[k];
        s->prev[4 * N + k] = c2[k];
    }
}

/* Restart from all six macros: populations at the equilibria of Eqs. (24),
 * (29)-(30) and (35) evaluated with the given phi, u, p, c1, c2; h shifted by
 * -/+ w_i dt S_1/2 so that Eq. (37) returns c1, c2 (as in orc_init_fields). */
void orc_init_macros(orc_sim* s, const double* phi, const double* ux, const double* uy,
                     const double* pr, const double* c1, const double* c2) {
    const orc_params* p = &s->p;
    const int N = s->N, qs = p->scalar_q;
    const double* ws = scalar_weights(qs);
    memset(s->h1, 0, 9 * (size_t)N * sizeof(double));
    memset(s->h2, 0, 9 * (size_t)N * sizeof(double));
    for (int k = 0; k < N; ++k) {
        cell_in c;
        cell_out o;
        memset(&c, 0, sizeof(c));
        c.phi = phi[k]; c.ux = ux[k]; c.uy = uy[k]; c.p = pr[k]; c.c1 = c1[k]; c.c2 = c2[k];
        discrete_functions(p, &c, &o);
        const double S1 = exchange_source(p, phi[k], c1[k], c2[k]);
        for (int i = 0; i < 9; ++i) {
            s->f[i * N + k] = o.feq[i];
            s->g[i * N + k] = o.geq[i];
        }
        s->prev[0 * N + k] = phi[k];
        s->prev[1 * N + k] = ux[k];
        s->prev[2 * N + k] = uy[k];
        if (p->scalar_model == 1) {
            const double c = c1[k] + c2[k], ke = k_eff(p, phi[k]);
            for (int i = 0; i < qs; ++i) {
                const double cuv = CX[i] * ux[k] + CY[i] * uy[k];
                s->h1[i * N + k] = (i == 0 ? c + (ws[0] - 1.0) * c / ke : ws[i] * c / ke) + ws[i] * cuv * c / CS2;
            }
            s->prev[3 * N + k] = c;
            s->prev[4 * N + k] = 0.0;
            continue;
        }
        for (int i = 0; i < qs; ++i) {
            s->h1[i * N + k] = o.h1eq[i] - ws[i] * 0.5 * DT * S1;
            s->h2[i * N + k] = o.h2eq[i] + ws[i] * 0.5 * DT * S1;
        }
        s->prev[3 * N + k] = c1[k];
        s->prev[4 * N + k] = c2[k];
    }
}

void orc_init(orc_sim* s, const double* sdf, double c1t, double c2t) {
    const int N = s->N;
    double* phi = malloc((size_t)N * sizeof(double));
    double* c1 = malloc((size_t)N * sizeof(double));
    double* c2 = malloc((size_t)N * sizeof(double));
    for (int k = 0; k < N; ++k) {
        /* Eq. (2) */
        phi[k] = 0.5 + 0.5 * tanh(2.0 * sdf[k] / s->p.W);
        c1[k] = c1t * phi[k];
        c2[k] = c2t * (1.0 - phi[k]);
    }
    orc_init_fields(s, phi, c1, c2);
    free(phi); free(c1); free(c2);
}

void orc_step(orc_sim* s, long nsteps) {
    const orc_params* p = &s->p;
    const int N = s->N;
    for (long n = 0; n < nsteps; ++n) {
        zeroth_moments(s);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) collide_cell(s, x, y);
        /* the previous-step macros are replaced only after every cell has collided */
        memcpy(s->prev, s->cur, 5 * (size_t)N * sizeof(double));
        stream_lattice(s, s->fc, s->f, 9);
        stream_lattice(s, s->gc, s->g, 9);
        stream_lattice(s, s->h1c, s->h1, p->scalar_q);
        stream_lattice(s, s->h2c, s->h2, p->scalar_q);
    }
}

void orc_get_fields(orc_sim* s, double* out) {
    const orc_params* p = &s->p;
    const int N = s->N;
    zeroth_moments(s);
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            cell_macros m;
            macros_of_cell(s, x, y, &m);
            const int k = y * p->nx + x;
            out[ORC_PHI * N + k] = m.in.phi;
            out[ORC_UX * N + k] = m.in.ux;
            out[ORC_UY * N + k] = m.in.uy;
            out[ORC_P * N + k] = m.in.p;
            out[ORC_C1 * N + k] = m.in.c1;
            out[ORC_C2 * N + k] = m.in.c2;
            out[ORC_RHO * N + k] = m.rho;
            out[ORC_MU * N + k] = m.mu;
        }
}

void orc_get_stencils(orc_sim* s, double* out) {
    const orc_params* p = &s->p;
    const int N = s->N;
    zeroth_moments(s);
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            cell_macros m;
            macros_of_cell(s, x, y, &m);
            const int k = y * p->nx + x;
            if (p->grad_scheme >= 1 && p->scalar_model == 0) {
                /* the time derivatives the collision would use */
                cell_in* c = &m.in;
                const double* pv = s->prev;
                c->dtc1ux = (c->c1 * c->ux - pv[3 * N + k] * pv[1 * N + k]) / DT;
                c->dtc1uy = (c->c1 * c->uy - pv[3 * N + k] * pv[2 * N + k]) / DT;
                c->dtc2ux = (c->c2 * c->ux - pv[4 * N + k] * pv[1 * N + k]) / DT;
                c->dtc2uy = (c->c2 * c->uy - pv[4 * N + k] * pv[2 * N + k]) / DT;
                local_scalar_gradients(s, k, c);
            }
            out[0 * N + k] = m.in.dphix;
            out[1 * N + k] = m.in.dphiy;
            out[2 * N + k] = m.in.lap;
            out[3 * N + k] = m.in.dc1x;
            out[4 * N + k] = m.in.dc1y;
            out[5 * N + k] = m.in.dc2x;
            out[6 * N + k] = m.in.dc2y;
        }
}

void orc_conserved(orc_sim* s, double out[2]) {
    zeroth_moments(s);
    double a = 0.0, b = 0.0;
    for (int k = 0; k < s->N; ++k) {
        a += s->phi[k];
        b += s->c1[k] + s->c2[k];
    }
    out[0] = a;
    out[1] = b;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n < 1 ? 1 : n);
#else
    (void)n;
#endif
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_taus(const orc_sim* s, double out[3]) {
    out[0] = s->tau_f;
    out[1] = s->tau_h1;
    out[2] = s->tau_h2;
}

void orc_cell_functions(const orc_params* p, const double* in, double* out) {
    cell_in c;
    c.phi = in[0]; c.ux = in[1]; c.uy = in[2]; c.p = in[3]; c.c1 = in[4]; c.c2 = in[5];
    c.dphix = in[6]; c.dphiy = in[7]; c.lap = in[8];
    c.dc1x = in[9]; c.dc1y = in[10]; c.dc2x = in[11]; c.dc2y = in[12];
    c.dtpux = in[13]; c.dtpuy = in[14]; c.dtc1ux = in[15]; c.dtc1uy = in[16];
    c.dtc2ux = in[17]; c.dtc2uy = in[18];
    cell_out o;
    discrete_functions(p, &c, &o);
    const double* blocks[10] = {o.feq, o.F, o.geq, o.G, o.h1eq, o.h2eq, o.H1, o.H2, o.Ht1, o.Ht2};
    for (int b = 0; b < 10; ++b) memcpy(out + 9 * b, blocks[b], 9 * sizeof(double));
}

void orc_solve_scalars(const orc_params* p, const double* in, double* out) {
    solve_scalars(p, in[0], in[1], in[2], &out[0], &out[1]);
}
