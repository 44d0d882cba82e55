/*
 * FP64 CPU oracle for the phase-field lattice Boltzmann method with
 * interfacial mass/heat transfer (Chen, Zhan, Chai & Shi, arXiv 2402.15752).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct restatement of the paper's time step that the GPU path is checked
 * against.  Only the test suite, the package's smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library.
 *
 * Units: lattice units, dx = dt = 1, cs^2 = 1/3.
 * Layout of every field: row-major, index = y * nx + x.
 */
#ifndef PFLBM_ORACLE_H
#define PFLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Physical parameters, as the paper states the problem (Sec. II, Sec. III). */
typedef struct {
    int nx, ny;
    int wall_x, wall_y;   /* 0: periodic, 1: half-way bounce-back walls     */
    int scalar_q;         /* 5 (D2Q5) or 9 (D2Q9) for the h1/h2 lattices     */
    double W, M, sigma;   /* interface width, mobility, surface tension     */
    double rho1, rho2;    /* densities of fluid 1 (phi=1) and fluid 2        */
    double mu1, mu2;      /* dynamic viscosities                             */
    double D1, D2;        /* scalar diffusivities                            */
    double Keq, A;        /* equilibrium jump K_eq, inverse time scale A     */
    double gx, gy;        /* acceleration: G += (rho - g_rho_ref) * g       */
    double g_rho_ref;
    double Fx, Fy;        /* constant body-force density: G += (Fx, Fy)     */
    int visc_model;       /* 0: linear in phi, 1: log mu = c1 log mu1 + c2 log mu2,
                             2: mu = mu_lin(phi) * exp(-visc_beta * (c1 + c2)) */
    double visc_beta;
    int scalar_model;     /* 0: two-scalar lattices h1, h2 (Sec. III C);
                             1: one-scalar lattice h3 for c = c1 + c2 (Sec. III D);
                             c1, c2 are then reported as the Henry split of c */
    int grad_scheme;      /* 0: grad phi, grad c1, grad c2 by the stencil of Eq. (41);
                             1: grad c1, grad c2 by the local scheme of Eq. (39);
                             2: also grad phi and |grad phi| by the local scheme
                                (Sec. III C, after Eq. 39); lap phi always Eq. (42) */
} orc_params;

typedef struct orc_sim orc_sim;

/* Output field indices for orc_get_fields (each field nx*ny doubles). */
enum { ORC_PHI = 0, ORC_UX, ORC_UY, ORC_P, ORC_C1, ORC_C2, ORC_RHO, ORC_MU, ORC_NFIELDS };

/* Returns NULL on invalid parameters (any relaxation time <= 1/2, etc.). */
orc_sim* orc_create(const orc_params* p);
void     orc_destroy(orc_sim* s);
/* phi from the signed distance (Eq. 2), c1 = c1t*phi, c2 = c2t*(1-phi). */
void     orc_init(orc_sim* s, const double* sdf, double c1t, double c2t);
/* General initial macros; u = 0, p = 0. */
void     orc_init_fields(orc_sim* s, const double* phi, const double* c1, const double* c2);
/* Restart from all six macros: populations at their equilibria (Eqs. 24, 29-30,
 * 35) for the given phi, u, p, c1, c2, h shifted by -/+ w_i S_1/2. */
void     orc_init_macros(orc_sim* s, const double* phi, const double* ux, const double* uy,
                         const double* p, const double* c1, const double* c2);
void     orc_step(orc_sim* s, long nsteps);
/* out: ORC_NFIELDS * nx * ny doubles, field-major. */
void     orc_get_fields(orc_sim* s, double* out);
/* Stencil values of the current state (Eqs. 41-42), 7 fields of nx*ny:
 * dphi_x, dphi_y, lap phi, dc1_x, dc1_y, dc2_x, dc2_y. */
void     orc_get_stencils(orc_sim* s, double* out);
/* {sum phi, sum (c1 + c2)} of the current state. */
void     orc_conserved(orc_sim* s, double out[2]);
/* Host threads of the per-node loops (1 = serial; results do not depend on it).
 * orc_threads() reports the current number (1 in a build without OpenMP). */
void     orc_set_threads(int n);
int      orc_threads(void);
/* Relaxation times {tau_f, tau_h1, tau_h2}. */
void     orc_taus(const orc_sim* s, double out[3]);

/*
 * Per-cell discrete functions for moment tests.  in[] holds
 *  0 phi, 1 ux, 2 uy, 3 p, 4 c1, 5 c2, 6 dphi_x, 7 dphi_y, 8 lap_phi,
 *  9 dc1_x, 10 dc1_y, 11 dc2_x, 12 dc2_y, 13 dt(phi ux), 14 dt(phi uy),
 *  15 dt(c1 ux), 16 dt(c1 uy), 17 dt(c2 ux), 18 dt(c2 uy)
 * out[] receives, each padded to 9 entries:
 *  feq, F, geq, G, h1eq, h2eq, H1, H2, Ht1, Ht2   (10 * 9 doubles)
 */
void     orc_cell_functions(const orc_params* p, const double* in, double* out);
/* 2x2 implicit scalar solve (Eq. 37): in {phi, P1, P2} -> out {c1, c2}. */
void     orc_solve_scalars(const orc_params* p, const double* in, double* out);

#ifdef __cplusplus
}
#endif
#endif
