/*
 * cdugks_oracle.h -- interface of the plain FP64 CPU oracle of the CDUGKS
 * step (arXiv:2208.09132, Sec. 2 and Sec. 2.1).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  The GPU library shares nothing with it.
 */
#ifndef CDUGKS_ORACLE_H
#define CDUGKS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_BC_PERIODIC 0
#define ORACLE_BC_SPECULAR 1
#define ORACLE_BC_DIRICHLET 2
#define ORACLE_MAX_NV1 4096

typedef struct {
    int D;                 /* spatial (= velocity) dimensions, 1..3 */
    int n[3];              /* cells per axis */
    double lo[3], hi[3];   /* domain per axis */
    int bc[3][2];          /* ORACLE_BC_* per axis, low/high side */
    int nv[3];             /* velocity nodes per axis */
    double vlo[3], vhi[3]; /* velocity range per axis (nodes include both ends) */
    int rule;              /* 0 trapezoid, 1 Boole (n = 4m+1) */
    double K;              /* internal degrees of freedom, gamma = (K+5)/(K+3) */
    double R;              /* gas constant */
    double mu_ref, T_ref, omega;   /* mu = mu_ref (T/T_ref)^omega */
    double Pr;             /* Prandtl number, tau_b = tau_g / Pr */
    double dt;             /* time step; <= 0: CFL rule with cfl below */
    double cfl;
    int recon;             /* 0: reconstruction R-c; 1: the face-gradient variant R-c2 */
    int collision;         /* 0: the paper's two relaxation times (TEDDF); 1: Shakhov S-model */
    double accel[3];       /* uniform external acceleration a (eqs. gsource, bsource); 0 = none */
} oracle_params;

typedef struct oracle oracle_t;

oracle_t *oracle_create(const oracle_params *p);
void oracle_destroy(oracle_t *o);
int oracle_init(oracle_t *o, const double *rho_u_T);          /* [Nc][2+D] */
int oracle_step(oracle_t *o, int nsteps);
void oracle_moments(const oracle_t *o, double *out);          /* [Nc][2+D] rho,u,T */
void oracle_conserved(const oracle_t *o, double *out);        /* [Nc][2+D] W */
void oracle_distributions(const oracle_t *o, double *g, double *b);   /* [Nc][Nv] */
void oracle_discrete_moments(const oracle_t *o, double *out); /* [Nc][2+D] */
void oracle_stress_heat_flux(const oracle_t *o, double *out); /* [Nc][D*D+D]: P row-major, q */
void oracle_equilibrium(const oracle_t *o, double rho, const double *u, double T, double *geq, double *beq);
void oracle_shakhov_equilibrium(const oracle_t *o, double rho, const double *u, double T, const double *q,
                                double *geq, double *beq);
void oracle_cell_heat_flux(const oracle_t *o, double *out);   /* [Nc][D] tracked q (collision = 1) */
int oracle_set_state(oracle_t *o, const double *g, const double *b, const double *W);
void oracle_face_W(const oracle_t *o, int a, double *out);
void oracle_face_moments(const oracle_t *o, int a, double *out);   /* moments of the face phi, as oracle_face_W */
void oracle_velocities(const oracle_t *o, double *xi, double *w);     /* [Nv][3], [Nv] */
double oracle_dt(const oracle_t *o);
int oracle_nv(const oracle_t *o);
long oracle_ncells(const oracle_t *o);
long oracle_steps(const oracle_t *o);
double oracle_vanleer(double s1, double s2);
int oracle_vgrid_1d(int n, double lo, double hi, int rule, double *nodes, double *weights);

#ifdef __cplusplus
}
#endif
#endif
