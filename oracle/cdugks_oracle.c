/*
 * cdugks_oracle.c -- plain FP64 CPU oracle of one CDUGKS time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The GPU
 * product path never calls it and shares no code, header or table with it.
 *
 * What it computes: the Coupled Discrete Unified Gas Kinetic Scheme of
 * Zamora, Slaughter & Abel (arXiv:2208.09132), Sec. 2 ("The Coupled Discrete
 * Unified Gas Kinetic Scheme") and Sec. 2.1 ("The Algorithm"), for the reduced
 * distributions g (VDF, eq. g) and b (TEDF, eq. b) on a uniform Cartesian grid
 * in D = 1, 2 or 3 dimensions with a tensor-product discrete velocity grid.
 * External acceleration: none by default; a uniform vector a (accel) turns
 * on the force terms of eqs. gsource/bsource (readings R-v below).
 *
 * Style: plain nested loops in the order the paper gives the steps, every
 * intermediate kept in a full array, std libm exp/pow, compensated
 * (Neumaier) summation for every velocity-space integral, explicit ghost
 * layers (two deep; three with recon = 1) filled before each step.  No
 * fusion, no reordering.
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   R-a  eq. implicit's phi^n_{j+1} is read as phi^n_j (eq. phiupdate agrees).
 *   R-b  rho*u = sum w xi g (the quadrature form of Sec. 2), not "u g".
 *   R-c  Face reconstruction: phi_bar(x_f, t+h) = phibar+_up + (x_f - h xi - x_up).sigma_up,
 *        the upwind cell chosen by the sign of xi along the face normal (Sec. 2,
 *        "piecewise upwind linear interpolation"; eq. relation).  The full
 *        D-vector slope is used, tangential components included.
 *   R-d  sigma1/sigma2 of eq. VanLeer are the one-sided differences
 *        (phi_j - phi_{j-1})/dx and (phi_{j+1} - phi_j)/dx; the limiter gives 0
 *        when they differ in sign or either is zero.
 *   R-e  The flux enters the conserved-variable update with a minus sign
 *        (outward normals), as in eq. implicit and eq. phiupdate.
 *   R-f  With a = 0 the velocity integral of S_b vanishes analytically and is
 *        omitted from eqs. rhoupdate-rhoEupdate.
 *   R-g  1/tau_bg = 1/tau_b - 1/tau_g (the same quantity as Sec. 2's
 *        tau_bg = tau_b tau_g/(tau_g - tau_b), finite at Pr = 1).
 *   R-h  xi . n = 0 at a face (odd velocity grids): the mean of the two
 *        one-sided reconstructions.
 *   R-i  S_b in phibar+ uses the cell's own tau^n and u^n; at a face, g is
 *        recovered first and b then uses that face g.
 *   R-j  Specular walls mirror the neighbouring interior cells with the
 *        normal velocity component reversed; Dirichlet ghosts hold the
 *        equilibrium of the initial state of the nearest interior cell.
 *   R-c2 (recon = 1, selectable) The paper's variant of the reconstruction
 *        (Sec. 2.1: the slopes themselves are reconstructed at the face from
 *        their own limited gradients): phibar+(x_f) = phibar+_up +
 *        (x_f - x_up).sigma_up, sigma_f = sigma_up + (x_f - x_up).grad sigma_up
 *        (the derivative along the face normal of each slope component, van
 *        Leer limited like the slopes), and phibar(x_f, t+h) = phibar+(x_f) -
 *        h xi.sigma_f.  It needs three ghost layers.
 *   R-s  (collision = 1, selectable) The Shakhov S-model in place of the
 *        paper's two relaxation times (Sec. 1 names it as the other route to
 *        Pr != 1; the paper gives no form, so it is taken from Shakhov's model
 *        of 1968 as the DUGKS literature applies it to reduced distributions):
 *        one relaxation time tau = mu/p for g and b, no b-source, and the
 *        equilibria carry the heat-flux correction (shakhov_equilibrium below).
 *   R-s1 The heat flux of a cell or face is taken relative to its conserved
 *        variables W: q_a = sum w xi_a b - u_a rho E - sum_b u_b (sum w xi_a
 *        xi_b g - rho u_a u_b), with rho, u, E from W (heat_flux below).
 *   R-s2 The heat flux in the equilibrium at t_{n+1} comes from the update's
 *        explicit part (every term of eq. phiupdate's numerator but the new
 *        equilibrium): the collision relaxes q at the rate Pr/tau, so the
 *        trapezoid rule gives q^{n+1} = q(explicit part)/(1 + dt Pr/(2 tau^{n+1})).
 *        At a face likewise q = q(phibar)/(1 + h Pr/(2 tau)).  The heat flux
 *        is tracked per cell like W; the initial Maxwellian state has q = 0,
 *        and so have Dirichlet ghosts.
 *   R-v  (accel != 0) The force terms of eqs. gsource/bsource, S_g = -a.grad_xi g
 *        and a.xi g - a.grad_xi b in S_b, with the velocity gradient by central
 *        differences on the velocity grid, the distribution taken as zero beyond
 *        its ends.  The source enters phibar+ with h/2 (eq. phibarplus) and the
 *        update with dt at t_n (the rectangle rule of Sec. 2).  The W update
 *        adds dt times the integrals of the sources taken analytically
 *        (eqs. rhoupdate-rhoEupdate): 0 for rho, rho^n a for rho u and
 *        (rho u)^n . a for rho E, as reading R-f takes the b-source's.
 *   R-v1 At a face, eqs. rhoubar/rhoEbar: rho u = sum w xi gbar + (h/2) rho a,
 *        then rho E = sum w bbar + (h/2) (rho u) . a with that rho u; the
 *        inverse of eq. phibar takes the velocity gradients of the force terms
 *        from phibar at the face and a.xi g with the face g (as R-i), so the
 *        face distributions carry exactly the face conserved variables.
 *   R-v3 At a specular wall face the wall takes the normal component of the
 *        force: it is left out of that face's W corrections and inversion, so
 *        the mirrored phibar and the face equilibrium stay symmetric and the
 *        wall passes no mass and no energy.
 *   R-v2 Ghost cells take phibar+ by the ghost rule itself: periodic copies,
 *        specular mirror images (the force mirrored with the cell: the image
 *        domain) and the Dirichlet equilibrium without a force term.
 *
 * Pinning (tests/test_oracle_pins.py): every step above is checked against a
 * closed form, an invariant or a textbook limit.  The S_b term of the
 * distribution update is pinned by the moving-frame sound-damping check; the
 * two O(h) shares of S_b (in phibar+ and in the face inversion), whose effect
 * stays below the discretisation error in every closed form, are pinned by
 * discrete Galilean invariance: without either, a drifting solution departs
 * from the resting one at first order in dt instead of second order.
 */
#include "cdugks_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG (o->ng)      /* ghost layers per side: 2 (stencil j-2 .. j+1), 3 with recon = 1 */
#define NW 5            /* stored conserved variables (rho, rho u[3], rho E) */

struct oracle {
    oracle_params p;
    int ng;             /* ghost layers per side */
    int D;
    int n[3];           /* interior cells per axis (1 for unused axes) */
    int ne[3];          /* extended cells per axis (with ghosts on active axes) */
    long Nc, Ne;        /* interior, extended cell counts */
    int Nv;
    double dx[3];
    int nv1[3];         /* velocity nodes per axis (1 for unused axes) */
    double dxi[3];      /* velocity grid spacing per axis */
    int accel;          /* a != 0 */
    double gam;         /* adiabatic index */
    double *xi;         /* [Nv][3] discrete velocities */
    double *w;          /* [Nv] quadrature weights */
    int *refl[3];       /* [Nv] index of the velocity with component a reversed */
    /* state */
    double *g, *b;      /* [Ne][Nv] */
    double *W;          /* [Ne][NW] */
    double *q;          /* [Ne][3] tracked heat flux at t_n (collision = 1, R-s2) */
    double *Wdir;       /* [Ne][NW] fixed Dirichlet ghost state */
    /* intermediates of the step, kept in full */
    double *geq, *beq, *Sb;     /* [Ne][Nv] cell equilibria and b-source at t_n */
    double *gp, *bp;            /* [Ne][Nv] phibar+ (eq. phibarplus) */
    double *sg, *sb;            /* [Ne][3][Nv] limited slopes (eq. VanLeer) */
    double *s2g, *s2b;          /* [Ne][3][3][Nv] limited derivative along a of slope b (recon = 1) */
    double *gfb, *bfb;          /* [3][Ne][Nv] phibar at faces, t + h (eq. relation) */
    double *Wf;                 /* [3][Ne][NW] face conserved variables (eqs. rhobar-rhoEbar) */
    double *gf, *bf;            /* [3][Ne][Nv] phi at faces, t + h (inverse of eq. phibar) */
    double *dFg, *dFb;          /* [Ne][Nv] net microflux per cell volume (eq. flux) */
    double *Wn;                 /* [Ne][NW] updated conserved variables */
    double *Fg, *Fb;            /* [Ne][Nv] force terms of the sources at t_n (accel, R-v) */
    double *qn;                 /* [Ne][3] heat flux at t_{n+1} (collision = 1) */
    long steps;
};

/* ------------------------------------------------------------------ helpers */

typedef struct { double s, c; } nsum;   /* Neumaier compensated sum */
static void nsum_add(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_val(const nsum *a) { return a->s + a->c; }

static long cidx(const struct oracle *o, int x, int y, int z) {
    return (long)x + (long)o->ne[0] * ((long)y + (long)o->ne[1] * (long)z);
}
static void ccoord(const struct oracle *o, long c, int q[3]) {
    q[0] = (int)(c % o->ne[0]);
    q[1] = (int)((c / o->ne[0]) % o->ne[1]);
    q[2] = (int)(c / ((long)o->ne[0] * o->ne[1]));
}
static int is_interior(const struct oracle *o, const int q[3]) {
    for (int a = 0; a < o->D; ++a)
        if (q[a] < NG || q[a] >= NG + o->n[a]) return 0;
    return 1;
}
static long step_of(const struct oracle *o, int a) {
    return a == 0 ? 1 : (a == 1 ? (long)o->ne[0] : (long)o->ne[0] * o->ne[1]);
}

/* Van Leer limiter, eq. VanLeer: (sgn s1 + sgn s2) |s1||s2| / (|s1| + |s2|). */
double oracle_vanleer(double s1, double s2) {
    double a1 = fabs(s1), a2 = fabs(s2);
    double sg = (s1 > 0) - (s1 < 0) + (s2 > 0) - (s2 < 0);
    if (a1 + a2 == 0.0) return 0.0;
    return sg * a1 * a2 / (a1 + a2);
}

/* One-dimensional velocity nodes and weights (Sec. 2, quadrature sum_k w_k).
 * Nodes include both ends: xi_k = lo + (hi - lo) k / (n - 1).
 * rule 0: composite trapezoid; rule 1: composite Boole (4th-order closed
 * Newton-Cotes, needs n = 4m + 1, as used in the paper's runs). */
int oracle_vgrid_1d(int n, double lo, double hi, int rule, double *nodes, double *weights) {
    if (n < 2 || !(hi > lo)) return -1;
    double d = (hi - lo) / (n - 1);
    for (int k = 0; k < n; ++k) nodes[k] = lo + (hi - lo) * (double)k / (double)(n - 1);
    if (rule == 0) {
        for (int k = 0; k < n; ++k) weights[k] = d;
        weights[0] = 0.5 * d;
        weights[n - 1] = 0.5 * d;
    } else if (rule == 1) {
        if ((n - 1) % 4 != 0) return -1;
        for (int k = 0; k < n; ++k) weights[k] = 0.0;
        for (int m = 0; m + 4 < n; m += 4) {   /* Boole on each panel of 4 intervals */
            weights[m + 0] += 14.0 * d / 45.0;
            weights[m + 1] += 64.0 * d / 45.0;
            weights[m + 2] += 24.0 * d / 45.0;
            weights[m + 3] += 64.0 * d / 45.0;
            weights[m + 4] += 14.0 * d / 45.0;
        }
    } else {
        return -1;
    }
    return 0;
}

/* rho, u, T from W = (rho, rho u, rho E) (Sec. 2: gamma = (K+5)/(K+3),
 * T = (gamma - 1)/R (E - u^2/2)). */
static void macro_from_W(const struct oracle *o, const double *W, double *rho, double u[3], double *T) {
    double r = W[0];
    double u2 = 0.0;
    for (int a = 0; a < 3; ++a) u[a] = 0.0;
    for (int a = 0; a < o->D; ++a) { u[a] = W[1 + a] / r; u2 += u[a] * u[a]; }
    double E = W[1 + o->D] / r;
    *rho = r;
    *T = (o->gam - 1.0) / o->p.R * (E - 0.5 * u2);
}

/* tau_g = mu/p with mu = mu_r (T/T_r)^w (eq. visc), tau_b = tau_g / Pr,
 * 1/tau_bg = 1/tau_b - 1/tau_g (reading R-g).  The Shakhov model (R-s) has
 * the one time tau_b = tau_g and no b-source. */
static void relax_times(const struct oracle *o, double rho, double T, double *tg, double *tb, double *inv_tbg) {
    double mu = o->p.mu_ref * pow(T / o->p.T_ref, o->p.omega);
    double p = rho * o->p.R * T;
    *tg = mu / p;
    *tb = o->p.collision ? *tg : *tg / o->p.Pr;
    *inv_tbg = 1.0 / *tb - 1.0 / *tg;
}

/* Equilibria, eqs. geq and beq. */
static void equilibrium(const struct oracle *o, double rho, const double u[3], double T,
                        const double *xi, double *geq, double *beq) {
    double RT = o->p.R * T;
    double c2 = 0.0, xi2 = 0.0;
    for (int a = 0; a < o->D; ++a) {
        c2 += (xi[a] - u[a]) * (xi[a] - u[a]);
        xi2 += xi[a] * xi[a];
    }
    double ge = rho / pow(2.0 * M_PI * RT, 0.5 * o->D) * exp(-c2 / (2.0 * RT));
    *geq = ge;
    *beq = 0.5 * (xi2 + (3.0 - o->D + o->p.K) * RT) * ge;
}

/* Z = xi . u - u^2/2 (Sec. 2, after eq. bPDE). */
static double zeta(const struct oracle *o, const double *xi, const double u[3]) {
    double xu = 0.0, u2 = 0.0;
    for (int a = 0; a < o->D; ++a) { xu += xi[a] * u[a]; u2 += u[a] * u[a]; }
    return xu - 0.5 * u2;
}

/* Shakhov S-model equilibrium of the reduced distributions (R-s).  With
 * eta the L = 3 - D + K velocity components and internal degrees of freedom
 * the D-dimensional grid does not resolve (N = 3 + K in all), the S-model
 * equilibrium of the full distribution is
 *     f_S = f_M [1 + (1 - Pr) c.q / ((N + 2) p RT) ((c^2 + eta^2)/RT - (N + 2))],
 * c = xi - u: Shakhov's form with the monatomic 5 read as N + 2, so that f_S
 * has the density, momentum, energy and pressure tensor of f_M and the heat
 * flux (1 - Pr) q.  g = int f deta and b = int (xi^2 + eta^2)/2 f deta with the
 * Gaussian moments of eta (<1> = 1, <eta^2> = L RT, <eta^4> = L (L+2) RT^2):
 *     g_S = g_M [1 + A c.q (c^2/RT - D - 2)],
 *     b_S = b_M + A c.q g_M [(xi^2/2)(c^2/RT - D - 2) + (L/2)(c^2 - D RT)],
 * A = (1 - Pr)/((K + 5) p RT). */
static void shakhov_equilibrium(const struct oracle *o, double rho, const double u[3], double T, const double q[3],
                                const double *xi, double *geq, double *beq) {
    double gM, bM;
    equilibrium(o, rho, u, T, xi, &gM, &bM);
    double RT = o->p.R * T;
    double c2 = 0.0, xi2 = 0.0, cq = 0.0;
    for (int a = 0; a < o->D; ++a) {
        double c = xi[a] - u[a];
        c2 += c * c;
        xi2 += xi[a] * xi[a];
        cq += c * q[a];
    }
    double A = (1.0 - o->p.Pr) / ((o->p.K + 5.0) * rho * RT * RT);
    double L = 3.0 - o->D + o->p.K;
    double P1 = c2 / RT - o->D - 2.0;
    *geq = gM * (1.0 + A * cq * P1);
    *beq = bM + A * cq * gM * (0.5 * xi2 * P1 + 0.5 * L * (c2 - o->D * RT));
}

/* The equilibria of the selected collision model at one place. */
static void model_equilibrium(const struct oracle *o, double rho, const double u[3], double T, const double q[3],
                              const double *xi, double *geq, double *beq) {
    if (o->p.collision) shakhov_equilibrium(o, rho, u, T, q, xi, geq, beq);
    else equilibrium(o, rho, u, T, xi, geq, beq);
}

/* Heat flux of distributions (g, b) [Nv] at one place relative to the
 * conserved variables W there (R-s1): with rho, u, E from W, the pressure
 * tensor P_ab = sum w xi_a xi_b g - rho u_a u_b and
 *     q_a = sum w xi_a b - u_a rho E - sum_b u_b P_ab. */
static void heat_flux(const struct oracle *o, const double *g, const double *b, const double *W, double q[3]) {
    int D = o->D;
    double rho, u[3], T;
    macro_from_W(o, W, &rho, u, &T);
    nsum mF[3], mP[3][3];
    memset(mF, 0, sizeof(mF));
    memset(mP, 0, sizeof(mP));
    for (long i = 0; i < o->Nv; ++i) {
        const double *xi = &o->xi[3 * i];
        for (int a = 0; a < D; ++a) {
            nsum_add(&mF[a], o->w[i] * xi[a] * b[i]);
            for (int bb = 0; bb < D; ++bb) nsum_add(&mP[a][bb], o->w[i] * xi[a] * xi[bb] * g[i]);
        }
    }
    for (int a = 0; a < 3; ++a) q[a] = 0.0;
    for (int a = 0; a < D; ++a) {
        q[a] = nsum_val(&mF[a]) - u[a] * W[1 + D];
        for (int bb = 0; bb < D; ++bb) q[a] -= u[bb] * (nsum_val(&mP[a][bb]) - rho * u[a] * u[bb]);
    }
}

/* The velocity-gradient parts of the force terms of eqs. gsource/bsource at
 * one place from its distributions (g, b) [Nv] (R-v): sg = -a.grad_xi g and
 * sb = -a.grad_xi b, the derivatives by central differences
 * (g(k+1) - g(k-1))/(2 dxi) with g = 0 beyond the ends of the velocity grid.
 * The whole force terms are S_g = sg and a.xi g + sb in S_b. */
static void force_gradients(const struct oracle *o, const double *acc, const double *g, const double *b, double *sg,
                            double *sb) {
    const int D = o->D;
    const long s1 = o->nv1[0], s2 = (long)o->nv1[0] * o->nv1[1];
    for (long i = 0; i < o->Nv; ++i) {
        const long k[3] = { i % o->nv1[0], (i / s1) % o->nv1[1], i / s2 };
        const long st[3] = { 1, s1, s2 };
        double G = 0.0, B = 0.0;
        for (int a = 0; a < D; ++a) {
            if (acc[a] == 0.0) continue;
            double gp = 0.0, gm = 0.0, bp = 0.0, bm = 0.0;
            if (k[a] + 1 < o->nv1[a]) { gp = g[i + st[a]]; bp = b[i + st[a]]; }
            if (k[a] - 1 >= 0) { gm = g[i - st[a]]; bm = b[i - st[a]]; }
            G += acc[a] * (gp - gm) / (2.0 * o->dxi[a]);
            B += acc[a] * (bp - bm) / (2.0 * o->dxi[a]);
        }
        sg[i] = -G;
        sb[i] = -B;
    }
}

/* acc . xi_i */
static double a_dot_xi(const struct oracle *o, const double *acc, long i) {
    double s = 0.0;
    for (int a = 0; a < o->D; ++a) s += acc[a] * o->xi[3 * i + a];
    return s;
}

/* ------------------------------------------------------------- ghost layers */

/* Fill the ghost cells of axis a over the full extent of the other axes
 * (so that corner ghosts are filled by the later axes). */
static void fill_axis(struct oracle *o, int a) {
    long Nv = o->Nv;
    int na = o->n[a];
    for (long c = 0; c < o->Ne; ++c) {
        int q[3];
        ccoord(o, c, q);
        int k = q[a];
        if (k >= NG && k < NG + na) continue;          /* not a ghost of this axis */
        int side = (k < NG) ? 0 : 1;
        int bc = o->p.bc[a][side];
        int src[3] = { q[0], q[1], q[2] };
        int mirror = 0;
        if (bc == ORACLE_BC_PERIODIC) {
            src[a] = NG + (((k - NG) % na) + na) % na;
        } else if (bc == ORACLE_BC_SPECULAR) {
            /* ghost NG-1-m mirrors interior NG+m; ghost NG+na+m mirrors NG+na-1-m */
            src[a] = (k < NG) ? (2 * NG - 1 - k) : (2 * (NG + na) - 1 - k);
            mirror = 1;
        } else { /* Dirichlet: fixed equilibrium of the initial state */
            memcpy(&o->W[c * NW], &o->Wdir[c * NW], NW * sizeof(double));
            for (int d = 0; d < 3; ++d) o->q[c * 3 + d] = 0.0;
            double rho, u[3], T;
            macro_from_W(o, &o->W[c * NW], &rho, u, &T);
            for (long i = 0; i < Nv; ++i)
                equilibrium(o, rho, u, T, &o->xi[3 * i], &o->g[c * Nv + i], &o->b[c * Nv + i]);
            continue;
        }
        long s = cidx(o, src[0], src[1], src[2]);
        memcpy(&o->W[c * NW], &o->W[s * NW], NW * sizeof(double));
        if (mirror) o->W[c * NW + 1 + a] = -o->W[s * NW + 1 + a];
        for (int d = 0; d < 3; ++d) o->q[c * 3 + d] = o->q[s * 3 + d];
        if (mirror) o->q[c * 3 + a] = -o->q[s * 3 + a];
        for (long i = 0; i < Nv; ++i) {
            long si = mirror ? o->refl[a][i] : i;
            o->g[c * Nv + i] = o->g[s * Nv + si];
            o->b[c * Nv + i] = o->b[s * Nv + si];
        }
    }
}

static void fill_ghosts(struct oracle *o) {
    for (int a = 0; a < o->D; ++a) fill_axis(o, a);
}

/* R-v2: phibar+ of the ghost cells of axis a by the ghost rule (the order
 * of fill_axis, so corners agree): periodic copy, specular mirror image,
 * Dirichlet equilibrium. */
static void fill_axis_phibar(struct oracle *o, int a) {
    long Nv = o->Nv;
    int na = o->n[a];
    for (long c = 0; c < o->Ne; ++c) {
        int q[3];
        ccoord(o, c, q);
        int k = q[a];
        if (k >= NG && k < NG + na) continue;
        int side = (k < NG) ? 0 : 1;
        int bc = o->p.bc[a][side];
        int src[3] = { q[0], q[1], q[2] };
        if (bc == ORACLE_BC_DIRICHLET) {
            memcpy(&o->gp[c * Nv], &o->geq[c * Nv], sizeof(double) * Nv);
            memcpy(&o->bp[c * Nv], &o->beq[c * Nv], sizeof(double) * Nv);
            continue;
        }
        int mirror = bc == ORACLE_BC_SPECULAR;
        if (mirror) src[a] = (k < NG) ? (2 * NG - 1 - k) : (2 * (NG + na) - 1 - k);
        else src[a] = NG + (((k - NG) % na) + na) % na;
        long s = cidx(o, src[0], src[1], src[2]);
        for (long i = 0; i < Nv; ++i) {
            long si = mirror ? o->refl[a][i] : i;
            o->gp[c * Nv + i] = o->gp[s * Nv + si];
            o->bp[c * Nv + i] = o->bp[s * Nv + si];
        }
    }
}

/* ----------------------------------------------------------------- create */

static void *xalloc(size_t n) { void *p = calloc(n ? n : 1, 1); return p; }

oracle_t *oracle_create(const oracle_params *p) {
    if (!p || p->D < 1 || p->D > 3 || p->collision < 0 || p->collision > 1) return NULL;
    struct oracle *o = (struct oracle *)xalloc(sizeof(*o));
    if (!o) return NULL;
    o->p = *p;
    o->ng = p->recon ? 3 : 2;
    o->accel = 0;
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(p->accel[a]) || (a >= p->D && p->accel[a] != 0.0)) { free(o); return NULL; }
        if (p->accel[a] != 0.0) o->accel = 1;
    }
    o->D = p->D;
    o->gam = (p->K + 5.0) / (p->K + 3.0);
    o->Nc = 1; o->Ne = 1; o->Nv = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < o->D) {
            if (p->n[a] < 1 || p->nv[a] < 2 || !(p->hi[a] > p->lo[a])) { free(o); return NULL; }
            o->n[a] = p->n[a];
            o->ne[a] = p->n[a] + 2 * NG;
            o->dx[a] = (p->hi[a] - p->lo[a]) / p->n[a];
            o->nv1[a] = p->nv[a];
            o->dxi[a] = (p->vhi[a] - p->vlo[a]) / (p->nv[a] - 1);
            o->Nv *= p->nv[a];
            for (int s = 0; s < 2; ++s) {
                if (p->bc[a][s] == ORACLE_BC_SPECULAR && (p->vlo[a] != -p->vhi[a] || p->n[a] < NG)) { free(o); return NULL; }
            }
            if ((p->bc[a][0] == ORACLE_BC_PERIODIC) != (p->bc[a][1] == ORACLE_BC_PERIODIC)) { free(o); return NULL; }
        } else {
            o->n[a] = 1; o->ne[a] = 1; o->dx[a] = 1.0; o->nv1[a] = 1; o->dxi[a] = 1.0;
        }
        o->Nc *= o->n[a];
        o->Ne *= o->ne[a];
    }
    long Nv = o->Nv, Ne = o->Ne;
    o->xi = (double *)xalloc(sizeof(double) * 3 * Nv);
    o->w = (double *)xalloc(sizeof(double) * Nv);
    for (int a = 0; a < 3; ++a) o->refl[a] = (int *)xalloc(sizeof(int) * Nv);
    /* tensor-product velocity grid, index i = k0 + nv0 (k1 + nv1 k2) */
    {
        double nodes[3][ORACLE_MAX_NV1], wts[3][ORACLE_MAX_NV1];
        int nv[3] = {1, 1, 1};
        for (int a = 0; a < o->D; ++a) {
            nv[a] = p->nv[a];
            if (nv[a] > ORACLE_MAX_NV1 ||
                oracle_vgrid_1d(nv[a], p->vlo[a], p->vhi[a], p->rule, nodes[a], wts[a]) != 0) {
                oracle_destroy(o);
                return NULL;
            }
        }
        for (int a = o->D; a < 3; ++a) { nodes[a][0] = 0.0; wts[a][0] = 1.0; }
        for (int k2 = 0; k2 < nv[2]; ++k2)
            for (int k1 = 0; k1 < nv[1]; ++k1)
                for (int k0 = 0; k0 < nv[0]; ++k0) {
                    long i = k0 + (long)nv[0] * (k1 + (long)nv[1] * k2);
                    o->xi[3 * i + 0] = nodes[0][k0];
                    o->xi[3 * i + 1] = nodes[1][k1];
                    o->xi[3 * i + 2] = nodes[2][k2];
                    o->w[i] = wts[0][k0] * wts[1][k1] * wts[2][k2];
                    o->refl[0][i] = (int)((nv[0] - 1 - k0) + (long)nv[0] * (k1 + (long)nv[1] * k2));
                    o->refl[1][i] = (int)(k0 + (long)nv[0] * ((nv[1] - 1 - k1) + (long)nv[1] * k2));
                    o->refl[2][i] = (int)(k0 + (long)nv[0] * (k1 + (long)nv[1] * (nv[2] - 1 - k2)));
                }
    }
    size_t F = sizeof(double) * (size_t)Ne * Nv;
    o->g = xalloc(F); o->b = xalloc(F);
    o->geq = xalloc(F); o->beq = xalloc(F); o->Sb = xalloc(F);
    o->gp = xalloc(F); o->bp = xalloc(F);
    o->sg = xalloc(3 * F); o->sb = xalloc(3 * F);
    if (p->recon) { o->s2g = xalloc(9 * F); o->s2b = xalloc(9 * F); }
    o->gfb = xalloc(3 * F); o->bfb = xalloc(3 * F);
    o->gf = xalloc(3 * F); o->bf = xalloc(3 * F);
    o->dFg = xalloc(F); o->dFb = xalloc(F);
    o->W = xalloc(sizeof(double) * NW * Ne);
    o->Wn = xalloc(sizeof(double) * NW * Ne);
    o->q = xalloc(sizeof(double) * 3 * Ne);
    o->qn = xalloc(sizeof(double) * 3 * Ne);
    o->Fg = xalloc(F); o->Fb = xalloc(F);
    o->Wdir = xalloc(sizeof(double) * NW * Ne);
    o->Wf = xalloc(sizeof(double) * 3 * NW * Ne);
    if (!o->g || !o->b || !o->geq || !o->beq || !o->Sb || !o->gp || !o->bp || !o->sg || !o->sb ||
        (p->recon && (!o->s2g || !o->s2b)) ||
        !o->gfb || !o->bfb || !o->gf || !o->bf || !o->dFg || !o->dFb || !o->W || !o->Wn || !o->q || !o->qn || !o->Fg || !o->Fb ||
        !o->Wdir || !o->Wf || !o->xi || !o->w) {
        oracle_destroy(o);
        return NULL;
    }
    /* time step: the fixed CFL rule of Sec. 4, dt = alpha dx_min / (2 |xi|_max),
     * |xi|_max the largest discrete speed, unless dt is given. */
    if (p->dt > 0) {
        o->p.dt = p->dt;
    } else {
        double dxmin = o->dx[0], vmax = 0.0;
        for (int a = 1; a < o->D; ++a) if (o->dx[a] < dxmin) dxmin = o->dx[a];
        for (long i = 0; i < Nv; ++i) {
            double s = 0.0;
            for (int a = 0; a < o->D; ++a) s += o->xi[3 * i + a] * o->xi[3 * i + a];
            if (sqrt(s) > vmax) vmax = sqrt(s);
        }
        o->p.dt = p->cfl * dxmin / (2.0 * vmax);
    }
    return o;
}

void oracle_destroy(oracle_t *o) {
    if (!o) return;
    free(o->xi); free(o->w);
    for (int a = 0; a < 3; ++a) free(o->refl[a]);
    free(o->g); free(o->b); free(o->geq); free(o->beq); free(o->Sb);
    free(o->gp); free(o->bp); free(o->sg); free(o->sb); free(o->s2g); free(o->s2b);
    free(o->gfb); free(o->bfb); free(o->gf); free(o->bf);
    free(o->dFg); free(o->dFb);
    free(o->W); free(o->Wn); free(o->Wdir); free(o->Wf); free(o->q); free(o->qn); free(o->Fg); free(o->Fb);
    free(o);
}

double oracle_dt(const oracle_t *o) { return o->p.dt; }
int oracle_nv(const oracle_t *o) { return o->Nv; }
long oracle_ncells(const oracle_t *o) { return o->Nc; }
long oracle_steps(const oracle_t *o) { return o->steps; }

void oracle_velocities(const oracle_t *o, double *xi, double *w) {
    for (long i = 0; i < o->Nv; ++i) {
        for (int a = 0; a < 3; ++a) xi[3 * i + a] = o->xi[3 * i + a];
        w[i] = o->w[i];
    }
}

/* ------------------------------------------------------------------- init */

/* Maxwell-Boltzmann initialisation from cell-centre rho, u, T (Sec. 3.4:
 * every problem starts from eqs. geq/beq given the moments).  W^0 is the
 * analytic (rho, rho u, rho (u^2/2 + c_v T)) with c_v = (3+K)R/2. */
int oracle_init(oracle_t *o, const double *rho_u_T) {
    int D = o->D;
    double cv = (3.0 + o->p.K) * o->p.R / 2.0;
    long Nv = o->Nv;
    long ic = 0;
    memset(o->W, 0, sizeof(double) * NW * o->Ne);
    memset(o->q, 0, sizeof(double) * 3 * o->Ne);   /* a Maxwellian carries no heat flux (R-s2) */
    for (int z = 0; z < o->n[2]; ++z)
        for (int y = 0; y < o->n[1]; ++y)
            for (int x = 0; x < o->n[0]; ++x, ++ic) {
                int q[3] = { x + (D > 0 ? NG : 0), y + (D > 1 ? NG : 0), z + (D > 2 ? NG : 0) };
                long c = cidx(o, q[0], q[1], q[2]);
                const double *m = &rho_u_T[ic * (2 + D)];
                double rho = m[0], u[3] = {0, 0, 0}, u2 = 0.0;
                for (int a = 0; a < D; ++a) { u[a] = m[1 + a]; u2 += u[a] * u[a]; }
                double T = m[1 + D];
                if (!(rho > 0) || !(T > 0)) return -1;
                o->W[c * NW + 0] = rho;
                for (int a = 0; a < D; ++a) o->W[c * NW + 1 + a] = rho * u[a];
                o->W[c * NW + 1 + D] = rho * (0.5 * u2 + cv * T);
                for (long i = 0; i < Nv; ++i)
                    equilibrium(o, rho, u, T, &o->xi[3 * i], &o->g[c * Nv + i], &o->b[c * Nv + i]);
            }
    /* Dirichlet ghost states: the initial state of the nearest interior cell */
    for (long c = 0; c < o->Ne; ++c) {
        int q[3];
        ccoord(o, c, q);
        int src[3] = { q[0], q[1], q[2] };
        for (int a = 0; a < D; ++a) {
            if (src[a] < NG) src[a] = NG;
            if (src[a] >= NG + o->n[a]) src[a] = NG + o->n[a] - 1;
        }
        long s = cidx(o, src[0], src[1], src[2]);
        memcpy(&o->Wdir[c * NW], &o->W[s * NW], NW * sizeof(double));
    }
    o->steps = 0;
    return 0;
}

/* ------------------------------------------------------------------- step */

static void one_step(struct oracle *o) {
    const int D = o->D;
    const long Nv = o->Nv, Ne = o->Ne;
    const double dt = o->p.dt;
    const double h = 0.5 * dt;                      /* h = dt/2 (after eq. phibar) */

    /* (0) ghost layers for the stencil */
    fill_ghosts(o);

    /* (1) cell equilibria, b-source and the quarter-step-advanced
     *     distributions phibar+ = (2tau-h)/(2tau) phi + h/(2tau) phi_eq + (h/2) S
     *     (eq. phibarplus; S_g = 0, S_b = Z/tau_bg (g - g_eq) for a = 0,
     *     eqs. gsource/bsource; Shakhov: phi_eq = phi_S with the cell's q, S_b = 0). */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < Ne; ++c) {
        double rho, u[3], T, tg, tb, itbg;
        macro_from_W(o, &o->W[c * NW], &rho, u, &T);
        relax_times(o, rho, T, &tg, &tb, &itbg);
        for (long i = 0; i < Nv; ++i) {
            long k = c * Nv + i;
            const double *xi = &o->xi[3 * i];
            model_equilibrium(o, rho, u, T, &o->q[c * 3], xi, &o->geq[k], &o->beq[k]);
            o->Sb[k] = zeta(o, xi, u) * itbg * (o->g[k] - o->geq[k]);
            o->gp[k] = (2.0 * tg - h) / (2.0 * tg) * o->g[k] + h / (2.0 * tg) * o->geq[k];
            o->bp[k] = (2.0 * tb - h) / (2.0 * tb) * o->b[k] + h / (2.0 * tb) * o->beq[k] + 0.5 * h * o->Sb[k];
        }
        if (o->accel) {   /* R-v: the force terms, h/2 of them in phibar+ */
            force_gradients(o, o->p.accel, &o->g[c * Nv], &o->b[c * Nv], &o->Fg[c * Nv], &o->Fb[c * Nv]);
            for (long i = 0; i < Nv; ++i) o->Fb[c * Nv + i] += a_dot_xi(o, o->p.accel, i) * o->g[c * Nv + i];
            for (long i = 0; i < Nv; ++i) {
                o->gp[c * Nv + i] += 0.5 * h * o->Fg[c * Nv + i];
                o->bp[c * Nv + i] += 0.5 * h * o->Fb[c * Nv + i];
            }
        }
    }
    if (o->accel)
        for (int a = 0; a < D; ++a) fill_axis_phibar(o, a);   /* R-v2 */

    /* (2) van Leer limited slopes of phibar+ along every axis (eq. VanLeer),
     *     for every cell whose two neighbours exist in the extended grid. */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < Ne; ++c) {
        int q[3];
        ccoord(o, c, q);
        int ok = 1;
        for (int a = 0; a < D; ++a) if (q[a] < 1 || q[a] > o->ne[a] - 2) ok = 0;
        if (!ok) continue;
        for (int a = 0; a < D; ++a) {
            long s = step_of(o, a);
            for (long i = 0; i < Nv; ++i) {
                long k = c * Nv + i;
                double s1g = (o->gp[k] - o->gp[k - s * Nv]) / o->dx[a];
                double s2g = (o->gp[k + s * Nv] - o->gp[k]) / o->dx[a];
                double s1b = (o->bp[k] - o->bp[k - s * Nv]) / o->dx[a];
                double s2b = (o->bp[k + s * Nv] - o->bp[k]) / o->dx[a];
                o->sg[(c * 3 + a) * Nv + i] = oracle_vanleer(s1g, s2g);
                o->sb[(c * 3 + a) * Nv + i] = oracle_vanleer(s1b, s2b);
            }
        }
    }

    /* (2b) recon = 1 (reading R-c2): the limited derivative along every axis a
     *      of every slope component b, in the same van Leer form, for every
     *      cell whose two neighbours along each axis have slopes. */
    if (o->p.recon) {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < Ne; ++c) {
            int q[3];
            ccoord(o, c, q);
            int ok = 1;
            for (int a = 0; a < D; ++a) if (q[a] < 2 || q[a] > o->ne[a] - 3) ok = 0;
            if (!ok) continue;
            for (int a = 0; a < D; ++a) {
                long s = step_of(o, a);
                for (int bax = 0; bax < D; ++bax)
                    for (long i = 0; i < Nv; ++i) {
                        long k0 = (c * 3 + bax) * Nv + i, km = ((c - s) * 3 + bax) * Nv + i, kp = ((c + s) * 3 + bax) * Nv + i;
                        long d = ((c * 3 + a) * 3 + bax) * Nv + i;
                        o->s2g[d] = oracle_vanleer((o->sg[k0] - o->sg[km]) / o->dx[a], (o->sg[kp] - o->sg[k0]) / o->dx[a]);
                        o->s2b[d] = oracle_vanleer((o->sb[k0] - o->sb[km]) / o->dx[a], (o->sb[kp] - o->sb[k0]) / o->dx[a]);
                    }
            }
        }
    }

    /* (3)-(5) every face of every interior cell.  The face of axis a with
     *     right cell R and left cell L = R - e_a is stored at index R.  Faces
     *     with R_a in [NG, NG + n_a] and interior tangential coordinates. */
    for (int a = 0; a < D; ++a) {
        long s = step_of(o, a);
#pragma omp parallel for schedule(static)
        for (long R = 0; R < Ne; ++R) {
            int q[3];
            ccoord(o, R, q);
            int ok = (q[a] >= NG && q[a] <= NG + o->n[a]);
            for (int bax = 0; bax < D; ++bax)
                if (bax != a && (q[bax] < NG || q[bax] >= NG + o->n[bax])) ok = 0;
            if (!ok) continue;
            long L = R - s;
            long fo = (long)a * Ne + R;          /* face slot */

            /* (3) phibar(x_f, t+h) = phibar+(x_f - h xi, t): upwind linear
             *     reconstruction along the characteristic (eq. relation, R-c). */
            for (long i = 0; i < Nv; ++i) {
                const double *xi = &o->xi[3 * i];
                double vg[2], vb[2];
                long ups[2] = { L, R };
                double dn[2] = { +0.5 * o->dx[a], -0.5 * o->dx[a] };   /* (x_f - x_up) along e_a */
                for (int side = 0; side < 2; ++side) {
                    long up = ups[side];
                    double rg = o->gp[up * Nv + i], rb = o->bp[up * Nv + i];
                    if (!o->p.recon) {
                        for (int bax = 0; bax < D; ++bax) {
                            double d = (bax == a ? dn[side] : 0.0) - h * xi[bax];
                            rg += d * o->sg[(up * 3 + bax) * Nv + i];
                            rb += d * o->sb[(up * 3 + bax) * Nv + i];
                        }
                    } else {
                        /* R-c2: phibar+ at the face from the upwind cell, the slope
                         * vector carried to the face along e_a, then back along the
                         * characteristic by h xi with that face slope */
                        rg += dn[side] * o->sg[(up * 3 + a) * Nv + i];
                        rb += dn[side] * o->sb[(up * 3 + a) * Nv + i];
                        for (int bax = 0; bax < D; ++bax) {
                            double sfg = o->sg[(up * 3 + bax) * Nv + i] + dn[side] * o->s2g[((up * 3 + a) * 3 + bax) * Nv + i];
                            double sfb = o->sb[(up * 3 + bax) * Nv + i] + dn[side] * o->s2b[((up * 3 + a) * 3 + bax) * Nv + i];
                            rg -= h * xi[bax] * sfg;
                            rb -= h * xi[bax] * sfb;
                        }
                    }
                    vg[side] = rg;
                    vb[side] = rb;
                }
                double G, B;
                if (xi[a] > 0) { G = vg[0]; B = vb[0]; }
                else if (xi[a] < 0) { G = vg[1]; B = vb[1]; }
                else { G = 0.5 * (vg[0] + vg[1]); B = 0.5 * (vb[0] + vb[1]); }   /* R-h */
                o->gfb[fo * Nv + i] = G;
                o->bfb[fo * Nv + i] = B;
            }

            /* (4) face conserved variables from phibar (eqs. rhobar-rhoEbar, a = 0) */
            nsum m[NW];
            memset(m, 0, sizeof(m));
            for (long i = 0; i < Nv; ++i) {
                double G = o->gfb[fo * Nv + i], B = o->bfb[fo * Nv + i];
                nsum_add(&m[0], o->w[i] * G);
                for (int bax = 0; bax < D; ++bax) nsum_add(&m[1 + bax], o->w[i] * o->xi[3 * i + bax] * G);
                nsum_add(&m[1 + D], o->w[i] * B);
            }
            double *Wf = &o->Wf[fo * NW];
            for (int k = 0; k < NW; ++k) Wf[k] = 0.0;
            for (int k = 0; k < 2 + D; ++k) Wf[k] = nsum_val(&m[k]);
            /* R-v3: the force at this face; a specular wall takes its normal component */
            double fa[3] = { o->p.accel[0], o->p.accel[1], o->p.accel[2] };
            if ((q[a] == NG && o->p.bc[a][0] == ORACLE_BC_SPECULAR) ||
                (q[a] == NG + o->n[a] && o->p.bc[a][1] == ORACLE_BC_SPECULAR))
                fa[a] = 0.0;
            if (o->accel) {   /* R-v1: eqs. rhoubar, rhoEbar */
                for (int bax = 0; bax < D; ++bax) Wf[1 + bax] += 0.5 * h * Wf[0] * fa[bax];
                for (int bax = 0; bax < D; ++bax) Wf[1 + D] += 0.5 * h * Wf[1 + bax] * fa[bax];
            }
            double qf[3] = {0.0, 0.0, 0.0};   /* Shakhov: the face heat flux (R-s1, R-s2) */
            if (o->p.collision) heat_flux(o, &o->gfb[fo * Nv], &o->bfb[fo * Nv], Wf, qf);

            /* (5) face tau and equilibria, then phi = inverse of eq. phibar:
             *     g_f = (2 tau_g gbar + h g_eq)/(2 tau_g + h),
             *     b_f = (2 tau_b bbar + h b_eq + h tau_b Z/tau_bg (g_f - g_eq))/(2 tau_b + h). */
            double rho, u[3], T, tg, tb, itbg;
            macro_from_W(o, Wf, &rho, u, &T);
            relax_times(o, rho, T, &tg, &tb, &itbg);
            for (int d = 0; d < 3; ++d) qf[d] /= 1.0 + h * o->p.Pr / (2.0 * tg);
            double *fsg = NULL, *fsb = NULL;   /* R-v1: force gradients of phibar at the face */
            if (o->accel) {
                fsg = (double *)calloc((size_t)2 * Nv, sizeof(double));
                fsb = fsg + Nv;
                force_gradients(o, fa, &o->gfb[fo * Nv], &o->bfb[fo * Nv], fsg, fsb);
            }
            for (long i = 0; i < Nv; ++i) {
                const double *xi = &o->xi[3 * i];
                double ge, be;
                model_equilibrium(o, rho, u, T, qf, xi, &ge, &be);
                double G = o->gfb[fo * Nv + i], B = o->bfb[fo * Nv + i];
                double gfv, bfv;
                if (!o->accel) {
                    gfv = (2.0 * tg * G + h * ge) / (2.0 * tg + h);
                    bfv = (2.0 * tb * B + h * be + h * tb * zeta(o, xi, u) * itbg * (gfv - ge)) / (2.0 * tb + h);
                } else {   /* the inverse of eq. phibar with the whole source S; a.xi g with the face g (R-i) */
                    gfv = (2.0 * tg * G + h * ge + h * tg * fsg[i]) / (2.0 * tg + h);
                    bfv = (2.0 * tb * B + h * be +
                           h * tb * (zeta(o, xi, u) * itbg * (gfv - ge) + a_dot_xi(o, fa, i) * gfv + fsb[i])) /
                          (2.0 * tb + h);
                }
                o->gf[fo * Nv + i] = gfv;
                o->bf[fo * Nv + i] = bfv;
            }
            free(fsg);
        }
    }

    /* (6)-(8) interior cells: net microflux (eq. flux, uniform grid so
     *     |A|/|V| = 1/dx_a), conserved-variable update (eqs. rhoupdate-
     *     rhoEupdate with readings R-e, R-f), then the distribution update
     *     eq. phiupdate with phi_eq and tau at t_{n+1} from W^{n+1}. */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < Ne; ++c) {
        int q[3];
        ccoord(o, c, q);
        if (!is_interior(o, q)) continue;
        for (long i = 0; i < Nv; ++i) {
            double Fg = 0.0, Fb = 0.0;
            for (int a = 0; a < D; ++a) {
                long fr = (long)a * Ne + (c + step_of(o, a));   /* right face of c */
                long fl = (long)a * Ne + c;                     /* left face of c */
                double xa = o->xi[3 * i + a];
                Fg += xa * (o->gf[fr * Nv + i] - o->gf[fl * Nv + i]) / o->dx[a];
                Fb += xa * (o->bf[fr * Nv + i] - o->bf[fl * Nv + i]) / o->dx[a];
            }
            o->dFg[c * Nv + i] = Fg;
            o->dFb[c * Nv + i] = Fb;
        }
        nsum m[NW];
        memset(m, 0, sizeof(m));
        for (long i = 0; i < Nv; ++i) {
            nsum_add(&m[0], o->w[i] * o->dFg[c * Nv + i]);
            for (int a = 0; a < D; ++a) nsum_add(&m[1 + a], o->w[i] * o->xi[3 * i + a] * o->dFg[c * Nv + i]);
            nsum_add(&m[1 + D], o->w[i] * o->dFb[c * Nv + i]);
        }
        for (int k = 0; k < NW; ++k) o->Wn[c * NW + k] = 0.0;
        for (int k = 0; k < 2 + D; ++k) o->Wn[c * NW + k] = o->W[c * NW + k] - dt * nsum_val(&m[k]);
        if (o->accel) {   /* R-v: dt times the integrals of the sources at t_n */
            for (int a = 0; a < D; ++a) {
                o->Wn[c * NW + 1 + a] += dt * o->W[c * NW] * o->p.accel[a];
                o->Wn[c * NW + 1 + D] += dt * o->W[c * NW + 1 + a] * o->p.accel[a];
            }
        }

        double rho0, u0[3], T0, tg0, tb0, itbg0;
        macro_from_W(o, &o->W[c * NW], &rho0, u0, &T0);
        relax_times(o, rho0, T0, &tg0, &tb0, &itbg0);
        double rho1, u1[3], T1, tg1, tb1, itbg1;
        macro_from_W(o, &o->Wn[c * NW], &rho1, u1, &T1);
        relax_times(o, rho1, T1, &tg1, &tb1, &itbg1);
        double *q1 = &o->qn[c * 3];
        for (int d = 0; d < 3; ++d) q1[d] = 0.0;
        if (o->p.collision) {
            /* R-s2: q^{n+1} from the explicit part of eq. phiupdate's numerator */
            double *eg = (double *)malloc(sizeof(double) * 2 * Nv), *eb = eg + Nv;
            for (long i = 0; i < Nv; ++i) {
                long k = c * Nv + i;
                eg[i] = o->g[k] + 0.5 * dt * (o->geq[k] - o->g[k]) / tg0 - dt * o->dFg[k];
                eb[i] = o->b[k] + 0.5 * dt * (o->beq[k] - o->b[k]) / tb0 - dt * o->dFb[k];
                if (o->accel) {
                    eg[i] += dt * o->Fg[k];
                    eb[i] += dt * o->Fb[k];
                }
            }
            heat_flux(o, eg, eb, &o->Wn[c * NW], q1);
            free(eg);
            for (int d = 0; d < 3; ++d) q1[d] /= 1.0 + dt * o->p.Pr / (2.0 * tg1);
        }
        for (long i = 0; i < Nv; ++i) {
            long k = c * Nv + i;
            double ge1, be1;
            model_equilibrium(o, rho1, u1, T1, q1, &o->xi[3 * i], &ge1, &be1);
            double gnew, bnew;
            if (!o->accel) {
                gnew = (o->g[k] + 0.5 * dt * (ge1 / tg1 + (o->geq[k] - o->g[k]) / tg0)
                        - dt * o->dFg[k]) / (1.0 + dt / (2.0 * tg1));
                bnew = (o->b[k] + 0.5 * dt * (be1 / tb1 + (o->beq[k] - o->b[k]) / tb0)
                        - dt * o->dFb[k] + dt * o->Sb[k]) / (1.0 + dt / (2.0 * tb1));
            } else {   /* eq. phiupdate with S^n = the b-source + the force terms */
                gnew = (o->g[k] + 0.5 * dt * (ge1 / tg1 + (o->geq[k] - o->g[k]) / tg0)
                        - dt * o->dFg[k] + dt * o->Fg[k]) / (1.0 + dt / (2.0 * tg1));
                bnew = (o->b[k] + 0.5 * dt * (be1 / tb1 + (o->beq[k] - o->b[k]) / tb0)
                        - dt * o->dFb[k] + dt * (o->Sb[k] + o->Fb[k])) / (1.0 + dt / (2.0 * tb1));
            }
            o->g[k] = gnew;
            o->b[k] = bnew;
        }
    }
    /* commit W^{n+1} for interior cells */
    for (long c = 0; c < Ne; ++c) {
        int q[3];
        ccoord(o, c, q);
        if (!is_interior(o, q)) continue;
        memcpy(&o->W[c * NW], &o->Wn[c * NW], NW * sizeof(double));
        memcpy(&o->q[c * 3], &o->qn[c * 3], 3 * sizeof(double));
    }
    o->steps += 1;
}

int oracle_step(oracle_t *o, int nsteps) {
    if (nsteps < 0) return -1;
    for (int s = 0; s < nsteps; ++s) one_step(o);
    return 0;
}

/* -------------------------------------------------------------- readback */

static long interior_ext(const struct oracle *o, long ic) {
    int x = (int)(ic % o->n[0]);
    int y = (int)((ic / o->n[0]) % o->n[1]);
    int z = (int)(ic / ((long)o->n[0] * o->n[1]));
    return cidx(o, x + (o->D > 0 ? NG : 0), y + (o->D > 1 ? NG : 0), z + (o->D > 2 ? NG : 0));
}

/* [Nc][2+D]: rho, u[D], T from the tracked conserved variables W (Sec. 2.1). */
void oracle_moments(const oracle_t *o, double *out) {
    int D = o->D;
    for (long ic = 0; ic < o->Nc; ++ic) {
        long c = interior_ext(o, ic);
        double rho, u[3], T;
        macro_from_W(o, &o->W[c * NW], &rho, u, &T);
        out[ic * (2 + D) + 0] = rho;
        for (int a = 0; a < D; ++a) out[ic * (2 + D) + 1 + a] = u[a];
        out[ic * (2 + D) + 1 + D] = T;
    }
}

/* [Nc][2+D]: W = (rho, rho u[D], rho E). */
void oracle_conserved(const oracle_t *o, double *out) {
    int D = o->D;
    for (long ic = 0; ic < o->Nc; ++ic) {
        long c = interior_ext(o, ic);
        for (int k = 0; k < 2 + D; ++k) out[ic * (2 + D) + k] = o->W[c * NW + k];
    }
}

/* g, b of the interior cells, [Nc][Nv] each. */
void oracle_distributions(const oracle_t *o, double *g, double *b) {
    long Nv = o->Nv;
    for (long ic = 0; ic < o->Nc; ++ic) {
        long c = interior_ext(o, ic);
        memcpy(&g[ic * Nv], &o->g[c * Nv], sizeof(double) * Nv);
        memcpy(&b[ic * Nv], &o->b[c * Nv], sizeof(double) * Nv);
    }
}

/* Discrete moments of g and b per interior cell, [Nc][2+D] (Sec. 2, sum_k w_k). */
void oracle_discrete_moments(const oracle_t *o, double *out) {
    int D = o->D;
    long Nv = o->Nv;
    for (long ic = 0; ic < o->Nc; ++ic) {
        long c = interior_ext(o, ic);
        nsum m[NW];
        memset(m, 0, sizeof(m));
        for (long i = 0; i < Nv; ++i) {
            nsum_add(&m[0], o->w[i] * o->g[c * Nv + i]);
            for (int a = 0; a < D; ++a) nsum_add(&m[1 + a], o->w[i] * o->xi[3 * i + a] * o->g[c * Nv + i]);
            nsum_add(&m[1 + D], o->w[i] * o->b[c * Nv + i]);
        }
        for (int k = 0; k < 2 + D; ++k) out[ic * (2 + D) + k] = nsum_val(&m[k]);
    }
}

/* Pressure tensor and heat flux of every cell from its distributions (a
 * diagnostic; the scheme itself does not use them).  With rho = sum w g,
 * rho u = sum w xi g and rho E = sum w b (the moments of Sec. 2), the pressure
 * tensor is the central second moment P_ab = sum w (xi - u)_a (xi - u)_b g,
 * and the heat flux q is what the flux of total energy sum w xi_a b carries
 * beyond convection and pressure work:
 *     q_a = sum w xi_a b - u_a rho E - sum_b P_ab u_b.
 * out: [Nc][D*D + D], P row-major, then q. */
void oracle_stress_heat_flux(const oracle_t *o, double *out) {
    int D = o->D;
    long Nv = o->Nv;
    for (long ic = 0; ic < o->Nc; ++ic) {
        long c = interior_ext(o, ic);
        const double *g = &o->g[c * Nv], *b = &o->b[c * Nv];
        nsum m0, m1[3], mE, mF[3], mP[3][3];
        memset(&m0, 0, sizeof(m0));
        memset(m1, 0, sizeof(m1));
        memset(&mE, 0, sizeof(mE));
        memset(mF, 0, sizeof(mF));
        memset(mP, 0, sizeof(mP));
        for (long i = 0; i < Nv; ++i) {
            nsum_add(&m0, o->w[i] * g[i]);
            nsum_add(&mE, o->w[i] * b[i]);
            for (int a = 0; a < D; ++a) {
                nsum_add(&m1[a], o->w[i] * o->xi[3 * i + a] * g[i]);
                nsum_add(&mF[a], o->w[i] * o->xi[3 * i + a] * b[i]);
            }
        }
        double rho = nsum_val(&m0), u[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) u[a] = nsum_val(&m1[a]) / rho;
        for (long i = 0; i < Nv; ++i)
            for (int a = 0; a < D; ++a)
                for (int bb = 0; bb < D; ++bb)
                    nsum_add(&mP[a][bb], o->w[i] * (o->xi[3 * i + a] - u[a]) * (o->xi[3 * i + bb] - u[bb]) * g[i]);
        double *dst = &out[ic * (D * D + D)];
        for (int a = 0; a < D; ++a)
            for (int bb = 0; bb < D; ++bb) dst[a * D + bb] = nsum_val(&mP[a][bb]);
        double rhoE = nsum_val(&mE);
        for (int a = 0; a < D; ++a) {
            double q = nsum_val(&mF[a]) - u[a] * rhoE;
            for (int bb = 0; bb < D; ++bb) q -= dst[a * D + bb] * u[bb];
            dst[D * D + a] = q;
        }
    }
}

/* Equilibria g_eq, b_eq at every node for one state (eqs. geq, beq). */
void oracle_equilibrium(const oracle_t *o, double rho, const double *u, double T, double *geq, double *beq) {
    double uu[3] = {0, 0, 0};
    for (int a = 0; a < o->D; ++a) uu[a] = u[a];
    for (long i = 0; i < o->Nv; ++i) equilibrium(o, rho, uu, T, &o->xi[3 * i], &geq[i], &beq[i]);
}

/* Overwrite the interior state (g, b [Nc][Nv], W [Nc][2+D]); for tests that
 * start from a non-equilibrium distribution. */
int oracle_set_state(oracle_t *o, const double *g, const double *b, const double *W) {
    int D = o->D;
    long Nv = o->Nv;
    for (long ic = 0; ic < o->Nc; ++ic) {
        long c = interior_ext(o, ic);
        memcpy(&o->g[c * Nv], &g[ic * Nv], sizeof(double) * Nv);
        memcpy(&o->b[c * Nv], &b[ic * Nv], sizeof(double) * Nv);
        for (int k = 0; k < NW; ++k) o->W[c * NW + k] = 0.0;
        for (int k = 0; k < 2 + D; ++k) o->W[c * NW + k] = W[ic * (2 + D) + k];
        for (int d = 0; d < 3; ++d) o->q[c * 3 + d] = 0.0;
        if (o->p.collision) heat_flux(o, &o->g[c * Nv], &o->b[c * Nv], &o->W[c * NW], &o->q[c * 3]);
    }
    return 0;
}

/* The Shakhov equilibria at every node for one state and heat flux q[D]. */
void oracle_shakhov_equilibrium(const oracle_t *o, double rho, const double *u, double T, const double *q,
                                double *geq, double *beq) {
    double uu[3] = {0, 0, 0}, qq[3] = {0, 0, 0};
    for (int a = 0; a < o->D; ++a) { uu[a] = u[a]; qq[a] = q[a]; }
    for (long i = 0; i < o->Nv; ++i) shakhov_equilibrium(o, rho, uu, T, qq, &o->xi[3 * i], &geq[i], &beq[i]);
}

/* The tracked heat flux q^n of every interior cell, [Nc][D] (collision = 1). */
void oracle_cell_heat_flux(const oracle_t *o, double *out) {
    for (long ic = 0; ic < o->Nc; ++ic) {
        long c = interior_ext(o, ic);
        for (int a = 0; a < o->D; ++a) out[ic * o->D + a] = o->q[c * 3 + a];
    }
}

/* Moments (rho, rho u, rho E) of the face distributions phi of the last step
 * (the inverse of eq. phibar), axis a, in the order of oracle_face_W. */
void oracle_face_moments(const oracle_t *o, int a, double *out) {
    int D = o->D;
    long k = 0, Nv = o->Nv;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = (d < D) ? NG : 0;
        hi[d] = (d < D) ? NG + o->n[d] : 1;
    }
    hi[a] += 1;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x, ++k) {
                long fo = (long)a * o->Ne + cidx(o, x, y, z);
                nsum m[NW];
                memset(m, 0, sizeof(m));
                for (long i = 0; i < Nv; ++i) {
                    double G = o->gf[fo * Nv + i];
                    nsum_add(&m[0], o->w[i] * G);
                    for (int b = 0; b < D; ++b) nsum_add(&m[1 + b], o->w[i] * o->xi[3 * i + b] * G);
                    nsum_add(&m[1 + D], o->w[i] * o->bf[fo * Nv + i]);
                }
                for (int m2 = 0; m2 < 2 + D; ++m2) out[k * (2 + D) + m2] = nsum_val(&m[m2]);
            }
}

/* Face conserved variables of the last step, axis a, [Nfaces_a][2+D] in the
 * order (x fastest) over faces R_a in [0, n_a], tangential interior. */
void oracle_face_W(const oracle_t *o, int a, double *out) {
    int D = o->D;
    long k = 0;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = (d < D) ? NG : 0;
        hi[d] = (d < D) ? NG + o->n[d] : 1;
    }
    hi[a] += 1;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x, ++k) {
                long R = cidx(o, x, y, z);
                for (int m = 0; m < 2 + D; ++m) out[k * (2 + D) + m] = o->Wf[((long)a * o->Ne + R) * NW + m];
            }
}
