// kernels.cuh -- sm_103a device code of the CDUGKS step (arXiv:2208.09132, Sec. 2.1).
//
// One time step is four kinds of launch on the caller's stream:
//
//   sweep A   per (tile of cells, group of velocity chunks): finalise phi^n from
//             the stored pre-update value phi* (the last factor of eq. phiupdate,
//             deferred until W^n is known), form phibar+ (eq. phibarplus) on the
//             tile and its two-cell halo in shared memory, van Leer slopes
//             (eq. VanLeer), reconstruct phibar at the owned faces along the
//             characteristic (eq. relation) and sum the face conserved variables
//             (eqs. rhobar-rhoEbar) over the group's velocities.
//   face      sum the groups' partial face W; face constants (u, T, tau).
//   sweep B   the face equilibrium (eqs. geq, beq), the inverse of eq. phibar,
//             the microflux xi.n phi (eq. flux), its moments (for W) and the
//             per-velocity net flux that gives phi* of eq. phiupdate, written to
//             the other state buffer.  In the face-store modes sweep A keeps the
//             reconstructed face values and sweep B is k_flux, which reads them;
//             otherwise sweep B reconstructs them again.
//
//   W update  W^{n+1} = W^n - dt sum_faces (M_right - M_left)/dx (eqs.
//             rhoupdate-rhoEupdate, outward normals), the status check and the
//             cell constants of W^{n+1}.
//
// Sweep modes (the mode of a tile shape) choose where the stencil work is done:
// on the halo box by the sweeps, once per point by a pre-pass (k_prep,
// k_shslope), and whether face values are stored; bit 3 selects the paper's
// face-gradient variant of the reconstruction (a three-cell halo), bit 4 the
// Shakhov collision model (with k_faceq and k_cellq for the heat flux), bit 5
// the external acceleration (force terms formed by k_prep).
//
// Layout in HBM: phi*[velocity chunk][cell][field g|b][VC], VC = 4 velocities,
// so one cell's chunk of g and b is one 32-byte sector (FP32) read with two
// 16-byte vector loads.  Boundaries are applied by index mapping while the
// halo is loaded (periodic wrap, mirror with reflected velocity, fixed
// equilibrium), not by ghost copies.  Sweep A stages the next chunk's halo box
// ahead of use: with tensor copies (TMA, completed on an mbarrier with a
// bounded wait) on 1D/2D tiles whose box lies inside the domain, per cell with
// cp.async elsewhere.  The kernels of a step are chained by programmatic
// dependent launch (pdl_wait before the first dependent read).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace cdg {

constexpr int VC = 4;             // velocities per chunk: the innermost run of the state layout

enum { BC_PERIODIC = 0, BC_SPECULAR = 1, BC_DIRICHLET = 2 };
enum { ST_NONFINITE = 1, ST_NEGATIVE = 2, ST_TIMEOUT = 4 };

// Tensor maps of the g and b halves of the input state buffer for the TMA
// staging of sweep A (one box of tile + halo cells per chunk), passed by value
// as a kernel parameter; on = 0 when the launch has none.
struct TmaPair {
    CUtensorMap g, b;
    int on;
};

// Problem geometry and physics, passed by value to every kernel.
struct Geo {
    int D;
    int n[3];
    int bc[3][2];
    long long Nc;
    int Nvp;          // padded velocity count (multiple of VC)
    int NVT;          // velocity chunks (Nvp / VC)
    int ntpg;         // velocity chunks per group
    int G;            // velocity groups
    int tiles[3];     // spatial tiles per axis
    int tile_id;      // which instantiated tile shape the sweeps use
    int fn[3][3];     // face-array extents per axis a: fn[a][b] = n[b] + (a == b)
    long long nf[3];  // faces per axis
    double dx[3];
    double hdx[3];    // h / dx_a
    double idx[3];    // 1 / dx_a
    double dt, h;
    double K, R, mu_ref, T_ref, omega, Pr;
    int shakhov;      // collision model: 0 the two relaxation times of Sec. 2, 1 the Shakhov S-model
    int accel;        // a uniform external acceleration is on (eqs. gsource, bsource)
    double acc[3];    // its components a_b (0 beyond D)
    int nv1[3];       // velocity nodes per axis (velocity i = k0 + nv1_0 (k1 + nv1_1 k2))
    double dxi[3];    // velocity spacing per axis
    int wait_log2;    // bounded waits give up after 2^wait_log2 tries
    int wait_test;    // test hook: sweep A issues no tensor copies, so its bounded wait runs out
    int nosrc;        // the b-source Z/tau_bg (g - g_eq) vanishes (Pr = 1, or the Shakhov model)
    // Separable Maxwellian factors (the lean shapes): per cell or face and axis b the
    // factors exp(-(xi_{b,k} - u_b)^2 / (2RT)) of every node k, formed in double; rows
    // of a table: axis 0 at [0, xrow[1]) (nv1_0 rounded up to VC), axis b >= 1 at
    // [xrow[b], xrow[b] + nv1_b); xrows rows in all.
    double vlo[3];    // first velocity node per axis
    int xrow[3];
    int xrows;
    int xal;          // nv1_0 is a multiple of VC: a chunk's four velocities share their other indices
};

template <typename T> struct CellC;
template <typename T> struct FaceC;

template <typename T>
struct Bufs {
    const T* phi_in;
    T* phi_out;
    T* phibar;            // phibar+ of every point (state layout), for the prepared and stored shapes
    T* sigma;             // van Leer slopes of every point, [chunk][cell][axis][g|b][VC] (stored shapes)
    T* face[3];           // reconstructed phibar at every face of axis a, [chunk][face][g|b][VC] (face-store shapes)
    double* W;            // [2+D][Nc] tracked conserved variables, updated in place
    CellC<T>* cellc;      // [Nc] constants of W^n (written by the W update / init)
    CellC<T>* cellc0;     // [Nc] constants of W^0 (Dirichlet ghosts)
    FaceC<T>* facec[3];   // [nf_a] constants of the face W (between the sweeps)
    double* wf[3];        // [G][2+D][nf_a] face W partial sums (sweep A)
    double* mf[3];        // [G][2+D][nf_a] face flux-moment partial sums (sweep B)
    const T* vel;         // [Nvp][8] per velocity: xi_0, xi_1, xi_2, w, |xi|^2/2, 2h xi_0/dx_0, 2h xi_1/dx_1,
                          // 2h xi_2/dx_2 (w = 0 on padding)
    const int* refl;      // [8][Nvp] velocity index with the components of mask reversed
    int* status;
    // Shakhov model only (null otherwise); NQ = D + D(D+1)/2 raw moments
    double* hq;           // [D][Nc] heat flux of the current time level, tracked like W
    double* qs;           // [G][NQ][Nc] raw velocity moments of phi* per velocity group
    double* qf[3];        // [G][NQ][nf_a] raw velocity moments of the face values per group
    T* force;             // acceleration only: force terms of the sources at t_n, state layout
    // lean shapes only (null otherwise): separable Maxwellian factor tables, layout of xaddr()
    T* xc;                // [rows][Nc] of W^n (written with the cell constants)
    T* xc0;               // [rows][Nc] of W^0 (Dirichlet ghosts)
    T* xf[3];             // [rows][nf_a] of the face W (written with the face constants)
};

// An instance as the kernels see it: geometry and both ping-pong orientations
// of its buffers (b[c] reads state buffer c and writes the other), kept in
// device memory.  Single-instance launches and batched launches read the same
// table, so a member computes the same numbers alone and inside a batch.
template <typename T>
struct Inst {
    Geo g;
    Bufs<T> b[2];
};
// Batched work items: one sweep CTA = (instance, tile, velocity group); one
// face/cell CTA = a range [start, start + count) of one instance.
struct Item {
    int inst, tile, grp, pad;
};
struct RItem {
    int inst, axis;
    long long start, count;
};
// Batched raw-moment work (Shakhov heat flux): faces [start, start + count) of
// one axis (axis >= 0) or cells (axis = -1) of one instance, one velocity group.
struct QItem {
    int inst, axis, grp, pad;
    long long start, count;
};

// ------------------------------------------------------------------ numerics

template <typename T> struct Num;
template <> struct Num<float> {
    // equilibrium exponent on base 2: exp(-c^2/(2RT)) = exp2(c^2 * cexp)
    static __device__ __forceinline__ float expo(float x) {
        float y;   // hardware base-2 exponential (relative error ~2^-22, subnormal results flushed)
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __host__ __device__ __forceinline__ double cexp_scale() { return 1.4426950408889634; }
    // 1/RT = cexp * irt_scale (cexp = -log2(e)/(2 RT))
    static __host__ __device__ __forceinline__ float irt_scale() { return -1.3862943611198906f; }
    // half the van Leer slope: s1 s2 / (s1 + s2) (the factor 2 is folded into the
    // reconstruction coefficients)
    static __device__ __forceinline__ float vanleer(float s1, float s2) {
        float p = s1 * s2;
        return p > 0.f ? __fdividef(p, s1 + s2) : 0.f;
    }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double expo(double x) { return exp(x); }
    static __host__ __device__ __forceinline__ double cexp_scale() { return 1.0; }
    static __host__ __device__ __forceinline__ double irt_scale() { return -2.0; }
    static __device__ __forceinline__ double vanleer(double s1, double s2) {
        double p = s1 * s2;
        return p > 0.0 ? p / (s1 + s2) : 0.0;
    }
};

// Per-cell constants for one cell state W (Sec. 2: T from E - u^2/2,
// tau_g = mu/p, tau_b = tau_g/Pr, 1/tau_bg = 1/tau_b - 1/tau_g), all
// formed in double and stored in the working precision.
template <typename T>
struct CellC {
    T u[3];
    T cexp, pref, eb, hu2;      // g_eq = pref exp(cexp |xi-u|^2), b_eq = (|xi|^2/2 + eb) g_eq, Z = xi.u - hu2
    T fa_g, fb_g, fa_b, fb_b;   // phi = fa phi* + fb phi_eq        (deferred end of eq. phiupdate)
    T kp_g, kp_b, kp_s;         // phibar+ = eq + kp (phi* - eq) [+ kp_s Z (g* - g_eq)] (eq. phibarplus with
                                //   phi - eq = fa (phi* - eq): kp = sa fa, kp_s = ssrc fa_g)
    T um_g, um_b, usrc;         // phi* = eq + um (phi - eq) [+ usrc Z (g - g_eq)] - dt dF (eq. phiupdate)
    T sq[3], e2;                // Shakhov: sq = (1 - Pr) q / ((K + 5) p RT), e2 = (3 - D + K) D RT / 2 (else 0)
};

// The phibar+ constants of a cell as packed in shared memory: u (D), cexp,
// pref, eb, hu2, kp_g, kp_b, kp_s, and with the Shakhov model sq (D), e2.
template <int D, bool SK = false>
struct CellPack {
    static constexpr int N = D + 7 + (SK ? D + 1 : 0);
    static constexpr int NV = (N + 3) / 4;
};

// Face constants from the face W (eq. phibar inverted: phi = eq + alpha (phibar - eq) [+ gb Z (g - g_eq)]).
template <typename T>
struct FaceC {
    T u[3];
    T cexp, pref, eb, hu2;
    T al_g, al_b, gam_b;
    T sq[3], e2;                // Shakhov constants of the face (as in CellC)
};

// Macroscopic state of a cell or face from its conserved variables (FP64).
struct Macro {
    double rho, u[3], T, RT;
};

// Explicitly rounded arithmetic in precision R (no multiply-add contraction),
// so every kernel that forms the constants below -- single instance or
// batched, any inlining context -- gets the same bits.
template <typename R> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double pow_(double a, double b) { return pow(a, b); }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float pow_(float a, float b) { return powf(a, b); }
};
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// x^omega for the viscosity law mu = mu_ref (T/T_ref)^omega: the hard-sphere
// (1/2) and Maxwell (1) exponents without the general power function.
template <typename R>
__device__ __forceinline__ R visc_power(R x, R omega) {
    return omega == R(0.5) ? Ar<R>::sqrt_(x) : (omega == R(1) ? x : Ar<R>::pow_(x, omega));
}
// x^(-D/2): the normalisation of a D-dimensional Maxwellian.
template <typename R>
__device__ __forceinline__ R gauss_norm(R x, int D) {
    using A = Ar<R>;
    return D == 2 ? A::div(R(1), x) : (D == 1 ? A::div(R(1), A::sqrt_(x)) : A::div(R(1), A::mul(x, A::sqrt_(x))));
}

__device__ __forceinline__ Macro macro_of(const Geo& g, const double* W) {
    Macro m;
    m.rho = W[0];
    const double irho = ddiv(1.0, m.rho);
    double u2 = 0.0;
    for (int a = 0; a < 3; ++a) m.u[a] = 0.0;
    for (int a = 0; a < g.D; ++a) {
        m.u[a] = dmul(W[1 + a], irho);
        u2 = dadd(u2, dmul(m.u[a], m.u[a]));
    }
    const double E = dmul(W[1 + g.D], irho);
    // T = (gamma - 1)/R (E - u^2/2), gamma = (K+5)/(K+3)
    m.T = dmul(ddiv(2.0, dmul(dadd(g.K, 3.0), g.R)), dsub(E, dmul(0.5, u2)));
    m.RT = dmul(g.R, m.T);
    return m;
}

// Inverse relaxation times in the storage precision R: 1/tau_g = p/mu,
// 1/tau_b = Pr/tau_g, 1/tau_b - 1/tau_g.  Inverse times stay finite in both
// limits (1/tau -> 0 as mu -> infinity), so every constant below is formed from
// them.  FP64 storage keeps all constants in FP64; FP32 storage forms them in
// FP32 from the FP64 macroscopic state (they are stored in FP32 either way).
template <typename R>
struct Relax {
    R itg, itb, itbg;
};
template <typename R>
__device__ __forceinline__ Relax<R> relax_of(const Geo& g, const Macro& m) {
    using A = Ar<R>;
    Relax<R> r;
    const R mu = A::mul((R)g.mu_ref, visc_power<R>(A::div((R)m.T, (R)g.T_ref), (R)g.omega));
    r.itg = A::div(A::mul((R)m.rho, (R)m.RT), mu);
    if (g.shakhov) {           // one relaxation time, no b-source
        r.itb = r.itg;
        r.itbg = R(0);
    } else {
        r.itb = A::mul((R)g.Pr, r.itg);
        r.itbg = A::mul(A::sub((R)g.Pr, R(1)), r.itg);
    }
    return r;
}

// The Shakhov S-model (the route to Pr != 1 that Sec. 1 names besides the
// two-time model; its form is Shakhov's, for all N = 3 + K degrees of freedom,
// integrated over the ones the velocity grid does not resolve):
//   g_S = g_M (1 + cq (c^2/RT - D - 2)),
//   b_S = g_M (|xi|^2/2 + eb + cq (|xi|^2/2 (c^2/RT - D - 2) + hL c^2 - e2)),
// c = xi - u, cq = sq . c, hL = (3 - D + K)/2.  Per cell or face (FP64 here):
// sq = (1 - Pr) q / ((K + 5) p RT) and e2 = hL D RT; q is the heat flux.
template <typename T>
__device__ __forceinline__ void shakhov_consts(const Geo& g, const Macro& m, const double* q, T sq[3], T& e2) {
    for (int a = 0; a < 3; ++a) sq[a] = T(0);
    e2 = T(0);
    if (!g.shakhov) return;
    const double A = ddiv(1.0 - g.Pr, dmul(dmul(g.K + 5.0, m.rho), dmul(m.RT, m.RT)));
    for (int a = 0; a < g.D; ++a) sq[a] = q ? (T)dmul(A, q[a]) : T(0);
    e2 = (T)dmul(dmul(0.5 * (3.0 - g.D + g.K), (double)g.D), m.RT);
}

// One velocity: the Shakhov equilibrium from the Maxwellian value gM.
template <typename T, int D>
__device__ __forceinline__ void shakhov_point(T gM, T c2, T cq, T irt, T hx, T eb, T hL, T e2, T& ge, T& be) {
    const T P1 = fma(c2, irt, T(-(D + 2)));
    ge = fma(gM * cq, P1, gM);
    be = gM * (hx + eb + cq * fma(hx, P1, fma(hL, c2, -e2)));
}

// Heat flux at a cell or face from the raw moments s = (sum w xi_a b [D],
// sum w xi_a xi_b g [a <= b]) of its distributions, relative to its conserved
// variables W (rho, u, E from W):
//   q_a = sum w xi_a b - u_a rho E - sum_b u_b (sum w xi_a xi_b g - rho u_a u_b).
template <int D>
__device__ __forceinline__ void heat_flux_raw(const Macro& m, const double* W, const double* s, double q[3]) {
    double Pi[3][3];
    int k = D;
    for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b) Pi[a][b] = Pi[b][a] = s[k++];
    for (int a = 0; a < 3; ++a) q[a] = 0.0;
    for (int a = 0; a < D; ++a) {
        double v = dsub(s[a], dmul(m.u[a], W[1 + D]));
        for (int b = 0; b < D; ++b) v = dsub(v, dmul(m.u[b], dsub(Pi[a][b], dmul(m.rho, dmul(m.u[a], m.u[b])))));
        q[a] = v;
    }
}

template <typename T>
__device__ __forceinline__ void eq_consts(const Geo& g, const Macro& m, T u[3], T& cexp, T& pref, T& eb, T& hu2) {
    using A = Ar<T>;
    double u2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        u[a] = (T)m.u[a];
        u2 = dadd(u2, dmul(m.u[a], m.u[a]));
    }
    const T RT = (T)m.RT;
    cexp = A::div((T)(-0.5 * Num<T>::cexp_scale()), RT);
    pref = A::mul((T)m.rho, gauss_norm<T>(A::mul((T)(2.0 * 3.14159265358979323846), RT), g.D));
    eb = A::mul((T)(0.5 * (3.0 - g.D + g.K)), RT);
    hu2 = (T)dmul(0.5, u2);
}

// Cell constants from W: equilibrium parameters and, with x = dt/(2 tau),
// fa = 1/(1 + x), fb = x fa (phi = fa phi* + fb phi_eq), kp = (1 - h/(2 tau)) fa,
// kp_s = (h/2)(1/tau_b - 1/tau_g) fa_g, um = 1 - x, usrc = dt (1/tau_b - 1/tau_g).
template <typename T>
__device__ __forceinline__ void make_cell(const Geo& g, const double* W, const double* q, CellC<T>& c) {
    using A = Ar<T>;
    const Macro m = macro_of(g, W);
    const Relax<T> r = relax_of<T>(g, m);
    eq_consts<T>(g, m, c.u, c.cexp, c.pref, c.eb, c.hu2);
    shakhov_consts<T>(g, m, q, c.sq, c.e2);
    const T dt = (T)g.dt, hh = (T)(0.5 * g.h), hdt = (T)(0.5 * g.dt);
    const T xg = A::mul(hdt, r.itg), xb = A::mul(hdt, r.itb);
    const T fa_g = A::div(T(1), A::add(T(1), xg)), fa_b = A::div(T(1), A::add(T(1), xb));
    c.fa_g = fa_g;
    c.fb_g = A::mul(xg, fa_g);
    c.fa_b = fa_b;
    c.fb_b = A::mul(xb, fa_b);
    c.kp_g = A::mul(A::sub(T(1), A::mul(hh, r.itg)), fa_g);
    c.kp_b = A::mul(A::sub(T(1), A::mul(hh, r.itb)), fa_b);
    c.kp_s = A::mul(A::mul(hh, r.itbg), fa_g);
    c.um_g = A::sub(T(1), xg);
    c.um_b = A::sub(T(1), xb);
    c.usrc = A::mul(dt, r.itbg);
}

// Face constants from the face W: equilibrium parameters, alpha = 1/(1 + h/(2 tau))
// (the inverse of eq. phibar) and gamma_b = (h/2)(1/tau_b - 1/tau_g) alpha_b.
template <typename T>
__device__ __forceinline__ void make_face(const Geo& g, const double* W, const double* q, FaceC<T>& f) {
    using A = Ar<T>;
    const Macro m = macro_of(g, W);
    const Relax<T> r = relax_of<T>(g, m);
    eq_consts<T>(g, m, f.u, f.cexp, f.pref, f.eb, f.hu2);
    shakhov_consts<T>(g, m, q, f.sq, f.e2);
    const T hh = (T)(0.5 * g.h);
    f.al_g = A::div(T(1), A::add(T(1), A::mul(hh, r.itg)));
    f.al_b = A::div(T(1), A::add(T(1), A::mul(hh, r.itb)));
    f.gam_b = A::mul(A::mul(hh, r.itbg), f.al_b);
}

// ---- separable Maxwellian factors (lean shapes)
//
// The Maxwellian of eq. geq factorises over the velocity axes:
//   g_eq(xi) = rho (2 pi RT)^{-D/2} prod_b exp(-(xi_b - u_b)^2 / (2RT)),
// so one place (a cell or a face) needs only sum_b nv1_b factors, not one
// exponential per velocity.  They are formed here in double for every node and
// stored in the working precision; the prefactor is folded into the factors of
// the last axis.  Per axis, from the node k* nearest u_b outward, the factors
// follow from E[k+1] = E[k] r_k, r_{k+1} = r_k q (and likewise downward) with
// r, s, q exponentials of the exact differences of the exponents, so the
// relative error of every factor is a few hundred double roundings at most,
// whatever c^2 / (2RT) is (high Mach).  Layout for n places:
//   axis 0 rows r < xrow[1]: [r / VC][n][VC] (a chunk's four factors are one vector),
//   rows r >= xrow[1]:       [r][n].
__host__ __device__ __forceinline__ size_t xaddr(const Geo& g, long long n, int r, long long item) {
    return r < g.xrow[1] ? ((size_t)(r / VC) * (size_t)n + (size_t)item) * VC + (size_t)(r % VC)
                         : (size_t)r * (size_t)n + (size_t)item;
}

template <typename T>
__device__ __forceinline__ void write_factors(const Geo& g, const Macro& m, T* __restrict__ X, long long n,
                                              long long item) {
    const double c = ddiv(0.5, m.RT);
    // rho (2 pi RT)^{-D/2}
    const double tp = dmul(2.0 * 3.14159265358979323846, m.RT);
    const double pref = ddiv(m.rho, g.D == 2 ? tp : (g.D == 1 ? sqrt(tp) : dmul(tp, sqrt(tp))));
    for (int b = 0; b < g.D; ++b) {
        const int nb = g.nv1[b];
        const double d = g.dxi[b], lo = g.vlo[b], ub = m.u[b];
        const int r0 = g.xrow[b];
        int ks = (int)rint((ub - lo) / d);
        ks = ks < 0 ? 0 : (ks > nb - 1 ? nb - 1 : ks);
        const double del = dsub(dadd(lo, dmul((double)ks, d)), ub);          // xi_{k*} - u_b
        const double q = exp(-dmul(2.0 * c, dmul(d, d)));
        double e0 = exp(-dmul(c, dmul(del, del)));
        if (b == g.D - 1) e0 = dmul(e0, pref);
        X[xaddr(g, n, r0 + ks, item)] = (T)e0;
        if (ks + 1 < nb) {
            double e = e0, r = exp(-dmul(c, dadd(dmul(2.0 * del, d), dmul(d, d))));
            for (int k = ks + 1; k < nb; ++k) {
                e = dmul(e, r);
                r = dmul(r, q);
                X[xaddr(g, n, r0 + k, item)] = (T)e;
            }
        }
        if (ks > 0) {
            double e = e0, s = exp(-dmul(c, dsub(dmul(d, d), dmul(2.0 * del, d))));
            for (int k = ks - 1; k >= 0; --k) {
                e = dmul(e, s);
                s = dmul(s, q);
                X[xaddr(g, n, r0 + k, item)] = (T)e;
            }
        }
        if (b == 0)
            for (int k = nb; k < g.xrow[1]; ++k) X[xaddr(g, n, k, item)] = T(0);   // padding of the last chunk
    }
}

// g_eq from the factors of one velocity, in the one order every kernel uses:
// x0 (x1 x2) in 3D, x0 x1 in 2D (the prefactor is inside x1 or x2).
template <typename T, int D>
__host__ __device__ __forceinline__ T lean_pair(T x1, T x2) {
    return D == 3 ? x1 * x2 : x1;
}
template <typename T, int D>
__host__ __device__ __forceinline__ T lean_geq(T x0, T x1, T x2) {
    return x0 * lean_pair<T, D>(x1, x2);
}

// g_eq of velocity i at cell c from the cell factor table (lean shapes).
template <typename T, int D>
__device__ __forceinline__ T table_geq(const Geo& g, const T* __restrict__ X, long long c, int i) {
    if (i >= g.nv1[0] * g.nv1[1] * g.nv1[2]) return T(0);
    const int k0 = i % g.nv1[0], k1 = (i / g.nv1[0]) % g.nv1[1], k2 = i / (g.nv1[0] * g.nv1[1]);
    const T x2 = D == 3 ? X[xaddr(g, g.Nc, g.xrow[2] + k2, c)] : T(1);
    return lean_geq<T, D>(X[xaddr(g, g.Nc, k0, c)], X[xaddr(g, g.Nc, g.xrow[1] + k1, c)], x2);
}

// Per-lane velocity data of one tile.
template <typename T, int D>
struct Vel {
    T xi[D];
    T nu[D];     // h xi_a / dx_a
    T w, hxi2;
};

template <typename T, int D>
__device__ __forceinline__ Vel<T, D> load_vel(const Geo& g, const Bufs<T>& bf, int i) {
    Vel<T, D> v;
    const T* rec = bf.vel + (size_t)i * 8;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        v.xi[a] = rec[a];
        v.nu[a] = (T)g.hdx[a] * v.xi[a];
    }
    v.w = rec[3];
    v.hxi2 = rec[4];
    return v;
}

// The equilibria of the collision model at one velocity (cell or face constants c).
template <typename T, int D, typename C>
__device__ __forceinline__ void equilibrium(const Geo& g, const C& c, const Vel<T, D>& v, T& geq, T& beq) {
    T c2 = T(0), cq = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        T d = v.xi[a] - c.u[a];
        c2 = fma(d, d, c2);
        cq = fma(c.sq[a], d, cq);
    }
    const T gM = c.pref * Num<T>::expo(c.cexp * c2);
    if (g.shakhov) {
        shakhov_point<T, D>(gM, c2, cq, c.cexp * Num<T>::irt_scale(), v.hxi2, c.eb, (T)(0.5 * (3.0 - D + g.K)), c.e2,
                            geq, beq);
    } else {
        geq = gM;
        beq = (v.hxi2 + c.eb) * geq;
    }
}


// ------------------------------------------------------------- accumulation

// Running sum of per-chunk partial sums: a Kahan pair in FP32, plain in FP64.
template <typename T> struct Kahan;
template <> struct Kahan<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct Kahan<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// ------------------------------------------------------------- geometry

// Map a cell coordinate that may lie in the ghost layers (two or three deep) onto the
// interior: axes resolved from the last to the first (the order in which
// ghost layers of later axes overwrite corners), periodic wrap, specular
// mirror (reflection bit set), Dirichlet clamp (flag).  Coordinates beyond the
// ghost layer (ragged tiles) are clamped; they are never read.
template <int D>
__device__ __forceinline__ void resolve(const Geo& g, int q[3], int& refl, bool& dir) {
    refl = 0;
    dir = false;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
        const int k = q[a], n = g.n[a];
        if (dir || (k >= 0 && k < n)) continue;
        const int bc = k < 0 ? g.bc[a][0] : g.bc[a][1];
        if (bc == BC_PERIODIC) {
            q[a] = ((k % n) + n) % n;
        } else if (bc == BC_SPECULAR) {
            q[a] = k < 0 ? -1 - k : 2 * n - 1 - k;
            refl ^= 1 << a;
        } else {
            dir = true;
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) q[a] = min(max(q[a], 0), g.n[a] - 1);
}

__device__ __forceinline__ long long cell_index(const Geo& g, const int q[3]) {
    return (long long)q[0] + (long long)g.n[0] * ((long long)q[1] + (long long)g.n[1] * q[2]);
}

__device__ __forceinline__ long long face_index(const Geo& g, int a, const int q[3]) {
    return (long long)q[0] + (long long)g.fn[a][0] * ((long long)q[1] + (long long)g.fn[a][1] * q[2]);
}

// Offset of (cell, velocity i, field) in the state layout [i/VC][cell][field][i%VC].
__device__ __forceinline__ size_t phi_addr(const Geo& g, long long cell, int i, int field) {
    return ((size_t)(i / VC) * (size_t)g.Nc + (size_t)cell) * (2 * VC) + (size_t)field * VC + (i % VC);
}

// A hint: fetch `bytes` (a multiple of 16, p 16-byte aligned, all inside one
// allocation) from global memory into L2.  No completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, int bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes));
}

// VC consecutive values as vector loads / stores (16-byte aligned by layout).
// NC = true reads through the non-coherent (read-only) path, for data no
// kernel of the running launch writes; the persistent batched step, whose
// items read what other items of the same launch wrote, loads coherently.
template <typename T> struct Chunk;
template <> struct Chunk<float> {
    template <bool NC = true>
    static __device__ __forceinline__ void load(const float* p, float (&v)[VC]) {
        const float4 a = NC ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    static __device__ __forceinline__ void store(float* p, const float (&v)[VC]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Chunk<double> {
    template <bool NC = true>
    static __device__ __forceinline__ void load(const double* p, double (&v)[VC]) {
        const double2 a = NC ? __ldg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
        const double2 b = NC ? __ldg(reinterpret_cast<const double2*>(p + 2)) : *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double* p, const double (&v)[VC]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};

// --------------------------------------------------------------- the sweep
//
// One CTA owns a tile of cells (one thread per cell) for the velocity tiles
// of its group and walks them VC velocities at a time.  Per chunk:
//   phase 1  phibar+ for the tile and its two-cell halo -> shared memory
//   phase 2  van Leer slopes (eq. VanLeer) of the cells one layer around
//            the tile -> shared memory
//   phase 3  per owned cell, its left faces (and right faces where no other
//            thread has them): upwind reconstruction (eq. relation).
//            Sweep A sums the face moments (eqs. rhobar-rhoEbar) in
//            registers; sweep B forms the face phi (eq. phibar inverted), the
//            flux xi_a phi and its moments, and stages the flux in shared memory
//   phase 4  (sweep B) per owned cell and velocity: net flux, phi* (eq. phiupdate).
// All threads of a warp hold the same velocity, so the upwind choice never
// diverges.

template <int D, int T0_, int T1_, int T2_, int HALO_ = 2>
struct Tile {
    static constexpr int T0 = T0_, T1 = D >= 2 ? T1_ : 1, T2 = D >= 3 ? T2_ : 1;
    static constexpr int NT = T0 * T1 * T2;                                   // threads = owned cells
    // halo box: local cells [-HALO, T + HALO - 1] per active axis (2, or 3 for the
    // face-gradient reconstruction, which also needs derivatives of the slopes)
    static constexpr int HALO = HALO_;
    static constexpr int E0 = T0 + 2 * HALO, E1 = D >= 2 ? T1 + 2 * HALO : 1, E2 = D >= 3 ? T2 + 2 * HALO : 1;
    static constexpr int BOX = E0 * E1 * E2;
    static constexpr int NH = BOX - NT;
    // slope box: local cells [-(HALO-1), T + HALO - 2] per active axis
    static constexpr int F0 = T0 + 2 * (HALO - 1), F1 = D >= 2 ? T1 + 2 * (HALO - 1) : 1;
    static constexpr int F2 = D >= 3 ? T2 + 2 * (HALO - 1) : 1;
    static constexpr int SB = F0 * F1 * F2;
    // slope-derivative box (HALO = 3): local cells [-1, T] per active axis
    static constexpr int G0 = T0 + 2, G1 = D >= 2 ? T1 + 2 : 1, G2 = D >= 3 ? T2 + 2 : 1;
    static constexpr int SB2 = G0 * G1 * G2;
    static constexpr int NF0 = (T0 + 1) * T1 * T2;
    static constexpr int NF1 = D >= 2 ? T0 * (T1 + 1) * T2 : 0;
    static constexpr int NF2 = D >= 3 ? T0 * T1 * (T2 + 1) : 0;
    static constexpr int NFT = NF0 + NF1 + NF2;
    __host__ __device__ static constexpr int bstride(int a) { return a == 0 ? 1 : (a == 1 ? E0 : E0 * E1); }
    __host__ __device__ static constexpr int sstride(int a) { return a == 0 ? 1 : (a == 1 ? F0 : F0 * F1); }
    __host__ __device__ static constexpr int s2stride(int a) { return a == 0 ? 1 : (a == 1 ? G0 : G0 * G1); }
    __host__ __device__ static constexpr int tdim(int a) { return a == 0 ? T0 : (a == 1 ? T1 : T2); }
    __host__ __device__ static constexpr int foff(int a) {
        return a == 0 ? 0 : (a == 1 ? NF0 : (a == 2 ? NF0 + NF1 : NFT));
    }
    // cells on a tile face normal to axis a, and where their slots start in a list over all axes
    __host__ __device__ static constexpr int plane(int a) { return NT / tdim(a); }
    __host__ __device__ static constexpr int poff(int a) {
        return (a > 0 ? plane(0) : 0) + (a > 1 && D >= 2 ? plane(1) : 0) + (a > 2 && D >= 3 ? plane(2) : 0);
    }
    static constexpr int NPL = (D >= 1 ? NT / T0 : 0) + (D >= 2 ? NT / T1 : 0) + (D >= 3 ? NT / T2 : 0);
    // this cell's slot on the tile face normal to axis a
    __device__ static __forceinline__ int plane_pos(int a, const int la[3]) {
        return a == 0 ? la[1] + T1 * la[2] : (a == 1 ? la[0] + T0 * la[2] : la[0] + T0 * la[1]);
    }
    __device__ static __forceinline__ int box_of(int l0, int l1, int l2) {
        return (l0 + HALO) + E0 * ((D >= 2 ? l1 + HALO : 0) + E1 * (D >= 3 ? l2 + HALO : 0));
    }
    __device__ static __forceinline__ int sbox_of(int l0, int l1, int l2) {
        constexpr int o = HALO - 1;
        return (l0 + o) + F0 * ((D >= 2 ? l1 + o : 0) + F1 * (D >= 3 ? l2 + o : 0));
    }
    __device__ static __forceinline__ int s2box_of(int l0, int l1, int l2) {
        return (l0 + 1) + G0 * ((D >= 2 ? l1 + 1 : 0) + G1 * (D >= 3 ? l2 + 1 : 0));
    }
    // local coordinates of slope-box cell s
    __device__ static __forceinline__ void sbox_local(int s, int l[3]) {
        l[0] = s % F0 - (HALO - 1);
        l[1] = D >= 2 ? (s / F0) % F1 - (HALO - 1) : 0;
        l[2] = D >= 3 ? s / (F0 * F1) - (HALO - 1) : 0;
    }
    // local face of axis a whose right cell has local coordinates l (l_a in [0, T_a])
    __device__ static __forceinline__ int face_local(int a, int l0, int l1, int l2) {
        const int d0 = T0 + (a == 0), d1 = T1 + (a == 1);
        return foff(a) + l0 + d0 * (l1 + d1 * l2);
    }
};

// Four values of the working precision: one velocity chunk of one cell, or
// four packed constants.  Aligned so that shared-memory traffic is 128-bit.
template <typename T>
struct alignas(4 * sizeof(T)) V4 {
    T v[4];
};

// Asynchronous global -> shared copies (cp.async): one VC chunk (16-byte
// pieces; both addresses 16-byte aligned by the layouts) or one element.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(__cvta_generic_to_global(gsrc))
                 : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_chunk(V4<T>* sdst, const T* gsrc) {
#pragma unroll
    for (int i = 0; i < (int)(sizeof(V4<T>) / 16); ++i)
        cp_async16(reinterpret_cast<char*>(sdst) + 16 * i, reinterpret_cast<const char*>(gsrc) + 16 * i);
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(__cvta_generic_to_global(gsrc)),
                 "n"((int)sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---- programmatic dependent launch: the kernels of a step are launched so
// that the next one may be scheduled while the previous one drains; each
// waits here, before it reads anything its predecessor wrote (a no-op when
// launched without the attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ---- TMA (cp.async.bulk.tensor) and mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// generic-proxy accesses of shared memory before async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];\n" ::
            "r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];\n" ::
            "r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}


// Sweep modes.  The low two bits say where sweep A (and a recomputing sweep
// B) takes phibar+ and the slopes from: 0 forms both on the halo box itself;
// 1 (prepared) loads phibar+ formed by k_prep and forms the slopes; 2 (stored)
// loads phibar+ and the slopes formed by k_shslope.  Bit 2 (face store):
// sweep A also writes the reconstructed face values, and sweep B is k_flux,
// which reads them instead of reconstructing them again.
// Bit 3 (face gradient): the paper's variant of the reconstruction, which also
// carries the slopes to the face with their own limited derivatives (three
// halo layers; fused face-store shapes only).
// Bit 4 (Shakhov): the sweeps and k_flux evaluate the Shakhov equilibria
// (face-store shapes only); k_faceq and k_cellq add the raw moments the heat
// flux needs.
// Bit 5 (acceleration): k_prep adds the force terms of the sources (prepared
// face-store shapes only) and k_flux takes them at the faces and in phi*.
// Bit 6 (launch-time, not a tile shape): the instance has no b-source, so
// sweep A and k_flux leave out Z = xi.u - u^2/2 and its terms (whose
// coefficients are then exactly 0: the same results, fewer instructions).
// Bit 7 (lean): the face-store shapes whose sweep A is lean.cuh's (D = 2, 3; the
// two-time model, upwind-cell reconstruction, velocity grids without a node at
// xi_a = 0): its cell equilibria are products of per-axis Maxwellian factors
// formed in double, kept in tables of every cell.  Bit 8 (face tables): sweep B
// is lean.cuh's as well and takes the face equilibria from factor tables of
// every face; without it sweep B is k_flux (an FP32 exponential per point).
enum {
    MODE_FUSED = 0, MODE_PREP = 1, MODE_STORED = 2, MODE_FACES = 4, MODE_R2 = 8, MODE_SK = 16, MODE_ACC = 32,
    MODE_NOSRC = 64, MODE_LEAN = 128, MODE_XF = 256
};
__host__ __device__ constexpr int mode_source(int mode) { return mode & 3; }
__host__ __device__ constexpr bool mode_faces(int mode) { return (mode & MODE_FACES) != 0; }
__host__ __device__ constexpr bool mode_r2(int mode) { return (mode & MODE_R2) != 0; }
__host__ __device__ constexpr bool mode_sk(int mode) { return (mode & MODE_SK) != 0; }
__host__ __device__ constexpr bool mode_acc(int mode) { return (mode & MODE_ACC) != 0; }
__host__ __device__ constexpr bool mode_nosrc(int mode) { return (mode & (MODE_NOSRC | MODE_SK)) != 0; }
__host__ __device__ constexpr int mode_halo(int mode) { return mode_r2(mode) ? 3 : 2; }
__host__ __device__ constexpr bool mode_lean(int mode) { return (mode & MODE_LEAN) != 0; }
__host__ __device__ constexpr bool mode_xf(int mode) { return (mode & MODE_XF) != 0; }

template <typename T, int D, int T0, int T1, int T2, int MODE = MODE_FUSED>
struct Smem {
    using TL = Tile<D, T0, T1, T2, mode_halo(MODE)>;
    static constexpr int NCCV = CellPack<D, mode_sk(MODE)>::NV;  // phase-1 constants per box cell, packed in V4
    static constexpr int NFC = D + 7;            // face constants
    static constexpr int NFCV = (NFC + 3) / 4;
    static constexpr int PN = mode_source(MODE) == MODE_STORED ? TL::SB : TL::BOX;   // cells of the phibar+ array
    static constexpr size_t nP = (size_t)2 * PN;                                    // V4 units
    static constexpr size_t nS = (size_t)D * 2 * TL::SB;
    static constexpr size_t nS2 = mode_r2(MODE) ? (size_t)D * D * 2 * TL::SB2 : 0;   // slope derivatives
    static constexpr size_t nCC = mode_source(MODE) == MODE_FUSED ? (size_t)NCCV * TL::BOX : 0;
    static constexpr size_t nFF = (size_t)2 * TL::NFT;
    static constexpr size_t nFC = (size_t)NFCV * TL::NFT;
    static constexpr size_t nInt = (size_t)2 * TL::BOX + TL::NH + 32;
    // Kahan sums of the faces at the domain's right end, [NM][plane slot] per axis (owned by the last cells)
    static constexpr size_t nRS = (size_t)TL::NPL * (2 + D);
    static constexpr size_t rs_bytes = nRS * sizeof(Kahan<T>);
    // CTAs per SM that a dynamic shared-memory size allows, and the limit of threads and >= 80 registers
    __host__ __device__ static constexpr int fit(size_t b) { return (int)((size_t)(228 * 1024) / (b + 1024)); }
    static constexpr int lim = (2048 / TL::NT) < (65536 / (TL::NT * 80)) ? (2048 / TL::NT) : (65536 / (TL::NT * 80));
    // staged phi* chunk per box cell: g at [0, BOXP), b at [BOXP, 2 BOXP) (BOXP: BOX rounded to 128 B
    // for TMA), then slack for the 128-byte alignment of TMA destinations and the mbarrier
    static constexpr int BOXP = (TL::BOX * (int)sizeof(V4<T>) + 127) / 128 * 128 / (int)sizeof(V4<T>);
    static constexpr size_t nST = (size_t)2 * BOXP + 256 / sizeof(V4<T>);
    static constexpr size_t a1 = (nP + nS + nS2 + nCC) * sizeof(V4<T>) + rs_bytes + sizeof(int) * nInt;   // sweep A
    static constexpr bool st_fits = fit(a1 + nST * sizeof(V4<T>)) >= (fit(a1) < lim ? fit(a1) : lim);
    // Sweep A of the fused shapes stages the next chunk's phi* of its halo box in
    // shared memory with asynchronous copies (where that costs no occupancy), so
    // the loads overlap phases 2-3 of the current chunk.
    __host__ __device__ static constexpr bool stage(bool B) {
        return !B && mode_source(MODE) == MODE_FUSED && st_fits;
    }
    __host__ __device__ static constexpr size_t vcount(bool B) {
        return nP + nS + nS2 + nCC + (B ? nFF + nFC : 0) + (stage(B) ? nST : 0);
    }
    __host__ __device__ static constexpr size_t bytes(bool B) {
        return vcount(B) * sizeof(V4<T>) + rs_bytes + sizeof(int) * nInt;
    }
};

// Offset of the chunk vt of face f (axis a) in the face-value layout.
__device__ __forceinline__ size_t face_addr(const Geo& g, int a, long long f, int vt) {
    return ((size_t)vt * (size_t)g.nf[a] + (size_t)f) * (2 * VC);
}

// Offset of (cell, velocity i, axis a, field f) in the slope layout.
template <int D>
__device__ __forceinline__ size_t sig_addr(const Geo& g, long long cell, int i, int a, int f) {
    return ((size_t)(i / VC) * (size_t)g.Nc + (size_t)cell) * (2 * D * VC) + (size_t)(a * 2 + f) * VC + (i % VC);
}

// phibar+ of one point (eq. phibarplus) from the stored phi* (gs, bs), the
// equilibrium (ge, be), Z = xi.u - |u|^2/2 and the cell constants.
// (NOSRC: kp_s = 0, the source term is left out.)
template <typename T, bool NOSRC = false>
__device__ __forceinline__ void phibar_plus(T ge, T be, T gs, T bs, T z, T kp_g, T kp_b, T kp_s, T& pg, T& pb) {
    const T dg = gs - ge;
    pg = fma(kp_g, dg, ge);
    if constexpr (NOSRC) pb = fma(kp_b, bs - be, be);
    else pb = fma(kp_s * z, dg, fma(kp_b, bs - be, be));
}

// Pack a cell's phibar+ constants (CellPack order; u and the heat flux with
// the components of a mirror image reversed) into V4 slots dst[j * stride].
template <typename T, int D, bool SK = false>
__device__ __forceinline__ void pack_cell(const CellC<T>& cs, int refl, V4<T>* dst, int stride) {
    using CP = CellPack<D, SK>;
    T cst[4 * CP::NV];
#pragma unroll
    for (int a = 0; a < D; ++a) cst[a] = (refl & (1 << a)) ? -cs.u[a] : cs.u[a];
    cst[D + 0] = cs.cexp;
    cst[D + 1] = cs.pref;
    cst[D + 2] = cs.eb;
    cst[D + 3] = cs.hu2;
    cst[D + 4] = cs.kp_g;
    cst[D + 5] = cs.kp_b;
    cst[D + 6] = cs.kp_s;
    if constexpr (SK) {
#pragma unroll
        for (int a = 0; a < D; ++a) cst[D + 7 + a] = (refl & (1 << a)) ? -cs.sq[a] : cs.sq[a];
        cst[2 * D + 7] = cs.e2;
    }
#pragma unroll
    for (int j = CP::N; j < 4 * CP::NV; ++j) cst[j] = T(0);
#pragma unroll
    for (int j = 0; j < CP::NV; ++j) {
        V4<T> qv;
#pragma unroll
        for (int e = 0; e < 4; ++e) qv.v[e] = cst[4 * j + e];
        dst[j * stride] = qv;
    }
}

// The equilibria at one velocity from packed constants cst (CellPack or
// FacePack order: u at 0, cexp at D, pref at D+1, eb at D+2, and with SK sq at
// D+7 and e2 at 2D+7) and the velocity xi (hx = |xi|^2/2); also Z = xi.u - hu2.
template <typename T, int D, bool SK, bool NOZ = false>
__device__ __forceinline__ void packed_eq(const T* cst, const T (&xi)[D], T hx, T hL, T& ge, T& be, T& z) {
    T c2 = T(0), cq = T(0);
    z = NOZ ? T(0) : -cst[D + 3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T d = xi[a] - cst[a];
        c2 = fma(d, d, c2);
        if constexpr (!NOZ) z = fma(xi[a], cst[a], z);
        if constexpr (SK) cq = fma(cst[D + 7 + a], d, cq);
    }
    const T gM = cst[D + 1] * Num<T>::expo(cst[D + 0] * c2);
    if constexpr (SK) {
        shakhov_point<T, D>(gM, c2, cq, cst[D + 0] * Num<T>::irt_scale(), hx, cst[D + 2], hL, cst[2 * D + 7], ge, be);
    } else {
        ge = gM;
        be = (hx + cst[D + 2]) * ge;
    }
}

// ---- external acceleration (eqs. gsource, bsource)
//
// The velocity-gradient parts of the force terms at velocity i of one place:
// fg = -sum_b a_b (g(i + s_b) - g(i - s_b)) / (2 dxi_b), fb likewise from b,
// central differences on the velocity grid with the distribution taken as 0
// beyond its ends (s_b the index stride of axis b).  val(j, g, b) supplies
// the distributions at velocity j; acc the force to use (a face at a
// specular wall leaves out its normal component).
template <typename T, int D, typename F>
__device__ __forceinline__ void force_gradient(const Geo& g, const double* acc, int i, F&& val, T& fg, T& fb) {
    fg = T(0);
    fb = T(0);
    int stride = 1;
#pragma unroll
    for (int b = 0; b < D; ++b) {
        const int k = (i / stride) % g.nv1[b];
        if (acc[b] != 0.0) {
            T gp = T(0), gm = T(0), bp = T(0), bm = T(0);
            if (k + 1 < g.nv1[b]) val(i + stride, gp, bp);
            if (k >= 1) val(i - stride, gm, bm);
            const T c = (T)(acc[b] / (2.0 * g.dxi[b]));
            fg = fma(-c, gp - gm, fg);
            fb = fma(-c, bp - bm, fb);
        }
        stride *= g.nv1[b];
    }
}

// The same for the four velocities of chunk vt at once, when every row of
// the velocity grid is whole chunks (nv1_0 a multiple of VC): the neighbour
// of a lane along axis b > 0 is the same lane of chunk vt +- s_b/VC, along
// axis 0 the next lane (or the end lane of chunk vt +- 1).  chunk(vn, gv, bv)
// loads the distributions of chunk vn; (gc, bc) are those of chunk vt.  Whole
// chunks are vector loads, coalesced across the cells (or faces) of a warp.
template <typename T, int D, typename F>
__device__ __forceinline__ void force_gradient_chunk(const Geo& g, const double* acc, int vt, F&& chunk,
                                                     const T (&gc)[VC], const T (&bc)[VC], T (&fg)[VC],
                                                     T (&fb)[VC]) {
#pragma unroll
    for (int v = 0; v < VC; ++v) fg[v] = fb[v] = T(0);
    int stride = 1;
#pragma unroll
    for (int b = 0; b < D; ++b) {
        if (acc[b] != 0.0) {
            const T c = (T)(acc[b] / (2.0 * g.dxi[b]));
            T gp[VC], gm[VC], bp[VC], bm[VC];
            const int k0 = ((vt * VC) / stride) % g.nv1[b];      // lane 0's index along b
            if (b == 0) {
                T gn[VC], bn[VC];
                const bool up = k0 + VC < g.nv1[0], dn = k0 >= 1;
                if (up) chunk(vt + 1, gn, bn);
#pragma unroll
                for (int v = 0; v < VC - 1; ++v) { gp[v] = gc[v + 1]; bp[v] = bc[v + 1]; }
                gp[VC - 1] = up ? gn[0] : T(0);
                bp[VC - 1] = up ? bn[0] : T(0);
                if (dn) chunk(vt - 1, gn, bn);
#pragma unroll
                for (int v = 1; v < VC; ++v) { gm[v] = gc[v - 1]; bm[v] = bc[v - 1]; }
                gm[0] = dn ? gn[VC - 1] : T(0);
                bm[0] = dn ? bn[VC - 1] : T(0);
            } else {                                          // the four lanes share their index along b
                const int sc = stride / VC;
                if (k0 + 1 < g.nv1[b]) chunk(vt + sc, gp, bp);
                else
#pragma unroll
                    for (int v = 0; v < VC; ++v) gp[v] = bp[v] = T(0);
                if (k0 >= 1) chunk(vt - sc, gm, bm);
                else
#pragma unroll
                    for (int v = 0; v < VC; ++v) gm[v] = bm[v] = T(0);
            }
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                fg[v] = fma(-c, gp[v] - gm[v], fg[v]);
                fb[v] = fma(-c, bp[v] - bm[v], fb[v]);
            }
        }
        stride *= g.nv1[b];
    }
}

// phibar+ (eq. phibarplus) of every point, for the prepared-shift shapes:
// one thread per cell over a run of velocity chunks, constants read once.
// With the acceleration (ACC) it also forms the force terms F^n of the
// sources from phi^n (= fa phi* + fb phi_eq) at the neighbouring velocities,
// adds h/2 of them to phibar+ and stores them for the update.
template <typename T, int D, bool ACC>
__device__ __forceinline__ void prep_body(const Geo& g, const Bufs<T>& bf, long long c, int vt0, int vt1) {
    const CellC<T> cs = bf.cellc[c];
    // phi^n of this cell at velocity j (the deferred end of eq. phiupdate)
    auto phin = [&](int j, T& gv, T& bv) {
        const T* rec = bf.vel + (size_t)j * 8;
        T c2 = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const T d = rec[a] - cs.u[a];
            c2 = fma(d, d, c2);
        }
        const T ge = cs.pref * Num<T>::expo(cs.cexp * c2);
        const T be = (rec[4] + cs.eb) * ge;
        gv = fma(cs.fa_g, bf.phi_in[phi_addr(g, c, j, 0)], cs.fb_g * ge);
        bv = fma(cs.fa_b, bf.phi_in[phi_addr(g, c, j, 1)], cs.fb_b * be);
    };
    // phi^n of this cell for the four velocities of chunk vn
    auto phin_chunk = [&](int vn, T (&gv)[VC], T (&bv)[VC]) {
        const size_t an = phi_addr(g, c, vn * VC, 0);
        T gsn[VC], bsn[VC];
        Chunk<T>::load(bf.phi_in + an, gsn);
        Chunk<T>::load(bf.phi_in + an + VC, bsn);
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const T* rec = bf.vel + (size_t)(vn * VC + v) * 8;
            T c2 = T(0);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const T d = rec[a] - cs.u[a];
                c2 = fma(d, d, c2);
            }
            const T ge = cs.pref * Num<T>::expo(cs.cexp * c2);
            const T be = (rec[4] + cs.eb) * ge;
            gv[v] = fma(cs.fa_g, gsn[v], cs.fb_g * ge);
            bv[v] = fma(cs.fa_b, bsn[v], cs.fb_b * be);
        }
    };
    const bool rows = g.nv1[0] % VC == 0;      // velocity rows are whole chunks
    for (int vt = vt0; vt < vt1; ++vt) {
        const size_t ad = phi_addr(g, c, vt * VC, 0);
        T gs[VC], bs[VC], pg[VC], pb[VC], fg[VC], fb[VC], gn0[VC], bn0[VC];
        Chunk<T>::load(bf.phi_in + ad, gs);
        Chunk<T>::load(bf.phi_in + ad + VC, bs);
        if constexpr (ACC) {
            if (rows) {
                phin_chunk(vt, gn0, bn0);
                force_gradient_chunk<T, D>(g, g.acc, vt, phin_chunk, gn0, bn0, fg, fb);
            }
        }
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const T* rec = bf.vel + (size_t)(vt * VC + v) * 8;
            T c2 = T(0), z = -cs.hu2;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const T d = rec[a] - cs.u[a];
                c2 = fma(d, d, c2);
                z = fma(rec[a], cs.u[a], z);
            }
            const T ge = cs.pref * Num<T>::expo(cs.cexp * c2);
            const T be = (rec[4] + cs.eb) * ge;
            phibar_plus<T>(ge, be, gs[v], bs[v], z, cs.kp_g, cs.kp_b, cs.kp_s, pg[v], pb[v]);
            if constexpr (ACC) {
                const int i = vt * VC + v;
                if (!rows) fg[v] = fb[v] = T(0);
                if (i < g.nv1[0] * g.nv1[1] * g.nv1[2]) {
                    if (!rows) force_gradient<T, D>(g, g.acc, i, phin, fg[v], fb[v]);
                    T ax = T(0);
#pragma unroll
                    for (int a = 0; a < D; ++a) ax = fma((T)g.acc[a], rec[a], ax);
                    const T gn = fma(cs.fa_g, gs[v], cs.fb_g * ge);      // phi^n at i
                    fb[v] = fma(ax, gn, fb[v]);
                }
                const T hh = (T)(0.5 * g.h);
                pg[v] = fma(hh, fg[v], pg[v]);
                pb[v] = fma(hh, fb[v], pb[v]);
            }
        }
        Chunk<T>::store(bf.phibar + ad, pg);
        Chunk<T>::store(bf.phibar + ad + VC, pb);
        if constexpr (ACC) {
            Chunk<T>::store(bf.force + ad, fg);
            Chunk<T>::store(bf.force + ad + VC, fb);
        }
    }
}

template <typename T, int D, bool ACC = false>
__global__ void k_prep(const Inst<T>* __restrict__ in, int cur, int chunks_per_thread) {
    pdl_wait();
    const Geo g = in->g;
    const Bufs<T> bf = in->b[cur];
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Nc) return;
    const int vt0 = blockIdx.y * chunks_per_thread;
    prep_body<T, D, ACC>(g, bf, c, vt0, min(g.NVT, vt0 + chunks_per_thread));
}

// Batched: one CTA per item = cells [start, start + count) of one instance and
// the run of kPrepChunks velocity chunks numbered axis (count <= blockDim).
// Both pre-pass launches use blocks of kPrepCells cells, one thread per cell.
constexpr int kPrepChunks = 8;
constexpr int kPrepCells = 128;
template <typename T, int D, bool ACC>
__global__ void k_prep_batch(const RItem* __restrict__ items, const Inst<T>* __restrict__ insts,
                             const int* __restrict__ cur) {
    pdl_wait();
    const RItem it = items[blockIdx.x];
    if (threadIdx.x >= it.count) return;
    const Inst<T>& in = insts[it.inst];
    const int vt0 = it.axis * kPrepChunks;
    prep_body<T, D, ACC>(in.g, in.b[cur[it.inst] & 1], it.start + threadIdx.x, vt0, min(in.g.NVT, vt0 + kPrepChunks));
}

// phibar+ and its van Leer slopes for every point, for the stored shapes: one
// CTA per tile of cells and group of velocity chunks, phibar+ formed on the
// tile and a one-cell halo in shared memory, slopes of the tile's own cells,
// both written in their layouts.
template <typename T, int D, int T0_, int T1_, int T2_, bool SK = false>
__host__ __device__ constexpr size_t shslope_smem_bytes() {
    using TL = Tile<D, T0_, T1_, T2_>;
    return ((size_t)2 * TL::SB + (size_t)CellPack<D, SK>::NV * TL::SB) * sizeof(V4<T>) + sizeof(int) * 2 * TL::SB;
}

template <typename T, int D, int T0_, int T1_, int T2_, bool SK = false>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT) k_shslope(const Inst<T>* __restrict__ in, int cur) {
    pdl_wait();
    using TL = Tile<D, T0_, T1_, T2_>;
    using Q = V4<T>;
    constexpr int SB = TL::SB, NCCV = CellPack<D, SK>::NV;
    extern __shared__ __align__(128) unsigned char smem[];
    const Geo g = in->g;
    const Bufs<T> bf = in->b[cur];
    Q* const P = reinterpret_cast<Q*>(smem);      // [2][SB]
    Q* const CC = P + 2 * SB;                     // [NCCV][SB]
    int* const csrc = reinterpret_cast<int*>(CC + NCCV * SB);
    int* const cfl = csrc + SB;
    const int t = threadIdx.x;
    int tb = blockIdx.x;
    int org[3] = {0, 0, 0};
    org[0] = (tb % g.tiles[0]) * TL::T0;
    tb /= g.tiles[0];
    if (D >= 2) { org[1] = (tb % g.tiles[1]) * TL::T1; tb /= g.tiles[1]; }
    if (D >= 3) org[2] = tb * TL::T2;
    const int vt0 = blockIdx.y * g.ntpg, vt1 = min(g.NVT, vt0 + g.ntpg);
    auto local = [&](int s2, int l[3]) {
        l[0] = s2 % TL::F0 - 1;
        l[1] = D >= 2 ? (s2 / TL::F0) % TL::F1 - 1 : 0;
        l[2] = D >= 3 ? s2 / (TL::F0 * TL::F1) - 1 : 0;
    };
    for (int s2 = t; s2 < SB; s2 += TL::NT) {
        int l[3];
        local(s2, l);
        int q[3] = {org[0] + l[0], org[1] + l[1], org[2] + l[2]};
        int refl;
        bool dir;
        resolve<D>(g, q, refl, dir);
        const long long c = cell_index(g, q);
        pack_cell<T, D, SK>(bf.cellc[c], refl, CC + s2, SB);
        csrc[s2] = (int)c;
        cfl[s2] = refl;
    }
    __syncthreads();
    const int la[3] = {t % TL::T0, D >= 2 ? (t / TL::T0) % TL::T1 : 0, D >= 3 ? t / (TL::T0 * TL::T1) : 0};
    const int qa[3] = {org[0] + la[0], org[1] + la[1], org[2] + la[2]};
    bool valid = true;
#pragma unroll
    for (int a = 0; a < D; ++a) valid = valid && qa[a] < g.n[a];
    const int sc = TL::sbox_of(la[0], la[1], la[2]);
    const long long own = valid ? cell_index(g, qa) : 0;
    const T hL = (T)(0.5 * (3.0 - D + g.K));
    for (int vt = vt0; vt < vt1; ++vt) {
        T xi[VC][D], hx[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const T* rec = bf.vel + (size_t)(vt * VC + v) * 8;
#pragma unroll
            for (int a = 0; a < D; ++a) xi[v][a] = rec[a];
            hx[v] = rec[4];
        }
        for (int s2 = t; s2 < SB; s2 += TL::NT) {
            const int rf = cfl[s2];
            const long long c = csrc[s2];
            T cst[4 * NCCV];
#pragma unroll
            for (int j = 0; j < NCCV; ++j) {
                const Q qv = CC[j * SB + s2];
#pragma unroll
                for (int e = 0; e < 4; ++e) cst[4 * j + e] = qv.v[e];
            }
            T gs[VC], bs[VC];
            if (rf) {
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    const int is = bf.refl[rf * g.Nvp + vt * VC + v];
                    gs[v] = bf.phi_in[phi_addr(g, c, is, 0)];
                    bs[v] = bf.phi_in[phi_addr(g, c, is, 1)];
                }
            } else {
                const size_t ad = phi_addr(g, c, vt * VC, 0);
                Chunk<T>::load(bf.phi_in + ad, gs);
                Chunk<T>::load(bf.phi_in + ad + VC, bs);
            }
            Q qg, qb;
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                T ge, be, z;
                packed_eq<T, D, SK>(cst, xi[v], hx[v], hL, ge, be, z);
                phibar_plus<T>(ge, be, gs[v], bs[v], z, cst[D + 4], cst[D + 5], cst[D + 6], qg.v[v], qb.v[v]);
            }
            P[0 * SB + s2] = qg;
            P[1 * SB + s2] = qb;
        }
        __syncthreads();
        if (valid) {
            const size_t ad = phi_addr(g, own, vt * VC, 0);
            Chunk<T>::store(bf.phibar + ad, P[0 * SB + sc].v);
            Chunk<T>::store(bf.phibar + ad + VC, P[1 * SB + sc].v);
            const size_t as = sig_addr<D>(g, own, vt * VC, 0, 0);
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const Q c = P[f * SB + sc];
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const int st = TL::sstride(a);
                    const Q l = P[f * SB + sc - st], r = P[f * SB + sc + st];
                    T o[VC];
#pragma unroll
                    for (int v = 0; v < VC; ++v) o[v] = Num<T>::vanleer(c.v[v] - l.v[v], r.v[v] - c.v[v]);
                    Chunk<T>::store(bf.sigma + as + (a * 2 + f) * VC, o);
                }
            }
        }
        __syncthreads();
    }
}

// ---- pieces shared by the recomputing sweep B and k_flux

// First owned cell of tile number `tile` (tiles numbered x fastest).
template <typename TL, int D>
__device__ __forceinline__ void tile_origin(const Geo& g, int tile, int org[3]) {
    int tb = tile;
    org[0] = (tb % g.tiles[0]) * TL::T0;
    org[1] = org[2] = 0;
    tb /= g.tiles[0];
    if (D >= 2) { org[1] = (tb % g.tiles[1]) * TL::T1; tb /= g.tiles[1]; }
    if (D >= 3) org[2] = tb * TL::T2;
}

// Face constants packed per face: u (D), cexp, pref, eb, hu2, alpha_g, alpha_b,
// gamma_b, and with the Shakhov model sq (D), e2.
template <int D, bool SK = false>
struct FacePack {
    static constexpr int N = D + 7 + (SK ? D + 1 : 0);
    static constexpr int NV = (N + 3) / 4;   // V4 units
};

// The packed constants of every face of the tile (both ends of each axis)
// into shared memory, FC[j * NFT + local face].
template <typename T, int D, typename TL, bool SK = false>
__device__ __forceinline__ void stage_face_consts(const Geo& g, const Bufs<T>& bf, const int org[3], V4<T>* FC) {
    constexpr int NFCV = FacePack<D, SK>::NV, NFT = TL::NFT;
#pragma unroll
    for (int a = 0; a < D; ++a)
    for (int r = threadIdx.x; r < TL::foff(a + 1) - TL::foff(a); r += TL::NT) {
        const int f = TL::foff(a) + r;
        const int d0 = TL::T0 + (a == 0), d1 = TL::T1 + (a == 1);
        int q[3] = {org[0] + r % d0, org[1] + (D >= 2 ? (r / d0) % d1 : 0), org[2] + (D >= 3 ? r / (d0 * d1) : 0)};
        bool ok = true;
#pragma unroll
        for (int b = 0; b < D; ++b) ok = ok && q[b] <= g.n[b] - (b == a ? 0 : 1);
        if (!ok) continue;
        const FaceC<T>& fs = bf.facec[a][face_index(g, a, q)];
        T cst[4 * NFCV];
#pragma unroll
        for (int b = 0; b < D; ++b) cst[b] = fs.u[b];
        cst[D + 0] = fs.cexp;
        cst[D + 1] = fs.pref;
        cst[D + 2] = fs.eb;
        cst[D + 3] = fs.hu2;
        cst[D + 4] = fs.al_g;
        cst[D + 5] = fs.al_b;
        cst[D + 6] = fs.gam_b;
        if constexpr (SK) {
#pragma unroll
            for (int b = 0; b < D; ++b) cst[D + 7 + b] = fs.sq[b];
            cst[2 * D + 7] = fs.e2;
        }
#pragma unroll
        for (int j = FacePack<D, SK>::N; j < 4 * NFCV; ++j) cst[j] = T(0);
#pragma unroll
        for (int j = 0; j < NFCV; ++j) {
            V4<T> qv;
#pragma unroll
            for (int e = 0; e < 4; ++e) qv.v[e] = cst[4 * j + e];
            FC[j * NFT + f] = qv;
        }
    }
}

// One face and chunk: the face equilibrium (eqs. geq, beq) from the packed
// constants fc, the inverse of eq. phibar applied to the reconstructed values
// (gb, bb), the microflux xi_a phi (eq. flux) into (fg, fb), and its moments
// with the quadrature weights added to sm.
// With the acceleration (ACC), the inverse of eq. phibar takes the whole
// source: alpha (h/2) fgg for g, and alpha_b (h/2) (a.xi g_f + fgb) for b, fgg
// and fgb the force gradients of phibar at the face, axi = a . xi.
template <typename T, int D, bool SK = false, bool ACC = false, bool NOSRC = false>
__device__ __forceinline__ void face_flux(const T* fc, const T (&xi)[VC][D], const T (&w)[VC], const T (&hx)[VC],
                                          int a, const T (&gb)[VC], const T (&bb)[VC], V4<T>& fg, V4<T>& fb,
                                          T* sm, T hL = T(0), const T* fgg = nullptr, const T* fgb = nullptr,
                                          const T* axi = nullptr, T hh = T(0)) {
    const T alg = fc[D + 4], alb = fc[D + 5], gmb = fc[D + 6];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        T ge, be, z;
        packed_eq<T, D, SK, SK || NOSRC>(fc, xi[v], hx[v], hL, ge, be, z);
        T gf = fma(alg, gb[v] - ge, ge);
        if constexpr (ACC) gf = fma(alg * hh, fgg[v], gf);
        T bfv;
        if constexpr (SK || NOSRC) bfv = fma(alb, bb[v] - be, be);
        else bfv = fma(gmb * z, gf - ge, fma(alb, bb[v] - be, be));
        if constexpr (ACC) bfv = fma(alb * hh, fma(axi[v], gf, fgb[v]), bfv);
        const T Fg = xi[v][a] * gf, Fb = xi[v][a] * bfv;
        fg.v[v] = Fg;
        fb.v[v] = Fb;
        const T wg = w[v] * Fg;
        sm[0] = Ar<T>::add(sm[0], wg);   // (explicitly rounded: the same bits in every kernel)
#pragma unroll
        for (int b = 0; b < D; ++b) sm[1 + b] = fma(xi[v][b], wg, sm[1 + b]);
        sm[1 + D] = fma(w[v], Fb, sm[1 + D]);
    }
}

// phi^n and phi_eq^n of one cell chunk: the deferred last factor of eq.
// phiupdate applied to the stored phi* (gs, bs) with the cell constants.
template <typename T, int D, bool SK = false>
__device__ __forceinline__ void own_state(const CellC<T>& own, const T (&xi)[VC][D], const T (&hx)[VC],
                                          const T (&gs)[VC], const T (&bs)[VC], T (&og)[VC], T (&ob)[VC],
                                          T (&oge)[VC], T (&obe)[VC], T hL = T(0)) {
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        T c2 = T(0), cq = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const T d = xi[v][a] - own.u[a];
            c2 = fma(d, d, c2);
            if constexpr (SK) cq = fma(own.sq[a], d, cq);
        }
        const T gM = own.pref * Num<T>::expo(own.cexp * c2);
        if constexpr (SK) {
            shakhov_point<T, D>(gM, c2, cq, own.cexp * Num<T>::irt_scale(), hx[v], own.eb, hL, own.e2, oge[v], obe[v]);
        } else {
            oge[v] = gM;
            obe[v] = (hx[v] + own.eb) * oge[v];
        }
        og[v] = fma(own.fa_g, gs[v], own.fb_g * oge[v]);
        ob[v] = fma(own.fa_b, bs[v], own.fb_b * obe[v]);
    }
}

// Net flux sum_a (F(right face) - F(left face)) / dx_a of the owned cell (local
// coordinates la) from the staged face fluxes FF[field * NFT + local face].
template <typename T, int D, typename TL>
__device__ __forceinline__ void net_flux(const T (&idxT)[3], const V4<T>* FF, const int la[3], T (&dFg)[VC], T (&dFb)[VC]) {
    constexpr int NFT = TL::NFT;
#pragma unroll
    for (int v = 0; v < VC; ++v) dFg[v] = dFb[v] = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int fl0 = TL::face_local(a, la[0], la[1], la[2]);
        const int fl1 = TL::face_local(a, la[0] + (a == 0), la[1] + (a == 1), la[2] + (a == 2));
        const V4<T> g0 = FF[0 * NFT + fl0], g1 = FF[0 * NFT + fl1];
        const V4<T> b0 = FF[1 * NFT + fl0], b1 = FF[1 * NFT + fl1];
        const T idx = idxT[a];
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            dFg[v] = fma(idx, g1.v[v] - g0.v[v], dFg[v]);
            dFb[v] = fma(idx, b1.v[v] - b0.v[v], dFb[v]);
        }
    }
}

// phi* = phi_eq + (1 - dt/2tau)(phi - phi_eq) [+ dt Z/tau_bg (g - g_eq)] - dt dF
// (eq. phiupdate, the last factor deferred) of one cell chunk, stored at dst.
template <typename T, int D, bool NOSRC = false>
__device__ __forceinline__ void store_phi_star(T dt, const T (&xi)[VC][D], const T (&u)[D], T hu2, T um_g,
                                               T um_b, T usrc, const T (&og)[VC], const T (&ob)[VC],
                                               const T (&oge)[VC], const T (&obe)[VC], const T (&dFg)[VC],
                                               const T (&dFb)[VC], T* dst) {
    T ng[VC], nb[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        const T dg = og[v] - oge[v];
        ng[v] = fma(-dt, dFg[v], fma(um_g, dg, oge[v]));
        if constexpr (NOSRC) {
            nb[v] = fma(-dt, dFb[v], fma(um_b, ob[v] - obe[v], obe[v]));
        } else {
            T z = -hu2;
#pragma unroll
            for (int a = 0; a < D; ++a) z = fma(xi[v][a], u[a], z);
            nb[v] = fma(-dt, dFb[v], fma(usrc * z, dg, fma(um_b, ob[v] - obe[v], obe[v])));
        }
    }
    Chunk<T>::store(dst, ng);
    Chunk<T>::store(dst + VC, nb);
}

// A group's partial sums of the faces a thread owns (its left faces, and its
// right faces at the domain's right end, summed in RS) into
// dst[a][(grp * (2+D) + m) * nf_a + face].
template <typename T, int D, typename TL>
__device__ __forceinline__ void write_face_sums(const Geo& g, double* const* dst, int grp, const int qa[3],
                                                const bool own_right[3], const Kahan<T> (&acc)[D][2 + D],
                                                const Kahan<T>* RS, const int pl[3]) {
    constexpr int NM = 2 + D;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const long long f0 = face_index(g, a, qa);
#pragma unroll
        for (int m = 0; m < NM; ++m) dst[a][((size_t)grp * NM + m) * g.nf[a] + f0] = acc[a][m].value();
        if (own_right[a]) {
            int qr[3] = {qa[0], qa[1], qa[2]};
            qr[a] += 1;
            const long long f1 = face_index(g, a, qr);
#pragma unroll
            for (int m = 0; m < NM; ++m)
                dst[a][((size_t)grp * NM + m) * g.nf[a] + f1] = RS[pl[a] + m * TL::plane(a)].value();
        }
    }
}

template <typename T, int D, int T0_, int T1_, int T2_, bool SWEEP_B, int MODE, bool PERS = false>
__device__ __forceinline__ void sweep_body(const Geo g, const Bufs<T> bf, int tile, int grp, unsigned char* smem,
                                           const TmaPair* tm = nullptr) {
    using TL = Tile<D, T0_, T1_, T2_, mode_halo(MODE)>;
    using SM = Smem<T, D, T0_, T1_, T2_, MODE>;
    constexpr bool PREP = mode_source(MODE) != MODE_FUSED;      // phibar+ comes from a prepared buffer
    constexpr bool STORED = mode_source(MODE) == MODE_STORED;   // ... and so do the slopes
    constexpr bool FACES = mode_faces(MODE);                     // sweep A stores the face values
    constexpr bool R2 = mode_r2(MODE);                           // face-gradient reconstruction
    constexpr bool SK = mode_sk(MODE);                           // Shakhov equilibria
    constexpr bool NOSRC = mode_nosrc(MODE);                     // no b-source (its terms left out)
    static_assert(!(SWEEP_B && FACES), "sweep B of the face-store shapes is k_flux");
    static_assert(!SK || (FACES && !R2 && mode_source(MODE) != MODE_PREP), "Shakhov shapes are fused or stored face-store shapes");
    static_assert(!R2 || (FACES && !PREP), "the face-gradient reconstruction is built for fused face-store shapes");
    constexpr int PN = SM::PN;
    using Q = V4<T>;
    constexpr int NM = 2 + D, BOX = TL::BOX, SB = TL::SB, NFT = TL::NFT;
    constexpr int NCCV = SM::NCCV, NFCV = SM::NFCV;
    static_assert(VC == 4, "the shared-memory layout packs one chunk in a V4");
    static_assert(TL::NT % 32 == 0, "whole warps");
    // The persistent step stages too, with cp.async only (no tensor maps): its
    // copies are issued after the item's acquire of the counts it waits for, and
    // read through the generic proxy (L2, or L1 after the acquire) -- coherent
    // like its direct loads, which take no read-only path.
    constexpr bool STAGE = SM::stage(SWEEP_B);
    constexpr bool NC = !PERS;
    Q* const P = reinterpret_cast<Q*>(smem);      // [2][PN] phibar+ chunk per cell
    Q* const S = P + SM::nP;                      // [D][2][SB] half van Leer slopes times dx
    Q* const S2 = S + SM::nS;                     // [D][D][2][SB2] their half van Leer differences (R2)
    Q* const CC = S2 + SM::nS2;                   // [NCCV][BOX] packed cell constants
    Q* const FF = CC + SM::nCC;                   // [2][NFT] face fluxes (sweep B)
    Q* const FC = FF + SM::nFF;                   // [NFCV][NFT] packed face constants (sweep B)
    // [2][BOXP] staged phi* (STAGE), 128-byte aligned for TMA, then the mbarrier of the TMA copies
    Q* const STraw = CC + SM::nCC + (SWEEP_B ? SM::nFF + SM::nFC : 0);
    Q* const ST = STraw + ((128u - (smem_u32(STraw) & 127u)) & 127u) / sizeof(Q);
    uint64_t* const tbar = reinterpret_cast<uint64_t*>(ST + 2 * SM::BOXP);
    constexpr int BOXP = SM::BOXP;
    constexpr int SB2 = TL::SB2;
    Kahan<T>* const RS = reinterpret_cast<Kahan<T>*>(smem + sizeof(Q) * SM::vcount(SWEEP_B));
    int* const csrc = reinterpret_cast<int*>(smem + sizeof(Q) * SM::vcount(SWEEP_B) + SM::rs_bytes);
    int* const cfl = csrc + BOX;
    int* const halo = cfl + BOX;
    int* const wcount = halo + TL::NH;            // [32] per-warp halo counts

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NW = TL::NT / 32;
    const T hL = (T)(0.5 * (3.0 - D + g.K));     // Shakhov: half the unresolved degrees of freedom
    // constants of the chunk loop in the working precision, converted once (the
    // conversions from double run on the FP64 pipe)
    const T dtT = (T)g.dt;
    const T idxT[3] = {(T)g.idx[0], (T)g.idx[1], (T)g.idx[2]};
    int org[3];
    tile_origin<TL, D>(g, tile, org);
    const int vt0 = grp * g.ntpg, vt1 = min(g.NVT, vt0 + g.ntpg);

    // this thread's cell
    const int la[3] = {t % TL::T0, D >= 2 ? (t / TL::T0) % TL::T1 : 0, D >= 3 ? t / (TL::T0 * TL::T1) : 0};
    const int qa[3] = {org[0] + la[0], org[1] + la[1], org[2] + la[2]};
    bool valid = true;
#pragma unroll
    for (int a = 0; a < D; ++a) valid = valid && qa[a] < g.n[a];
    const int kc = TL::box_of(la[0], la[1], la[2]);
    const int sc = TL::sbox_of(la[0], la[1], la[2]);
    const int s2c = TL::s2box_of(la[0], la[1], la[2]);

    auto box_local = [&](int k, int l[3]) {
        l[0] = k % TL::E0 - TL::HALO;
        l[1] = D >= 2 ? (k / TL::E0) % TL::E1 - TL::HALO : 0;
        l[2] = D >= 3 ? k / (TL::E0 * TL::E1) - TL::HALO : 0;
    };
    // The cells the tile's faces read: upwind of a face are the owned cells and
    // one layer below each axis, and one layer above an axis only where faces on
    // the tile's upper side are formed (the domain's end in sweep A, every tile
    // edge in sweep B); phibar+ is needed on those and on their neighbours
    // along every axis (the slopes).  Corners beyond that are never read.  The
    // shapes that load phibar+ (and the slopes) skip the rest; the fused ones
    // form the whole box (measured faster: fixed trip counts, no spills).
    constexpr bool PRUNE = PREP && !R2;
    bool rext[3] = {true, true, true};
#pragma unroll
    for (int a = 0; a < D; ++a) rext[a] = SWEEP_B || org[a] + TL::tdim(a) >= g.n[a];
    auto upwind_cell = [&](const int (&l)[3]) {
        int out = 0;
        bool ok = true;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            if (l[b] < -1 || l[b] > TL::tdim(b)) ok = false;
            else if (l[b] == -1) ++out;
            else if (l[b] == TL::tdim(b)) {
                ++out;
                ok = ok && rext[b];
            }
        }
        return ok && out <= 1;
    };
    auto needed_box = [&](const int (&l)[3]) {
        if (upwind_cell(l)) return true;
        bool any = false;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            int m[3] = {l[0], l[1], l[2]};
            m[b] = l[b] - 1;
            any = any || upwind_cell(m);
            m[b] = l[b] + 1;
            any = any || upwind_cell(m);
        }
        return any;
    };
    auto is_halo = [&](int k) {
        int l[3];
        box_local(k, l);
        bool inner = true;
#pragma unroll
        for (int a = 0; a < D; ++a) inner = inner && l[a] >= 0 && l[a] < TL::tdim(a);
        return !inner && (!PRUNE || needed_box(l));
    };
    // bit j: slope-box cell t + j NT is upwind of a face (its slopes are formed or loaded)
    static_assert((SB + TL::NT - 1) / TL::NT <= 32, "one mask bit per slope-box cell of a thread");
    unsigned smask = 0;
    for (int s2 = t, j = 0; s2 < SB; s2 += TL::NT, ++j) {
        int l[3];
        TL::sbox_local(s2, l);
        if (!PRUNE || upwind_cell(l)) smask |= 1u << j;
    }

    // ---- prologue: halo box (boundary mapping, packed constants), ordered halo list, face constants
    for (int k = t; k < BOX; k += TL::NT) {
        int l[3];
        box_local(k, l);
        int q[3] = {org[0] + l[0], org[1] + l[1], org[2] + l[2]};
        int refl;
        bool dir;
        resolve<D>(g, q, refl, dir);
        const long long c = cell_index(g, q);
        csrc[k] = (int)c;
        cfl[k] = refl | (dir ? 8 : 0);
        if (PREP) continue;
        pack_cell<T, D, SK>(dir ? bf.cellc0[c] : bf.cellc[c], refl, CC + k, BOX);
    }
    int nhalo = 0;      // length of the halo list
    {   // halo list in box order (warp ballots), so neighbouring threads touch neighbouring cells
        constexpr int PER = ((BOX + NW - 1) / NW + 31) / 32 * 32;
        const int k0 = warp * PER, k1 = min(BOX, k0 + PER);
        int cnt = 0;
        for (int kb = k0; kb < k1; kb += 32) {
            const int k = kb + lane;
            cnt += __popc(__ballot_sync(0xffffffffu, k < k1 && is_halo(k)));
        }
        if (lane == 0) wcount[warp] = cnt;
        __syncthreads();
        int base = 0;
        for (int w2 = 0; w2 < warp; ++w2) base += wcount[w2];
        for (int w2 = 0; w2 < NW; ++w2) nhalo += wcount[w2];
        for (int kb = k0; kb < k1; kb += 32) {
            const int k = kb + lane;
            const bool hk = k < k1 && is_halo(k);
            const unsigned m = __ballot_sync(0xffffffffu, hk);
            if (hk) halo[base + __popc(m & ((1u << lane) - 1u))] = k;
            base += __popc(m);
        }
    }
    if (SWEEP_B) stage_face_consts<T, D, TL>(g, bf, org, FC);
    // constants of the owned cell for the distribution update
    T um_g = T(0), um_b = T(0), usrc = T(0);
    CellC<T> own;       // all of them (prepared shapes: phase 4 recomputes phi and phi_eq)
    if (SWEEP_B && valid) {
        own = bf.cellc[cell_index(g, qa)];
        um_g = own.um_g;
        um_b = own.um_b;
        usrc = own.usrc;
    }
    // which faces this thread computes: left faces; right faces where no other thread does
    bool right[3] = {false, false, false};
    bool own_right[3] = {false, false, false};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        own_right[a] = valid && qa[a] == g.n[a] - 1;
        right[a] = valid && (SWEEP_B ? (la[a] == TL::tdim(a) - 1 || own_right[a]) : own_right[a]);
    }
    Kahan<T> acc[D][NM];          // the left faces; the domain's right end sums in RS
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[a][m].zero();
    int pl[3] = {0, 0, 0};        // this cell's slot in RS per axis
#pragma unroll
    for (int a = 0; a < D; ++a) pl[a] = TL::poff(a) * NM + TL::plane_pos(a, la);
    for (int k = t; k < (int)SM::nRS; k += TL::NT) RS[k].zero();
    // TMA staging (1D/2D): for a tile whose halo box lies inside the domain the
    // box of every chunk is one tensor copy of g and one of b, issued by thread 0
    // and completed on an mbarrier; the other tiles copy per cell (boundary
    // mapping).  Boxes are at most 256 cells per axis.
    bool tma = false;
    if constexpr (STAGE && D <= 2 && TL::E0 <= 256 && TL::E1 <= 256) {
        tma = tm != nullptr && tm->on;
#pragma unroll
        for (int a = 0; a < D; ++a) tma = tma && org[a] - TL::HALO >= 0 && org[a] + TL::tdim(a) + TL::HALO <= g.n[a];
        if (tma && t == 0) mbar_init(tbar, 1);
    }
    unsigned tphase = 0;
    auto fetch_tma = [&](int vt) {      // thread 0: both halves of chunk vt's box
        if (g.wait_test) return;        // (test hook) nothing arrives: the wait below runs out
        constexpr unsigned bytes = 2u * TL::BOX * sizeof(Q);
        mbar_expect_tx(tbar, bytes);
        if constexpr (D == 1) {
            tma_load_3d(ST, &tm->g, tbar, 0, org[0] - TL::HALO, vt);
            tma_load_3d(ST + BOXP, &tm->b, tbar, 0, org[0] - TL::HALO, vt);
        } else {
            tma_load_4d(ST, &tm->g, tbar, 0, org[0] - TL::HALO, org[1] - TL::HALO, vt);
            tma_load_4d(ST + BOXP, &tm->b, tbar, 0, org[0] - TL::HALO, org[1] - TL::HALO, vt);
        }
    };
    bool tma_late = false;              // a bounded wait gave up (then the CTA reports and stops)
    __syncthreads();
    const int NH = PRUNE ? nhalo : TL::NH;

    // Asynchronous copies of chunk vt's phi* for the box cells this thread forms
    // in phase 1 (its own cell and its halo cells), into its own ST slots: a
    // mirror image takes the reflected velocities element by element, a
    // Dirichlet ghost needs none.  Each thread reads back only what it copied.
    auto fetch = [&](int vt) {
        auto one = [&](int k) {
            const int fl = cfl[k];
            if (fl & 8) return;
            const long long c = csrc[k];
            if (fl & 7) {
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    const int is = bf.refl[(fl & 7) * g.Nvp + vt * VC + v];
                    cp_async_elem(&ST[k].v[v], bf.phi_in + phi_addr(g, c, is, 0));
                    cp_async_elem(&ST[BOXP + k].v[v], bf.phi_in + phi_addr(g, c, is, 1));
                }
            } else {
                const size_t ad = phi_addr(g, c, vt * VC, 0);
                cp_async_chunk(&ST[k], bf.phi_in + ad);
                cp_async_chunk(&ST[BOXP + k], bf.phi_in + ad + VC);
            }
        };
        one(kc);
        for (int h = t; h < NH; h += TL::NT) one(halo[h]);
        cp_async_commit();
    };
    __syncthreads();                    // the mbarrier's initialisation is visible
    if (STAGE && vt0 < vt1) {
        if (tma) {
            if (t == 0) fetch_tma(vt0);
        } else {
            fetch(vt0);
        }
    }

    for (int vt = vt0; vt < vt1; ++vt) {
        if (STAGE) {
            if (tma) {                                 // the box of chunk vt has landed
                bool done = false;
                for (int it = 0; it < (1 << g.wait_log2) && !done; ++it) done = mbar_try_wait(tbar, tphase);
                tma_late = tma_late || !done;
                tphase ^= 1u;
            } else {
                cp_async_wait_all();                   // this thread's copies of chunk vt have landed
            }
        }
        // velocity records of the chunk (same for every thread); nu = 2 h xi / dx
        T xi[VC][D], nu[VC][D], w[VC], hx[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const Q* rec = reinterpret_cast<const Q*>(bf.vel + (size_t)(vt * VC + v) * 8);
            const Q r0 = rec[0], r1 = rec[1];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                xi[v][a] = r0.v[a];
                nu[v][a] = a == 0 ? r1.v[1] : (a == 1 ? r1.v[2] : r1.v[3]);
            }
            w[v] = r0.v[3];
            hx[v] = r1.v[0];
        }
        // per axis: +1 / -1 when the chunk's four xi_a share a strict sign, else 0
        int sgn[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            bool pos = true, neg = true;
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                pos = pos && xi[v][a] > T(0);
                neg = neg && xi[v][a] < T(0);
            }
            sgn[a] = pos ? 1 : (neg ? -1 : 0);
        }

        // ---- phase 1: phibar+ = eq + sa (phi - eq) [+ ssrc Z (g - g_eq)] on the box (eq. phibarplus)
        T og[VC], ob[VC], oge[VC], obe[VC];   // the owned cell's phi and phi_eq (sweep B)
        auto cell = [&](int k, bool keep) {
            const int fl = cfl[k];
            const long long c = csrc[k];
            T cst[4 * NCCV];
#pragma unroll
            for (int j = 0; j < NCCV; ++j) {
                const Q qv = CC[j * BOX + k];
#pragma unroll
                for (int e = 0; e < 4; ++e) cst[4 * j + e] = qv.v[e];
            }
            T gs[VC], bs[VC];
            if (fl & 8) {
#pragma unroll
                for (int v = 0; v < VC; ++v) gs[v] = bs[v] = T(0);
            } else if (STAGE) {
                const Q sg = ST[k], sb = ST[BOXP + k];
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    gs[v] = sg.v[v];
                    bs[v] = sb.v[v];
                }
            } else if (fl & 7) {
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    const int is = bf.refl[(fl & 7) * g.Nvp + vt * VC + v];
                    gs[v] = bf.phi_in[phi_addr(g, c, is, 0)];
                    bs[v] = bf.phi_in[phi_addr(g, c, is, 1)];
                }
            } else {
                const size_t ad = phi_addr(g, c, vt * VC, 0);
                Chunk<T>::template load<NC>(bf.phi_in + ad, gs);
                Chunk<T>::template load<NC>(bf.phi_in + ad + VC, bs);
            }
            const T kp_g = cst[D + 4], kp_b = cst[D + 5], kp_s = cst[D + 6];
            Q qg, qb;
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                T ge, be, z;
                packed_eq<T, D, SK, NOSRC>(cst, xi[v], hx[v], hL, ge, be, z);
                if (fl & 8) {
                    qg.v[v] = ge;
                    qb.v[v] = be;
                } else {
                    phibar_plus<T, NOSRC>(ge, be, gs[v], bs[v], z, kp_g, kp_b, kp_s, qg.v[v], qb.v[v]);
                    if (SWEEP_B && keep) {   // phi^n of the owned cell (the deferred end of eq. phiupdate)
                        og[v] = fma(own.fa_g, gs[v], own.fb_g * ge);
                        ob[v] = fma(own.fa_b, bs[v], own.fb_b * be);
                        oge[v] = ge;
                        obe[v] = be;
                    }
                }
            }
            P[0 * BOX + k] = qg;
            P[1 * BOX + k] = qb;
        };
        // prepared shapes: phibar+ comes from the prepared buffer (Dirichlet ghosts: their equilibrium)
        auto pcell = [&](int k) {
            const int fl = cfl[k];
            const long long c = csrc[k];
            Q qg, qb;
            if (fl & 8) {
                const CellC<T> cs = bf.cellc0[c];
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    T c2 = T(0);
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        const T ua = (fl & (1 << a)) ? -cs.u[a] : cs.u[a];
                        const T d = xi[v][a] - ua;
                        c2 = fma(d, d, c2);
                    }
                    qg.v[v] = cs.pref * Num<T>::expo(cs.cexp * c2);
                    qb.v[v] = (hx[v] + cs.eb) * qg.v[v];
                }
            } else if (fl & 7) {
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    const int is = bf.refl[(fl & 7) * g.Nvp + vt * VC + v];
                    qg.v[v] = bf.phibar[phi_addr(g, c, is, 0)];
                    qb.v[v] = bf.phibar[phi_addr(g, c, is, 1)];
                }
            } else {
                const size_t ad = phi_addr(g, c, vt * VC, 0);
                Chunk<T>::template load<NC>(bf.phibar + ad, qg.v);
                Chunk<T>::template load<NC>(bf.phibar + ad + VC, qb.v);
            }
            P[0 * BOX + k] = qg;
            P[1 * BOX + k] = qb;
        };
        if (STORED) {
            // phibar+ and slopes of the cells [-1, T] around the tile from the stored arrays;
            // a mirrored cell takes the reflected velocity and flips the mirrored slope components
            for (int s2 = t, j = 0; s2 < SB; s2 += TL::NT, ++j) {
                if (PRUNE && !((smask >> j) & 1u)) continue;
                int sl[3];
                TL::sbox_local(s2, sl);
                const int k = TL::box_of(sl[0], sl[1], sl[2]);
                const int rf = cfl[k] & 7;
                const long long c = csrc[k];
                Q qg, qb, qs[D][2];
                if (rf == 0) {
                    const size_t ad = phi_addr(g, c, vt * VC, 0);
                    Chunk<T>::template load<NC>(bf.phibar + ad, qg.v);
                    Chunk<T>::template load<NC>(bf.phibar + ad + VC, qb.v);
                    const size_t as = sig_addr<D>(g, c, vt * VC, 0, 0);
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        Chunk<T>::template load<NC>(bf.sigma + as + (a * 2 + 0) * VC, qs[a][0].v);
                        Chunk<T>::template load<NC>(bf.sigma + as + (a * 2 + 1) * VC, qs[a][1].v);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        const int is = bf.refl[rf * g.Nvp + vt * VC + v];
                        qg.v[v] = bf.phibar[phi_addr(g, c, is, 0)];
                        qb.v[v] = bf.phibar[phi_addr(g, c, is, 1)];
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            const T sgn_a = (rf & (1 << a)) ? T(-1) : T(1);
                            qs[a][0].v[v] = sgn_a * bf.sigma[sig_addr<D>(g, c, is, a, 0)];
                            qs[a][1].v[v] = sgn_a * bf.sigma[sig_addr<D>(g, c, is, a, 1)];
                        }
                    }
                }
                P[0 * PN + s2] = qg;
                P[1 * PN + s2] = qb;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    S[(a * 2 + 0) * SB + s2] = qs[a][0];
                    S[(a * 2 + 1) * SB + s2] = qs[a][1];
                }
            }
        } else if (PREP) {
            pcell(kc);
            for (int h = t; h < NH; h += TL::NT) pcell(halo[h]);
        } else {
            cell(kc, valid);
            for (int h = t; h < NH; h += TL::NT) cell(halo[h], false);
            if (STAGE && !tma && vt + 1 < vt1) fetch(vt + 1);    // this thread's slots are read: refill them
        }
        if (tma) {
            // every thread has read the box: the next chunk's copies may overwrite it
            if (__syncthreads_or(tma_late)) {
                if (t == 0) atomicOr(bf.status, ST_TIMEOUT);
                return;
            }
            if (t == 0 && vt + 1 < vt1) {
                fence_proxy_async_smem();
                fetch_tma(vt + 1);
            }
        } else {
            __syncthreads();
        }

        // ---- phase 2: half van Leer slopes (times dx) of the cells [-1, T] around the tile
        for (int s = t, j = 0; s < (STORED ? 0 : SB); s += TL::NT, ++j) {
            if (PRUNE && !((smask >> j) & 1u)) continue;
            int sl[3];
            TL::sbox_local(s, sl);
            const int k = TL::box_of(sl[0], sl[1], sl[2]);
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const Q c = P[f * BOX + k];
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const int st = TL::bstride(a);
                    const Q l = P[f * BOX + k - st], r = P[f * BOX + k + st];
                    Q o;
#pragma unroll
                    for (int v = 0; v < VC; ++v) o.v[v] = Num<T>::vanleer(c.v[v] - l.v[v], r.v[v] - c.v[v]);
                    S[(a * 2 + f) * SB + s] = o;
                }
            }
        }
        if (!STORED) __syncthreads();

        // ---- phase 2b (face gradient): half van Leer differences along every axis a
        //      of every slope component b, on the cells [-1, T] (the upwind cells)
        if constexpr (R2) {
            for (int s2 = t; s2 < SB2; s2 += TL::NT) {
                const int l0 = s2 % TL::G0 - 1, l1 = D >= 2 ? (s2 / TL::G0) % TL::G1 - 1 : 0;
                const int l2 = D >= 3 ? s2 / (TL::G0 * TL::G1) - 1 : 0;
                const int ks = TL::sbox_of(l0, l1, l2);
#pragma unroll
                for (int f = 0; f < 2; ++f)
#pragma unroll
                    for (int b = 0; b < D; ++b) {
                        const Q c = S[(b * 2 + f) * SB + ks];
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            const int st = TL::sstride(a);
                            const Q l = S[(b * 2 + f) * SB + ks - st], r = S[(b * 2 + f) * SB + ks + st];
                            Q o;
#pragma unroll
                            for (int v = 0; v < VC; ++v) o.v[v] = Num<T>::vanleer(c.v[v] - l.v[v], r.v[v] - c.v[v]);
                            S2[((a * D + b) * 2 + f) * SB2 + s2] = o;
                        }
                    }
            }
            __syncthreads();
        }

        // ---- phase 3: faces of the owned cell
        if (valid) {
#pragma unroll
            for (int a = 0; a < D; ++a) {
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (side == 1 && !right[a]) continue;
                    const int Lb = kc + (side - 1) * TL::bstride(a), Rb = Lb + TL::bstride(a);
                    const int Ls = sc + (side - 1) * TL::sstride(a), Rs = Ls + TL::sstride(a);
                    const int L2 = s2c + (side - 1) * TL::s2stride(a), R2i = L2 + TL::s2stride(a);
                    int lf[3] = {la[0], la[1], la[2]};
                    lf[a] += side;
                    const int fl = TL::face_local(a, lf[0], lf[1], lf[2]);
                    const bool own = side == 0 || own_right[a];
                    // phibar at the face, t + h: upwind value + (x_f - h xi - x_up) . sigma_up
                    T gb[VC], bb[VC];
                    if (sgn[a] != 0) {
                        const bool lft = sgn[a] > 0;
                        const int up = lft ? Lb : Rb, ups = lft ? Ls : Rs;
                        const int pu = STORED ? ups : up;
                        const Q pg = P[0 * PN + pu], pb = P[1 * PN + pu];
                        Q sg[D], sb[D];
#pragma unroll
                        for (int b = 0; b < D; ++b) {
                            sg[b] = S[(b * 2 + 0) * SB + ups];
                            sb[b] = S[(b * 2 + 1) * SB + ups];
                        }
                        const T one = lft ? T(1) : T(-1);   // (x_f - x_up)/(dx/2) along the normal
                        Q dg[R2 ? D : 1], db[R2 ? D : 1];   // slope derivatives along a at the upwind cell
                        if constexpr (R2) {
                            const int up2 = lft ? L2 : R2i;
#pragma unroll
                            for (int b = 0; b < D; ++b) {
                                dg[b] = S2[((a * D + b) * 2 + 0) * SB2 + up2];
                                db[b] = S2[((a * D + b) * 2 + 1) * SB2 + up2];
                            }
                        }
#pragma unroll
                        for (int v = 0; v < VC; ++v) {
                            T rg = pg.v[v], rb = pb.v[v];
#pragma unroll
                            for (int b = 0; b < D; ++b) {
                                const T k = (b == a) ? one - nu[v][a] : -nu[v][b];
                                rg = fma(k, sg[b].v[v], rg);
                                rb = fma(k, sb[b].v[v], rb);
                            }
                            if constexpr (R2) {   // - h xi . (x_f - x_up) grad sigma
#pragma unroll
                                for (int b = 0; b < D; ++b) {
                                    rg = fma(-one * nu[v][b], dg[b].v[v], rg);
                                    rb = fma(-one * nu[v][b], db[b].v[v], rb);
                                }
                            }
                            gb[v] = rg;
                            bb[v] = rb;
                        }
                    } else {
                        const T* Ps = reinterpret_cast<const T*>(P);
                        const T* Ss = reinterpret_cast<const T*>(S);
                        const T* S2s = reinterpret_cast<const T*>(S2);
                        // side one: +1 for the left cell upwind, -1 for the right
                        auto recon = [&](int v, int up, int ups, int up2, T one, T& rg, T& rb) {
                            const int pu = STORED ? ups : up;
                            rg = Ps[(0 * PN + pu) * VC + v];
                            rb = Ps[(1 * PN + pu) * VC + v];
#pragma unroll
                            for (int b = 0; b < D; ++b) {
                                const T k = (b == a) ? one - nu[v][a] : -nu[v][b];
                                rg = fma(k, Ss[((b * 2 + 0) * SB + ups) * VC + v], rg);
                                rb = fma(k, Ss[((b * 2 + 1) * SB + ups) * VC + v], rb);
                            }
                            if constexpr (R2) {
#pragma unroll
                                for (int b = 0; b < D; ++b) {
                                    rg = fma(-one * nu[v][b], S2s[(((a * D + b) * 2 + 0) * SB2 + up2) * VC + v], rg);
                                    rb = fma(-one * nu[v][b], S2s[(((a * D + b) * 2 + 1) * SB2 + up2) * VC + v], rb);
                                }
                            }
                        };
#pragma unroll
                        for (int v = 0; v < VC; ++v) {
                            const T x = xi[v][a];
                            if (x != T(0)) {
                                const bool lft = x > T(0);
                                recon(v, lft ? Lb : Rb, lft ? Ls : Rs, lft ? L2 : R2i, lft ? T(1) : T(-1), gb[v], bb[v]);
                            } else {   // xi . n = 0: mean of both one-sided values
                                T g1, b1, g2, b2;
                                recon(v, Lb, Ls, L2, T(1), g1, b1);
                                recon(v, Rb, Rs, R2i, T(-1), g2, b2);
                                gb[v] = T(0.5) * (g1 + g2);
                                bb[v] = T(0.5) * (b1 + b2);
                            }
                        }
                    }
                    T sm[NM];
#pragma unroll
                    for (int m = 0; m < NM; ++m) sm[m] = T(0);
                    if (FACES) {   // sweep A computes each face once: keep it for k_flux
                        int qf[3] = {qa[0], qa[1], qa[2]};
                        qf[a] += side;
                        T* const dst = bf.face[a] + face_addr(g, a, face_index(g, a, qf), vt);
                        Chunk<T>::store(dst, gb);
                        Chunk<T>::store(dst + VC, bb);
                    }
                    if (!SWEEP_B) {
                        // face conserved variables (eqs. rhobar-rhoEbar, a = 0)
#pragma unroll
                        for (int v = 0; v < VC; ++v) {
                            const T wg = w[v] * gb[v];
                            sm[0] = Ar<T>::add(sm[0], wg);   // (explicitly rounded: the same bits in every kernel)
#pragma unroll
                            for (int b = 0; b < D; ++b) sm[1 + b] = fma(xi[v][b], wg, sm[1 + b]);
                            sm[1 + D] = fma(w[v], bb[v], sm[1 + D]);
                        }
                    } else {
                        // face equilibrium, inverse of eq. phibar, microflux xi_a phi
                        T fcst[4 * NFCV];
#pragma unroll
                        for (int j = 0; j < NFCV; ++j) {
                            const Q qv = FC[j * NFT + fl];
#pragma unroll
                            for (int e = 0; e < 4; ++e) fcst[4 * j + e] = qv.v[e];
                        }
                        Q fg, fb;
                        face_flux<T, D, false, false, NOSRC>(fcst, xi, w, hx, a, gb, bb, fg, fb, sm);
                        FF[0 * NFT + fl] = fg;
                        FF[1 * NFT + fl] = fb;
                    }
                    if (side == 0) {
#pragma unroll
                        for (int m = 0; m < NM; ++m) acc[a][m].add(sm[m]);
                    } else if (own) {           // the domain's right end
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            Kahan<T> k = RS[pl[a] + m * TL::plane(a)];
                            k.add(sm[m]);
                            RS[pl[a] + m * TL::plane(a)] = k;
                        }
                    }
                }
            }
        }

        if (SWEEP_B) {
            __syncthreads();
            // ---- phase 4: phi* = phi_eq + (1 - dt/2tau)(phi - phi_eq) [+ dt Z/tau_bg (g - g_eq)] - dt dF
            if (valid) {
                T dFg[VC], dFb[VC];
                net_flux<T, D, TL>(idxT, FF, la, dFg, dFb);
                T u[D], hu2;
                if (PREP) {
#pragma unroll
                    for (int a = 0; a < D; ++a) u[a] = own.u[a];
                    hu2 = own.hu2;
                    // phi and phi_eq of the owned cell (not kept from phase 1 on this path)
                    T gs[VC], bs[VC];
                    const size_t ad0 = phi_addr(g, cell_index(g, qa), vt * VC, 0);
                    Chunk<T>::template load<NC>(bf.phi_in + ad0, gs);
                    Chunk<T>::template load<NC>(bf.phi_in + ad0 + VC, bs);
                    own_state<T, D>(own, xi, hx, gs, bs, og, ob, oge, obe);
                } else {
#pragma unroll
                    for (int a = 0; a < D; ++a) u[a] = reinterpret_cast<const T*>(&CC[(a / 4) * BOX + kc])[a % 4];
                    hu2 = reinterpret_cast<const T*>(&CC[((D + 3) / 4) * BOX + kc])[(D + 3) % 4];
                }
                store_phi_star<T, D, NOSRC>(dtT, xi, u, hu2, um_g, um_b, usrc, og, ob, oge, obe, dFg, dFb,
                                     bf.phi_out + phi_addr(g, cell_index(g, qa), vt * VC, 0));
            }
        }
        __syncthreads();   // before the next chunk overwrites P and S
    }

    // ---- epilogue: this group's partial face sums
    if (valid) write_face_sums<T, D, TL>(g, SWEEP_B ? bf.mf : bf.wf, grp, qa, own_right, acc, RS, pl);
}

// CTAs per SM that the shared memory of a sweep allows (at least 1, at most 4);
// the launch bounds ask the compiler to fit the registers to the same count.
template <typename T, int D, int T0_, int T1_, int T2_, bool SWEEP_B, int MODE>
struct Occ {
    static constexpr size_t kSmemPerSM = 228 * 1024;
    static constexpr size_t per = Smem<T, D, T0_, T1_, T2_, MODE>::bytes(SWEEP_B) + 1024;
    static constexpr int by_smem = (int)(kSmemPerSM / per);
    static constexpr int by_threads = 2048 / Tile<D, T0_, T1_, T2_>::NT;
    static constexpr int by_regs = 65536 / (Tile<D, T0_, T1_, T2_>::NT * 80);   // keep >= 80 registers
    static constexpr int v1 = by_smem < by_threads ? by_smem : by_threads;
    static constexpr int v0 = v1 < by_regs ? v1 : by_regs;
    static constexpr int value = v0 < 1 ? 1 : (v0 > 4 ? 4 : v0);
};

// One problem instance: grid (tiles, velocity groups).
template <typename T, int D, int T0_, int T1_, int T2_, bool SWEEP_B, int MODE>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (Occ<T, D, T0_, T1_, T2_, SWEEP_B, MODE>::value))
    k_sweep(const Inst<T>* __restrict__ in, int cur, const __grid_constant__ TmaPair tm) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    sweep_body<T, D, T0_, T1_, T2_, SWEEP_B, MODE>(in->g, in->b[cur], blockIdx.x, blockIdx.y, smem, &tm);
}

// ---- sweep B of the face-store shapes
//
// One CTA per (tile, velocity group), one thread per owned cell, the tiling
// of the sweeps.  Per chunk each thread reads the stored values of both faces
// of its cell along every axis, forms their fluxes and phi* of its cell from
// the net flux.  A face shared by two cells is formed by both, from the same
// values with the same arithmetic, so both see the same flux; there is no
// exchange between threads and no barrier inside the chunk loop.  A face's
// moments are summed by its owner (the cell on its right; the last cell for
// the domain's right end), in chunk order.

template <typename T, int D, int T0_, int T1_, int T2_, bool SK = false>
struct FluxSmem {
    using TL = Tile<D, T0_, T1_, T2_>;
    static constexpr int NPL = TL::NPL;
    __host__ __device__ static constexpr int plane(int a) { return TL::plane(a); }
    __host__ __device__ static constexpr int poff(int a) { return TL::poff(a); }
    static_assert(TL::poff(D) == TL::NPL, "one slot per cell of each tile face");
    static constexpr size_t nV4 = (size_t)FacePack<D, SK>::NV * TL::NFT;
    static constexpr size_t bytes = nV4 * sizeof(V4<T>) + (size_t)NPL * (2 + D) * sizeof(Kahan<T>);
};

template <typename T, int D, int T0_, int T1_, int T2_, bool SK = false, bool ACC = false, bool NOSRC = false,
          bool PERS = false>
__device__ __forceinline__ void flux_body(const Geo g, const Bufs<T> bf, int tile, int grp, unsigned char* smem) {
    constexpr bool NC = !PERS;      // the persistent batched step reads coherently
    using TL = Tile<D, T0_, T1_, T2_>;
    using FS = FluxSmem<T, D, T0_, T1_, T2_, SK>;
    using Q = V4<T>;
    constexpr int NM = 2 + D, NFT = TL::NFT, NFCV = FacePack<D, SK>::NV;
    Q* const FC = reinterpret_cast<Q*>(smem);     // [NFCV][NFT] packed face constants
    // running sums of the faces at the domain's right end, [NM][plane cell] per axis
    Kahan<T>* const RS = reinterpret_cast<Kahan<T>*>(smem + FS::nV4 * sizeof(Q));
    const int t = threadIdx.x;
    int org[3];
    tile_origin<TL, D>(g, tile, org);
    const int vt0 = grp * g.ntpg, vt1 = min(g.NVT, vt0 + g.ntpg);
    const int la[3] = {t % TL::T0, D >= 2 ? (t / TL::T0) % TL::T1 : 0, D >= 3 ? t / (TL::T0 * TL::T1) : 0};
    const int qa[3] = {org[0] + la[0], org[1] + la[1], org[2] + la[2]};
    bool valid = true;
#pragma unroll
    for (int a = 0; a < D; ++a) valid = valid && qa[a] < g.n[a];
    stage_face_consts<T, D, TL, SK>(g, bf, org, FC);
    for (int k = t; k < FS::NPL * NM; k += TL::NT) RS[k].zero();
    __syncthreads();
    if (!valid) return;          // no barrier below

    const CellC<T> own = bf.cellc[cell_index(g, qa)];
    const T hL = (T)(0.5 * (3.0 - D + g.K));
    const T dtT = (T)g.dt;                        // converted once, outside the chunk loop
    const T idxT[3] = {(T)g.idx[0], (T)g.idx[1], (T)g.idx[2]};
    const size_t cell_ad = phi_addr(g, cell_index(g, qa), 0, 0);
    const size_t chunk_stride = (size_t)g.Nc * (2 * VC);
    bool own_right[3] = {false, false, false};
    int ff[3];                   // global left face per axis (the right one is ff + face stride; < 2^31)
#pragma unroll
    for (int a = 0; a < D; ++a) {
        own_right[a] = qa[a] == g.n[a] - 1;
        ff[a] = (int)face_index(g, a, qa);
    }
    Kahan<T> acc[D][NM];         // the left faces
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[a][m].zero();
    // The first thread of each x-row of the tile asks L2 for the row's data of
    // the next chunk while this one is formed: its cells' phi*, its left faces
    // along every axis (along x the row's right end too), and along y / z the
    // faces above the tile's last row.  Rows are contiguous in every layout.
    // (Not with the force terms, whose reads of neighbouring velocity chunks
    // measured slower with it.)
    const bool row_lead = !ACC && la[0] == 0;
    const int nrow = min(TL::T0, g.n[0] - org[0]);
    constexpr int RB = 2 * VC * (int)sizeof(T);     // bytes per cell or face and chunk
    const int tdim[3] = {TL::T0, TL::T1, TL::T2};

    for (int vt = vt0; vt < vt1; ++vt) {
        if (row_lead && vt + 1 < vt1) {
            prefetch_l2(bf.phi_in + cell_ad + (size_t)(vt + 1) * chunk_stride, nrow * RB);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const T* fb = bf.face[a] + face_addr(g, a, ff[a], vt + 1);
                prefetch_l2(fb, (nrow + (a == 0 ? 1 : 0)) * RB);
                if (a > 0 && (la[a] == tdim[a] - 1 || own_right[a])) {
                    const int fs = a == 1 ? g.fn[1][0] : g.fn[2][0] * g.fn[2][1];
                    prefetch_l2(fb + (size_t)fs * (2 * VC), nrow * RB);
                }
            }
        }
        T xi[VC][D], w[VC], hx[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const Q* rec = reinterpret_cast<const Q*>(bf.vel + (size_t)(vt * VC + v) * 8);
            const Q r0 = rec[0];
#pragma unroll
            for (int a = 0; a < D; ++a) xi[v][a] = r0.v[a];
            w[v] = r0.v[3];
            hx[v] = rec[1].v[0];
        }
        const size_t ad = cell_ad + (size_t)vt * chunk_stride;
        T gs[VC], bs[VC];
        Chunk<T>::template load<NC>(bf.phi_in + ad, gs);
        Chunk<T>::template load<NC>(bf.phi_in + ad + VC, bs);
        T dFg[VC], dFb[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v) dFg[v] = dFb[v] = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            Q F[2][2];           // [side][g|b]
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                // the right face of axis a is the left face of the next cell along a
                const int fs = a == 0 ? 1 : (a == 1 ? g.fn[1][0] : g.fn[2][0] * g.fn[2][1]);
                const T* src = bf.face[a] + face_addr(g, a, ff[a] + side * fs, vt);
                T gb[VC], bb[VC];
                Chunk<T>::template load<NC>(src, gb);
                Chunk<T>::template load<NC>(src + VC, bb);
                const int fl = TL::face_local(a, la[0] + (a == 0 ? side : 0), la[1] + (a == 1 ? side : 0),
                                              la[2] + (a == 2 ? side : 0));
                T fcst[4 * NFCV];
#pragma unroll
                for (int j = 0; j < NFCV; ++j) {
                    const Q qv = FC[j * NFT + fl];
#pragma unroll
                    for (int e = 0; e < 4; ++e) fcst[4 * j + e] = qv.v[e];
                }
                T sm[NM];
#pragma unroll
                for (int m = 0; m < NM; ++m) sm[m] = T(0);
                if constexpr (ACC) {
                    // the force at this face (a specular wall takes the normal component),
                    // its gradients from the face values at the neighbouring velocities
                    double fac[3] = {g.acc[0], g.acc[1], g.acc[2]};
                    if ((side == 0 && qa[a] == 0 && g.bc[a][0] == BC_SPECULAR) ||
                        (side == 1 && own_right[a] && g.bc[a][1] == BC_SPECULAR))
                        fac[a] = 0.0;
                    const long long fidx = (long long)ff[a] + side * fs;
                    const T* fbase = bf.face[a];
                    auto val = [&](int j, T& gv, T& bv) {
                        const size_t fa0 = face_addr(g, a, fidx, j / VC) + (j % VC);
                        gv = fbase[fa0];
                        bv = fbase[fa0 + VC];
                    };
                    T fgg[VC], fgb[VC], axi[VC];
                    if (g.nv1[0] % VC == 0) {        // velocity rows are whole chunks: vector loads
                        auto chunk = [&](int vn, T (&gv)[VC], T (&bv)[VC]) {
                            const T* p = fbase + face_addr(g, a, fidx, vn);
                            Chunk<T>::template load<NC>(p, gv);
                            Chunk<T>::template load<NC>(p + VC, bv);
                        };
                        force_gradient_chunk<T, D>(g, fac, vt, chunk, gb, bb, fgg, fgb);
                    }
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        const int i = vt * VC + v;
                        if (g.nv1[0] % VC != 0) {
                            fgg[v] = fgb[v] = T(0);
                            if (i < g.nv1[0] * g.nv1[1] * g.nv1[2])
                                force_gradient<T, D>(g, fac, i, val, fgg[v], fgb[v]);
                        }
                        axi[v] = T(0);
#pragma unroll
                        for (int b = 0; b < D; ++b) axi[v] = fma((T)fac[b], xi[v][b], axi[v]);
                    }
                    face_flux<T, D, SK, true, NOSRC>(fcst, xi, w, hx, a, gb, bb, F[side][0], F[side][1], sm, hL, fgg,
                                                     fgb, axi, (T)(0.5 * g.h));
                } else {
                    face_flux<T, D, SK, false, NOSRC>(fcst, xi, w, hx, a, gb, bb, F[side][0], F[side][1], sm, hL);
                }
                if (side == 0) {
#pragma unroll
                    for (int m = 0; m < NM; ++m) acc[a][m].add(sm[m]);
                } else if (own_right[a]) {
                    const int pl = FS::poff(a) * NM + TL::plane_pos(a, la);
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        Kahan<T> k = RS[pl + m * FS::plane(a)];
                        k.add(sm[m]);
                        RS[pl + m * FS::plane(a)] = k;
                    }
                }
            }
            const T idx = idxT[a];
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                dFg[v] = fma(idx, F[1][0].v[v] - F[0][0].v[v], dFg[v]);
                dFb[v] = fma(idx, F[1][1].v[v] - F[0][1].v[v], dFb[v]);
            }
        }
        if constexpr (ACC) {     // + dt F^n of the own cell (eq. phiupdate's source, rectangle rule)
            T fgo[VC], fbo[VC];
            Chunk<T>::template load<NC>(bf.force + ad, fgo);
            Chunk<T>::template load<NC>(bf.force + ad + VC, fbo);
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                dFg[v] -= fgo[v];
                dFb[v] -= fbo[v];
            }
        }
        T og[VC], ob[VC], oge[VC], obe[VC];
        own_state<T, D, SK>(own, xi, hx, gs, bs, og, ob, oge, obe, hL);
        T u[D];
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = own.u[a];
        store_phi_star<T, D, SK || NOSRC>(dtT, xi, u, own.hu2, own.um_g, own.um_b, own.usrc, og, ob, oge, obe, dFg,
                                          dFb, bf.phi_out + ad);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
        for (int m = 0; m < NM; ++m) bf.mf[a][((size_t)grp * NM + m) * g.nf[a] + ff[a]] = acc[a][m].value();
        if (own_right[a]) {
            const int fs = a == 0 ? 1 : (a == 1 ? g.fn[1][0] : g.fn[2][0] * g.fn[2][1]);
            const int pl = FS::poff(a) * NM + TL::plane_pos(a, la);
#pragma unroll
            for (int m = 0; m < NM; ++m)
                bf.mf[a][((size_t)grp * NM + m) * g.nf[a] + ff[a] + fs] = RS[pl + m * FS::plane(a)].value();
        }
    }
}

// CTAs per SM for k_flux: shared memory and threads, keeping >= 80 registers.
template <typename T, int D, int T0_, int T1_, int T2_, bool SK = false>
struct FluxOcc {
    static constexpr size_t per = FluxSmem<T, D, T0_, T1_, T2_, SK>::bytes + 1024;
    static constexpr int by_smem = (int)((228 * 1024) / per);
    static constexpr int by_threads = 2048 / Tile<D, T0_, T1_, T2_>::NT;
    static constexpr int by_regs = 65536 / (Tile<D, T0_, T1_, T2_>::NT * 128);
    static constexpr int v1 = by_smem < by_threads ? by_smem : by_threads;
    static constexpr int v0 = v1 < by_regs ? v1 : by_regs;
    static constexpr int value = v0 < 1 ? 1 : (v0 > 8 ? 8 : v0);
};

template <typename T, int D, int T0_, int T1_, int T2_, bool SK = false, bool ACC = false, bool NOSRC = false>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (FluxOcc<T, D, T0_, T1_, T2_, SK>::value))
    k_flux(const Inst<T>* __restrict__ in, int cur) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    flux_body<T, D, T0_, T1_, T2_, SK, ACC, NOSRC>(in->g, in->b[cur], blockIdx.x, blockIdx.y, smem);
}

// Many instances in one launch: the device table of instances and a work list
// of items, one per CTA.  The current parity of each instance lives on the
// device and the W-update kernel flips it, so a captured graph replays.

template <typename T, int D, int T0_, int T1_, int T2_, bool SWEEP_B, int MODE = MODE_FUSED>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (Occ<T, D, T0_, T1_, T2_, SWEEP_B, MODE>::value))
    k_sweep_batch(const Item* __restrict__ items, const Inst<T>* __restrict__ insts, const int* __restrict__ cur) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    const Item it = items[blockIdx.x];
    const Inst<T>& in = insts[it.inst];
    sweep_body<T, D, T0_, T1_, T2_, SWEEP_B, MODE>(in.g, in.b[cur[it.inst] & 1], it.tile, it.grp, smem);
}

template <typename T, int D, int T0_, int T1_, int T2_, bool SK = false, bool ACC = false>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (FluxOcc<T, D, T0_, T1_, T2_, SK>::value))
    k_flux_batch(const Item* __restrict__ items, const Inst<T>* __restrict__ insts, const int* __restrict__ cur) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    const Item it = items[blockIdx.x];
    const Inst<T>& in = insts[it.inst];
    flux_body<T, D, T0_, T1_, T2_, SK, ACC>(in.g, in.b[cur[it.inst] & 1], it.tile, it.grp, smem);
}

// ---- Shakhov model: raw velocity moments for the heat flux
//
// Per item (a face of one axis, or a cell) of a [chunk][item][g|b][VC] array
// and velocity group: s = (sum w xi_a b [D], sum w xi_a xi_b g [a <= b]) over
// the group's chunks, in chunk order (per-chunk sums folded into Kahan pairs
// in FP32), into dst[(grp * NQ + m) * n + item].  k_faceq reads the stored
// face values (phibar at the faces), k_cellq the phi* just written (the
// explicit part of eq. phiupdate).
template <int D>
struct NQ {
    static constexpr int value = D + D * (D + 1) / 2;
};

template <typename T, int D>
__device__ __forceinline__ void raw_moments(const Geo& g, const T* __restrict__ vel, const T* __restrict__ src,
                                            long long n, long long item, int grp, double* __restrict__ dst) {
    constexpr int M = NQ<D>::value;
    Kahan<T> acc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m].zero();
    const int vt0 = grp * g.ntpg, vt1 = min(g.NVT, vt0 + g.ntpg);
    for (int vt = vt0; vt < vt1; ++vt) {
        T gv[VC], bv[VC];
        const T* p = src + ((size_t)vt * (size_t)n + (size_t)item) * (2 * VC);
        Chunk<T>::load(p, gv);
        Chunk<T>::load(p + VC, bv);
        T sm[M];
#pragma unroll
        for (int m = 0; m < M; ++m) sm[m] = T(0);
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const T* rec = vel + (size_t)(vt * VC + v) * 8;
            T xi[D];
#pragma unroll
            for (int a = 0; a < D; ++a) xi[a] = rec[a];
            const T wg = rec[3] * gv[v], wb = rec[3] * bv[v];
            int k = D;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                sm[a] = fma(xi[a], wb, sm[a]);
#pragma unroll
                for (int b = a; b < D; ++b, ++k) sm[k] = fma(xi[a] * xi[b], wg, sm[k]);
            }
        }
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m].add(sm[m]);
    }
#pragma unroll
    for (int m = 0; m < M; ++m) dst[((size_t)grp * M + m) * (size_t)n + item] = acc[m].value();
}

// grid (faces / blockDim, velocity groups, axes)
template <typename T, int D>
__global__ void k_faceq(const Inst<T>* __restrict__ in, int cur) {
    pdl_wait();
    // the axis is a launch index: read what it selects from the record, copy nothing
    const Geo& g = in->g;
    const Bufs<T>& bf = in->b[cur];
    const int a = blockIdx.z;
    if (a >= D) return;
    const long long nf = g.nf[a];
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < nf) raw_moments<T, D>(g, bf.vel, bf.face[a], nf, f, blockIdx.y, bf.qf[a]);
}

// grid (cells / blockDim, velocity groups)
template <typename T, int D>
__global__ void k_cellq(const Inst<T>* __restrict__ in, int cur) {
    pdl_wait();
    const Geo g = in->g;
    const Bufs<T> bf = in->b[cur];
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.Nc) raw_moments<T, D>(g, bf.vel, bf.phi_out, g.Nc, c, blockIdx.y, bf.qs);
}

// Batched raw moments: one CTA per item (faces of one axis, or cells, of one
// instance and one velocity group); faces read the stored face values, cells
// the phi* that sweep B has just written.
template <typename T, int D>
__global__ void k_rawq_batch(const QItem* __restrict__ items, const Inst<T>* __restrict__ insts,
                             const int* __restrict__ cur) {
    pdl_wait();
    const QItem it = items[blockIdx.x];
    const Geo& g = insts[it.inst].g;
    const Bufs<T>& bf = insts[it.inst].b[cur[it.inst] & 1];
    const T* src = it.axis >= 0 ? bf.face[it.axis] : bf.phi_out;
    double* dst = it.axis >= 0 ? bf.qf[it.axis] : bf.qs;
    const long long n = it.axis >= 0 ? g.nf[it.axis] : g.Nc;
    for (long long k = threadIdx.x; k < it.count; k += blockDim.x)
        raw_moments<T, D>(g, bf.vel, src, n, it.start + k, it.grp, dst);
}

// Sums over the velocity groups of M per-group partial sums of one item
// (src[(gg M + m) n], src at the item), added in group order; the loads of
// four groups are issued before their additions, so a thread waits for one
// memory round trip per four groups, not per group.
template <int M>
__device__ __forceinline__ void group_sums(const double* __restrict__ src, size_t n, int G, double (&s)[M]) {
    constexpr int UG = 4;
#pragma unroll
    for (int m = 0; m < M; ++m) s[m] = 0.0;
    int gg = 0;
    for (; gg + UG <= G; gg += UG) {
        double v[UG][M];
#pragma unroll
        for (int u = 0; u < UG; ++u)
#pragma unroll
            for (int m = 0; m < M; ++m) v[u][m] = src[((size_t)(gg + u) * M + m) * n];
#pragma unroll
        for (int u = 0; u < UG; ++u)
#pragma unroll
            for (int m = 0; m < M; ++m) s[m] = dadd(s[m], v[u][m]);
    }
    for (; gg < G; ++gg)
#pragma unroll
        for (int m = 0; m < M; ++m) s[m] = dadd(s[m], src[((size_t)gg * M + m) * n]);
}

// Group sums of the raw moments of one item (fixed order), then its heat flux
// relative to W divided by 1 + x Pr/tau: x = h/2 at a face (phibar relaxes the
// heat flux by that factor), dt/2 at a cell (phi* against phi^{n+1}).
template <typename T, int D>
__device__ __forceinline__ void shakhov_heat_flux(const Geo& g, const double* src, long long n, long long item,
                                                  const double* W, double x, double q[3]) {
    constexpr int M = NQ<D>::value;
    double s[M];
    group_sums<M>(src + item, (size_t)n, g.G, s);
    const Macro mc = macro_of(g, W);
    heat_flux_raw<D>(mc, W, s, q);
    const Relax<double> r = relax_of<double>(g, mc);
    const double div = dadd(1.0, dmul(dmul(x, g.Pr), r.itg));
    for (int a = 0; a < D; ++a) q[a] = ddiv(q[a], div);
}

// Face constants from the group-summed face W (fixed summation order).
template <typename T, int D>
__device__ __forceinline__ void facec_body(const Geo& g, const Bufs<T>& bf, int a, long long f) {
    constexpr int NM = 2 + D;
    double W[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    {
        double s[NM];
        group_sums<NM>(bf.wf[a] + f, (size_t)g.nf[a], g.G, s);
        for (int m = 0; m < NM; ++m) W[m] = s[m];
    }
    if (g.accel) {   // eqs. rhoubar, rhoEbar: + (h/2) rho a, then + (h/2) (rho u) . a
        double fac[3] = {g.acc[0], g.acc[1], g.acc[2]};
        const long long st = a == 0 ? 1 : (a == 1 ? (long long)g.fn[a][0] : (long long)g.fn[a][0] * g.fn[a][1]);
        const int qn = (int)((f / st) % g.fn[a][a]);
        if ((qn == 0 && g.bc[a][0] == BC_SPECULAR) || (qn == g.n[a] && g.bc[a][1] == BC_SPECULAR))
            fac[a] = 0.0;    // a specular wall takes the normal component of the force
        const double hh = 0.5 * g.h;
        for (int b = 0; b < D; ++b) W[1 + b] = dadd(W[1 + b], dmul(dmul(hh, W[0]), fac[b]));
        for (int b = 0; b < D; ++b) W[1 + D] = dadd(W[1 + D], dmul(dmul(hh, W[1 + b]), fac[b]));
    }
    double q[3] = {0.0, 0.0, 0.0};
    if (g.shakhov) shakhov_heat_flux<T, D>(g, bf.qf[a], g.nf[a], f, W, 0.5 * g.h, q);
    make_face<T>(g, W, q, bf.facec[a][f]);
    if (bf.xf[a]) write_factors<T>(g, macro_of(g, W), bf.xf[a], g.nf[a], f);
}

// grid (faces / blockDim, axes): every axis in one launch
template <typename T, int D>
__global__ void k_facec(const Inst<T>* __restrict__ in, int cur) {
    pdl_wait();
    const int a = blockIdx.y;
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < D && f < in->g.nf[a]) facec_body<T, D>(in->g, in->b[cur], a, f);
}

template <typename T, int D>
__global__ void k_facec_batch(const RItem* __restrict__ items, const Inst<T>* __restrict__ insts,
                              const int* __restrict__ cur) {
    pdl_wait();
    const RItem it = items[blockIdx.x];
    // the member's record read from the table (the ranges are whole blocks of
    // about one face per thread: a copy of the record per thread costs more
    // than the aliasing reloads it avoids)
    const Inst<T>& in = insts[it.inst];
    const int c = cur[it.inst] & 1;
    for (long long k = threadIdx.x; k < it.count; k += blockDim.x) facec_body<T, D>(in.g, in.b[c], it.axis, it.start + k);
}

// W^{n+1} = W^n - dt sum_a (M_a(right face) - M_a(left face)) / dx_a (outward
// normals), the status check, and the cell constants of W^{n+1}.
template <typename T, int D>
__device__ __forceinline__ void wupdate_body(const Geo& g, const Bufs<T>& bf, long long c) {
    constexpr int NM = 2 + D;
    int q[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((long long)g.n[0] * g.n[1]))};
    double dW[NM];
    for (int m = 0; m < NM; ++m) dW[m] = 0.0;
    for (int a = 0; a < D; ++a) {
        const long long fl = face_index(g, a, q);
        int qr[3] = {q[0], q[1], q[2]};
        qr[a] += 1;
        const long long fr = face_index(g, a, qr);
        double sr[NM], sl[NM];
        group_sums<NM>(bf.mf[a] + fr, (size_t)g.nf[a], g.G, sr);
        group_sums<NM>(bf.mf[a] + fl, (size_t)g.nf[a], g.G, sl);
        for (int m = 0; m < NM; ++m) dW[m] = __fma_rn(dsub(sr[m], sl[m]), g.idx[a], dW[m]);
    }
    double W[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < NM; ++m) W[m] = __fma_rn(-g.dt, dW[m], bf.W[(size_t)m * g.Nc + c]);
    if (g.accel) {   // + dt times the source integrals at t_n: rho^n a, (rho u)^n . a
        const double rho0 = bf.W[c];
        for (int b = 0; b < D; ++b) {
            W[1 + b] = dadd(W[1 + b], dmul(dmul(g.dt, rho0), g.acc[b]));
            W[1 + D] = dadd(W[1 + D], dmul(dmul(g.dt, bf.W[(size_t)(1 + b) * g.Nc + c]), g.acc[b]));
        }
    }
    bool finite = true;
    for (int m = 0; m < NM; ++m) {
        finite = finite && isfinite(W[m]);
        bf.W[(size_t)m * g.Nc + c] = W[m];
    }
    // internal energy rho e = rho E - |rho u|^2 / (2 rho) > 0  <=>  2 rho (rho E) > |rho u|^2 (rho > 0)
    double m2 = 0.0;
    for (int a = 0; a < D; ++a) m2 += W[1 + a] * W[1 + a];
    int st = 0;
    if (!finite) st |= ST_NONFINITE;
    else if (!(W[0] > 0.0) || !(2.0 * W[0] * W[1 + D] > m2)) st |= ST_NEGATIVE;
    if (st) atomicOr(bf.status, st);
    double hq[3] = {0.0, 0.0, 0.0};      // Shakhov: the heat flux of t_{n+1}
    if (g.shakhov) {
        shakhov_heat_flux<T, D>(g, bf.qs, g.Nc, c, W, 0.5 * g.dt, hq);
        for (int a = 0; a < D; ++a) bf.hq[(size_t)a * g.Nc + c] = hq[a];
    }
    make_cell<T>(g, W, hq, bf.cellc[c]);
    if (bf.xc) write_factors<T>(g, macro_of(g, W), bf.xc, g.Nc, c);
}

template <typename T, int D>
__global__ void k_wupdate(const Inst<T>* __restrict__ in, int cur) {
    pdl_wait();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < in->g.Nc) wupdate_body<T, D>(in->g, in->b[cur], c);
}

// Batched W update; the item that starts at cell 0 of an instance flips its
// buffer parity (no other kernel of the step reads it afterwards).
template <typename T, int D>
__global__ void k_wupdate_batch(const RItem* __restrict__ items, const Inst<T>* __restrict__ insts,
                                int* __restrict__ cur) {
    pdl_wait();
    const RItem it = items[blockIdx.x];
    // The member's first block flips its buffer index when done, so a later
    // block of the same member may read either value: the two records differ
    // only in the phi buffers, which the W update does not touch.
    const int c0 = cur[it.inst] & 1;
    const Inst<T>& in = insts[it.inst];
    for (long long k = threadIdx.x; k < it.count; k += blockDim.x) wupdate_body<T, D>(in.g, in.b[c0], it.start + k);
    if (it.start == 0) {
        __syncthreads();
        if (threadIdx.x == 0) cur[it.inst] = c0 ^ 1;
    }
}

// Cell constants from the stored W (after a state restore).
template <typename T, int D>
__global__ void k_cellc(const Inst<T>* __restrict__ in, int cur) {
    const Geo g = in->g;
    const Bufs<T> bf = in->b[cur];
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Nc) return;
    double W[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < 2 + D; ++m) W[m] = bf.W[(size_t)m * g.Nc + c];
    double q[3] = {0.0, 0.0, 0.0};
    if (g.shakhov)
        for (int a = 0; a < D; ++a) q[a] = bf.hq[(size_t)a * g.Nc + c];
    make_cell<T>(g, W, q, bf.cellc[c]);
    if (bf.xc) write_factors<T>(g, macro_of(g, W), bf.xc, g.Nc, c);
}

// Maxwell-Boltzmann initial state: W^0 from (rho, u, T), its constants (also
// kept as the Dirichlet ghost constants), phi* = phi_eq(W^0) (the stored
// pre-update value whose finalisation gives phi^0 = phi_eq).
template <typename T, int D>
__global__ void k_init(const Inst<T>* __restrict__ in, int cur, const double* __restrict__ fields) {
    const Geo g = in->g;
    const Bufs<T> bf = in->b[cur];
    constexpr int NM = 2 + D;
    const long long c = blockIdx.x;
    const double* f = fields + (size_t)c * NM;
    double Wc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double cv = (3.0 + g.K) * g.R / 2.0;
    double u2 = 0.0;
    Wc[0] = f[0];
    for (int a = 0; a < D; ++a) {
        Wc[1 + a] = f[0] * f[1 + a];
        u2 += f[1 + a] * f[1 + a];
    }
    Wc[1 + D] = f[0] * (0.5 * u2 + cv * f[1 + D]);
    if (threadIdx.x < NM) bf.W[(size_t)threadIdx.x * g.Nc + c] = Wc[threadIdx.x];
    if (g.shakhov && threadIdx.x < D) bf.hq[(size_t)threadIdx.x * g.Nc + c] = 0.0;   // a Maxwellian: q = 0
    __shared__ CellC<T> shc;
    if (threadIdx.x == 0) {       // the FP64 constants once per cell, not once per thread
        make_cell<T>(g, Wc, nullptr, shc);
        bf.cellc[c] = shc;
        bf.cellc0[c] = shc;
        if (bf.xc) {              // lean shapes: the separable factors of W^0
            const Macro m0 = macro_of(g, Wc);
            write_factors<T>(g, m0, bf.xc, g.Nc, c);
            write_factors<T>(g, m0, bf.xc0, g.Nc, c);
        }
    }
    __syncthreads();
    const CellC<T> cc = shc;
    for (int i = threadIdx.x; i < g.Nvp; i += blockDim.x) {
        const Vel<T, D> v = load_vel<T, D>(g, bf, i);
        T ge, be;
        if (bf.xc) {              // the equilibrium as the lean sweeps form it: the product of the factors
            ge = table_geq<T, D>(g, bf.xc, c, i);
            be = (v.hxi2 + cc.eb) * ge;
        } else {
            equilibrium<T, D>(g, cc, v, ge, be);
        }
        const size_t ad = phi_addr(g, c, i, 0);
        bf.phi_out[ad] = ge;
        bf.phi_out[ad + VC] = be;
    }
}

// rho, u, T per cell from W (Sec. 2), or W itself, [Nc][2+D].
template <int D>
__global__ void k_moments(Geo g, const double* __restrict__ W, double* __restrict__ out, int conserved) {
    constexpr int NM = 2 + D;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Nc) return;
    double Wc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < NM; ++m) Wc[m] = W[(size_t)m * g.Nc + c];
    if (conserved) {
        for (int m = 0; m < NM; ++m) out[(size_t)c * NM + m] = Wc[m];
        return;
    }
    Macro mc = macro_of(g, Wc);
    out[(size_t)c * NM] = mc.rho;
    for (int a = 0; a < D; ++a) out[(size_t)c * NM + 1 + a] = mc.u[a];
    out[(size_t)c * NM + 1 + D] = mc.T;
}

// Pressure tensor and heat flux of every cell from its finalised distributions
// (a diagnostic output; the step does not use them).  One CTA per cell sums
// the raw moments over the velocities in FP64 (tree of fixed order), then
//   P_ab = sum w xi_a xi_b g - rho u_a u_b  (= sum w (xi - u)_a (xi - u)_b g),
//   q_a  = sum w xi_a b - u_a rho E - sum_b P_ab u_b,
// with rho, rho u, rho E the moments of the same distributions.
// out: [Nc][D*D + D], P row-major, then q.
constexpr int kStressThreads = 128;
template <typename T, int D>
__global__ void __launch_bounds__(kStressThreads) k_stress(const Inst<T>* __restrict__ in, int cur,
                                                           double* __restrict__ out) {
    constexpr int NA = 1 + D + D * (D + 1) / 2 + 1 + D;     // rho, rho u, second moments, rho E, energy flux
    __shared__ double red[NA][kStressThreads];
    const Geo g = in->g;
    const Bufs<T> bf = in->b[cur];
    const long long c = blockIdx.x;
    const int t = threadIdx.x;
    const CellC<T> cc = bf.cellc[c];
    double acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = 0.0;
    for (int i = t; i < g.Nvp; i += kStressThreads) {
        const Vel<T, D> v = load_vel<T, D>(g, bf, i);
        T ge, be;
        if (bf.xc) {
            ge = table_geq<T, D>(g, bf.xc, c, i);
            be = (v.hxi2 + cc.eb) * ge;
        } else {
            equilibrium<T, D>(g, cc, v, ge, be);
        }
        const size_t ad = phi_addr(g, c, i, 0);
        const double gv = (double)fma(cc.fa_g, bf.phi_in[ad], cc.fb_g * ge);
        const double bv = (double)fma(cc.fa_b, bf.phi_in[ad + VC], cc.fb_b * be);
        const double wg = (double)v.w * gv, wb = (double)v.w * bv;
        int k = 0;
        acc[k++] += wg;
#pragma unroll
        for (int a = 0; a < D; ++a) acc[k++] += (double)v.xi[a] * wg;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b2 = a; b2 < D; ++b2) acc[k++] += (double)v.xi[a] * (double)v.xi[b2] * wg;
        acc[k++] += wb;
#pragma unroll
        for (int a = 0; a < D; ++a) acc[k++] += (double)v.xi[a] * wb;
    }
#pragma unroll
    for (int k = 0; k < NA; ++k) red[k][t] = acc[k];
    __syncthreads();
    for (int s2 = kStressThreads / 2; s2 > 0; s2 >>= 1) {
        if (t < s2)
#pragma unroll
            for (int k = 0; k < NA; ++k) red[k][t] += red[k][t + s2];
        __syncthreads();
    }
    if (t != 0) return;
    const double rho = red[0][0];
    double u[D], P[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = red[1 + a][0] / rho;
    int k = 1 + D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b2 = a; b2 < D; ++b2) {
            P[a][b2] = red[k++][0] - rho * u[a] * u[b2];
            P[b2][a] = P[a][b2];
        }
    const double rhoE = red[k++][0];
    double* dst = out + (size_t)c * (D * D + D);
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
        for (int b2 = 0; b2 < D; ++b2) dst[a * D + b2] = P[a][b2];
        double q = red[k + a][0] - u[a] * rhoE;
#pragma unroll
        for (int b2 = 0; b2 < D; ++b2) q -= P[a][b2] * u[b2];
        dst[D * D + a] = q;
    }
}

// The finalised distributions phi = fa phi* + fb phi_eq at the current time
// level, written in the state layout into the idle buffer.
template <typename T, int D>
__global__ void k_finalise(const Inst<T>* __restrict__ in, int cur) {
    const Geo g = in->g;
    const Bufs<T> bf = in->b[cur];
    const long long c = blockIdx.x;
    const CellC<T> cc = bf.cellc[c];
    for (int i = threadIdx.x; i < g.Nvp; i += blockDim.x) {
        const Vel<T, D> v = load_vel<T, D>(g, bf, i);
        T ge, be;
        if (bf.xc) {
            ge = table_geq<T, D>(g, bf.xc, c, i);
            be = (v.hxi2 + cc.eb) * ge;
        } else {
            equilibrium<T, D>(g, cc, v, ge, be);
        }
        const size_t ad = phi_addr(g, c, i, 0);
        bf.phi_out[ad] = fma(cc.fa_g, bf.phi_in[ad], cc.fb_g * ge);
        bf.phi_out[ad + VC] = fma(cc.fa_b, bf.phi_in[ad + VC], cc.fb_b * be);
    }
}

}  // namespace cdg
