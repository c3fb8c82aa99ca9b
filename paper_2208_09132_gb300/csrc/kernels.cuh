// kernels.cuh -- sm_103a device code of the CDUGKS step (arXiv:2208.09132, Sec. 2.1).
//
// One time step is three launches on the caller's stream:
//
//   sweep A  per (spatial tile, velocity group): finalise phi^n from the stored
//            pre-update value phi* (the last factor of eq. phiupdate, deferred
//            until W^n is known), form phibar+ (eq. phibarplus) on the tile and
//            a two-cell halo in shared memory, reconstruct phibar at every
//            owned face along the characteristic (eqs. VanLeer, relation) and
//            reduce the face conserved variables (eqs. rhobar-rhoEbar) over the
//            group's velocities: warp butterfly per 32-velocity tile, then a
//            compensated accumulator per face in shared memory.
//   sweep B  the same reconstruction, then the face equilibrium (eqs. geq,
//            beq) from the face W, inversion of eq. phibar, the microflux
//            xi.n phi (eq. flux), the face moments of the flux (for W) and the
//            per-velocity net flux, which feeds phi* of eq. phiupdate, written
//            to the other state buffer.
//   W update W^{n+1} = W^n - dt sum_faces (M_right - M_left)/dx (eqs.
//            rhoupdate-rhoEupdate, outward normals), with the status check.
//
// Layout in HBM: phi*[velocity tile][cell][field g|b][32 lanes], so a warp
// reads 2 x 128 contiguous bytes (FP32) per cell and a tile of cells of one
// velocity tile is a dense slab.  Boundaries are applied by index mapping
// while the halo is loaded (periodic wrap, mirror with reflected velocity,
// fixed equilibrium), not by ghost copies.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace cdg {

constexpr int VI = 32;            // velocities per tile = lanes of a warp
constexpr int NWARPS = 8;
constexpr int NTHREADS = VI * NWARPS;

enum { BC_PERIODIC = 0, BC_SPECULAR = 1, BC_DIRICHLET = 2 };
enum { ST_NONFINITE = 1, ST_NEGATIVE = 2 };

// Problem geometry and physics, passed by value to every kernel.
struct Geo {
    int D;
    int n[3];
    int bc[3][2];
    long long Nc;
    int Nvp;          // padded velocity count (multiple of VI)
    int NVT;          // velocity tiles
    int ntpg;         // velocity tiles per group
    int G;            // velocity groups
    int tiles[3];     // spatial tiles per axis
    int fn[3][3];     // face-array extents per axis a: fn[a][b] = n[b] + (a == b)
    long long nf[3];  // faces per axis
    double dx[3];
    double hdx[3];    // h / dx_a
    double idx[3];    // 1 / dx_a
    double dt, h;
    double K, R, mu_ref, T_ref, omega, Pr;
};

template <typename T> struct CellC;
template <typename T> struct FaceC;

template <typename T>
struct Bufs {
    const T* phi_in;
    T* phi_out;
    double* W;            // [2+D][Nc] tracked conserved variables, updated in place
    CellC<T>* cellc;      // [Nc] constants of W^n (written by the W update / init)
    CellC<T>* cellc0;     // [Nc] constants of W^0 (Dirichlet ghosts)
    FaceC<T>* facec[3];   // [nf_a] constants of the face W (between the sweeps)
    double* wf[3];        // [G][2+D][nf_a] face W partial sums (sweep A)
    double* mf[3];        // [G][2+D][nf_a] face flux-moment partial sums (sweep B)
    const T* xi;          // [3][Nvp]
    const T* w;           // [Nvp] quadrature weights (0 on padding)
    const T* hxi2;        // [Nvp] |xi|^2 / 2
    const int* refl;      // [8][Nvp] velocity index with the components of mask reversed
    int* status;
};

// ------------------------------------------------------------------ numerics

template <typename T> struct Num;
template <> struct Num<float> {
    // equilibrium exponent on base 2: exp(-c^2/(2RT)) = exp2(c^2 * cexp)
    static __device__ __forceinline__ float expo(float x) { return exp2f(x); }
    static __host__ __device__ __forceinline__ double cexp_scale() { return 1.4426950408889634; }
    static __device__ __forceinline__ float vanleer(float s1, float s2) {
        float p = s1 * s2;
        return p > 0.f ? __fdividef(2.f * p, s1 + s2) : 0.f;
    }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double expo(double x) { return exp(x); }
    static __host__ __device__ __forceinline__ double cexp_scale() { return 1.0; }
    static __device__ __forceinline__ double vanleer(double s1, double s2) {
        double p = s1 * s2;
        return p > 0.0 ? 2.0 * p / (s1 + s2) : 0.0;
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
    T sa_g, sa_b, ssrc;         // phibar+ = eq + sa (phi - eq) [+ ssrc Z (g - g_eq)]   (eq. phibarplus)
    T um_g, um_b, usrc;         // phi* = eq + um (phi - eq) [+ usrc Z (g - g_eq)] - dt dF (eq. phiupdate)
};

// Face constants from the face W (eq. phibar inverted: phi = eq + alpha (phibar - eq) [+ gb Z (g - g_eq)]).
template <typename T>
struct FaceC {
    T u[3];
    T cexp, pref, eb, hu2;
    T al_g, al_b, gam_b;
};

struct Macro {
    double rho, u[3], T, RT, tg, tb, itbg;
};

__device__ __forceinline__ Macro macro_of(const Geo& g, const double* W) {
    Macro m;
    m.rho = W[0];
    double u2 = 0.0;
    for (int a = 0; a < 3; ++a) m.u[a] = 0.0;
    for (int a = 0; a < g.D; ++a) {
        m.u[a] = W[1 + a] / m.rho;
        u2 += m.u[a] * m.u[a];
    }
    double E = W[1 + g.D] / m.rho;
    double gam = (g.K + 5.0) / (g.K + 3.0);
    m.T = (gam - 1.0) / g.R * (E - 0.5 * u2);
    m.RT = g.R * m.T;
    double mu = g.mu_ref * pow(m.T / g.T_ref, g.omega);
    m.tg = mu / (m.rho * m.RT);
    m.tb = m.tg / g.Pr;
    m.itbg = 1.0 / m.tb - 1.0 / m.tg;
    return m;
}

template <typename T>
__device__ __forceinline__ void eq_consts(const Geo& g, const Macro& m, T u[3], T& cexp, T& pref, T& eb, T& hu2) {
    double u2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        u[a] = (T)m.u[a];
        u2 += m.u[a] * m.u[a];
    }
    cexp = (T)(-Num<T>::cexp_scale() / (2.0 * m.RT));
    pref = (T)(m.rho * pow(2.0 * 3.14159265358979323846 * m.RT, -0.5 * g.D));
    eb = (T)(0.5 * (3.0 - g.D + g.K) * m.RT);
    hu2 = (T)(0.5 * u2);
}

template <typename T>
__device__ __forceinline__ void make_cell(const Geo& g, const double* W, CellC<T>& c) {
    Macro m = macro_of(g, W);
    eq_consts<T>(g, m, c.u, c.cexp, c.pref, c.eb, c.hu2);
    const double dt = g.dt, h = g.h;
    c.fa_g = (T)(2.0 * m.tg / (2.0 * m.tg + dt));
    c.fb_g = (T)(dt / (2.0 * m.tg + dt));
    c.fa_b = (T)(2.0 * m.tb / (2.0 * m.tb + dt));
    c.fb_b = (T)(dt / (2.0 * m.tb + dt));
    c.sa_g = (T)(1.0 - h / (2.0 * m.tg));
    c.sa_b = (T)(1.0 - h / (2.0 * m.tb));
    c.ssrc = (T)(0.5 * h * m.itbg);
    c.um_g = (T)(1.0 - dt / (2.0 * m.tg));
    c.um_b = (T)(1.0 - dt / (2.0 * m.tb));
    c.usrc = (T)(dt * m.itbg);
}

template <typename T>
__device__ __forceinline__ void make_face(const Geo& g, const double* W, FaceC<T>& f) {
    Macro m = macro_of(g, W);
    eq_consts<T>(g, m, f.u, f.cexp, f.pref, f.eb, f.hu2);
    const double h = g.h;
    f.al_g = (T)(2.0 * m.tg / (2.0 * m.tg + h));
    f.al_b = (T)(2.0 * m.tb / (2.0 * m.tb + h));
    f.gam_b = (T)(h * m.tb * m.itbg / (2.0 * m.tb + h));
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
#pragma unroll
    for (int a = 0; a < D; ++a) {
        v.xi[a] = bf.xi[a * g.Nvp + i];
        v.nu[a] = (T)g.hdx[a] * v.xi[a];
    }
    v.w = bf.w[i];
    v.hxi2 = bf.hxi2[i];
    return v;
}

template <typename T, int D, typename C>
__device__ __forceinline__ void equilibrium(const C& c, const Vel<T, D>& v, T& geq, T& beq) {
    T c2 = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        T d = v.xi[a] - c.u[a];
        c2 = fma(d, d, c2);
    }
    geq = c.pref * Num<T>::expo(c.cexp * c2);
    beq = (v.hxi2 + c.eb) * geq;
}

template <typename T, int D, typename C>
__device__ __forceinline__ T zeta(const C& c, const Vel<T, D>& v) {
    T z = -c.hu2;
#pragma unroll
    for (int a = 0; a < D; ++a) z = fma(v.xi[a], c.u[a], z);
    return z;
}

// ------------------------------------------------------- warp reductions

// Sum NM values over the 32 lanes.  Returns, in every lane, the total of one
// moment; moment_of_lane() says which.  Recursive halving: at each of the
// first log2(NP) steps a lane keeps half of its values and receives the
// partner's half of the other values.
template <typename T, int NM>
struct WarpSum {
    static constexpr int NP = NM <= 2 ? 2 : (NM <= 4 ? 4 : 8);
    static constexpr int LG = NP == 2 ? 1 : (NP == 4 ? 2 : 3);
    static __device__ __forceinline__ T run(const T (&vin)[NM], int lane) {
        T v[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) v[k] = k < NM ? vin[k] : T(0);
        int cnt = NP;
#pragma unroll
        for (int s = 0; s < LG; ++s) {
            const int mask = 16 >> s;
            const bool hi = (lane & mask) != 0;
            cnt >>= 1;
#pragma unroll
            for (int k = 0; k < NP / 2; ++k) {
                if (k < cnt) {
                    T keep = hi ? v[k + cnt] : v[k];
                    T send = hi ? v[k] : v[k + cnt];
                    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
                }
            }
        }
        T r = v[0];
#pragma unroll
        for (int s = LG; s < 5; ++s) r += __shfl_xor_sync(0xffffffffu, r, 16 >> s);
        return r;
    }
    // lane bits 4, 3, 2 (most significant first) select the value index
    static __device__ __forceinline__ int moment_of_lane(int lane) {
        int m = 0;
#pragma unroll
        for (int s = 0; s < LG; ++s) m = (m << 1) | ((lane >> (4 - s)) & 1);
        return m;
    }
    static __device__ __forceinline__ bool writer(int lane) {
        return (lane & ((1 << (5 - LG)) - 1)) == 0;
    }
};

// Compensated accumulation of per-tile sums (FP32: Kahan pair; FP64: plain).
template <typename T> struct Acc;
template <> struct Acc<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct Acc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// ------------------------------------------------------------- geometry

// Map a cell coordinate that may lie in the two-deep ghost layer onto the
// interior: axes resolved from the last to the first (the order in which
// ghost layers of later axes overwrite corners), periodic wrap, specular
// mirror (reflection bit set), Dirichlet clamp (flag).  Coordinates beyond the
// ghost layer (ragged tiles) are clamped; they are never read.
__device__ __forceinline__ void resolve(const Geo& g, int q[3], int& refl, bool& dir) {
    refl = 0;
    dir = false;
    for (int a = g.D - 1; a >= 0; --a) {
        const int k = q[a], n = g.n[a];
        if (k >= 0 && k < n) continue;
        const int bc = g.bc[a][k < 0 ? 0 : 1];
        if (bc == BC_PERIODIC) {
            q[a] = ((k % n) + n) % n;
        } else if (bc == BC_SPECULAR) {
            q[a] = k < 0 ? -1 - k : 2 * n - 1 - k;
            refl ^= 1 << a;
        } else {
            dir = true;
            break;
        }
    }
    for (int a = 0; a < g.D; ++a) q[a] = min(max(q[a], 0), g.n[a] - 1);
}

__device__ __forceinline__ long long cell_index(const Geo& g, const int q[3]) {
    return (long long)q[0] + (long long)g.n[0] * ((long long)q[1] + (long long)g.n[1] * q[2]);
}

__device__ __forceinline__ long long face_index(const Geo& g, int a, const int q[3]) {
    return (long long)q[0] + (long long)g.fn[a][0] * ((long long)q[1] + (long long)g.fn[a][1] * q[2]);
}

template <typename T>
__device__ __forceinline__ size_t phi_addr(const Geo& g, long long cell, int i, int field) {
    return ((size_t)(i / VI) * (size_t)g.Nc + (size_t)cell) * (2 * VI) + (size_t)field * VI + (i % VI);
}

// --------------------------------------------------------------- the sweep

template <int D, int TX, int TY, int TZ>
struct Tile {
    static constexpr int T0 = TX, T1 = D >= 2 ? TY : 1, T2 = D >= 3 ? TZ : 1;
    // tile + halo: local cells [-2, T+1] per active axis (the right face of the
    // last cell reads the slope at local T, which needs local T+1)
    static constexpr int E0 = T0 + 4, E1 = D >= 2 ? T1 + 4 : 1, E2 = D >= 3 ? T2 + 4 : 1;
    static constexpr int BOX = E0 * E1 * E2;
    static constexpr int OWN = T0 * T1 * T2;
    static constexpr int NM = 2 + D;
    static constexpr int NF0 = (T0 + 1) * T1 * T2;
    static constexpr int NF1 = D >= 2 ? T0 * (T1 + 1) * T2 : 0;
    static constexpr int NF2 = D >= 3 ? T0 * T1 * (T2 + 1) : 0;
    static constexpr int NFT = NF0 + NF1 + NF2;         // local face table
    static __host__ __device__ constexpr int stride(int a) { return a == 0 ? 1 : (a == 1 ? E0 : E0 * E1); }
    static __host__ __device__ constexpr int tdim(int a) { return a == 0 ? T0 : (a == 1 ? T1 : T2); }
    static __host__ __device__ constexpr int foff(int a) { return a == 0 ? 0 : (a == 1 ? NF0 : NF0 + NF1); }
    // local face (axis a) with right cell at local coords l (l_a in [0, T_a])
    static __device__ __forceinline__ int face_local(int a, int l0, int l1, int l2) {
        const int d0 = T0 + (a == 0), d1 = T1 + (a == 1);
        return foff(a) + l0 + d0 * (l1 + d1 * l2);
    }
    static __device__ __forceinline__ int box_of(int l0, int l1, int l2) {
        return (l0 + 2) + E0 * ((D >= 2 ? l1 + 2 : 0) + E1 * (D >= 3 ? l2 + 2 : 0));
    }
};

template <typename T, int D, int TX, int TY, int TZ>
struct SweepSmem {
    using TL = Tile<D, TX, TY, TZ>;
    static constexpr size_t off_P = 0;                                              // [BOX][2][VI] T
    static constexpr size_t off_cc = off_P + sizeof(T) * TL::BOX * 2 * VI;          // [BOX] CellC
    static constexpr size_t off_src = off_cc + sizeof(CellC<T>) * TL::BOX;          // [BOX] long long
    static constexpr size_t off_fl = off_src + sizeof(long long) * TL::BOX;         // [BOX] int flags
    static constexpr size_t off_fc = ((off_fl + sizeof(int) * TL::BOX + 15) / 16) * 16;  // [NFT] FaceC
    static constexpr size_t off_acc = ((off_fc + sizeof(FaceC<T>) * TL::NFT + 15) / 16) * 16;  // [NFT][NM] Acc
    static constexpr size_t bytes = off_acc + sizeof(Acc<T>) * TL::NFT * TL::NM;
};

// Reconstruct phibar at the face between box cells L = R - e_a and R along
// axis a for this lane's velocity: the upwind cell by the sign of xi_a,
// value phibar+_up + (x_f - h xi - x_up) . sigma_up with the van Leer slope
// vector of phibar+ at the upwind cell (eq. relation; eq. VanLeer).
template <typename T, int D, typename TL>
__device__ __forceinline__ void reconstruct(const T* __restrict__ P, int L, int R, int a, const Vel<T, D>& v,
                                            int lane, T& gb, T& bb) {
    auto one = [&](int up, T ka, T& og, T& ob) {
        const T* pg = P + (size_t)up * 2 * VI + lane;
        T cg = pg[0], cb = pg[VI];
        T rg = cg, rb = cb;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const int s = TL::stride(b) * 2 * VI;
            T lg = pg[-s], lb = pg[VI - s], hg = pg[s], hb = pg[VI + s];
            T k = (b == a) ? ka : -v.nu[b];
            rg = fma(k, Num<T>::vanleer(cg - lg, hg - cg), rg);
            rb = fma(k, Num<T>::vanleer(cb - lb, hb - cb), rb);
        }
        og = rg;
        ob = rb;
    };
    const T xa = v.xi[a];
    const bool left = xa > T(0);
    const int up = left ? L : R;
    const T ka = (left ? T(0.5) : T(-0.5)) - v.nu[a];
    one(up, ka, gb, bb);
    if (__any_sync(0xffffffffu, xa == T(0))) {   // xi . n = 0: mean of both one-sided values
        if (xa == T(0)) {
            T g2, b2;
            one(L, T(0.5), gb, bb);
            one(R, T(-0.5), g2, b2);
            gb = T(0.5) * (gb + g2);
            bb = T(0.5) * (bb + b2);
        }
    }
}

template <typename T, int D, int TX, int TY, int TZ, bool SWEEP_B>
__global__ void __launch_bounds__(NTHREADS) k_sweep(Geo g, Bufs<T> bf) {
    using TL = Tile<D, TX, TY, TZ>;
    using SM = SweepSmem<T, D, TX, TY, TZ>;
    constexpr int NM = TL::NM;
    extern __shared__ __align__(16) unsigned char smem[];
    T* P = reinterpret_cast<T*>(smem + SM::off_P);
    CellC<T>* cc = reinterpret_cast<CellC<T>*>(smem + SM::off_cc);
    long long* csrc = reinterpret_cast<long long*>(smem + SM::off_src);
    int* cfl = reinterpret_cast<int*>(smem + SM::off_fl);
    FaceC<T>* fc = reinterpret_cast<FaceC<T>*>(smem + SM::off_fc);
    Acc<T>* acc = reinterpret_cast<Acc<T>*>(smem + SM::off_acc);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int tb = blockIdx.x;
    int org[3] = {0, 0, 0};
    org[0] = (tb % g.tiles[0]) * TL::T0;
    tb /= g.tiles[0];
    if (D >= 2) { org[1] = (tb % g.tiles[1]) * TL::T1; tb /= g.tiles[1]; }
    if (D >= 3) { org[2] = tb * TL::T2; }
    const int grp = blockIdx.y;
    const int vt0 = grp * g.ntpg, vt1 = min(g.NVT, vt0 + g.ntpg);

    // ---- prologue: box cells (BC mapping, cell constants), face constants, accumulators
    for (int k = tid; k < TL::BOX; k += NTHREADS) {
        int l[3] = {k % TL::E0 - 2, D >= 2 ? (k / TL::E0) % TL::E1 - 2 : 0, D >= 3 ? k / (TL::E0 * TL::E1) - 2 : 0};
        int q[3] = {org[0] + l[0], org[1] + l[1], org[2] + l[2]};
        int refl;
        bool dir;
        resolve(g, q, refl, dir);
        const long long c = cell_index(g, q);
        CellC<T> cst = dir ? bf.cellc0[c] : bf.cellc[c];
        for (int a = 0; a < D; ++a)
            if (refl & (1 << a)) cst.u[a] = -cst.u[a];
        cc[k] = cst;
        csrc[k] = c;
        cfl[k] = refl | (dir ? 8 : 0);
    }
    for (int k = tid; k < TL::NFT * NM; k += NTHREADS) acc[k].zero();
    if (SWEEP_B) {
        for (int f = tid; f < TL::NFT; f += NTHREADS) {
            int a = f < TL::NF0 ? 0 : (f < TL::NF0 + TL::NF1 ? 1 : 2);
            int r = f - TL::foff(a);
            const int d0 = TL::T0 + (a == 0), d1 = TL::T1 + (a == 1);
            int q[3] = {org[0] + r % d0, org[1] + (D >= 2 ? (r / d0) % d1 : 0), org[2] + (D >= 3 ? r / (d0 * d1) : 0)};
            bool ok = true;
            for (int b = 0; b < D; ++b) ok = ok && q[b] <= g.n[b] - (b == a ? 0 : 1);
            if (ok) fc[f] = bf.facec[a][face_index(g, a, q)];
        }
    }
    __syncthreads();

    for (int vt = vt0; vt < vt1; ++vt) {
        const int i = vt * VI + lane;
        const Vel<T, D> v = load_vel<T, D>(g, bf, i);

        // ---- phase 1: phibar+ on the box (eq. phibarplus) from the finalised phi
        for (int k = warp; k < TL::BOX; k += NWARPS) {
            const CellC<T>& c = cc[k];
            const int fl = cfl[k];
            T ge, be;
            equilibrium<T, D>(c, v, ge, be);
            T pg, pb;
            if (fl & 8) {
                pg = ge;
                pb = be;
            } else {
                const int is = (fl & 7) ? bf.refl[(fl & 7) * g.Nvp + i] : i;
                const size_t ad = phi_addr<T>(g, csrc[k], is, 0);
                const T sg = bf.phi_in[ad], sb = bf.phi_in[ad + VI];
                const T gg = fma(c.fa_g, sg, c.fb_g * ge);
                const T bb = fma(c.fa_b, sb, c.fb_b * be);
                const T dg = gg - ge;
                pg = fma(c.sa_g, dg, ge);
                pb = fma(c.ssrc * zeta<T, D>(c, v), dg, fma(c.sa_b, bb - be, be));
            }
            P[(size_t)k * 2 * VI + lane] = pg;
            P[(size_t)k * 2 * VI + VI + lane] = pb;
        }
        __syncthreads();

        // ---- phase 2: owned cells
        for (int o = warp; o < TL::OWN; o += NWARPS) {
            const int l0 = o % TL::T0, l1 = D >= 2 ? (o / TL::T0) % TL::T1 : 0, l2 = D >= 3 ? o / (TL::T0 * TL::T1) : 0;
            const int q0 = org[0] + l0, q1 = org[1] + l1, q2 = org[2] + l2;
            if (q0 >= g.n[0] || (D >= 2 && q1 >= g.n[1]) || (D >= 3 && q2 >= g.n[2])) continue;
            const int kc = TL::box_of(l0, l1, l2);
            const int qa[3] = {q0, q1, q2};
            const int la[3] = {l0, l1, l2};
            T dFg = T(0), dFb = T(0);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int s = TL::stride(a);
                const bool last = qa[a] == g.n[a] - 1;
#pragma unroll
                for (int side = 0; side < 2; ++side) {     // 0: left face of the cell, 1: right face
                    if (!SWEEP_B && side == 1 && !last) continue;
                    const int R = kc + side * s, L = R - s;
                    T gb, bb;
                    reconstruct<T, D, TL>(P, L, R, a, v, lane, gb, bb);
                    int lf[3] = {la[0], la[1], la[2]};
                    lf[a] += side;
                    const int fl = TL::face_local(a, lf[0], lf[1], lf[2]);
                    const bool own = side == 0 || last;
                    T mom[NM];
                    if (!SWEEP_B) {
                        // face conserved variables (eqs. rhobar-rhoEbar with a = 0)
                        const T wg = v.w * gb;
                        mom[0] = wg;
#pragma unroll
                        for (int b = 0; b < D; ++b) mom[1 + b] = v.xi[b] * wg;
                        mom[1 + D] = v.w * bb;
                    } else {
                        // face equilibrium and inversion of eq. phibar, then the microflux
                        const FaceC<T>& f = fc[fl];
                        T ge, be;
                        equilibrium<T, D>(f, v, ge, be);
                        const T gf = fma(f.al_g, gb - ge, ge);
                        const T bf_ = fma(f.gam_b * zeta<T, D>(f, v), gf - ge, fma(f.al_b, bb - be, be));
                        const T Fg = v.xi[a] * gf, Fb = v.xi[a] * bf_;
                        const T idx = (T)g.idx[a];
                        if (side == 0) {
                            dFg = fma(-idx, Fg, dFg);
                            dFb = fma(-idx, Fb, dFb);
                        } else {
                            dFg = fma(idx, Fg, dFg);
                            dFb = fma(idx, Fb, dFb);
                        }
                        const T wg = v.w * Fg;
                        mom[0] = wg;
#pragma unroll
                        for (int b = 0; b < D; ++b) mom[1 + b] = v.xi[b] * wg;
                        mom[1 + D] = v.w * Fb;
                    }
                    if (own) {
                        const T r = WarpSum<T, NM>::run(mom, lane);
                        const int m = WarpSum<T, NM>::moment_of_lane(lane);
                        if (WarpSum<T, NM>::writer(lane) && m < NM) acc[fl * NM + m].add(r);
                    }
                }
            }
            if (SWEEP_B) {
                // distribution update (eq. phiupdate) up to its last factor:
                // phi* = phi_eq + (1 - dt/2tau)(phi - phi_eq) + dt S - dt dF
                const CellC<T>& c = cc[kc];
                T ge, be;
                equilibrium<T, D>(c, v, ge, be);
                const long long cell = csrc[kc];
                const size_t ad = phi_addr<T>(g, cell, i, 0);
                const T sg = bf.phi_in[ad], sb = bf.phi_in[ad + VI];
                const T gg = fma(c.fa_g, sg, c.fb_g * ge);
                const T bb = fma(c.fa_b, sb, c.fb_b * be);
                const T dg = gg - ge;
                const T dt = (T)g.dt;
                const T ng = fma(-dt, dFg, fma(c.um_g, dg, ge));
                const T nb = fma(-dt, dFb, fma(c.usrc * zeta<T, D>(c, v), dg, fma(c.um_b, bb - be, be)));
                bf.phi_out[ad] = ng;
                bf.phi_out[ad + VI] = nb;
            }
        }
        __syncthreads();
    }

    // ---- epilogue: write this group's partial face sums
    double* const* dst = SWEEP_B ? bf.mf : bf.wf;
    for (int k = tid; k < TL::NFT * NM; k += NTHREADS) {
        const int f = k / NM, m = k % NM;
        int a = f < TL::NF0 ? 0 : (f < TL::NF0 + TL::NF1 ? 1 : 2);
        if (a >= D) continue;
        int r = f - TL::foff(a);
        const int d0 = TL::T0 + (a == 0), d1 = TL::T1 + (a == 1);
        int l[3] = {r % d0, D >= 2 ? (r / d0) % d1 : 0, D >= 3 ? r / (d0 * d1) : 0};
        int q[3] = {org[0] + l[0], org[1] + l[1], org[2] + l[2]};
        bool own = true;
        for (int b = 0; b < D; ++b) {
            if (b == a) own = own && q[b] <= g.n[b] && (l[b] < TL::tdim(b) || q[b] == g.n[b]);
            else own = own && q[b] < g.n[b];
        }
        if (!own) continue;
        dst[a][((size_t)grp * NM + m) * g.nf[a] + face_index(g, a, q)] = acc[k].value();
    }
}

// Face constants from the group-summed face W (fixed summation order).
template <typename T, int D>
__global__ void k_facec(Geo g, Bufs<T> bf, int a) {
    constexpr int NM = 2 + D;
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.nf[a]) return;
    double W[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < NM; ++m) {
        double s = 0.0;
        for (int gg = 0; gg < g.G; ++gg) s += bf.wf[a][((size_t)gg * NM + m) * g.nf[a] + f];
        W[m] = s;
    }
    make_face<T>(g, W, bf.facec[a][f]);
}

// W^{n+1} = W^n - dt sum_a (M_a(right face) - M_a(left face)) / dx_a (outward
// normals), the status check, and the cell constants of W^{n+1}.
template <typename T, int D>
__global__ void k_wupdate(Geo g, Bufs<T> bf) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Nc) return;
    constexpr int NM = 2 + D;
    int q[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((long long)g.n[0] * g.n[1]))};
    double dW[NM];
    for (int m = 0; m < NM; ++m) dW[m] = 0.0;
    for (int a = 0; a < D; ++a) {
        const long long fl = face_index(g, a, q);
        int qr[3] = {q[0], q[1], q[2]};
        qr[a] += 1;
        const long long fr = face_index(g, a, qr);
        for (int m = 0; m < NM; ++m) {
            double sr = 0.0, sl = 0.0;
            for (int gg = 0; gg < g.G; ++gg) {
                sr += bf.mf[a][((size_t)gg * NM + m) * g.nf[a] + fr];
                sl += bf.mf[a][((size_t)gg * NM + m) * g.nf[a] + fl];
            }
            dW[m] += (sr - sl) * g.idx[a];
        }
    }
    double W[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    bool finite = true;
    for (int m = 0; m < NM; ++m) {
        W[m] = bf.W[(size_t)m * g.Nc + c] - g.dt * dW[m];
        finite = finite && isfinite(W[m]);
        bf.W[(size_t)m * g.Nc + c] = W[m];
    }
    double u2 = 0.0;
    for (int a = 0; a < D; ++a) u2 += (W[1 + a] / W[0]) * (W[1 + a] / W[0]);
    const double e = W[1 + D] / W[0] - 0.5 * u2;
    int st = 0;
    if (!finite) st |= ST_NONFINITE;
    else if (!(W[0] > 0.0) || !(e > 0.0)) st |= ST_NEGATIVE;
    if (st) atomicOr(bf.status, st);
    make_cell<T>(g, W, bf.cellc[c]);
}

// Cell constants from the stored W (after a state restore).
template <typename T, int D>
__global__ void k_cellc(Geo g, Bufs<T> bf) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.Nc) return;
    double W[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < 2 + D; ++m) W[m] = bf.W[(size_t)m * g.Nc + c];
    make_cell<T>(g, W, bf.cellc[c]);
}

// Maxwell-Boltzmann initial state: W^0 from (rho, u, T), its constants (also
// kept as the Dirichlet ghost constants), phi* = phi_eq(W^0) (the stored
// pre-update value whose finalisation gives phi^0 = phi_eq).
template <typename T, int D>
__global__ void k_init(Geo g, Bufs<T> bf, const double* __restrict__ fields) {
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
    CellC<T> cc;
    make_cell<T>(g, Wc, cc);
    if (threadIdx.x == 0) {
        bf.cellc[c] = cc;
        bf.cellc0[c] = cc;
    }
    for (int i = threadIdx.x; i < g.Nvp; i += blockDim.x) {
        const Vel<T, D> v = load_vel<T, D>(g, bf, i);
        T ge, be;
        equilibrium<T, D>(cc, v, ge, be);
        const size_t ad = phi_addr<T>(g, c, i, 0);
        bf.phi_out[ad] = ge;
        bf.phi_out[ad + VI] = be;
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

// The finalised distributions phi = fa phi* + fb phi_eq at the current time
// level, written in the state layout into the idle buffer.
template <typename T, int D>
__global__ void k_finalise(Geo g, Bufs<T> bf) {
    const long long c = blockIdx.x;
    const CellC<T> cc = bf.cellc[c];
    for (int i = threadIdx.x; i < g.Nvp; i += blockDim.x) {
        const Vel<T, D> v = load_vel<T, D>(g, bf, i);
        T ge, be;
        equilibrium<T, D>(cc, v, ge, be);
        const size_t ad = phi_addr<T>(g, c, i, 0);
        bf.phi_out[ad] = fma(cc.fa_g, bf.phi_in[ad], cc.fb_g * ge);
        bf.phi_out[ad + VI] = fma(cc.fa_b, bf.phi_in[ad + VI], cc.fb_b * be);
    }
}

}  // namespace cdg
