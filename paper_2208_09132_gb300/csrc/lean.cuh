// lean.cuh -- the "lean" face-store shapes of the CDUGKS step (arXiv:2208.09132,
// Sec. 2.1) for D = 2 and 3.
//
// They compute the same scheme as the fused face-store shapes (two relaxation
// times, upwind-cell reconstruction; the velocity grid has no node at xi_a = 0)
// with three differences in how:
//
//  * The equilibria (eqs. geq, beq) are products of separable factors: the
//    Maxwellian of a place is rho (2 pi RT)^{-D/2} prod_b exp(-(xi_b - u_b)^2 / 2RT),
//    and the per-axis factors of every cell and face are formed in double by the
//    FP64 kernels (write_factors: W update, face constants, init) into tables.
//    A point's g_eq is then D - 1 multiplications of table entries -- no
//    exponential per point, and the exponent is exact to double rounding at any
//    Mach number.
//  * Sweep A forms phibar+ only on the cells that some face's reconstruction
//    reads (the upwind cells U of the tile's faces and their axis neighbours),
//    and each upwind cell reconstructs the values of the faces it is upwind of
//    (one limited slope vector per cell, each face value formed once) into
//    shared memory; the owners of the faces then sum the face moments.
//  * Sweep B (k_lflux) reads the stored face values of both faces of its cell
//    along every axis and takes their equilibria from the face factor tables;
//    no barrier in its chunk loop (a shared face is formed by both cells).
#pragma once

#include "kernels.cuh"

namespace cdg {

// Shared memory of lean sweep A.  Box layout (Tile, two halo layers) for
// phibar+; the region cells (R_max of them at most, in box order) carry their
// constants, source cell and flags; FV holds the reconstructed values of the
// tile's faces (Tile face layout); RS the Kahan sums of the domain-end faces.
template <typename T, int D, int T0_, int T1_, int T2_>
struct LeanA {
    using TL = Tile<D, T0_, T1_, T2_, 2>;
    static constexpr int BOX = TL::BOX, NT = TL::NT, NFT = TL::NFT;
    // upwind cells: owned, one layer below each axis, one layer at the domain end of each axis
    static constexpr int UMAX = NT + 2 * TL::NPL;
    // region: U and its axis neighbours (two layers beyond U per axis, and the edges)
    static constexpr int EDGES = D == 2 ? 4 : 4 * (TL::T0 + TL::T1 + TL::T2);
    static constexpr int RMAX_ = NT + 4 * TL::NPL + EDGES;
    static constexpr int RMAX = RMAX_ < BOX ? RMAX_ : BOX;
    static constexpr size_t nP = (size_t)2 * BOX;      // V4
    static constexpr size_t nCC = (size_t)2 * RMAX;    // V4: u0 u1 u2 hu2 | eb kp_g kp_b kp_s
    static constexpr size_t nFV = (size_t)2 * NFT;     // V4
    static constexpr size_t v4bytes = (nP + nCC + nFV) * sizeof(V4<T>);
    static constexpr size_t rs_bytes = (size_t)TL::NPL * (2 + D) * sizeof(Kahan<T>);
    // region slot: source cell (int), box index (u16), flags (u8), prefetch run length (u8);
    // U slot: box index | kind << 12 (u16), the FV slots of its faces per axis
    // (side -, side +; 0xffff none); 32 ints of scratch
    static constexpr size_t off_rbox = (size_t)RMAX * 4;
    static constexpr size_t off_ulist = off_rbox + (size_t)RMAX * 2;
    static constexpr size_t off_ufs = off_ulist + (size_t)UMAX * 2;
    static constexpr size_t off_rfl = off_ufs + (size_t)UMAX * 2 * D * 2;
    static constexpr size_t off_rrun = off_rfl + (size_t)RMAX;
    static constexpr size_t off_wcnt = (off_rrun + (size_t)RMAX + 3) / 4 * 4;
    static constexpr size_t int_bytes = off_wcnt + 32 * 4;
    static constexpr size_t bytes = v4bytes + rs_bytes + (int_bytes + 15) / 16 * 16;
    static_assert(BOX < 4096, "box index in 12 bits");
};

template <typename T, int D, int T0_, int T1_, int T2_>
struct LeanAOcc {
    static constexpr size_t per = LeanA<T, D, T0_, T1_, T2_>::bytes + 1024;
    static constexpr int by_smem = (int)((228 * 1024) / per);
    static constexpr int by_threads = 2048 / Tile<D, T0_, T1_, T2_>::NT;
    // keep >= 80 registers (FP32) or >= 168 (FP64 values take two registers)
    static constexpr int by_regs = 65536 / (Tile<D, T0_, T1_, T2_>::NT * (sizeof(T) == 8 ? 168 : 80));
    static constexpr int v1 = by_smem < by_threads ? by_smem : by_threads;
    static constexpr int v0 = v1 < by_regs ? v1 : by_regs;
    static constexpr int value = v0 < 1 ? 1 : (v0 > 4 ? 4 : v0);
};

// In-order compaction of the box cells k in [0, n) that satisfy pred(k) into
// list[], in box order (every thread of the CTA calls it; cnt: [32] scratch).
template <int NT, typename L, typename F>
__device__ __forceinline__ int compact_box(int n, L* list, int* cnt, F&& pred, unsigned tag_of_k_shift = 0) {
    constexpr int NW = NT / 32;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = ((n + NW - 1) / NW + 31) / 32 * 32;
    const int k0 = warp * per, k1 = min(n, k0 + per);
    int c = 0;
    for (int kb = k0; kb < k1; kb += 32) {
        const int k = kb + lane;
        c += __popc(__ballot_sync(0xffffffffu, k < k1 && pred(k) >= 0));
    }
    if (lane == 0) cnt[warp] = c;
    __syncthreads();
    int base = 0, total = 0;
    for (int w = 0; w < NW; ++w) {
        base += w < warp ? cnt[w] : 0;
        total += cnt[w];
    }
    for (int kb = k0; kb < k1; kb += 32) {
        const int k = kb + lane;
        const int v = k < k1 ? pred(k) : -1;
        const unsigned m = __ballot_sync(0xffffffffu, v >= 0);
        if (v >= 0) list[base + __popc(m & ((1u << lane) - 1u))] = (L)(k | (v << tag_of_k_shift));
        base += __popc(m);
    }
    __syncthreads();
    return total;
}

// Factor-table rows of the current chunk (aligned velocity grids: nv1_0 a
// multiple of VC, so a chunk's four velocities share k1, k2): the first row of
// its axis-0 block and its rows of axes 1 and 2, direct and with the axis
// mirrored (k -> n - 1 - k).  Advanced chunk by chunk without divisions.
struct LeanRows {
    int c0, k1, k2;               // chunk index along axis 0 (of nv1_0 / VC), k1, k2
    int r0, r1, r2, r0m, r1m, r2m;
};
__device__ __forceinline__ void lean_rows_set(const Geo& g, LeanRows& R) {
    const int n0c = g.nv1[0] / VC;
    R.r0 = R.c0 * VC;
    R.r0m = (n0c - 1 - R.c0) * VC;
    R.r1 = g.xrow[1] + R.k1;
    R.r1m = g.xrow[1] + g.nv1[1] - 1 - R.k1;
    R.r2 = g.xrow[2] + R.k2;
    R.r2m = g.xrow[2] + g.nv1[2] - 1 - R.k2;
}
// The lean kernels visit the chunks of a group in the order j = vt0 .. vt1 - 1
// of a numbering in which the axis-0 chunk index c0 varies slowest (aligned
// grids): chunk j is vt = c0 + (nv1_0 / VC) (k1 + nv1_1 k2) with c0 = j / (nv1_1 nv1_2)
// and k1 + nv1_1 k2 = j mod (nv1_1 nv1_2).  A place's four axis-0 factors then
// stay the same over long runs of chunks (cache hits) and only the scalar
// factor of axis 1 changes from chunk to chunk.  Any split of the chunks into
// groups gives the same scheme (the groups' sums are added in a fixed order).
__device__ __forceinline__ int lean_vt(const Geo& g, const LeanRows& R) {
    return R.c0 + (g.nv1[0] / VC) * (R.k1 + g.nv1[1] * R.k2);
}
__device__ __forceinline__ LeanRows lean_rows(const Geo& g, int j) {
    LeanRows R;
    const int m = g.nv1[1] * g.nv1[2];
    R.c0 = j / m;
    R.k1 = (j % m) % g.nv1[1];
    R.k2 = (j % m) / g.nv1[1];
    lean_rows_set(g, R);
    return R;
}
__device__ __forceinline__ void lean_rows_next(const Geo& g, LeanRows& R) {
    if (++R.k1 == g.nv1[1]) {
        R.k1 = 0;
        if (++R.k2 == g.nv1[2]) {
            R.k2 = 0;
            ++R.c0;
        }
    }
    lean_rows_set(g, R);
}
__device__ __forceinline__ int lean_vt_next(const Geo& g, LeanRows R) {
    lean_rows_next(g, R);
    return lean_vt(g, R);
}

// g_eq of the four lanes of chunk vt at table place `item` (n places), with the
// velocity components of the mirror axes (bits of refl) reflected.  Aligned
// grids: one vector and one or two scalar loads (rows of R); otherwise each
// lane's indices are found from its velocity number.
template <typename T, int D>
__device__ __forceinline__ void lean_geq4(const Geo& g, const T* __restrict__ X, long long n, long long item,
                                          int refl, int vt, const LeanRows& R, T (&ge)[VC]) {
    const size_t nn = (size_t)n, it = (size_t)item;
    if (g.xal) {
        const int r0 = (refl & 1) ? R.r0m : R.r0;
        const int r1 = (refl & 2) ? R.r1m : R.r1;
        T x0[VC];
        Chunk<T>::load(X + (size_t)r0 * nn + VC * it, x0);      // = xaddr(g, n, r0, item), r0 a multiple of VC
        const T x1 = __ldg(X + (size_t)r1 * nn + it);
        T x2 = T(1);
        if (D == 3) x2 = __ldg(X + (size_t)((refl & 4) ? R.r2m : R.r2) * nn + it);
        const T pr = lean_pair<T, D>(x1, x2);
#pragma unroll
        for (int v = 0; v < VC; ++v) ge[v] = ((refl & 1) ? x0[VC - 1 - v] : x0[v]) * pr;
    } else {
        const int nv = g.nv1[0] * g.nv1[1] * g.nv1[2];
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            const int i = vt * VC + v;
            ge[v] = T(0);
            if (i < nv) {
                int k0 = i % g.nv1[0], k1 = (i / g.nv1[0]) % g.nv1[1], k2 = i / (g.nv1[0] * g.nv1[1]);
                if (refl & 1) k0 = g.nv1[0] - 1 - k0;
                if (refl & 2) k1 = g.nv1[1] - 1 - k1;
                if (refl & 4) k2 = g.nv1[2] - 1 - k2;
                const T x2 = D == 3 ? __ldg(X + xaddr(g, n, g.xrow[2] + k2, item)) : T(1);
                ge[v] = lean_geq<T, D>(__ldg(X + xaddr(g, n, k0, item)), __ldg(X + xaddr(g, n, g.xrow[1] + k1, item)),
                                       x2);
            }
        }
    }
}

// ---------------------------------------------------------------- sweep A
template <typename T, int D, int T0_, int T1_, int T2_, bool NOSRC>
__device__ __forceinline__ void lean_a_body(const Geo& g, const Bufs<T>& bf, int tile, int grp, unsigned char* smem) {
    using LA = LeanA<T, D, T0_, T1_, T2_>;
    using TL = typename LA::TL;
    using Q = V4<T>;
    constexpr int NM = 2 + D, BOX = TL::BOX, NT = TL::NT, NFT = TL::NFT, RMAX = LA::RMAX;
    constexpr unsigned short NONE = 0xffffu;
    static_assert(NT % 32 == 0, "whole warps");
    Q* const P = reinterpret_cast<Q*>(smem);                // [2][BOX]
    Q* const CC = P + LA::nP;                              // [2][RMAX]
    Q* const FV = CC + LA::nCC;                            // [2][NFT]
    Kahan<T>* const RS = reinterpret_cast<Kahan<T>*>(smem + LA::v4bytes);
    unsigned char* ip = smem + LA::v4bytes + LA::rs_bytes;
    int* const rsrc = reinterpret_cast<int*>(ip);                                    // [RMAX]
    unsigned short* const rbox = reinterpret_cast<unsigned short*>(ip + LA::off_rbox);    // [RMAX]
    unsigned short* const ulist = reinterpret_cast<unsigned short*>(ip + LA::off_ulist);  // [UMAX]
    unsigned short* const ufs = reinterpret_cast<unsigned short*>(ip + LA::off_ufs);      // [UMAX][2D]
    unsigned char* const rfl = ip + LA::off_rfl;                                     // [RMAX]
    unsigned char* const rrun = ip + LA::off_rrun;                                   // [RMAX]
    int* const wcnt = reinterpret_cast<int*>(ip + LA::off_wcnt);                     // [32]

    const int t = threadIdx.x;
    int org[3];
    tile_origin<TL, D>(g, tile, org);
    const int vt0 = grp * g.ntpg, vt1 = min(g.NVT, vt0 + g.ntpg);
    const int la[3] = {t % TL::T0, D >= 2 ? (t / TL::T0) % TL::T1 : 0, D >= 3 ? t / (TL::T0 * TL::T1) : 0};
    const int qa[3] = {org[0] + la[0], org[1] + la[1], org[2] + la[2]};
    bool valid = true;
#pragma unroll
    for (int a = 0; a < D; ++a) valid = valid && qa[a] < g.n[a];
    int ext[3];     // local coordinate of the domain end along each axis (> T_a: beyond the tile)
#pragma unroll
    for (int a = 0; a < 3; ++a) ext[a] = a < D ? g.n[a] - org[a] : 1;

    auto box_local = [&](int k, int l[3]) {
        l[0] = k % TL::E0 - 2;
        l[1] = D >= 2 ? (k / TL::E0) % TL::E1 - 2 : 0;
        l[2] = D >= 3 ? k / (TL::E0 * TL::E1) - 2 : 0;
    };
    // kind of an upwind cell at local l: 0 owned, 1 + a layer below axis a, 4 + a
    // the ghost beyond the domain end of axis a; -1 none
    auto ukind = [&](const int (&l)[3]) {
        int out = -1, nout = 0;
        bool ok = true;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const int tb = TL::tdim(b) < ext[b] ? TL::tdim(b) : ext[b];     // owned extent along b
            if (l[b] >= 0 && l[b] < tb) continue;
            ++nout;
            if (l[b] == -1) out = 1 + b;
            else if (l[b] == ext[b] && ext[b] <= TL::tdim(b)) out = 4 + b;
            else ok = false;
        }
        if (!ok || nout > 1) return -1;
        return nout == 0 ? 0 : out;
    };
    auto region = [&](int k) {
        int l[3];
        box_local(k, l);
        if (ukind(l) >= 0) return 0;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            int m[3] = {l[0], l[1], l[2]};
            m[b] = l[b] - 1;
            if (ukind(m) >= 0) return 0;
            m[b] = l[b] + 1;
            if (ukind(m) >= 0) return 0;
        }
        return -1;
    };
    auto upred = [&](int k) {
        int l[3];
        box_local(k, l);
        return ukind(l);
    };
    // ---- prologue: region list (box order) with source cells, flags, constants and
    // prefetch runs; U list with the FV slots of the faces each upwind cell forms
    const int NR = compact_box<NT>(BOX, rbox, wcnt, region);
    const int NU = compact_box<NT>(BOX, ulist, wcnt, upred, 12);
    for (int r = t; r < NR; r += NT) {
        const int k = rbox[r];
        int l[3];
        box_local(k, l);
        int q[3] = {org[0] + l[0], org[1] + l[1], org[2] + l[2]};
        int refl;
        bool dir;
        resolve<D>(g, q, refl, dir);
        const long long c = cell_index(g, q);
        rsrc[r] = (int)c;
        rfl[r] = (unsigned char)(refl | (dir ? 8 : 0));
        const CellC<T>& cs = dir ? bf.cellc0[c] : bf.cellc[c];
        Q c0, c1;
#pragma unroll
        for (int a = 0; a < 3; ++a) c0.v[a] = a < D ? ((refl & (1 << a)) ? -cs.u[a] : cs.u[a]) : T(0);
        c0.v[3] = cs.hu2;
        c1.v[0] = cs.eb;
        c1.v[1] = cs.kp_g;
        c1.v[2] = cs.kp_b;
        c1.v[3] = cs.kp_s;
        CC[r] = c0;
        CC[RMAX + r] = c1;
    }
    for (int u = t; u < NU; u += NT) {
        const int e = ulist[u];
        const int k = e & 0xfff, kind = e >> 12;
        int l[3];
        box_local(k, l);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            unsigned short fneg = NONE, fpos = NONE;
            int lf[3] = {l[0], l[1], l[2]};
            if (kind == 0) {
                fneg = (unsigned short)TL::face_local(a, lf[0], lf[1], lf[2]);          // its left face
                if (l[a] + 1 < TL::tdim(a) || l[a] + 1 == ext[a]) {                     // its right face, if owned
                    lf[a] += 1;
                    fpos = (unsigned short)TL::face_local(a, lf[0], lf[1], lf[2]);
                }
            } else if (kind == 1 + a) {                                              // below the tile
                lf[a] += 1;
                fpos = (unsigned short)TL::face_local(a, lf[0], lf[1], lf[2]);
            } else if (kind == 4 + a) {                                              // beyond the domain end
                fneg = (unsigned short)TL::face_local(a, lf[0], lf[1], lf[2]);
            }
            ufs[u * 2 * D + 2 * a] = fneg;
            ufs[u * 2 * D + 2 * a + 1] = fpos;
        }
    }
    __syncthreads();
    // prefetch runs: a region slot that starts a run of slots whose source cells
    // are consecutive plain cells (no mirror, no Dirichlet ghost) records the run length
    for (int r = t; r < NR; r += NT) {
        int len = 0;
        const bool start = rfl[r] == 0 && (r == 0 || rfl[r - 1] != 0 || rsrc[r - 1] + 1 != rsrc[r]);
        if (start) {
            len = 1;
            while (r + len < NR && len < 255 && rfl[r + len] == 0 && rsrc[r + len] == rsrc[r] + len) ++len;
        }
        rrun[r] = (unsigned char)len;
    }
    // this thread's faces: left faces, and the domain's end where it is the last cell
    bool own_right[3] = {false, false, false};
    int fl_left[3] = {0, 0, 0}, fl_end[3] = {0, 0, 0};      // FV slots
    long long gf_left[3] = {0, 0, 0}, gf_end[3] = {0, 0, 0};  // global face numbers
#pragma unroll
    for (int a = 0; a < D; ++a) {
        own_right[a] = valid && qa[a] == g.n[a] - 1;
        int lf[3] = {la[0], la[1], la[2]};
        fl_left[a] = TL::face_local(a, lf[0], lf[1], lf[2]);
        gf_left[a] = valid ? face_index(g, a, qa) : 0;
        lf[a] += 1;
        fl_end[a] = TL::face_local(a, lf[0], lf[1], lf[2]);
        int qf[3] = {qa[0], qa[1], qa[2]};
        qf[a] += 1;
        gf_end[a] = own_right[a] ? face_index(g, a, qf) : 0;
    }
    Kahan<T> acc[D][NM];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[a][m].zero();
    int pl[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) pl[a] = TL::poff(a) * NM + TL::plane_pos(a, la);
    for (int k = t; k < TL::NPL * NM; k += NT) RS[k].zero();
    __syncthreads();

    LeanRows R = lean_rows(g, g.xal ? vt0 : 0);
    const size_t chunk_stride = (size_t)g.Nc * (2 * VC);
    for (int j = vt0; j < vt1; ++j) {
        const int vt = g.xal ? lean_vt(g, R) : j;                 // chunk j of the visiting order
        const int vtn = j + 1 < vt1 ? (g.xal ? lean_vt_next(g, R) : j + 1) : -1;   // the next one (prefetch)
        // velocity records of the chunk (the same for every thread): xi, w, |xi|^2/2, nu = 2 h xi / dx
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
        // lanes whose velocity points along +axis (the rest, padding included, count as -)
        unsigned pos[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            pos[a] = 0;
#pragma unroll
            for (int v = 0; v < VC; ++v) pos[a] |= (xi[v][a] > T(0) ? 1u : 0u) << v;
        }
        const T* const phic = bf.phi_in + (size_t)vt * chunk_stride;

        // ---- phase 1: phibar+ on the region (eq. phibarplus), separable equilibrium
        for (int r = t; r < NR; r += NT) {
            const int k = rbox[r], fl = rfl[r];
            const int c = rsrc[r];
            const int run = rrun[r];
            if (run && vtn >= 0)               // L2 hint: this run's cells of the next chunk
                prefetch_l2(bf.phi_in + (size_t)vtn * chunk_stride + (size_t)c * (2 * VC),
                            run * 2 * VC * (int)sizeof(T));
            const Q c1 = CC[RMAX + r];
            T ge[VC], be[VC];
            lean_geq4<T, D>(g, (fl & 8) ? bf.xc0 : bf.xc, g.Nc, c, fl & 7, vt, R, ge);
#pragma unroll
            for (int v = 0; v < VC; ++v) be[v] = (hx[v] + c1.v[0]) * ge[v];
            Q pg, pb;
            if (fl & 8) {              // Dirichlet ghost: the equilibrium of its initial state
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    pg.v[v] = ge[v];
                    pb.v[v] = be[v];
                }
            } else {
                T gs[VC], bs[VC];
                if (fl & 7) {
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        const int is = bf.refl[(fl & 7) * g.Nvp + vt * VC + v];
                        gs[v] = bf.phi_in[phi_addr(g, c, is, 0)];
                        bs[v] = bf.phi_in[phi_addr(g, c, is, 1)];
                    }
                } else {
                    const T* src = phic + (size_t)c * (2 * VC);
                    Chunk<T>::load(src, gs);
                    Chunk<T>::load(src + VC, bs);
                }
                T z[VC];
                if constexpr (!NOSRC) {
                    const Q c0 = CC[r];
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        T zz = -c0.v[3];
#pragma unroll
                        for (int a = 0; a < D; ++a) zz = fma(xi[v][a], c0.v[a], zz);
                        z[v] = zz;
                    }
                }
#pragma unroll
                for (int v = 0; v < VC; ++v)
                    phibar_plus<T, NOSRC>(ge[v], be[v], gs[v], bs[v], NOSRC ? T(0) : z[v], c1.v[1], c1.v[2], c1.v[3],
                                          pg.v[v], pb.v[v]);
            }
            P[k] = pg;
            P[BOX + k] = pb;
        }
        __syncthreads();

        // ---- phase 2: per upwind cell, the limited slope vector and the values of
        //      the faces it is upwind of (eq. relation), into FV
        for (int u = t; u < NU; u += NT) {
            const int k = ulist[u] & 0xfff;
            T base[2][VC], hs[2][D][VC];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const Q c = P[f * BOX + k];
#pragma unroll
                for (int v = 0; v < VC; ++v) base[f][v] = c.v[v];
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    const int st = TL::bstride(b);
                    const Q lo = P[f * BOX + k - st], hi = P[f * BOX + k + st];
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        hs[f][b][v] = Num<T>::vanleer(c.v[v] - lo.v[v], hi.v[v] - c.v[v]);
                        base[f][v] = fma(-nu[v][b], hs[f][b][v], base[f][v]);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const unsigned lanes = side ? pos[a] : (~pos[a] & 0xFu);
                    const unsigned short fi = ufs[u * 2 * D + 2 * a + side];
                    if (!lanes || fi == NONE) continue;
                    const T one = side ? T(1) : T(-1);     // the face on the + or - side of the cell
                    Q vg, vb;
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        vg.v[v] = fma(one, hs[0][a][v], base[0][v]);
                        vb.v[v] = fma(one, hs[1][a][v], base[1][v]);
                    }
                    if (lanes == 0xFu) {
                        FV[fi] = vg;
                        FV[NFT + fi] = vb;
                    } else {
                        T* fg = reinterpret_cast<T*>(&FV[fi]);
                        T* fb = reinterpret_cast<T*>(&FV[NFT + fi]);
#pragma unroll
                        for (int v = 0; v < VC; ++v)
                            if (lanes & (1u << v)) {
                                fg[v] = vg.v[v];
                                fb[v] = vb.v[v];
                            }
                    }
                }
            }
        }
        __syncthreads();

        // ---- phase 3: the owned faces to the face store, and their moments (eqs. rhobar-rhoEbar)
        if (valid) {
#pragma unroll
            for (int a = 0; a < D; ++a) {
                T* const fbase = bf.face[a] + (size_t)vt * (size_t)g.nf[a] * (2 * VC);
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (side == 1 && !own_right[a]) continue;
                    const int fi = side ? fl_end[a] : fl_left[a];
                    const Q vg = FV[fi], vb = FV[NFT + fi];
                    T* const dst = fbase + (size_t)(side ? gf_end[a] : gf_left[a]) * (2 * VC);
                    Chunk<T>::store(dst, vg.v);
                    Chunk<T>::store(dst + VC, vb.v);
                    T sm[NM];
#pragma unroll
                    for (int m = 0; m < NM; ++m) sm[m] = T(0);
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        const T wg = w[v] * vg.v[v];
                        sm[0] = Ar<T>::add(sm[0], wg);   // (explicitly rounded: the same bits in every kernel)
#pragma unroll
                        for (int b = 0; b < D; ++b) sm[1 + b] = fma(xi[v][b], wg, sm[1 + b]);
                        sm[1 + D] = fma(w[v], vb.v[v], sm[1 + D]);
                    }
                    if (side == 0) {
#pragma unroll
                        for (int m = 0; m < NM; ++m) acc[a][m].add(sm[m]);
                    } else {
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            Kahan<T> kk = RS[pl[a] + m * TL::plane(a)];
                            kk.add(sm[m]);
                            RS[pl[a] + m * TL::plane(a)] = kk;
                        }
                    }
                }
            }
        }
        if (g.xal) lean_rows_next(g, R);
        // (the next chunk's phase 1 writes P only; its barrier orders phase 2's FV
        // writes after every thread's phase 3 reads)
    }
    if (valid) write_face_sums<T, D, TL>(g, bf.wf, grp, qa, own_right, acc, RS, pl);
}

template <typename T, int D, int T0_, int T1_, int T2_, bool NOSRC>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (LeanAOcc<T, D, T0_, T1_, T2_>::value))
    k_lsweep(const Inst<T>* __restrict__ in, int cur) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    lean_a_body<T, D, T0_, T1_, T2_, NOSRC>(in->g, in->b[cur], blockIdx.x, blockIdx.y, smem);
}

template <typename T, int D, int T0_, int T1_, int T2_, bool NOSRC>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (LeanAOcc<T, D, T0_, T1_, T2_>::value))
    k_lsweep_batch(const Item* __restrict__ items, const Inst<T>* __restrict__ insts, const int* __restrict__ cur) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    const Item it = items[blockIdx.x];
    const Inst<T>& in = insts[it.inst];
    lean_a_body<T, D, T0_, T1_, T2_, NOSRC>(in.g, in.b[cur[it.inst] & 1], it.tile, it.grp, smem);
}

// ---------------------------------------------------------------- sweep B
//
// One CTA per (tile, velocity group), one thread per owned cell, no barrier in
// the chunk loop.  Per chunk each thread reads the stored values of both faces
// of its cell along every axis, forms their fluxes (face equilibrium from the
// face factor tables, the inverse of eq. phibar, xi_a phi: eq. flux) and phi*
// of its cell from the net flux (eq. phiupdate, its last factor deferred).  A
// face shared by two cells is formed by both from the same values with the same
// arithmetic; its moments are summed by its owner only (the cell on its right,
// the last cell for the domain's end).
template <typename T, int D, int T0_, int T1_, int T2_>
struct LeanB {
    using TL = Tile<D, T0_, T1_, T2_, 2>;
    static constexpr int NFT = TL::NFT, NT = TL::NT, NPL = TL::NPL;
    static constexpr size_t nFC = (size_t)2 * NFT;      // V4: u0 u1 u2 hu2 | eb al_g al_b gam_b
    static constexpr size_t bytes = nFC * sizeof(V4<T>) + (size_t)NPL * (2 + D) * sizeof(Kahan<T>);
};

template <typename T, int D, int T0_, int T1_, int T2_>
struct LeanBOcc {
    static constexpr size_t per = LeanB<T, D, T0_, T1_, T2_>::bytes + 1024;
    static constexpr int by_smem = (int)((228 * 1024) / per);
    static constexpr int by_threads = 2048 / Tile<D, T0_, T1_, T2_>::NT;
    // keep >= 128 registers (FP32) or >= 200 (FP64)
    static constexpr int by_regs = 65536 / (Tile<D, T0_, T1_, T2_>::NT * (sizeof(T) == 8 ? 200 : 128));
    static constexpr int v1 = by_smem < by_threads ? by_smem : by_threads;
    static constexpr int v0 = v1 < by_regs ? v1 : by_regs;
    static constexpr int value = v0 < 1 ? 1 : (v0 > 8 ? 8 : v0);
};

// The flux of one face and chunk from its stored value (src): face equilibrium
// (separable factors of the face), inverse of eq. phibar, xi_a phi; with
// MOM its moments (quadrature weights applied) are added to sm.
template <typename T, int D, bool NOSRC, bool MOM>
__device__ __forceinline__ void lean_face_flux(const Geo& g, const Bufs<T>& bf, int a, long long fidx, int vt,
                                               const LeanRows& R, const T* src, const V4<T>& fc0, const V4<T>& fc1,
                                               const T (&xi)[VC][D], const T (&w)[VC], const T (&hx)[VC],
                                               T (&Fg)[VC], T (&Fb)[VC], T* sm) {
    T gb[VC], bb[VC], ge[VC];
    Chunk<T>::load(src, gb);
    Chunk<T>::load(src + VC, bb);
    lean_geq4<T, D>(g, bf.xf[a], g.nf[a], fidx, 0, vt, R, ge);
    const T eb = fc1.v[0], alg = fc1.v[1], alb = fc1.v[2], gmb = fc1.v[3];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        const T be = (hx[v] + eb) * ge[v];
        const T gf = fma(alg, gb[v] - ge[v], ge[v]);
        T bfv = fma(alb, bb[v] - be, be);
        if constexpr (!NOSRC) {
            T z = -fc0.v[3];
#pragma unroll
            for (int b = 0; b < D; ++b) z = fma(xi[v][b], fc0.v[b], z);
            bfv = fma(gmb * z, gf - ge[v], bfv);
        }
        const T fg = xi[v][a] * gf, fb = xi[v][a] * bfv;
        Fg[v] = fg;
        Fb[v] = fb;
        if constexpr (MOM) {
            const T wg = w[v] * fg;
            sm[0] = Ar<T>::add(sm[0], wg);   // (explicitly rounded: the same bits in every kernel)
#pragma unroll
            for (int b = 0; b < D; ++b) sm[1 + b] = fma(xi[v][b], wg, sm[1 + b]);
            sm[1 + D] = fma(w[v], fb, sm[1 + D]);
        }
    }
}

template <typename T, int D, int T0_, int T1_, int T2_, bool NOSRC>
__device__ __forceinline__ void lean_b_body(const Geo& g, const Bufs<T>& bf, int tile, int grp, unsigned char* smem) {
    using LB = LeanB<T, D, T0_, T1_, T2_>;
    using TL = typename LB::TL;
    using Q = V4<T>;
    constexpr int NM = 2 + D, NFT = TL::NFT, NT = TL::NT;
    Q* const FC = reinterpret_cast<Q*>(smem);      // [2][NFT]
    Kahan<T>* const RS = reinterpret_cast<Kahan<T>*>(smem + LB::nFC * sizeof(Q));   // domain-end faces
    const int t = threadIdx.x;
    int org[3];
    tile_origin<TL, D>(g, tile, org);
    const int vt0 = grp * g.ntpg, vt1 = min(g.NVT, vt0 + g.ntpg);
    const int la[3] = {t % TL::T0, D >= 2 ? (t / TL::T0) % TL::T1 : 0, D >= 3 ? t / (TL::T0 * TL::T1) : 0};
    const int qa[3] = {org[0] + la[0], org[1] + la[1], org[2] + la[2]};
    bool valid = true;
#pragma unroll
    for (int a = 0; a < D; ++a) valid = valid && qa[a] < g.n[a];
    // ---- face constants of the tile's faces (those inside the domain)
    for (int fi = t; fi < NFT; fi += NT) {
        int a = 0;
#pragma unroll
        for (int b = 1; b < D; ++b) a += fi >= TL::foff(b) ? 1 : 0;
        const int r = fi - TL::foff(a);
        const int d0 = TL::T0 + (a == 0), d1 = TL::T1 + (a == 1);
        int q[3] = {org[0] + r % d0, org[1] + (D >= 2 ? (r / d0) % d1 : 0), org[2] + (D >= 3 ? r / (d0 * d1) : 0)};
        bool ok = true;
#pragma unroll
        for (int b = 0; b < D; ++b) ok = ok && q[b] <= g.n[b] - (b == a ? 0 : 1);
        if (!ok) continue;
        const FaceC<T>& fs = bf.facec[a][face_index(g, a, q)];
        Q c0, c1;
#pragma unroll
        for (int b = 0; b < 3; ++b) c0.v[b] = b < D ? fs.u[b] : T(0);
        c0.v[3] = fs.hu2;
        c1.v[0] = fs.eb;
        c1.v[1] = fs.al_g;
        c1.v[2] = fs.al_b;
        c1.v[3] = fs.gam_b;
        FC[fi] = c0;
        FC[NFT + fi] = c1;
    }
    for (int k = t; k < TL::NPL * NM; k += NT) RS[k].zero();
    __syncthreads();
    if (!valid) return;          // no barrier below

    const CellC<T> own = bf.cellc[cell_index(g, qa)];
    const int cidx = (int)cell_index(g, qa);
    const size_t chunk_stride = (size_t)g.Nc * (2 * VC);
    const T dtT = (T)g.dt;                           // converted once (conversions from double use the FP64 pipe)
    T idxT[D];
#pragma unroll
    for (int a = 0; a < D; ++a) idxT[a] = (T)g.idx[a];
    bool own_right[3] = {false, false, false};
    int ff[3] = {0, 0, 0}, fs_[3] = {0, 0, 0};     // left face number, stride to the right face
    int fl[3][2];                                   // local face slots (FC) of both faces
    size_t fstride[3] = {0, 0, 0};                  // elements per chunk of each axis' face array
#pragma unroll
    for (int a = 0; a < D; ++a) {
        own_right[a] = qa[a] == g.n[a] - 1;
        ff[a] = (int)face_index(g, a, qa);
        fs_[a] = a == 0 ? 1 : (a == 1 ? g.fn[1][0] : g.fn[2][0] * g.fn[2][1]);
        fl[a][0] = TL::face_local(a, la[0], la[1], la[2]);
        fl[a][1] = TL::face_local(a, la[0] + (a == 0), la[1] + (a == 1), la[2] + (a == 2));
        fstride[a] = (size_t)g.nf[a] * (2 * VC);
    }
    Kahan<T> acc[D][NM];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[a][m].zero();
    const bool row_lead = la[0] == 0;
    const int nrow = min(TL::T0, g.n[0] - org[0]);
    constexpr int RB = 2 * VC * (int)sizeof(T);
    const int tdim[3] = {TL::T0, TL::T1, TL::T2};

    LeanRows R = lean_rows(g, g.xal ? vt0 : 0);
    for (int j = vt0; j < vt1; ++j) {
        const int vt = g.xal ? lean_vt(g, R) : j;                 // chunk j of the visiting order
        const int vtn = j + 1 < vt1 ? (g.xal ? lean_vt_next(g, R) : j + 1) : -1;
        if (row_lead && vtn >= 0) {          // L2 hints for the next chunk's rows
            prefetch_l2(bf.phi_in + (size_t)vtn * chunk_stride + (size_t)cidx * (2 * VC), nrow * RB);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const T* fb = bf.face[a] + (size_t)vtn * fstride[a] + (size_t)ff[a] * (2 * VC);
                prefetch_l2(fb, (nrow + (a == 0 ? 1 : 0)) * RB);
                if (a > 0 && (la[a] == tdim[a] - 1 || own_right[a])) prefetch_l2(fb + (size_t)fs_[a] * (2 * VC), nrow * RB);
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
        const size_t ad = (size_t)vt * chunk_stride + (size_t)cidx * (2 * VC);
        T gs[VC], bs[VC], oge[VC];
        Chunk<T>::load(bf.phi_in + ad, gs);
        Chunk<T>::load(bf.phi_in + ad + VC, bs);
        lean_geq4<T, D>(g, bf.xc, g.Nc, cidx, 0, vt, R, oge);
        T dFg[VC], dFb[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v) dFg[v] = dFb[v] = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const T* fb0 = bf.face[a] + (size_t)vt * fstride[a] + (size_t)ff[a] * (2 * VC);
            T F0g[VC], F0b[VC], F1g[VC], F1b[VC];
            {   // the left face: owned, moments summed
                T sm[NM];
#pragma unroll
                for (int m = 0; m < NM; ++m) sm[m] = T(0);
                lean_face_flux<T, D, NOSRC, true>(g, bf, a, ff[a], vt, R, fb0, FC[fl[a][0]], FC[NFT + fl[a][0]], xi, w,
                                                  hx, F0g, F0b, sm);
#pragma unroll
                for (int m = 0; m < NM; ++m) acc[a][m].add(sm[m]);
            }
            // the right face: the next cell's left face (its moments summed there), or the domain's end
            const long long fr = (long long)ff[a] + fs_[a];
            const T* fb1 = fb0 + (size_t)fs_[a] * (2 * VC);
            if (own_right[a]) {
                T sm[NM];
#pragma unroll
                for (int m = 0; m < NM; ++m) sm[m] = T(0);
                lean_face_flux<T, D, NOSRC, true>(g, bf, a, fr, vt, R, fb1, FC[fl[a][1]], FC[NFT + fl[a][1]], xi, w, hx,
                                                  F1g, F1b, sm);
                const int pl = TL::poff(a) * NM + TL::plane_pos(a, la);
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    Kahan<T> k = RS[pl + m * TL::plane(a)];
                    k.add(sm[m]);
                    RS[pl + m * TL::plane(a)] = k;
                }
            } else {
                lean_face_flux<T, D, NOSRC, false>(g, bf, a, fr, vt, R, fb1, FC[fl[a][1]], FC[NFT + fl[a][1]], xi, w,
                                                   hx, F1g, F1b, nullptr);
            }
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                dFg[v] = fma(idxT[a], F1g[v] - F0g[v], dFg[v]);
                dFb[v] = fma(idxT[a], F1b[v] - F0b[v], dFb[v]);
            }
        }
        // ---- phi* of the owned cell from the net flux (eq. phiupdate)
        T obe[VC], og[VC], ob[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            obe[v] = (hx[v] + own.eb) * oge[v];
            og[v] = fma(own.fa_g, gs[v], own.fb_g * oge[v]);
            ob[v] = fma(own.fa_b, bs[v], own.fb_b * obe[v]);
        }
        T u[D];
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = own.u[a];
        store_phi_star<T, D, NOSRC>(dtT, xi, u, own.hu2, own.um_g, own.um_b, own.usrc, og, ob, oge, obe, dFg, dFb,
                                    bf.phi_out + ad);
        if (g.xal) lean_rows_next(g, R);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
        for (int m = 0; m < NM; ++m) bf.mf[a][((size_t)grp * NM + m) * g.nf[a] + ff[a]] = acc[a][m].value();
        if (own_right[a]) {
            const int pl = TL::poff(a) * NM + TL::plane_pos(a, la);
#pragma unroll
            for (int m = 0; m < NM; ++m)
                bf.mf[a][((size_t)grp * NM + m) * g.nf[a] + ff[a] + fs_[a]] = RS[pl + m * TL::plane(a)].value();
        }
    }
}

template <typename T, int D, int T0_, int T1_, int T2_, bool NOSRC>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (LeanBOcc<T, D, T0_, T1_, T2_>::value))
    k_lflux(const Inst<T>* __restrict__ in, int cur) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    lean_b_body<T, D, T0_, T1_, T2_, NOSRC>(in->g, in->b[cur], blockIdx.x, blockIdx.y, smem);
}

template <typename T, int D, int T0_, int T1_, int T2_, bool NOSRC>
__global__ void __launch_bounds__(Tile<D, T0_, T1_, T2_>::NT, (LeanBOcc<T, D, T0_, T1_, T2_>::value))
    k_lflux_batch(const Item* __restrict__ items, const Inst<T>* __restrict__ insts, const int* __restrict__ cur) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    const Item it = items[blockIdx.x];
    const Inst<T>& in = insts[it.inst];
    lean_b_body<T, D, T0_, T1_, T2_, NOSRC>(in.g, in.b[cur[it.inst] & 1], it.tile, it.grp, smem);
}

}  // namespace cdg
