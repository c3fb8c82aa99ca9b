// api.cu -- the C ABI of include/cdugks.h: problem validation, workspace layout
// in caller-owned device memory, velocity tables, and the per-step launch
// sequence of the CDUGKS update (arXiv:2208.09132, Sec. 2.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/cdugks.h"
#include "launch.cuh"
#include "persist.cuh"

using cdg::BatchPlan;
using cdg::Bufs;
using cdg::CellC;
using cdg::FaceC;
using cdg::Geo;
using cdg::Inst;
using cdg::Item;
using cdg::PHead;
using cdg::PItem;
using cdg::PState;
using cdg::QItem;
using cdg::RItem;
using cdg::VC;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(CDUGKS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t phi[2], pb, sg, fv[3], W, cellc, cellc0, facec[3], wf[3], mf[3], vel, refl, io, status, inst;
    size_t hq, qs, qf[3];     // Shakhov model only
    size_t force;             // acceleration only
    size_t xc, xc0, xf[3];    // lean shapes only: separable factor tables
    size_t total;
};

// Optional workspace buffers, by the sweep modes that need them.
enum { BUF_PHIBAR = 1, BUF_SLOPES = 2, BUF_FACES = 4, BUF_FORCE = 8, BUF_XTAB = 16 };
int buffers_of(int mode) {
    int b = 0;
    if (cdg::mode_lean(mode)) b |= BUF_XTAB;
    if (cdg::mode_acc(mode)) b |= BUF_FORCE;
    if (cdg::mode_source(mode) != cdg::MODE_FUSED) b |= BUF_PHIBAR;
    if (cdg::mode_source(mode) == cdg::MODE_STORED) b |= BUF_SLOPES;
    if (cdg::mode_faces(mode)) b |= BUF_FACES;
    return b;
}

}  // namespace

struct cdugks {
    cdugks_grid grid;
    cdugks_vgrid vgrid;
    cdugks_phys phys;
    Geo g;
    int prec;              // CDUGKS_FP64 / CDUGKS_FP32
    size_t elt;            // bytes of one stored value
    size_t cellc_bytes, facec_bytes;
    int Nv;
    int gcap;              // velocity groups the workspace is laid out for
    int bufs_cap;          // optional buffers the workspace holds (BUF_* bits)
    int gsel;              // requested groups (0 = auto)
    int recon;             // CDUGKS_RECON_UPWIND_CELL or CDUGKS_RECON_FACE_GRADIENT
    int collision;         // CDUGKS_COLLISION_TEDDF or CDUGKS_COLLISION_SHAKHOV
    bool zero_node;        // some active velocity axis has a node at xi = 0 (no lean shapes)
    Layout lay;
    unsigned char* base;
    size_t bound_bytes;
    cudaStream_t stream;
    bool bound, initialised;
    int cur;               // state buffer holding phi* of the current time level
    long long steps;
    std::vector<double> vel;  // [Nvp][8]: xi_0, xi_1, xi_2, w, |xi|^2/2, 0, 0, 0
    std::vector<float> vel32; // the same table rounded to float (FP32 storage)
    std::vector<int> refl;    // [8][Nvp]
    // captured steps (cdugks_capture): one graph per parity of the state buffer it starts from
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_steps = 0;
};

namespace {

// 1D nodes (both ends included) and weights, Sec. 2 quadrature sum_k w_k.
bool vgrid_1d(int n, double lo, double hi, int rule, std::vector<double>& x, std::vector<double>& w) {
    if (n < 2 || !(hi > lo)) return false;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double d = (hi - lo) / (n - 1);
    for (int k = 0; k < n; ++k) x[k] = lo + (hi - lo) * (double)k / (double)(n - 1);
    if (rule == CDUGKS_RULE_TRAPEZOID) {
        for (int k = 0; k < n; ++k) w[k] = (k == 0 || k == n - 1) ? 0.5 * d : d;
    } else if (rule == CDUGKS_RULE_BOOLE) {
        if ((n - 1) % 4 != 0) return false;
        const double c[5] = {14.0, 64.0, 24.0, 64.0, 14.0};
        for (int p = 0; p + 4 < n; p += 4)
            for (int j = 0; j < 5; ++j) w[p + j] += c[j] * d / 45.0;
    } else {
        return false;
    }
    return true;
}

cdg::TileShape tile_of(int prec, int D, int id) {
    return prec == CDUGKS_FP32 ? cdg::tile_shape_f32(D, id) : cdg::tile_shape_f64(D, id);
}
int tile_count(int prec, int D) { return prec == CDUGKS_FP32 ? cdg::tile_count_f32(D) : cdg::tile_count_f64(D); }
int tile_mode(int prec, int D, int id) {
    return prec == CDUGKS_FP32 ? cdg::tile_mode_f32(D, id) : cdg::tile_mode_f64(D, id);
}

void set_tiles(cdugks* h, int id) {
    Geo& g = h->g;
    g.tile_id = id;
    const cdg::TileShape ts = tile_of(h->prec, g.D, id);
    for (int a = 0; a < 3; ++a) g.tiles[a] = a < g.D ? (g.n[a] + ts.t[a] - 1) / ts.t[a] : 1;
}

int groups_for(const cdugks* h, int requested) {
    const Geo& g = h->g;
    if (requested > 0) return std::min(requested, g.NVT);
    // enough CTAs for a few full waves over 152 SMs (at least 2 resident per SM)
    const long long tiles = (long long)g.tiles[0] * g.tiles[1] * g.tiles[2];
    const long long want = 152LL * 2 * 4;
    long long G = (want + tiles - 1) / tiles;
    G = std::max(1LL, std::min<long long>(G, g.NVT));
    G = std::min<long long>(G, 64);
    return (int)G;
}

void set_groups(cdugks* h, int G) {
    Geo& g = h->g;
    g.ntpg = (g.NVT + G - 1) / G;
    g.G = (g.NVT + g.ntpg - 1) / g.ntpg;
}

void make_layout(cdugks* h) {
    const Geo& g = h->g;
    const int NM = 2 + g.D;
    Layout& L = h->lay;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t state = (size_t)g.Nvp * (size_t)g.Nc * 2 * h->elt;
    L.phi[0] = take(state);
    L.phi[1] = take(state);
    L.pb = (h->bufs_cap & BUF_PHIBAR) ? take(state) : 0;
    L.force = (h->bufs_cap & BUF_FORCE) ? take(state) : 0;
    L.sg = (h->bufs_cap & BUF_SLOPES) ? take(state * g.D) : 0;
    for (int a = 0; a < 3; ++a)
        L.fv[a] = (h->bufs_cap & BUF_FACES) && a < g.D ? take((size_t)g.Nvp * (size_t)g.nf[a] * 2 * h->elt) : 0;
    L.W = take(sizeof(double) * NM * g.Nc);
    L.cellc = take(h->cellc_bytes * g.Nc);
    L.cellc0 = take(h->cellc_bytes * g.Nc);
    for (int a = 0; a < 3; ++a) {
        const long long nf = a < g.D ? g.nf[a] : 0;
        L.facec[a] = take(h->facec_bytes * nf);
        L.wf[a] = take(sizeof(double) * (size_t)h->gcap * NM * nf);
        L.mf[a] = take(sizeof(double) * (size_t)h->gcap * NM * nf);
    }
    L.vel = take(h->elt * 8 * g.Nvp);
    L.refl = take(sizeof(int) * 8 * g.Nvp);
    L.io = take(sizeof(double) * std::max(NM, g.D * g.D + g.D) * g.Nc);   // moments, or P and q
    const bool sk = h->collision == CDUGKS_COLLISION_SHAKHOV;
    const int NQ = g.D + g.D * (g.D + 1) / 2;
    L.hq = sk ? take(sizeof(double) * g.D * g.Nc) : 0;
    L.qs = sk ? take(sizeof(double) * (size_t)h->gcap * NQ * g.Nc) : 0;
    for (int a = 0; a < 3; ++a) L.qf[a] = sk && a < g.D ? take(sizeof(double) * (size_t)h->gcap * NQ * g.nf[a]) : 0;
    const bool xt = (h->bufs_cap & BUF_XTAB) != 0;
    L.xc = xt ? take(h->elt * (size_t)g.xrows * g.Nc) : 0;
    L.xc0 = xt ? take(h->elt * (size_t)g.xrows * g.Nc) : 0;
    for (int a = 0; a < 3; ++a) L.xf[a] = xt && a < g.D ? take(h->elt * (size_t)g.xrows * g.nf[a]) : 0;
    L.status = take(256);
    L.inst = take(std::max(sizeof(Inst<float>), sizeof(Inst<double>)));
    L.total = off;
}

template <typename T>
Bufs<T> bufs(const cdugks* h, int in) {
    Bufs<T> b;
    unsigned char* p = h->base;
    const Layout& L = h->lay;
    b.phi_in = reinterpret_cast<const T*>(p + L.phi[in]);
    b.phi_out = reinterpret_cast<T*>(p + L.phi[1 - in]);
    b.phibar = (h->bufs_cap & BUF_PHIBAR) ? reinterpret_cast<T*>(p + L.pb) : nullptr;
    b.force = (h->bufs_cap & BUF_FORCE) ? reinterpret_cast<T*>(p + L.force) : nullptr;
    b.sigma = (h->bufs_cap & BUF_SLOPES) ? reinterpret_cast<T*>(p + L.sg) : nullptr;
    for (int a = 0; a < 3; ++a)
        b.face[a] = (h->bufs_cap & BUF_FACES) && a < h->g.D ? reinterpret_cast<T*>(p + L.fv[a]) : nullptr;
    b.W = reinterpret_cast<double*>(p + L.W);
    b.cellc = reinterpret_cast<CellC<T>*>(p + L.cellc);
    b.cellc0 = reinterpret_cast<CellC<T>*>(p + L.cellc0);
    for (int a = 0; a < 3; ++a) {
        b.facec[a] = reinterpret_cast<FaceC<T>*>(p + L.facec[a]);
        b.wf[a] = reinterpret_cast<double*>(p + L.wf[a]);
        b.mf[a] = reinterpret_cast<double*>(p + L.mf[a]);
    }
    b.vel = reinterpret_cast<const T*>(p + L.vel);
    b.refl = reinterpret_cast<const int*>(p + L.refl);
    b.status = reinterpret_cast<int*>(p + L.status);
    const bool sk = h->collision == CDUGKS_COLLISION_SHAKHOV;
    b.hq = sk ? reinterpret_cast<double*>(p + L.hq) : nullptr;
    b.qs = sk ? reinterpret_cast<double*>(p + L.qs) : nullptr;
    for (int a = 0; a < 3; ++a) b.qf[a] = sk && a < h->g.D ? reinterpret_cast<double*>(p + L.qf[a]) : nullptr;
    // the factor tables exist (and are kept up to date) only while a lean shape is selected
    const bool xt = (h->bufs_cap & BUF_XTAB) && cdg::mode_lean(tile_mode(h->prec, h->g.D, h->g.tile_id));
    b.xc = xt ? reinterpret_cast<T*>(p + L.xc) : nullptr;
    b.xc0 = xt ? reinterpret_cast<T*>(p + L.xc0) : nullptr;
    const bool xft = xt && cdg::mode_xf(tile_mode(h->prec, h->g.D, h->g.tile_id));   // face tables: lean sweep B only
    for (int a = 0; a < 3; ++a) b.xf[a] = xft && a < h->g.D ? reinterpret_cast<T*>(p + L.xf[a]) : nullptr;
    return b;
}

void drop_graphs(cdugks* h) {
    for (int c = 0; c < 2; ++c) {
        if (h->gexec[c]) cudaGraphExecDestroy(h->gexec[c]);
        if (h->graph[c]) cudaGraphDestroy(h->graph[c]);
        h->gexec[c] = nullptr;
        h->graph[c] = nullptr;
    }
    h->graph_steps = 0;
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double>& v) {
    std::vector<T> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
    return o;
}

template <typename T>
Inst<T> inst_of(const cdugks* h) {
    Inst<T> in;
    in.g = h->g;
    in.b[0] = bufs<T>(h, 0);
    in.b[1] = bufs<T>(h, 1);
    return in;
}

// The instance record every kernel of this handle reads (geometry + buffers).
int upload_inst(cdugks* h) {
    cudaError_t e;
    if (h->prec == CDUGKS_FP32) {
        const Inst<float> in = inst_of<float>(h);
        e = cudaMemcpyAsync(h->base + h->lay.inst, &in, sizeof(in), cudaMemcpyHostToDevice, h->stream);
        if (!e) e = cudaStreamSynchronize(h->stream);
    } else {
        const Inst<double> in = inst_of<double>(h);
        e = cudaMemcpyAsync(h->base + h->lay.inst, &in, sizeof(in), cudaMemcpyHostToDevice, h->stream);
        if (!e) e = cudaStreamSynchronize(h->stream);
    }
    if (e) return cuda_fail(e, "upload instance record");
    return CDUGKS_OK;
}

template <typename T>
const Inst<T>* dinst(const cdugks* h) {
    return reinterpret_cast<const Inst<T>*>(h->base + h->lay.inst);
}

int check_ready(const cdugks* h, bool need_init) {
    if (!h) return fail(CDUGKS_ERR_INVALID, "null handle");
    if (!h->bound) return fail(CDUGKS_ERR_UNBOUND, "no workspace bound (cdugks_bind)");
    if (need_init && !h->initialised) return fail(CDUGKS_ERR_UNBOUND, "state not initialised (cdugks_init)");
    return CDUGKS_OK;
}

struct StateHeader {
    char magic[8];
    int dim, prec, Nvp, collision;
    long long Nc, steps;
    double dt;
};

}  // namespace

extern "C" {

int cdugks_create(const cdugks_grid* grid, const cdugks_vgrid* vgrid, const cdugks_phys* phys, cdugks_t** out) {
    if (!out) return fail(CDUGKS_ERR_INVALID, "null output pointer");
    *out = nullptr;
    if (!grid || !vgrid || !phys) return fail(CDUGKS_ERR_INVALID, "null description");
    const int D = grid->dim;
    if (D < 1 || D > 3) return fail(CDUGKS_ERR_INVALID, "dim must be 1, 2 or 3");
    if (phys->precision != CDUGKS_FP64 && phys->precision != CDUGKS_FP32)
        return fail(CDUGKS_ERR_INVALID, "precision must be CDUGKS_FP64 or CDUGKS_FP32");
    if (!(phys->R > 0) || !(phys->mu_ref > 0) || !(phys->T_ref > 0) || !(phys->Pr > 0) || !(phys->K >= 0) ||
        !std::isfinite(phys->omega))
        return fail(CDUGKS_ERR_INVALID, "physics parameters must be positive (K >= 0)");
    cdugks* h = new (std::nothrow) cdugks();
    if (!h) return fail(CDUGKS_ERR_OOM, "host allocation failed");
    h->grid = *grid;
    h->vgrid = *vgrid;
    h->phys = *phys;
    h->prec = phys->precision;
    h->elt = h->prec == CDUGKS_FP32 ? sizeof(float) : sizeof(double);
    h->cellc_bytes = h->prec == CDUGKS_FP32 ? sizeof(CellC<float>) : sizeof(CellC<double>);
    h->facec_bytes = h->prec == CDUGKS_FP32 ? sizeof(FaceC<float>) : sizeof(FaceC<double>);
    Geo& g = h->g;
    std::memset(&g, 0, sizeof(g));
    g.D = D;
    g.Nc = 1;
    std::vector<double> nodes[3], wts[3];
    int nv[3] = {1, 1, 1};
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            if (grid->n[a] < 1 || !(grid->hi[a] > grid->lo[a])) {
                delete h;
                return fail(CDUGKS_ERR_INVALID, "each active axis needs n >= 1 and hi > lo");
            }
            for (int s = 0; s < 2; ++s) {
                const int bc = grid->bc[a][s];
                if (bc < 0 || bc > 2) {
                    delete h;
                    return fail(CDUGKS_ERR_INVALID, "unknown boundary condition");
                }
                if (bc == CDUGKS_BC_SPECULAR && (grid->n[a] < 2 || vgrid->lo[a] != -vgrid->hi[a])) {
                    delete h;
                    return fail(CDUGKS_ERR_INVALID, "specular walls need n >= 2 and a symmetric velocity range");
                }
            }
            if ((grid->bc[a][0] == CDUGKS_BC_PERIODIC) != (grid->bc[a][1] == CDUGKS_BC_PERIODIC)) {
                delete h;
                return fail(CDUGKS_ERR_INVALID, "periodic must be set on both sides of an axis");
            }
            if (!vgrid_1d(vgrid->n[a], vgrid->lo[a], vgrid->hi[a], vgrid->rule, nodes[a], wts[a])) {
                delete h;
                return fail(CDUGKS_ERR_INVALID, "bad velocity grid (n >= 2, hi > lo, Boole needs n = 4m+1)");
            }
            nv[a] = vgrid->n[a];
            g.nv1[a] = vgrid->n[a];
            g.dxi[a] = (vgrid->hi[a] - vgrid->lo[a]) / (vgrid->n[a] - 1);
            g.vlo[a] = vgrid->lo[a];
            for (double x : nodes[a]) h->zero_node = h->zero_node || x == 0.0;
            g.n[a] = grid->n[a];
            g.bc[a][0] = grid->bc[a][0];
            g.bc[a][1] = grid->bc[a][1];
            g.dx[a] = (grid->hi[a] - grid->lo[a]) / grid->n[a];
        } else {
            nodes[a].assign(1, 0.0);
            wts[a].assign(1, 1.0);
            g.nv1[a] = 1;
            g.dxi[a] = 1.0;
            g.vlo[a] = 0.0;
            g.n[a] = 1;
            g.dx[a] = 1.0;
        }
        g.Nc *= g.n[a];
    }
    const long long Nv = (long long)nv[0] * nv[1] * nv[2];
    if (Nv > (1LL << 26) || g.Nc > (1LL << 31)) {
        delete h;
        return fail(CDUGKS_ERR_INVALID, "problem too large");
    }
    h->Nv = (int)Nv;
    g.NVT = (int)((Nv + VC - 1) / VC);
    g.Nvp = g.NVT * VC;
    // rows of the separable factor tables: axis 0 padded to whole chunks, then the other axes
    g.xrow[0] = 0;
    g.xrow[1] = (nv[0] + VC - 1) / VC * VC;
    g.xrow[2] = g.xrow[1] + (D >= 2 ? nv[1] : 0);
    g.xrows = g.xrow[2] + (D >= 3 ? nv[2] : 0);
    g.xal = nv[0] % VC == 0;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) g.fn[a][b] = g.n[b] + (a == b && a < D ? 1 : 0);
        g.nf[a] = (long long)g.fn[a][0] * g.fn[a][1] * g.fn[a][2];
        if (g.nf[a] >= (1LL << 31)) {      // cell and face numbers are 32-bit in the kernels
            delete h;
            return fail(CDUGKS_ERR_INVALID, "problem too large");
        }
    }
    // velocity tables (padding: xi = 0, w = 0)
    h->vel.assign(8 * (size_t)g.Nvp, 0.0);
    h->refl.assign(8 * (size_t)g.Nvp, 0);
    double vmax = 0.0;
    for (int k2 = 0; k2 < nv[2]; ++k2)
        for (int k1 = 0; k1 < nv[1]; ++k1)
            for (int k0 = 0; k0 < nv[0]; ++k0) {
                const long long i = k0 + (long long)nv[0] * (k1 + (long long)nv[1] * k2);
                const double x[3] = {nodes[0][k0], nodes[1][k1], nodes[2][k2]};
                double s = 0.0;
                for (int a = 0; a < D; ++a) {
                    h->vel[(size_t)i * 8 + a] = x[a];
                    s += x[a] * x[a];
                }
                h->vel[(size_t)i * 8 + 3] = wts[0][k0] * wts[1][k1] * wts[2][k2];
                h->vel[(size_t)i * 8 + 4] = 0.5 * s;
                vmax = std::max(vmax, std::sqrt(s));
                for (int m = 0; m < 8; ++m) {
                    const int r0 = (m & 1) ? nv[0] - 1 - k0 : k0;
                    const int r1 = (m & 2) ? nv[1] - 1 - k1 : k1;
                    const int r2 = (m & 4) ? nv[2] - 1 - k2 : k2;
                    h->refl[(size_t)m * g.Nvp + i] = (int)(r0 + (long long)nv[0] * (r1 + (long long)nv[1] * r2));
                }
            }
    for (long long i = Nv; i < g.Nvp; ++i)
        for (int m = 0; m < 8; ++m) h->refl[(size_t)m * g.Nvp + i] = (int)i;
    // time step: fixed CFL rule of Sec. 4 unless given
    double dt = phys->dt;
    if (!(dt > 0)) {
        double dxmin = g.dx[0];
        for (int a = 1; a < D; ++a) dxmin = std::min(dxmin, g.dx[a]);
        if (!(phys->cfl > 0) || !(vmax > 0)) {
            delete h;
            return fail(CDUGKS_ERR_INVALID, "need dt > 0 or cfl > 0 with a nonzero velocity grid");
        }
        dt = phys->cfl * dxmin / (2.0 * vmax);
    }
    g.dt = dt;
    g.h = 0.5 * dt;
    for (int a = 0; a < 3; ++a) {
        g.hdx[a] = g.h / g.dx[a];
        g.idx[a] = 1.0 / g.dx[a];
    }
    // reconstruction coefficients 2 h xi_a / dx_a in the velocity records
    for (long long i = 0; i < Nv; ++i)
        for (int a = 0; a < D; ++a) h->vel[(size_t)i * 8 + 5 + a] = 2.0 * g.hdx[a] * h->vel[(size_t)i * 8 + a];
    g.wait_log2 = 22;
    g.K = phys->K;
    g.R = phys->R;
    g.mu_ref = phys->mu_ref;
    g.T_ref = phys->T_ref;
    g.omega = phys->omega;
    g.Pr = phys->Pr;
    // with Pr = 1 the TEDDF b-source coefficient (Pr - 1)/tau vanishes exactly
    g.nosrc = phys->Pr == 1.0;
    set_tiles(h, 0);
    h->vel32 = cast_vec<float>(h->vel);
    h->gsel = 0;
    h->gcap = groups_for(h, 0);
    set_groups(h, h->gcap);
    make_layout(h);
    h->stream = nullptr;
    h->cur = 0;
    *out = h;
    return CDUGKS_OK;
}

int cdugks_set_velocity_groups(cdugks_t* h, int groups) {
    if (!h || groups < 0) return fail(CDUGKS_ERR_INVALID, "bad velocity group count");
    const int G = groups_for(h, groups);
    if (h->bound && G > h->gcap)
        return fail(CDUGKS_ERR_INVALID, "more velocity groups than the bound workspace was laid out for");
    if (!h->bound && G > h->gcap) {
        h->gcap = G;
        make_layout(h);
    }
    drop_graphs(h);
    h->gsel = groups;
    set_groups(h, G);
    if (h->bound) return upload_inst(h);
    return CDUGKS_OK;
}

int cdugks_tile_count(int precision, int dim) {
    if ((precision != CDUGKS_FP32 && precision != CDUGKS_FP64) || dim < 1 || dim > 3) return 0;
    return tile_count(precision, dim);
}

int cdugks_tile_shape(int precision, int dim, int tile_id, int* out) {
    if (!out || (precision != CDUGKS_FP32 && precision != CDUGKS_FP64) || dim < 1 || dim > 3 || tile_id < 0 ||
        tile_id >= tile_count(precision, dim))
        return fail(CDUGKS_ERR_INVALID, "unknown tile");
    const cdg::TileShape ts = tile_of(precision, dim, tile_id);
    for (int a = 0; a < 3; ++a) out[a] = ts.t[a];
    out[3] = tile_mode(precision, dim, tile_id);
    return CDUGKS_OK;
}

int cdugks_set_tile(cdugks_t* h, int tile_id) {
    if (!h) return fail(CDUGKS_ERR_INVALID, "null handle");
    if (tile_id < 0 || tile_id >= tile_count(h->prec, h->g.D)) return fail(CDUGKS_ERR_INVALID, "unknown tile id");
    const int mode = tile_mode(h->prec, h->g.D, tile_id);
    if (cdg::mode_r2(mode) != (h->recon == CDUGKS_RECON_FACE_GRADIENT))
        return fail(CDUGKS_ERR_INVALID, "tile shape does not implement the selected reconstruction");
    if (cdg::mode_sk(mode) != (h->collision == CDUGKS_COLLISION_SHAKHOV))
        return fail(CDUGKS_ERR_INVALID, "tile shape does not implement the selected collision model");
    if (cdg::mode_acc(mode) != (h->g.accel != 0))
        return fail(CDUGKS_ERR_INVALID, "tile shape does not implement the selected external acceleration");
    if (cdg::mode_source(mode) == cdg::MODE_STORED)
        for (int a = 0; a < h->g.D; ++a)
            if (h->g.bc[a][0] == CDUGKS_BC_DIRICHLET || h->g.bc[a][1] == CDUGKS_BC_DIRICHLET)
                return fail(CDUGKS_ERR_INVALID, "stored-slope shapes support periodic and specular boundaries only");
    if (cdg::mode_lean(mode) && h->zero_node)
        return fail(CDUGKS_ERR_INVALID, "lean shapes need a velocity grid without a node at xi = 0");
    if (cdg::mode_lean(mode) && h->bound && h->initialised && !cdg::mode_lean(tile_mode(h->prec, h->g.D, h->g.tile_id)))
        return fail(CDUGKS_ERR_INVALID, "select a lean shape before cdugks_init (its factor tables start there)");
    drop_graphs(h);
    const int need = buffers_of(mode);
    if (need & ~h->bufs_cap) {
        if (h->bound)
            return fail(CDUGKS_ERR_INVALID, "this shape needs more workspace buffers: select it before cdugks_bind");
        h->bufs_cap |= need;
        make_layout(h);
    }
    set_tiles(h, tile_id);
    const int G = groups_for(h, h->gsel);
    if (h->bound && G > h->gcap) set_groups(h, h->gcap);
    else {
        if (!h->bound && G > h->gcap) {
            h->gcap = G;
            make_layout(h);
        }
        set_groups(h, G);
    }
    if (h->bound) return upload_inst(h);
    return CDUGKS_OK;
}

int cdugks_workspace_bytes(const cdugks_t* h, size_t* bytes) {
    if (!h || !bytes) return fail(CDUGKS_ERR_INVALID, "null argument");
    *bytes = h->lay.total;
    return CDUGKS_OK;
}

int cdugks_set_reconstruction(cdugks_t* h, int recon) {
    if (!h) return fail(CDUGKS_ERR_INVALID, "null handle");
    if (recon != CDUGKS_RECON_UPWIND_CELL && recon != CDUGKS_RECON_FACE_GRADIENT)
        return fail(CDUGKS_ERR_INVALID, "unknown reconstruction");
    if (h->bound) return fail(CDUGKS_ERR_INVALID, "select the reconstruction before cdugks_bind");
    int id = -1;
    for (int t = 0; t < tile_count(h->prec, h->g.D) && id < 0; ++t) {
        const int m = tile_mode(h->prec, h->g.D, t);
        if (cdg::mode_r2(m) == (recon == CDUGKS_RECON_FACE_GRADIENT) &&
            cdg::mode_sk(m) == (h->collision == CDUGKS_COLLISION_SHAKHOV) && cdg::mode_acc(m) == (h->g.accel != 0))
            id = t;
    }
    if (id < 0)
        return fail(CDUGKS_ERR_INVALID,
                    "no tile shape implements this reconstruction with this collision model for this dimension");
    if (recon == CDUGKS_RECON_FACE_GRADIENT)   // a mirror image three cells deep
        for (int a = 0; a < h->g.D; ++a)
            for (int s2 = 0; s2 < 2; ++s2)
                if (h->g.bc[a][s2] == CDUGKS_BC_SPECULAR && h->g.n[a] < 3)
                    return fail(CDUGKS_ERR_INVALID, "the face-gradient reconstruction needs 3 cells next to a specular wall");
    h->recon = recon;
    return cdugks_set_tile(h, id);
}

int cdugks_set_collision(cdugks_t* h, int model) {
    if (!h) return fail(CDUGKS_ERR_INVALID, "null handle");
    if (model != CDUGKS_COLLISION_TEDDF && model != CDUGKS_COLLISION_SHAKHOV)
        return fail(CDUGKS_ERR_INVALID, "unknown collision model");
    if (h->bound) return fail(CDUGKS_ERR_INVALID, "select the collision model before cdugks_bind");
    int id = -1;
    for (int t = 0; t < tile_count(h->prec, h->g.D) && id < 0; ++t) {
        const int m = tile_mode(h->prec, h->g.D, t);
        if (cdg::mode_sk(m) == (model == CDUGKS_COLLISION_SHAKHOV) &&
            cdg::mode_r2(m) == (h->recon == CDUGKS_RECON_FACE_GRADIENT) && cdg::mode_acc(m) == (h->g.accel != 0))
            id = t;
    }
    if (id < 0)
        return fail(CDUGKS_ERR_INVALID, "no tile shape implements this collision model with this reconstruction");
    if (model == CDUGKS_COLLISION_SHAKHOV && cdg::mode_source(tile_mode(h->prec, h->g.D, id)) == cdg::MODE_STORED)
        for (int a = 0; a < h->g.D; ++a)
            if (h->g.bc[a][0] == CDUGKS_BC_DIRICHLET || h->g.bc[a][1] == CDUGKS_BC_DIRICHLET)
                return fail(CDUGKS_ERR_INVALID, "the Shakhov shapes of this dimension support periodic and specular boundaries only");
    const int old = h->collision;
    h->collision = model;
    h->g.shakhov = model == CDUGKS_COLLISION_SHAKHOV;
    make_layout(h);
    const int rc = cdugks_set_tile(h, id);
    if (rc) {
        h->collision = old;
        h->g.shakhov = old == CDUGKS_COLLISION_SHAKHOV;
        make_layout(h);
    }
    return rc;
}

int cdugks_set_acceleration(cdugks_t* h, const double* a) {
    if (!h) return fail(CDUGKS_ERR_INVALID, "null handle");
    if (h->bound) return fail(CDUGKS_ERR_INVALID, "set the acceleration before cdugks_bind");
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 3 && a; ++b) {
        if (!std::isfinite(a[b]) || (b >= h->g.D && a[b] != 0.0))
            return fail(CDUGKS_ERR_INVALID, "acceleration components must be finite, and 0 beyond dim");
        acc[b] = a[b];
    }
    const int on = acc[0] != 0.0 || acc[1] != 0.0 || acc[2] != 0.0;
    int id = -1;
    for (int t = 0; t < tile_count(h->prec, h->g.D) && id < 0; ++t) {
        const int m = tile_mode(h->prec, h->g.D, t);
        if (cdg::mode_acc(m) == (on != 0) && cdg::mode_sk(m) == (h->collision == CDUGKS_COLLISION_SHAKHOV) &&
            cdg::mode_r2(m) == (h->recon == CDUGKS_RECON_FACE_GRADIENT))
            id = t;
    }
    if (id < 0)
        return fail(CDUGKS_ERR_INVALID,
                    "no tile shape implements the acceleration with this collision model and reconstruction");
    const Geo old = h->g;
    for (int b = 0; b < 3; ++b) h->g.acc[b] = acc[b];
    h->g.accel = on;
    const int rc = cdugks_set_tile(h, id);
    if (rc) h->g = old;
    return rc;
}

int cdugks_test_wait_timeout(cdugks_t* h, int on) {
    if (!h) return fail(CDUGKS_ERR_INVALID, "null handle");
    drop_graphs(h);
    h->g.wait_test = on ? 1 : 0;
    h->g.wait_log2 = on ? 10 : 22;
    if (h->bound) return upload_inst(h);
    return CDUGKS_OK;
}

int cdugks_bind(cdugks_t* h, void* device_ptr, size_t bytes, void* cuda_stream) {
    if (!h || !device_ptr) return fail(CDUGKS_ERR_INVALID, "null argument");
    drop_graphs(h);
    if (((uintptr_t)device_ptr) % kAlign) return fail(CDUGKS_ERR_INVALID, "workspace must be 256-byte aligned");
    if (bytes < h->lay.total) return fail(CDUGKS_ERR_OOM, "workspace smaller than cdugks_workspace_bytes");
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, device_ptr);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(CDUGKS_ERR_INVALID, "workspace is not device memory");
    h->base = static_cast<unsigned char*>(device_ptr);
    h->bound_bytes = bytes;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    const Geo& g = h->g;
    // velocity table in the storage precision
    if (h->prec == CDUGKS_FP32) {
        if ((e = cudaMemcpyAsync(h->base + h->lay.vel, h->vel32.data(), h->vel32.size() * 4, cudaMemcpyHostToDevice,
                                 h->stream)))
            return cuda_fail(e, "upload velocity table");
    } else {
        if ((e = cudaMemcpyAsync(h->base + h->lay.vel, h->vel.data(), h->vel.size() * 8, cudaMemcpyHostToDevice,
                                 h->stream)))
            return cuda_fail(e, "upload velocity table");
    }
    if ((e = cudaMemcpyAsync(h->base + h->lay.refl, h->refl.data(), h->refl.size() * sizeof(int),
                             cudaMemcpyHostToDevice, h->stream)))
        return cuda_fail(e, "upload reflection table");
    if ((e = cudaMemsetAsync(h->base + h->lay.status, 0, 256, h->stream))) return cuda_fail(e, "clear status");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "cudaStreamSynchronize");
    (void)g;
    h->bound = true;
    h->initialised = false;
    return upload_inst(h);
}

int cdugks_init(cdugks_t* h, const double* rho_u_T) {
    int rc = check_ready(h, false);
    if (rc) return rc;
    if (!rho_u_T) return fail(CDUGKS_ERR_INVALID, "null fields");
    const Geo& g = h->g;
    const int NM = 2 + g.D;
    for (long long c = 0; c < g.Nc; ++c) {
        const double rho = rho_u_T[c * NM], T = rho_u_T[c * NM + 1 + g.D];
        if (!(rho > 0) || !(T > 0)) return fail(CDUGKS_ERR_INVALID, "density and temperature must be positive");
        for (int m = 0; m < NM; ++m)
            if (!std::isfinite(rho_u_T[c * NM + m])) return fail(CDUGKS_ERR_INVALID, "non-finite field");
    }
    cudaError_t e;
    double* io = reinterpret_cast<double*>(h->base + h->lay.io);
    if ((e = cudaMemcpyAsync(io, rho_u_T, sizeof(double) * NM * g.Nc, cudaMemcpyHostToDevice, h->stream)))
        return cuda_fail(e, "upload fields");
    // initial state goes to buffer 0: launch with phi_in = buffer 1, phi_out = buffer 0
    if (h->prec == CDUGKS_FP32) e = cdg::launch_init_f32(g, dinst<float>(h), 1, io, h->stream);
    else e = cdg::launch_init_f64(g, dinst<double>(h), 1, io, h->stream);
    if (e) return cuda_fail(e, "init kernel");
    if ((e = cudaMemsetAsync(h->base + h->lay.status, 0, 256, h->stream))) return cuda_fail(e, "clear status");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "init");
    h->cur = 0;
    h->steps = 0;
    h->initialised = true;
    return CDUGKS_OK;
}

namespace {
cudaError_t launch_one_step(cdugks* h) {
    const void* phi_in = h->base + h->lay.phi[h->cur];
    if (h->prec == CDUGKS_FP32) return cdg::launch_step_f32(h->g, dinst<float>(h), h->cur, h->stream, nullptr, phi_in);
    return cdg::launch_step_f64(h->g, dinst<double>(h), h->cur, h->stream, nullptr, phi_in);
}
}  // namespace

int cdugks_step(cdugks_t* h, int nsteps) {
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (nsteps < 0) return fail(CDUGKS_ERR_INVALID, "nsteps < 0");
    int done = 0;
    cudaError_t e;
    if (h->graph_steps > 0)
        for (; done + h->graph_steps <= nsteps; done += h->graph_steps) {
            if ((e = cudaGraphLaunch(h->gexec[h->cur], h->stream))) return cuda_fail(e, "cudaGraphLaunch");
            h->cur ^= h->graph_steps & 1;
            h->steps += h->graph_steps;
        }
    for (; done < nsteps; ++done) {
        if ((e = launch_one_step(h))) return cuda_fail(e, "step launch");
        h->cur = 1 - h->cur;
        h->steps += 1;
    }
    return CDUGKS_OK;
}

int cdugks_capture(cdugks_t* h, int steps_per_graph) {
    int rc = check_ready(h, false);
    if (rc) return rc;
    if (steps_per_graph < 0 || steps_per_graph > 4096) return fail(CDUGKS_ERR_INVALID, "steps_per_graph in [0, 4096]");
    drop_graphs(h);
    if (steps_per_graph == 0) return CDUGKS_OK;
    if (!h->stream) return fail(CDUGKS_ERR_INVALID, "graph capture needs a non-default stream");
    const int cur0 = h->cur;
    for (int c = 0; c < 2; ++c) {          // a graph for each parity the state can start from
        h->cur = c;
        cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e) {
            h->cur = cur0;
            drop_graphs(h);
            return cuda_fail(e, "cudaStreamBeginCapture");
        }
        for (int s = 0; s < steps_per_graph && e == cudaSuccess; ++s) {
            e = launch_one_step(h);
            h->cur = 1 - h->cur;
        }
        const cudaError_t e2 = cudaStreamEndCapture(h->stream, &h->graph[c]);
        if (!e && !e2) e = cudaGraphInstantiate(&h->gexec[c], h->graph[c], 0);
        if (e || e2) {
            h->cur = cur0;
            drop_graphs(h);
            return cuda_fail(e ? e : e2, "capture steps");
        }
    }
    h->cur = cur0;
    h->graph_steps = steps_per_graph;
    return CDUGKS_OK;
}

int cdugks_profile_step(cdugks_t* h, int nsteps, double* ms_out) {
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (nsteps < 1 || nsteps > 100000 || !ms_out) return fail(CDUGKS_ERR_INVALID, "need 1 <= nsteps <= 1e5 and ms_out");
    // all events exist before the first launch, so the device never waits on the host
    std::vector<cudaEvent_t> ev((size_t)nsteps * 5);
    cudaError_t e = cudaSuccess;
    size_t made = 0;
    for (; made < ev.size(); ++made)
        if ((e = cudaEventCreate(&ev[made]))) break;
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
        cudaEvent_t* es = &ev[(size_t)s * 5];
        const void* phi_in = h->base + h->lay.phi[h->cur];
        if (h->prec == CDUGKS_FP32) e = cdg::launch_step_f32(h->g, dinst<float>(h), h->cur, h->stream, es, phi_in);
        else e = cdg::launch_step_f64(h->g, dinst<double>(h), h->cur, h->stream, es, phi_in);
        if (e) break;
        h->cur = 1 - h->cur;
        h->steps += 1;
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[(size_t)s * 5 + k], ev[(size_t)s * 5 + k + 1]);
            acc[k] += ms;
        }
    for (size_t k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    if (e) return cuda_fail(e, "profile_step");
    for (int k = 0; k < 4; ++k) ms_out[k] = acc[k] / nsteps;
    return CDUGKS_OK;
}

int cdugks_sync_status(cdugks_t* h) {
    int rc = check_ready(h, false);
    if (rc) return rc;
    int st = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&st, h->base + h->lay.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream)))
        return cuda_fail(e, "read status");
    if ((e = cudaMemsetAsync(h->base + h->lay.status, 0, 256, h->stream))) return cuda_fail(e, "clear status");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "cudaStreamSynchronize");
    if (st & cdg::ST_TIMEOUT)
        return fail(CDUGKS_ERR_TIMEOUT, "a bounded device wait (tensor-copy barrier) gave up; that step is incomplete");
    if (st & cdg::ST_NONFINITE) return fail(CDUGKS_ERR_NONFINITE, "a conserved variable became non-finite");
    if (st & cdg::ST_NEGATIVE) return fail(CDUGKS_ERR_NEGATIVE, "density or internal energy became <= 0");
    return CDUGKS_OK;
}

static int fetch_cells(cdugks_t* h, double* out, int conserved) {
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!out) return fail(CDUGKS_ERR_INVALID, "null output");
    const Geo& g = h->g;
    double* io = reinterpret_cast<double*>(h->base + h->lay.io);
    cudaError_t e = cdg::launch_moments(g, reinterpret_cast<double*>(h->base + h->lay.W), io, conserved, h->stream);
    if (e) return cuda_fail(e, "moments kernel");
    if ((e = cudaMemcpyAsync(out, io, sizeof(double) * (2 + g.D) * g.Nc, cudaMemcpyDeviceToHost, h->stream)))
        return cuda_fail(e, "download moments");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "moments");
    return CDUGKS_OK;
}

int cdugks_moments(cdugks_t* h, double* out) { return fetch_cells(h, out, 0); }

int cdugks_stress_heat_flux(cdugks_t* h, double* out) {
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!out) return fail(CDUGKS_ERR_INVALID, "null output");
    const Geo& g = h->g;
    double* io = reinterpret_cast<double*>(h->base + h->lay.io);
    cudaError_t e;
    if (h->prec == CDUGKS_FP32) e = cdg::launch_stress_f32(g, dinst<float>(h), h->cur, io, h->stream);
    else e = cdg::launch_stress_f64(g, dinst<double>(h), h->cur, io, h->stream);
    if (e) return cuda_fail(e, "stress kernel");
    if ((e = cudaMemcpyAsync(out, io, sizeof(double) * (g.D * g.D + g.D) * g.Nc, cudaMemcpyDeviceToHost,
                             h->stream)))
        return cuda_fail(e, "download stress and heat flux");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "stress and heat flux");
    return CDUGKS_OK;
}
int cdugks_conserved(cdugks_t* h, double* out) { return fetch_cells(h, out, 1); }

int cdugks_distributions(cdugks_t* h, double* gout, double* bout) {
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!gout || !bout) return fail(CDUGKS_ERR_INVALID, "null output");
    const Geo& g = h->g;
    cudaError_t e;
    if (h->prec == CDUGKS_FP32) e = cdg::launch_finalise_f32(g, dinst<float>(h), h->cur, h->stream);
    else e = cdg::launch_finalise_f64(g, dinst<double>(h), h->cur, h->stream);
    if (e) return cuda_fail(e, "finalise kernel");
    const size_t n = (size_t)g.Nvp * g.Nc * 2;
    std::vector<unsigned char> host(n * h->elt);
    if ((e = cudaMemcpyAsync(host.data(), h->base + h->lay.phi[1 - h->cur], host.size(), cudaMemcpyDeviceToHost,
                             h->stream)))
        return cuda_fail(e, "download distributions");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "distributions");
    // layout marshalling only: [tile][cell][field][lane] -> [cell][velocity]
    for (long long c = 0; c < g.Nc; ++c)
        for (int i = 0; i < h->Nv; ++i) {
            const size_t ad = ((size_t)(i / VC) * g.Nc + c) * (2 * VC) + (i % VC);
            double gv, bv;
            if (h->prec == CDUGKS_FP32) {
                gv = reinterpret_cast<const float*>(host.data())[ad];
                bv = reinterpret_cast<const float*>(host.data())[ad + VC];
            } else {
                gv = reinterpret_cast<const double*>(host.data())[ad];
                bv = reinterpret_cast<const double*>(host.data())[ad + VC];
            }
            gout[(size_t)c * h->Nv + i] = gv;
            bout[(size_t)c * h->Nv + i] = bv;
        }
    return CDUGKS_OK;
}

int cdugks_cell_distributions(cdugks_t* h, const long long* cells, int n, double* gout, double* bout) {
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!cells || n < 0 || (n > 0 && (!gout || !bout))) return fail(CDUGKS_ERR_INVALID, "bad arguments");
    const Geo& g = h->g;
    for (int k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= g.Nc) return fail(CDUGKS_ERR_INVALID, "cell index out of range");
    cudaError_t e;
    if (h->prec == CDUGKS_FP32) e = cdg::launch_finalise_f32(g, dinst<float>(h), h->cur, h->stream);
    else e = cdg::launch_finalise_f64(g, dinst<double>(h), h->cur, h->stream);
    if (e) return cuda_fail(e, "finalise kernel");
    // one cell's chunks are 2*VC values every Nc*2*VC values: one strided copy per cell
    const size_t row = 2 * VC * h->elt, pitch = (size_t)g.Nc * row;
    std::vector<unsigned char> host((size_t)g.NVT * row);
    const unsigned char* src = h->base + h->lay.phi[1 - h->cur];
    for (int k = 0; k < n; ++k) {
        if ((e = cudaMemcpy2DAsync(host.data(), row, src + (size_t)cells[k] * row, pitch, row, (size_t)g.NVT,
                                   cudaMemcpyDeviceToHost, h->stream)))
            return cuda_fail(e, "download cell");
        if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "cell distributions");
        for (int i = 0; i < h->Nv; ++i) {
            const size_t ad = (size_t)(i / VC) * (2 * VC) + (i % VC);
            double gv, bv;
            if (h->prec == CDUGKS_FP32) {
                gv = reinterpret_cast<const float*>(host.data())[ad];
                bv = reinterpret_cast<const float*>(host.data())[ad + VC];
            } else {
                gv = reinterpret_cast<const double*>(host.data())[ad];
                bv = reinterpret_cast<const double*>(host.data())[ad + VC];
            }
            gout[(size_t)k * h->Nv + i] = gv;
            bout[(size_t)k * h->Nv + i] = bv;
        }
    }
    return CDUGKS_OK;
}

int cdugks_state_bytes(const cdugks_t* h, size_t* bytes) {
    if (!h || !bytes) return fail(CDUGKS_ERR_INVALID, "null argument");
    const Geo& g = h->g;
    const size_t nq = h->collision == CDUGKS_COLLISION_SHAKHOV ? (size_t)g.D : 0;   // the tracked heat flux
    *bytes = sizeof(StateHeader) + (size_t)g.Nvp * g.Nc * 2 * h->elt + sizeof(double) * (2 + g.D + nq) * g.Nc;
    return CDUGKS_OK;
}

int cdugks_get_state(cdugks_t* h, void* host, size_t bytes) {
    int rc = check_ready(h, true);
    if (rc) return rc;
    size_t need;
    cdugks_state_bytes(h, &need);
    if (!host || bytes < need) return fail(CDUGKS_ERR_INVALID, "state buffer too small");
    const Geo& g = h->g;
    StateHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "CDUGKS1", 8);
    hd.dim = g.D;
    hd.prec = h->prec;
    hd.Nvp = g.Nvp;
    hd.Nc = g.Nc;
    hd.steps = h->steps;
    hd.dt = g.dt;
    hd.collision = h->collision;
    unsigned char* p = static_cast<unsigned char*>(host);
    std::memcpy(p, &hd, sizeof(hd));
    const size_t sb = (size_t)g.Nvp * g.Nc * 2 * h->elt;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(p + sizeof(hd), h->base + h->lay.phi[h->cur], sb, cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaMemcpyAsync(p + sizeof(hd) + sb, h->base + h->lay.W, sizeof(double) * (2 + g.D) * g.Nc,
                             cudaMemcpyDeviceToHost, h->stream)))
        return cuda_fail(e, "download state");
    if (h->collision == CDUGKS_COLLISION_SHAKHOV &&
        (e = cudaMemcpyAsync(p + sizeof(hd) + sb + sizeof(double) * (2 + g.D) * g.Nc, h->base + h->lay.hq,
                             sizeof(double) * g.D * g.Nc, cudaMemcpyDeviceToHost, h->stream)))
        return cuda_fail(e, "download heat flux");
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "get_state");
    return CDUGKS_OK;
}

int cdugks_set_state(cdugks_t* h, const void* host, size_t bytes) {
    int rc = check_ready(h, false);
    if (rc) return rc;
    size_t need;
    cdugks_state_bytes(h, &need);
    if (!host || bytes < need) return fail(CDUGKS_ERR_INVALID, "state buffer too small");
    const Geo& g = h->g;
    StateHeader hd;
    std::memcpy(&hd, host, sizeof(hd));
    if (std::memcmp(hd.magic, "CDUGKS1", 8) || hd.dim != g.D || hd.prec != h->prec || hd.Nvp != g.Nvp ||
        hd.Nc != g.Nc || hd.dt != g.dt || hd.collision != h->collision)
        return fail(CDUGKS_ERR_INVALID, "state image does not match this problem");
    const unsigned char* p = static_cast<const unsigned char*>(host);
    const size_t sb = (size_t)g.Nvp * g.Nc * 2 * h->elt;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->base + h->lay.phi[0], p + sizeof(hd), sb, cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaMemcpyAsync(h->base + h->lay.W, p + sizeof(hd) + sb, sizeof(double) * (2 + g.D) * g.Nc,
                             cudaMemcpyHostToDevice, h->stream)))
        return cuda_fail(e, "upload state");
    if (h->collision == CDUGKS_COLLISION_SHAKHOV &&
        (e = cudaMemcpyAsync(h->base + h->lay.hq, p + sizeof(hd) + sb + sizeof(double) * (2 + g.D) * g.Nc,
                             sizeof(double) * g.D * g.Nc, cudaMemcpyHostToDevice, h->stream)))
        return cuda_fail(e, "upload heat flux");
    h->cur = 0;
    if (h->prec == CDUGKS_FP32) e = cdg::launch_cellc_f32(g, dinst<float>(h), 0, h->stream);
    else e = cdg::launch_cellc_f64(g, dinst<double>(h), 0, h->stream);
    if (e) return cuda_fail(e, "cell constants");
    if (!h->initialised) {
        // Dirichlet ghost constants: the restored state stands in for the initial one
        if ((e = cudaMemcpyAsync(h->base + h->lay.cellc0, h->base + h->lay.cellc, h->cellc_bytes * g.Nc,
                                 cudaMemcpyDeviceToDevice, h->stream)))
            return cuda_fail(e, "copy constants");
        if ((h->bufs_cap & BUF_XTAB) &&
            (e = cudaMemcpyAsync(h->base + h->lay.xc0, h->base + h->lay.xc, h->elt * (size_t)g.xrows * g.Nc,
                                 cudaMemcpyDeviceToDevice, h->stream)))
            return cuda_fail(e, "copy factor tables");
    }
    if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "set_state");
    h->steps = hd.steps;
    h->initialised = true;
    return CDUGKS_OK;
}

int cdugks_info(const cdugks_t* h, cdugks_info_t* info) {
    if (!h || !info) return fail(CDUGKS_ERR_INVALID, "null argument");
    info->dim = h->g.D;
    info->ncells = h->g.Nc;
    info->nvel = h->Nv;
    info->nvel_padded = h->g.Nvp;
    info->dt = h->g.dt;
    info->steps = h->steps;
    info->precision = h->prec;
    info->velocity_groups = h->g.G;
    info->tile_id = h->g.tile_id;
    {
        const cdg::TileShape ts = tile_of(h->prec, h->g.D, h->g.tile_id);
        for (int a = 0; a < 3; ++a) info->tile[a] = ts.t[a];
    }
    info->state_bytes = (double)h->g.Nvp * (double)h->g.Nc * 2.0 * (double)h->elt;
    return CDUGKS_OK;
}

void cdugks_destroy(cdugks_t* h) {
    if (!h) return;
    drop_graphs(h);
    delete h;
}

const char* cdugks_strerror(int code) {
    switch (code) {
        case CDUGKS_OK: return "ok";
        case CDUGKS_ERR_INVALID: return "invalid argument";
        case CDUGKS_ERR_OOM: return "workspace too small";
        case CDUGKS_ERR_CUDA: return "CUDA error";
        case CDUGKS_ERR_NONFINITE: return "non-finite conserved variable";
        case CDUGKS_ERR_TIMEOUT: return "device wait timed out";
        case CDUGKS_ERR_UNBOUND: return "workspace not bound or state not initialised";
        case CDUGKS_ERR_NEGATIVE: return "non-positive density or temperature";
        default: return "unknown error";
    }
}

const char* cdugks_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------ batches

}  // extern "C"

struct cdugks_batch {
    std::vector<cdugks*> mem;
    int prec, D;
    std::vector<int> tile_ids;                 // distinct tile shapes, in plan order
    std::vector<std::vector<Item>> sweep_items;
    std::vector<RItem> face_items, cell_items;
    std::vector<RItem> prep_items;             // acceleration members: the pre-pass
    std::vector<QItem> faceq_items, cellq_items;   // Shakhov members: raw moments
    std::vector<unsigned char> insts;          // host image of the Inst<T> table
    std::vector<int> cur;
    size_t off_insts, off_cur, off_sweep[cdg::kMaxBatchShapes], off_face, off_cell, total;
    size_t off_prep, off_faceq, off_cellq;
    unsigned char* base;
    cudaStream_t stream;
    bool bound;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_steps;
    long long steps;
    // the persistent step (cdugks_batch_set_persistent): one launch per call or graph
    bool pers;
    int pcap_mem;                              // members and items per step the workspace holds
    long long pcap_items;
    std::vector<PItem> pitems;
    std::vector<int> pper;                     // [member][4] items of each kind per step
    size_t off_phead, off_pitems, off_pstate;
    int wait_log2, test_hook;
};

namespace {

template <typename T>
void fill_insts(cdugks_batch* b) {
    b->insts.assign(sizeof(Inst<T>) * b->mem.size(), 0);
    Inst<T>* in = reinterpret_cast<Inst<T>*>(b->insts.data());
    for (size_t i = 0; i < b->mem.size(); ++i) {
        in[i].g = b->mem[i]->g;
        in[i].b[0] = bufs<T>(b->mem[i], 0);
        in[i].b[1] = bufs<T>(b->mem[i], 1);
    }
}

BatchPlan plan_of(const cdugks_batch* b) {
    BatchPlan p;
    std::memset(&p, 0, sizeof(p));
    p.D = b->D;
    p.ntile = (int)b->tile_ids.size();
    for (int k = 0; k < p.ntile; ++k) {
        p.tile_id[k] = b->tile_ids[k];
        p.sweep_items[k] = reinterpret_cast<const Item*>(b->base + b->off_sweep[k]);
        p.n_sweep[k] = (int)b->sweep_items[k].size();
    }
    p.face_items = reinterpret_cast<const RItem*>(b->base + b->off_face);
    p.n_face = (int)b->face_items.size();
    p.cell_items = reinterpret_cast<const RItem*>(b->base + b->off_cell);
    p.n_cell = (int)b->cell_items.size();
    p.prep_items = reinterpret_cast<const RItem*>(b->base + b->off_prep);
    p.n_prep = (int)b->prep_items.size();
    p.faceq_items = reinterpret_cast<const QItem*>(b->base + b->off_faceq);
    p.n_faceq = (int)b->faceq_items.size();
    p.cellq_items = reinterpret_cast<const QItem*>(b->base + b->off_cellq);
    p.n_cellq = (int)b->cellq_items.size();
    return p;
}

// nsteps persistent steps in one launch (the counters are cleared first).
cudaError_t batch_persist_launch(cdugks_batch* b, int nsteps) {
    const PHead* h = reinterpret_cast<const PHead*>(b->base + b->off_phead);
    const PItem* it = reinterpret_cast<const PItem*>(b->base + b->off_pitems);
    PState* st = reinterpret_cast<PState*>(b->base + b->off_pstate);
    int* cur = reinterpret_cast<int*>(b->base + b->off_cur);
    const int tile = b->tile_ids[0];
    if (b->prec == CDUGKS_FP32)
        return cdg::launch_batch_persist_f32(b->D, tile, h, it, reinterpret_cast<const Inst<float>*>(b->base + b->off_insts),
                                             cur, st, nsteps, b->wait_log2, b->test_hook, b->stream);
    return cdg::launch_batch_persist_f64(b->D, tile, h, it, reinterpret_cast<const Inst<double>*>(b->base + b->off_insts),
                                         cur, st, nsteps, b->wait_log2, b->test_hook, b->stream);
}

cudaError_t batch_launch(cdugks_batch* b) {
    if (b->pers) return batch_persist_launch(b, 1);
    const BatchPlan p = plan_of(b);
    int* cur = reinterpret_cast<int*>(b->base + b->off_cur);
    if (b->prec == CDUGKS_FP32)
        return cdg::launch_batch_step_f32(p, reinterpret_cast<const Inst<float>*>(b->base + b->off_insts), cur,
                                          b->stream);
    return cdg::launch_batch_step_f64(p, reinterpret_cast<const Inst<double>*>(b->base + b->off_insts), cur,
                                      b->stream);
}

void batch_advance_host(cdugks_batch* b, int nsteps) {
    for (cdugks* m : b->mem) {
        m->cur ^= (nsteps & 1);
        m->steps += nsteps;
    }
    b->steps += nsteps;
}

void batch_drop_graph(cdugks_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_steps = 0;
}

// A handle that may join a batch of this precision and dimension.
int batch_member_ok(const cdugks* m, int prec, int D) {
    if (!m || !m->bound || !m->initialised) return fail(CDUGKS_ERR_UNBOUND, "every member must be bound and initialised");
    if (m->prec != prec || m->g.D != D) return fail(CDUGKS_ERR_INVALID, "members must share precision and dim");
    const int mode = tile_mode(m->prec, m->g.D, m->g.tile_id);
    if (cdg::mode_source(mode) != cdg::MODE_FUSED && !cdg::mode_acc(mode))
        return fail(CDUGKS_ERR_INVALID, "prepared and stored tile shapes are not batched; choose another shape");
    return CDUGKS_OK;
}

// Before the membership changes: finish the work in flight on the batch stream
// (the members' state must be final) and drop the binding and the graph.
int batch_unbind(cdugks_batch* b) {
    if (b->bound && b->stream) {
        const cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e) return cuda_fail(e, "batch sync before a membership change");
    }
    batch_drop_graph(b);
    b->bound = false;
    b->base = nullptr;
    return CDUGKS_OK;
}

// Work lists and workspace layout of the current members: sweep items grouped
// by tile shape (largest per-item work first), face and cell ranges, the
// instance table.
int batch_plan(cdugks_batch* b) {
    const int n = (int)b->mem.size(), D = b->D;
    b->tile_ids.clear();
    for (int i = 0; i < n; ++i) {
        const int id = b->mem[i]->g.tile_id;
        if (std::find(b->tile_ids.begin(), b->tile_ids.end(), id) == b->tile_ids.end()) b->tile_ids.push_back(id);
    }
    std::sort(b->tile_ids.begin(), b->tile_ids.end());
    if (b->tile_ids.size() > (size_t)cdg::kMaxBatchShapes)     // before any per-shape table is filled
        return fail(CDUGKS_ERR_INVALID, "too many tile shapes in one batch");
    b->sweep_items.assign(b->tile_ids.size(), {});
    for (int i = 0; i < n; ++i) {
        const Geo& g = b->mem[i]->g;
        const int k = (int)(std::find(b->tile_ids.begin(), b->tile_ids.end(), g.tile_id) - b->tile_ids.begin());
        const int tiles = g.tiles[0] * g.tiles[1] * g.tiles[2];
        for (int t = 0; t < tiles; ++t)
            for (int gr = 0; gr < g.G; ++gr) b->sweep_items[k].push_back(Item{i, t, gr, 0});
    }
    for (auto& v : b->sweep_items)
        std::stable_sort(v.begin(), v.end(), [&](const Item& x, const Item& y) {
            const Geo& gx = b->mem[x.inst]->g;
            const Geo& gy = b->mem[y.inst]->g;
            const int wx = std::min(gx.ntpg, gx.NVT - x.grp * gx.ntpg), wy = std::min(gy.ntpg, gy.NVT - y.grp * gy.ntpg);
            return wx > wy;
        });
    // face and cell ranges: whole blocks of the kernel that runs them (64 threads,
    // or the persistent shape's threads), sized so that the batch has about 2048
    // of each (a few ranges of a lone member would leave most SMs idle while
    // each thread loops over FP64 work; many members need no smaller ones)
    long long unit = 64;
    if (b->pers) {
        const cdg::TileShape ts = tile_of(b->prec, D, b->tile_ids[0]);
        unit = (long long)ts.t[0] * ts.t[1] * ts.t[2];
    }
    long long tot_f = 0, tot_c = 0;
    for (int i = 0; i < n; ++i) {
        const Geo& g = b->mem[i]->g;
        for (int a = 0; a < D; ++a) tot_f += g.nf[a];
        tot_c += g.Nc;
    }
    auto range_size = [&](long long tot) {
        const long long r = (tot / 2048 + unit - 1) / unit * unit;
        return std::max(unit, std::min(r, std::max(unit, 1024 / unit * unit)));
    };
    const long long RF = range_size(tot_f), RC = range_size(tot_c);
    b->face_items.clear();
    b->cell_items.clear();
    for (int i = 0; i < n; ++i) {
        const Geo& g = b->mem[i]->g;
        for (int a = 0; a < D; ++a)
            for (long long s0 = 0; s0 < g.nf[a]; s0 += RF)
                b->face_items.push_back(RItem{i, a, s0, std::min(RF, g.nf[a] - s0)});
        for (long long s0 = 0; s0 < g.Nc; s0 += RC) b->cell_items.push_back(RItem{i, 0, s0, std::min(RC, g.Nc - s0)});
    }
    // the pre-pass of acceleration members (cells x runs of chunks) and the raw
    // moments of Shakhov members (ranges x velocity groups), by member
    b->prep_items.clear();
    b->faceq_items.clear();
    b->cellq_items.clear();
    const long long RP = cdg::kPrepCells, RQ = 512;
    for (int i = 0; i < n; ++i) {
        const Geo& g = b->mem[i]->g;
        if (g.accel) {
            const int runs = (g.NVT + cdg::kPrepChunks - 1) / cdg::kPrepChunks;
            for (int r = 0; r < runs; ++r)
                for (long long s0 = 0; s0 < g.Nc; s0 += RP) b->prep_items.push_back(RItem{i, r, s0, std::min(RP, g.Nc - s0)});
        }
        if (g.shakhov) {
            for (int gr = 0; gr < g.G; ++gr) {
                for (int a = 0; a < D; ++a)
                    for (long long s0 = 0; s0 < g.nf[a]; s0 += RQ)
                        b->faceq_items.push_back(QItem{i, a, gr, 0, s0, std::min(RQ, g.nf[a] - s0)});
                for (long long s0 = 0; s0 < g.Nc; s0 += RQ)
                    b->cellq_items.push_back(QItem{i, -1, gr, 0, s0, std::min(RQ, g.Nc - s0)});
            }
        }
    }
    if (b->prec == CDUGKS_FP32) fill_insts<float>(b);
    else fill_insts<double>(b);
    b->cur.assign(n, 0);
    if (b->pers) {
        // one list per step: every member's sweep A items, then the face, sweep B and W items
        if (b->tile_ids.size() != 1) return fail(CDUGKS_ERR_INVALID, "a persistent batch needs one tile shape");
        b->pitems.clear();
        b->pper.assign((size_t)n * 4, 0);
        for (const Item& x : b->sweep_items[0]) {
            b->pitems.push_back(PItem{x.inst, cdg::PK_A, x.tile, x.grp, 0, 0});
            ++b->pper[(size_t)x.inst * 4 + cdg::PK_A];
        }
        for (const RItem& x : b->face_items) {
            b->pitems.push_back(PItem{x.inst, cdg::PK_F, x.axis, 0, x.start, x.count});
            ++b->pper[(size_t)x.inst * 4 + cdg::PK_F];
        }
        for (const Item& x : b->sweep_items[0]) {
            b->pitems.push_back(PItem{x.inst, cdg::PK_B, x.tile, x.grp, 0, 0});
            ++b->pper[(size_t)x.inst * 4 + cdg::PK_B];
        }
        for (const RItem& x : b->cell_items) {
            b->pitems.push_back(PItem{x.inst, cdg::PK_W, 0, 0, x.start, x.count});
            ++b->pper[(size_t)x.inst * 4 + cdg::PK_W];
        }
        if (n > cdg::kPMaxMembers) return fail(CDUGKS_ERR_INVALID, "too many members for a persistent batch");
        if (n > b->pcap_mem || (long long)b->pitems.size() > b->pcap_items) {
            // bound (an in-place rewrite): no room; unbound: grow the reservation
            if (b->bound) return fail(CDUGKS_ERR_INVALID, "the persistent batch holds more members or items than reserved");
            b->pcap_mem = std::max(b->pcap_mem, n);
            b->pcap_items = std::max(b->pcap_items, (long long)b->pitems.size());
        }
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    if (b->pers) {
        // room for the reserved member and item capacity, at offsets that do not
        // depend on the members: a membership change rewrites the tables in place
        const size_t inst_bytes = b->prec == CDUGKS_FP32 ? sizeof(Inst<float>) : sizeof(Inst<double>);
        b->off_insts = take(inst_bytes * (size_t)b->pcap_mem);
        b->off_cur = take(sizeof(int) * (size_t)b->pcap_mem);
        b->off_phead = take(sizeof(PHead));
        b->off_pitems = take(sizeof(PItem) * (size_t)b->pcap_items);
        b->off_pstate = take(sizeof(PState));
        b->total = off;
        return CDUGKS_OK;
    }
    b->off_insts = take(b->insts.size());
    b->off_cur = take(sizeof(int) * n);
    for (size_t k = 0; k < b->sweep_items.size(); ++k) b->off_sweep[k] = take(sizeof(Item) * b->sweep_items[k].size());
    b->off_face = take(sizeof(RItem) * b->face_items.size());
    b->off_cell = take(sizeof(RItem) * b->cell_items.size());
    b->off_prep = take(sizeof(RItem) * b->prep_items.size());
    b->off_faceq = take(sizeof(QItem) * b->faceq_items.size());
    b->off_cellq = take(sizeof(QItem) * b->cellq_items.size());
    b->total = off;
    return CDUGKS_OK;
}

// The persistent plan's device tables (instance table, parities, head, items).
cudaError_t batch_upload_persist(cdugks_batch* b) {
    PHead* hd = new (std::nothrow) PHead;
    if (!hd) return cudaErrorMemoryAllocation;
    std::memset(hd, 0, sizeof(PHead));
    hd->nmem = (int)b->mem.size();
    hd->nitems = (int)b->pitems.size();
    for (size_t m = 0; m < b->mem.size(); ++m)
        for (int k = 0; k < 4; ++k) hd->per[m][k] = b->pper[m * 4 + k];
    cudaError_t e = cudaMemcpyAsync(b->base + b->off_phead, hd, sizeof(PHead), cudaMemcpyHostToDevice, b->stream);
    if (!e) e = cudaMemcpyAsync(b->base + b->off_pitems, b->pitems.data(), sizeof(PItem) * b->pitems.size(),
                                cudaMemcpyHostToDevice, b->stream);
    if (!e) e = cudaStreamSynchronize(b->stream);      // (the host copies are pageable: staged before return)
    delete hd;
    return e;
}

// A persistent batch that is bound: rewrite its device tables for the current
// members in place (the binding and any captured graph stay valid).
int batch_rewrite_in_place(cdugks_batch* b) {
    cudaError_t e;
    for (size_t i = 0; i < b->mem.size(); ++i) b->cur[i] = b->mem[i]->cur;
    if ((e = cudaMemcpyAsync(b->base + b->off_insts, b->insts.data(), b->insts.size(), cudaMemcpyHostToDevice,
                             b->stream)) ||
        (e = cudaMemcpyAsync(b->base + b->off_cur, b->cur.data(), sizeof(int) * b->cur.size(), cudaMemcpyHostToDevice,
                             b->stream)) ||
        (e = batch_upload_persist(b)))
        return cuda_fail(e, "rewrite persistent plan");
    return CDUGKS_OK;
}

}  // namespace

extern "C" {

int cdugks_batch_create(cdugks_t* const* members, int n, cdugks_batch_t** out) {
    if (!out) return fail(CDUGKS_ERR_INVALID, "null output pointer");
    *out = nullptr;
    if (!members || n < 1) return fail(CDUGKS_ERR_INVALID, "a batch needs at least one member");
    const int prec = members[0] ? members[0]->prec : -1, D = members[0] ? members[0]->g.D : -1;
    for (int i = 0; i < n; ++i) {
        const int rc = batch_member_ok(members[i], prec, D);
        if (rc) return rc;
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return fail(CDUGKS_ERR_INVALID, "a member appears twice");
    }
    cdugks_batch* b = new (std::nothrow) cdugks_batch();
    if (!b) return fail(CDUGKS_ERR_OOM, "host allocation failed");
    b->mem.assign(members, members + n);
    b->prec = prec;
    b->D = D;
    const int rc = batch_plan(b);
    if (rc) {
        delete b;
        return rc;
    }
    *out = b;
    return CDUGKS_OK;
}

int cdugks_batch_admit(cdugks_batch_t* b, cdugks_t* member) {
    if (!b) return fail(CDUGKS_ERR_INVALID, "null batch");
    int rc = batch_member_ok(member, b->prec, b->D);
    if (rc) return rc;
    if (std::find(b->mem.begin(), b->mem.end(), member) != b->mem.end())
        return fail(CDUGKS_ERR_INVALID, "already a member");
    const cudaError_t e = cudaStreamSynchronize(member->stream);   // its own work lands before the batch's
    if (e) return cuda_fail(e, "member sync before admission");
    if (b->pers && b->bound && b->tile_ids.size() == 1 && member->g.tile_id == b->tile_ids[0]) {
        // a persistent batch rewrites its tables in place if they fit
        const cudaError_t e2 = cudaStreamSynchronize(b->stream);
        if (e2) return cuda_fail(e2, "batch sync before admission");
        b->mem.push_back(member);
        if (batch_plan(b) == CDUGKS_OK) return batch_rewrite_in_place(b);
        b->mem.pop_back();
        batch_plan(b);
    }
    if ((rc = batch_unbind(b))) return rc;
    b->mem.push_back(member);
    if ((rc = batch_plan(b))) {
        b->mem.pop_back();
        batch_plan(b);
        return rc;
    }
    return CDUGKS_OK;
}

int cdugks_batch_retire(cdugks_batch_t* b, cdugks_t* member) {
    if (!b || !member) return fail(CDUGKS_ERR_INVALID, "null argument");
    const auto it = std::find(b->mem.begin(), b->mem.end(), member);
    if (it == b->mem.end()) return fail(CDUGKS_ERR_INVALID, "not a member");
    if (b->mem.size() == 1) return fail(CDUGKS_ERR_INVALID, "a batch needs at least one member");
    if (b->pers && b->bound) {
        // a persistent batch rewrites its tables in place
        const cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e) return cuda_fail(e, "batch sync before retirement");
        b->mem.erase(it);
        const int rc = batch_plan(b);
        if (rc) return rc;
        return batch_rewrite_in_place(b);
    }
    int rc = batch_unbind(b);
    if (rc) return rc;
    b->mem.erase(it);
    return batch_plan(b);
}

int cdugks_batch_workspace_bytes(const cdugks_batch_t* b, size_t* bytes) {
    if (!b || !bytes) return fail(CDUGKS_ERR_INVALID, "null argument");
    *bytes = b->total;
    return CDUGKS_OK;
}

int cdugks_batch_bind(cdugks_batch_t* b, void* device_ptr, size_t bytes, void* cuda_stream) {
    if (!b || !device_ptr) return fail(CDUGKS_ERR_INVALID, "null argument");
    if (((uintptr_t)device_ptr) % kAlign) return fail(CDUGKS_ERR_INVALID, "workspace must be 256-byte aligned");
    if (bytes < b->total) return fail(CDUGKS_ERR_OOM, "workspace smaller than cdugks_batch_workspace_bytes");
    batch_drop_graph(b);
    b->base = static_cast<unsigned char*>(device_ptr);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    for (size_t i = 0; i < b->mem.size(); ++i) b->cur[i] = b->mem[i]->cur;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->base + b->off_insts, b->insts.data(), b->insts.size(), cudaMemcpyHostToDevice,
                             b->stream)) ||
        (e = cudaMemcpyAsync(b->base + b->off_cur, b->cur.data(), sizeof(int) * b->cur.size(),
                             cudaMemcpyHostToDevice, b->stream)))
        return cuda_fail(e, "upload batch tables");
    for (size_t k = 0; k < b->sweep_items.size() && !b->pers; ++k)
        if ((e = cudaMemcpyAsync(b->base + b->off_sweep[k], b->sweep_items[k].data(),
                                 sizeof(Item) * b->sweep_items[k].size(), cudaMemcpyHostToDevice, b->stream)))
            return cuda_fail(e, "upload sweep items");
    if (!b->pers &&
        ((e = cudaMemcpyAsync(b->base + b->off_face, b->face_items.data(), sizeof(RItem) * b->face_items.size(),
                              cudaMemcpyHostToDevice, b->stream)) ||
         (e = cudaMemcpyAsync(b->base + b->off_cell, b->cell_items.data(), sizeof(RItem) * b->cell_items.size(),
                              cudaMemcpyHostToDevice, b->stream)) ||
         (!b->prep_items.empty() &&
          (e = cudaMemcpyAsync(b->base + b->off_prep, b->prep_items.data(), sizeof(RItem) * b->prep_items.size(),
                               cudaMemcpyHostToDevice, b->stream))) ||
         (!b->faceq_items.empty() &&
          (e = cudaMemcpyAsync(b->base + b->off_faceq, b->faceq_items.data(), sizeof(QItem) * b->faceq_items.size(),
                               cudaMemcpyHostToDevice, b->stream))) ||
         (!b->cellq_items.empty() &&
          (e = cudaMemcpyAsync(b->base + b->off_cellq, b->cellq_items.data(), sizeof(QItem) * b->cellq_items.size(),
                               cudaMemcpyHostToDevice, b->stream)))))
        return cuda_fail(e, "upload range items");
    if (b->pers && (e = batch_upload_persist(b))) return cuda_fail(e, "upload persistent plan");
    // members' own streams may still be working on their state
    for (cdugks* m : b->mem)
        if ((e = cudaStreamSynchronize(m->stream))) return cuda_fail(e, "member stream");
    if ((e = cudaStreamSynchronize(b->stream))) return cuda_fail(e, "batch bind");
    b->bound = true;
    return CDUGKS_OK;
}


int cdugks_batch_capture(cdugks_batch_t* b, int steps_per_graph) {
    if (!b || !b->bound) return fail(CDUGKS_ERR_UNBOUND, "batch not bound");
    if (steps_per_graph < 0 || steps_per_graph > 4096) return fail(CDUGKS_ERR_INVALID, "steps_per_graph in [0, 4096]");
    batch_drop_graph(b);
    if (steps_per_graph == 0) return CDUGKS_OK;
    if (!b->stream) return fail(CDUGKS_ERR_INVALID, "graph capture needs a non-default stream");
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e) return cuda_fail(e, "cudaStreamBeginCapture");
    if (b->pers) e = batch_persist_launch(b, steps_per_graph);
    else
        for (int s = 0; s < steps_per_graph && e == cudaSuccess; ++s) e = batch_launch(b);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e || e2) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e ? e : e2, "capture batch steps");
    }
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaGraphInstantiate(&exec, graph, 0))) {
        cudaGraphDestroy(graph);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    b->graph = graph;
    b->exec = exec;
    b->graph_steps = steps_per_graph;
    return CDUGKS_OK;
}

int cdugks_batch_step(cdugks_batch_t* b, int nsteps) {
    if (!b || !b->bound) return fail(CDUGKS_ERR_UNBOUND, "batch not bound");
    if (nsteps < 0) return fail(CDUGKS_ERR_INVALID, "nsteps < 0");
    int done = 0;
    cudaError_t e = cudaSuccess;
    if (b->exec)
        for (; done + b->graph_steps <= nsteps; done += b->graph_steps)
            if ((e = cudaGraphLaunch(b->exec, b->stream))) return cuda_fail(e, "cudaGraphLaunch");
    if (b->pers && done < nsteps) {
        if ((e = batch_persist_launch(b, nsteps - done))) return cuda_fail(e, "persistent batch step launch");
        done = nsteps;
    }
    for (; done < nsteps; ++done)
        if ((e = batch_launch(b))) return cuda_fail(e, "batch step launch");
    batch_advance_host(b, nsteps);
    return CDUGKS_OK;
}

int cdugks_batch_set_persistent(cdugks_batch_t* b, int on, int max_members, long long max_items) {
    if (!b) return fail(CDUGKS_ERR_INVALID, "null batch");
    int rc = batch_unbind(b);
    if (rc) return rc;
    if (on) {
        if (b->tile_ids.size() != 1) return fail(CDUGKS_ERR_INVALID, "a persistent batch needs one tile shape");
        const bool ok = b->prec == CDUGKS_FP32 ? cdg::batch_persistent_f32(b->D, b->tile_ids[0])
                                               : cdg::batch_persistent_f64(b->D, b->tile_ids[0]);
        if (!ok) return fail(CDUGKS_ERR_INVALID, "this tile shape has no persistent batched step");
        const int pcap = std::max((int)b->mem.size(), max_members);
        if (pcap > cdg::kPMaxMembers) return fail(CDUGKS_ERR_INVALID, "too many members for a persistent batch");
        b->pers = true;
        b->pcap_mem = pcap;
        b->pcap_items = (long long)1 << 40;           // first the current list, then its size sets the room
        b->wait_log2 = b->wait_log2 ? b->wait_log2 : 26;
        rc = batch_plan(b);
        if (rc == CDUGKS_OK) {
            b->pcap_items = std::max((long long)b->pitems.size(), max_items);
            rc = batch_plan(b);
        }
        if (rc) {
            b->pers = false;
            batch_plan(b);
        }
        return rc;
    }
    b->pers = false;
    return batch_plan(b);
}

int cdugks_batch_bound(const cdugks_batch_t* b) { return b && b->bound ? 1 : 0; }

int cdugks_batch_step_members(cdugks_batch_t* b, const int* steps, int n) {
    if (!b || !b->bound) return fail(CDUGKS_ERR_UNBOUND, "batch not bound");
    if (!b->pers) return fail(CDUGKS_ERR_INVALID, "per-member step counts need the persistent step");
    if (!steps || n != (int)b->mem.size()) return fail(CDUGKS_ERR_INVALID, "one step count per member");
    int mx = 0;
    for (int i = 0; i < n; ++i) {
        if (steps[i] < 0) return fail(CDUGKS_ERR_INVALID, "negative step count");
        mx = std::max(mx, steps[i]);
    }
    if (mx == 0) return CDUGKS_OK;
    // the limits, then the launch, then limits off again (all stream-ordered; the
    // host copies are pageable, so they are staged before each call returns)
    PHead* h = reinterpret_cast<PHead*>(b->base + b->off_phead);
    const int on = 1, off = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->lim, steps, sizeof(int) * n, cudaMemcpyHostToDevice, b->stream)) ||
        (e = cudaMemcpyAsync(&h->use_lim, &on, sizeof(int), cudaMemcpyHostToDevice, b->stream)) ||
        (e = batch_persist_launch(b, mx)) ||
        (e = cudaMemcpyAsync(&h->use_lim, &off, sizeof(int), cudaMemcpyHostToDevice, b->stream)))
        return cuda_fail(e, "per-member batch step");
    for (int i = 0; i < n; ++i) {
        b->mem[i]->cur ^= (steps[i] & 1);
        b->mem[i]->steps += steps[i];
    }
    b->steps += mx;
    return CDUGKS_OK;
}

int cdugks_batch_test_wait_timeout(cdugks_batch_t* b, int on) {
    if (!b) return fail(CDUGKS_ERR_INVALID, "null batch");
    batch_drop_graph(b);
    b->test_hook = on ? 1 : 0;
    b->wait_log2 = on ? 12 : 26;
    return CDUGKS_OK;
}

int cdugks_batch_sync(cdugks_batch_t* b) {
    if (!b || !b->bound) return fail(CDUGKS_ERR_UNBOUND, "batch not bound");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e) return cuda_fail(e, "batch sync");
    int worst = CDUGKS_OK;
    for (cdugks* m : b->mem) {
        const int rc = cdugks_sync_status(m);
        if (rc != CDUGKS_OK && worst == CDUGKS_OK) worst = rc;
    }
    return worst;
}

void cdugks_batch_destroy(cdugks_batch_t* b) {
    if (!b) return;
    batch_drop_graph(b);
    delete b;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free step.  Some callers cannot allocate device memory: code that
// runs inside a host framework whose memory pool owns all of the GPU and only
// lends out buffers it already holds, or a latency-critical loop in which a
// device allocation (which may synchronise the whole device, or fail once the
// pool is fragmented) is not acceptable.  For them cdugks_step_noalloc takes
// the state buffers from the caller and keeps every other piece of device
// scratch (cell and face constants, face-moment partial sums, velocity
// tables, status word) in the fixed array below.  The array lives in every
// process that loads this library, on every GPU it touches, until exit.
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kNoallocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices];

// Device address of the scratch array on the current device.  In host code the
// symbol is only a stand-in; its device address is looked up once per device,
// with that device current, and cached.
int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(CDUGKS_ERR_INVALID, "device index too large");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return CDUGKS_OK;
}

template <typename T>
int noalloc_run(cdugks* h, const void* phi_in, void* phi_out, double* W, cudaStream_t st) {
    Geo g = h->g;
    if (h->recon != CDUGKS_RECON_UPWIND_CELL)
        return fail(CDUGKS_ERR_INVALID, "the allocation-free step implements the upwind-cell reconstruction only");
    if (tile_mode(h->prec, g.D, g.tile_id) != cdg::MODE_FUSED) {   // no room for phibar+ / slope / face buffers here
        g.tile_id = 0;
        const cdg::TileShape ts = tile_of(h->prec, g.D, 0);
        for (int a = 0; a < 3; ++a) g.tiles[a] = a < g.D ? (g.n[a] + ts.t[a] - 1) / ts.t[a] : 1;
    }
    const int NM = 2 + g.D;
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(reinterpret_cast<void**>(&base));
    if (rc) return rc;
    // scratch layout; fewer velocity groups when the partial sums would not fit
    size_t need = 0, off_cellc = 0, off_facec[3] = {0, 0, 0}, off_wf[3] = {0, 0, 0}, off_mf[3] = {0, 0, 0};
    size_t off_vel = 0, off_refl = 0, off_status = 0, off_inst = 0;
    for (int G = std::max(1, g.G);; G = std::max(1, G / 2)) {
        g.ntpg = (g.NVT + G - 1) / G;
        g.G = (g.NVT + g.ntpg - 1) / g.ntpg;
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t o = off;
            off = align_up(off + bytes);
            return o;
        };
        off_cellc = take(h->cellc_bytes * (size_t)g.Nc);
        for (int a = 0; a < 3; ++a) {
            const size_t nf = a < g.D ? (size_t)g.nf[a] : 0;
            off_facec[a] = take(h->facec_bytes * nf);
            off_wf[a] = take(sizeof(double) * (size_t)g.G * NM * nf);
            off_mf[a] = take(sizeof(double) * (size_t)g.G * NM * nf);
        }
        off_vel = take(sizeof(T) * 8 * (size_t)g.Nvp);
        off_refl = take(sizeof(int) * 8 * (size_t)g.Nvp);
        off_status = take(256);
        off_inst = take(sizeof(Inst<T>));
        need = off;
        if (need <= kNoallocScratchBytes || G == 1) break;
    }
    if (need > kNoallocScratchBytes) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "problem needs %zu bytes of scratch; the allocation-free step has %zu (use cdugks_step)", need,
                      kNoallocScratchBytes);
        return fail(CDUGKS_ERR_INVALID, msg);
    }
    Bufs<T> b;
    std::memset(&b, 0, sizeof(b));      // no optional buffers (factor tables, Shakhov, force) on this path
    b.phi_in = static_cast<const T*>(phi_in);
    b.phi_out = static_cast<T*>(phi_out);
    b.phibar = nullptr;
    b.sigma = nullptr;
    for (int a = 0; a < 3; ++a) b.face[a] = nullptr;
    b.W = W;
    b.cellc = reinterpret_cast<CellC<T>*>(base + off_cellc);
    b.cellc0 = b.cellc;   // no Dirichlet ghosts on this path
    for (int a = 0; a < 3; ++a) {
        b.facec[a] = reinterpret_cast<FaceC<T>*>(base + off_facec[a]);
        b.wf[a] = reinterpret_cast<double*>(base + off_wf[a]);
        b.mf[a] = reinterpret_cast<double*>(base + off_mf[a]);
    }
    b.vel = reinterpret_cast<const T*>(base + off_vel);
    b.refl = reinterpret_cast<const int*>(base + off_refl);
    b.status = reinterpret_cast<int*>(base + off_status);
    // the array keeps whatever the last call left: reload the tables and the
    // instance record, clear the status word
    Inst<T> in;
    in.g = g;
    in.b[0] = b;
    in.b[1] = b;
    cudaError_t e;
    const void* vel = h->prec == CDUGKS_FP32 ? static_cast<const void*>(h->vel32.data())
                                             : static_cast<const void*>(h->vel.data());
    if ((e = cudaMemcpyAsync(base + off_vel, vel, sizeof(T) * 8 * (size_t)g.Nvp, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + off_refl, h->refl.data(), sizeof(int) * h->refl.size(), cudaMemcpyHostToDevice,
                             st)) ||
        (e = cudaMemsetAsync(base + off_status, 0, 256, st)) ||
        (e = cudaMemcpyAsync(base + off_inst, &in, sizeof(in), cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "prepare scratch");
    const Inst<T>* din = reinterpret_cast<const Inst<T>*>(base + off_inst);
    if constexpr (std::is_same<T, float>::value) {
        e = cdg::launch_cellc_f32(g, din, 0, st);
        if (!e) e = cdg::launch_step_f32(g, din, 0, st);
    } else {
        e = cdg::launch_cellc_f64(g, din, 0, st);
        if (!e) e = cdg::launch_step_f64(g, din, 0, st);
    }
    if (e) return cuda_fail(e, "allocation-free step launch");
    // (copies from pageable host memory return once the source has been staged,
    // so the stack copy of the instance record may go out of scope here)
    return CDUGKS_OK;
}

}  // namespace

extern "C" {

int cdugks_step_noalloc(cdugks_t* h, const void* phi_in, void* phi_out, double* W, void* cuda_stream) {
    if (!h || !phi_in || !phi_out || !W) return fail(CDUGKS_ERR_INVALID, "null argument");
    if (phi_in == phi_out) return fail(CDUGKS_ERR_INVALID, "phi_in and phi_out must be different buffers");
    if (h->collision != CDUGKS_COLLISION_TEDDF || h->g.accel)
        return fail(CDUGKS_ERR_INVALID,
                    "the allocation-free step implements the two-time collision model without acceleration only");
    for (int a = 0; a < h->g.D; ++a)
        if (h->g.bc[a][0] == CDUGKS_BC_DIRICHLET || h->g.bc[a][1] == CDUGKS_BC_DIRICHLET)
            return fail(CDUGKS_ERR_INVALID, "the allocation-free step supports periodic and specular boundaries only");
    if ((((uintptr_t)phi_in) | ((uintptr_t)phi_out)) % 32 || ((uintptr_t)W) % 8)
        return fail(CDUGKS_ERR_INVALID, "state buffers must be 32-byte aligned and W 8-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (h->prec == CDUGKS_FP32) return noalloc_run<float>(h, phi_in, phi_out, W, st);
    return noalloc_run<double>(h, phi_in, phi_out, W, st);
}

double cdugks_mu_from_kn(double kn, double rho_ref, double T_ref, double R, double length) {
    return 5.0 / 16.0 * kn * length * rho_ref * std::sqrt(2.0 * 3.14159265358979323846 * R * T_ref);
}

}  // extern "C"
