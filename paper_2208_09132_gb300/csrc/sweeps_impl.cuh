// sweeps_impl.cuh -- launch helpers shared by the two precision translation units.
#pragma once

#include "launch.cuh"

namespace cdg {

// Block size of the per-face and per-cell kernels: small, so that the FP64
// constant computations of a small problem spread over many SMs.
constexpr int kSmallBlock = 64;

// One instantiated tile shape of the sweeps and its launches.
template <typename T, int D, int TX, int TY, int TZ>
struct Shape {
    using SM = Smem<T, D, TX, TY, TZ>;
    using TL = Tile<D, TX, TY, TZ>;

    static cudaError_t configure() {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_sweep<T, D, TX, TY, TZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SM::bytes(false))))
            return e;
        if ((e = cudaFuncSetAttribute(k_sweep<T, D, TX, TY, TZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SM::bytes(true))))
            return e;
        if ((e = cudaFuncSetAttribute(k_sweep_batch<T, D, TX, TY, TZ, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes(false))))
            return e;
        if ((e = cudaFuncSetAttribute(k_sweep_batch<T, D, TX, TY, TZ, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes(true))))
            return e;
        done = true;
        return cudaSuccess;
    }

    static cudaError_t step(const Geo& g, const Inst<T>* in, int cur, cudaStream_t s, cudaEvent_t* ev) {
        cudaError_t e = configure();
        if (e) return e;
        const dim3 grid(g.tiles[0] * g.tiles[1] * g.tiles[2], g.G);
        if (ev) cudaEventRecord(ev[0], s);
        k_sweep<T, D, TX, TY, TZ, false><<<grid, TL::NT, SM::bytes(false), s>>>(in, cur);
        if (ev) cudaEventRecord(ev[1], s);
        for (int a = 0; a < D; ++a) {
            const unsigned blocks = (unsigned)((g.nf[a] + kSmallBlock - 1) / kSmallBlock);
            k_facec<T, D><<<blocks, kSmallBlock, 0, s>>>(in, cur, a);
        }
        if (ev) cudaEventRecord(ev[2], s);
        k_sweep<T, D, TX, TY, TZ, true><<<grid, TL::NT, SM::bytes(true), s>>>(in, cur);
        if (ev) cudaEventRecord(ev[3], s);
        k_wupdate<T, D><<<(unsigned)((g.Nc + kSmallBlock - 1) / kSmallBlock), kSmallBlock, 0, s>>>(in, cur);
        if (ev) cudaEventRecord(ev[4], s);
        return cudaGetLastError();
    }

    static cudaError_t sweep_batch(bool B, const Item* items, int n, const Inst<T>* insts, const int* cur,
                                   cudaStream_t s) {
        cudaError_t e = configure();
        if (e) return e;
        if (n <= 0) return cudaSuccess;
        if (B) k_sweep_batch<T, D, TX, TY, TZ, true><<<n, TL::NT, SM::bytes(true), s>>>(items, insts, cur);
        else k_sweep_batch<T, D, TX, TY, TZ, false><<<n, TL::NT, SM::bytes(false), s>>>(items, insts, cur);
        return cudaGetLastError();
    }
};

// The shapes of one precision, indexed by tile id: Shapes<...>::get(D, id).
template <typename T, typename S1a, typename S1b, typename S1c, typename S2a, typename S2b, typename S3a>
struct ShapeTable {
    static int count(int D) { return D == 1 ? 3 : (D == 2 ? 2 : 1); }
    static TileShape shape(int D, int id) {
        if (D == 1) {
            const int t[3] = {S1a::TL::T0, S1b::TL::T0, S1c::TL::T0};
            return {{t[id < 3 ? id : 0], 1, 1}};
        }
        if (D == 2) {
            if (id == 1) return {{S2b::TL::T0, S2b::TL::T1, 1}};
            return {{S2a::TL::T0, S2a::TL::T1, 1}};
        }
        return {{S3a::TL::T0, S3a::TL::T1, S3a::TL::T2}};
    }
    static size_t smem(int D, int id) {
        if (D == 1) return id == 1 ? S1b::SM::bytes(true) : (id == 2 ? S1c::SM::bytes(true) : S1a::SM::bytes(true));
        if (D == 2) return id == 1 ? S2b::SM::bytes(true) : S2a::SM::bytes(true);
        return S3a::SM::bytes(true);
    }
    static cudaError_t step(const Geo& g, const Inst<T>* in, int cur, cudaStream_t s, cudaEvent_t* ev) {
        if (g.D == 1) {
            if (g.tile_id == 1) return S1b::step(g, in, cur, s, ev);
            if (g.tile_id == 2) return S1c::step(g, in, cur, s, ev);
            return S1a::step(g, in, cur, s, ev);
        }
        if (g.D == 2) return g.tile_id == 1 ? S2b::step(g, in, cur, s, ev) : S2a::step(g, in, cur, s, ev);
        return S3a::step(g, in, cur, s, ev);
    }
    static cudaError_t sweep_batch(int D, int id, bool B, const Item* it, int n, const Inst<T>* in, const int* cur,
                                   cudaStream_t s) {
        if (D == 1) {
            if (id == 1) return S1b::sweep_batch(B, it, n, in, cur, s);
            if (id == 2) return S1c::sweep_batch(B, it, n, in, cur, s);
            return S1a::sweep_batch(B, it, n, in, cur, s);
        }
        if (D == 2) return id == 1 ? S2b::sweep_batch(B, it, n, in, cur, s) : S2a::sweep_batch(B, it, n, in, cur, s);
        return S3a::sweep_batch(B, it, n, in, cur, s);
    }
};

template <typename Table, typename T>
cudaError_t run_batch_step(const BatchPlan& p, const Inst<T>* insts, int* cur, cudaStream_t s) {
    cudaError_t e;
    for (int k = 0; k < p.ntile; ++k)
        if ((e = Table::sweep_batch(p.D, p.tile_id[k], false, p.sweep_items[k], p.n_sweep[k], insts, cur, s)))
            return e;
    if (p.n_face > 0) {
        switch (p.D) {
            case 1: k_facec_batch<T, 1><<<p.n_face, kSmallBlock, 0, s>>>(p.face_items, insts, cur); break;
            case 2: k_facec_batch<T, 2><<<p.n_face, kSmallBlock, 0, s>>>(p.face_items, insts, cur); break;
            default: k_facec_batch<T, 3><<<p.n_face, kSmallBlock, 0, s>>>(p.face_items, insts, cur); break;
        }
    }
    for (int k = 0; k < p.ntile; ++k)
        if ((e = Table::sweep_batch(p.D, p.tile_id[k], true, p.sweep_items[k], p.n_sweep[k], insts, cur, s)))
            return e;
    if (p.n_cell > 0) {
        switch (p.D) {
            case 1: k_wupdate_batch<T, 1><<<p.n_cell, kSmallBlock, 0, s>>>(p.cell_items, insts, cur); break;
            case 2: k_wupdate_batch<T, 2><<<p.n_cell, kSmallBlock, 0, s>>>(p.cell_items, insts, cur); break;
            default: k_wupdate_batch<T, 3><<<p.n_cell, kSmallBlock, 0, s>>>(p.cell_items, insts, cur); break;
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_init(const Geo& g, const Inst<T>* in, int cur, const double* fields, cudaStream_t s) {
    const dim3 grid((unsigned)g.Nc);
    switch (g.D) {
        case 1: k_init<T, 1><<<grid, 128, 0, s>>>(in, cur, fields); break;
        case 2: k_init<T, 2><<<grid, 128, 0, s>>>(in, cur, fields); break;
        default: k_init<T, 3><<<grid, 128, 0, s>>>(in, cur, fields); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_cellc(const Geo& g, const Inst<T>* in, int cur, cudaStream_t s) {
    const unsigned blocks = (unsigned)((g.Nc + kSmallBlock - 1) / kSmallBlock);
    switch (g.D) {
        case 1: k_cellc<T, 1><<<blocks, kSmallBlock, 0, s>>>(in, cur); break;
        case 2: k_cellc<T, 2><<<blocks, kSmallBlock, 0, s>>>(in, cur); break;
        default: k_cellc<T, 3><<<blocks, kSmallBlock, 0, s>>>(in, cur); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_finalise(const Geo& g, const Inst<T>* in, int cur, cudaStream_t s) {
    const dim3 grid((unsigned)g.Nc);
    switch (g.D) {
        case 1: k_finalise<T, 1><<<grid, 128, 0, s>>>(in, cur); break;
        case 2: k_finalise<T, 2><<<grid, 128, 0, s>>>(in, cur); break;
        default: k_finalise<T, 3><<<grid, 128, 0, s>>>(in, cur); break;
    }
    return cudaGetLastError();
}

}  // namespace cdg
