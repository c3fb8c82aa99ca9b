// sweeps_impl.cuh -- launch helpers shared by the two precision translation units.
#pragma once

#include "launch.cuh"

namespace cdg {

template <typename T, int D, int TX, int TY, int TZ>
cudaError_t run_step(const Geo& g, const Bufs<T>& b, cudaStream_t s, cudaEvent_t* ev) {
    using SM = Smem<T, D, TX, TY, TZ>;
    using TL = Tile<D, TX, TY, TZ>;
    static bool configured = false;
    cudaError_t e;
    if (!configured) {
        e = cudaFuncSetAttribute(k_sweep<T, D, TX, TY, TZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SM::bytes(false));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_sweep<T, D, TX, TY, TZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SM::bytes(true));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid(g.tiles[0] * g.tiles[1] * g.tiles[2], g.G);
    if (ev) cudaEventRecord(ev[0], s);
    k_sweep<T, D, TX, TY, TZ, false><<<grid, TL::NT, SM::bytes(false), s>>>(g, b);
    if (ev) cudaEventRecord(ev[1], s);
    for (int a = 0; a < D; ++a) {
        const unsigned blocks = (unsigned)((g.nf[a] + 127) / 128);
        k_facec<T, D><<<blocks, 128, 0, s>>>(g, b, a);
    }
    if (ev) cudaEventRecord(ev[2], s);
    k_sweep<T, D, TX, TY, TZ, true><<<grid, TL::NT, SM::bytes(true), s>>>(g, b);
    if (ev) cudaEventRecord(ev[3], s);
    k_wupdate<T, D><<<(unsigned)((g.Nc + 127) / 128), 128, 0, s>>>(g, b);
    if (ev) cudaEventRecord(ev[4], s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_init(const Geo& g, const Bufs<T>& b, const double* fields, cudaStream_t s) {
    const dim3 grid((unsigned)g.Nc);
    switch (g.D) {
        case 1: k_init<T, 1><<<grid, 128, 0, s>>>(g, b, fields); break;
        case 2: k_init<T, 2><<<grid, 128, 0, s>>>(g, b, fields); break;
        default: k_init<T, 3><<<grid, 128, 0, s>>>(g, b, fields); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_cellc(const Geo& g, const Bufs<T>& b, cudaStream_t s) {
    const unsigned blocks = (unsigned)((g.Nc + 127) / 128);
    switch (g.D) {
        case 1: k_cellc<T, 1><<<blocks, 128, 0, s>>>(g, b); break;
        case 2: k_cellc<T, 2><<<blocks, 128, 0, s>>>(g, b); break;
        default: k_cellc<T, 3><<<blocks, 128, 0, s>>>(g, b); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_finalise(const Geo& g, const Bufs<T>& b, cudaStream_t s) {
    const dim3 grid((unsigned)g.Nc);
    switch (g.D) {
        case 1: k_finalise<T, 1><<<grid, 128, 0, s>>>(g, b); break;
        case 2: k_finalise<T, 2><<<grid, 128, 0, s>>>(g, b); break;
        default: k_finalise<T, 3><<<grid, 128, 0, s>>>(g, b); break;
    }
    return cudaGetLastError();
}

}  // namespace cdg
