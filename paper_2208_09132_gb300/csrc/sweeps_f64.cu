// sweeps_f64.cu -- FP64 instantiations of the CDUGKS step (the plain method),
// plus the precision-independent moment kernel and the tile table.
#include "sweeps_impl.cuh"

namespace cdg {

TileShape tile_shape(int precision, int D) {
    if (precision == 1) {
        if (D == 1) return {{256, 1, 1}};
        if (D == 2) return {{32, 8, 1}};
        return {{8, 4, 4}};
    }
    if (D == 1) return {{256, 1, 1}};
    if (D == 2) return {{16, 8, 1}};
    return {{4, 4, 4}};
}

size_t sweep_smem_bytes(int precision, int D) {
    if (precision == 1) {
        if (D == 1) return Smem<float, 1, 256, 1, 1>::bytes(true);
        if (D == 2) return Smem<float, 2, 32, 8, 1>::bytes(true);
        return Smem<float, 3, 8, 4, 4>::bytes(true);
    }
    if (D == 1) return Smem<double, 1, 256, 1, 1>::bytes(true);
    if (D == 2) return Smem<double, 2, 16, 8, 1>::bytes(true);
    return Smem<double, 3, 4, 4, 4>::bytes(true);
}

cudaError_t launch_step_f64(const Geo& g, const Bufs<double>& b, cudaStream_t s, cudaEvent_t* ev) {
    switch (g.D) {
        case 1: return run_step<double, 1, 256, 1, 1>(g, b, s, ev);
        case 2: return run_step<double, 2, 16, 8, 1>(g, b, s, ev);
        default: return run_step<double, 3, 4, 4, 4>(g, b, s, ev);
    }
}
cudaError_t launch_init_f64(const Geo& g, const Bufs<double>& b, const double* f, cudaStream_t s) {
    return run_init<double>(g, b, f, s);
}
cudaError_t launch_cellc_f64(const Geo& g, const Bufs<double>& b, cudaStream_t s) {
    return run_cellc<double>(g, b, s);
}
cudaError_t launch_finalise_f64(const Geo& g, const Bufs<double>& b, cudaStream_t s) {
    return run_finalise<double>(g, b, s);
}

cudaError_t launch_moments(const Geo& g, const double* W, double* out, int conserved, cudaStream_t s) {
    const unsigned blocks = (unsigned)((g.Nc + 255) / 256);
    switch (g.D) {
        case 1: k_moments<1><<<blocks, 256, 0, s>>>(g, W, out, conserved); break;
        case 2: k_moments<2><<<blocks, 256, 0, s>>>(g, W, out, conserved); break;
        default: k_moments<3><<<blocks, 256, 0, s>>>(g, W, out, conserved); break;
    }
    return cudaGetLastError();
}

}  // namespace cdg
