// launch.cuh -- host-side launch interface between the C ABI (api.cu) and the
// per-precision translation units that instantiate the kernels.
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"

namespace cdg {

struct TileShape {
    int t[3];
};

// Tile shape and dynamic shared memory of the sweeps for a precision (0 FP64, 1 FP32) and dimension.
TileShape tile_shape(int precision, int D);
size_t sweep_smem_bytes(int precision, int D);

// One time step: sweep A, face constants, sweep B, W update (+ cell constants of W^{n+1}).
// ev: null, or five events recorded before, between and after the four phases.
cudaError_t launch_step_f32(const Geo& g, const Bufs<float>& b, cudaStream_t s, cudaEvent_t* ev = nullptr);
cudaError_t launch_step_f64(const Geo& g, const Bufs<double>& b, cudaStream_t s, cudaEvent_t* ev = nullptr);
// Maxwellian initial state from device fields [Nc][2+D] (rho, u, T).
cudaError_t launch_init_f32(const Geo& g, const Bufs<float>& b, const double* fields, cudaStream_t s);
cudaError_t launch_init_f64(const Geo& g, const Bufs<double>& b, const double* fields, cudaStream_t s);
// Cell constants from the stored W.
cudaError_t launch_cellc_f32(const Geo& g, const Bufs<float>& b, cudaStream_t s);
cudaError_t launch_cellc_f64(const Geo& g, const Bufs<double>& b, cudaStream_t s);
// Finalised distributions into phi_out.
cudaError_t launch_finalise_f32(const Geo& g, const Bufs<float>& b, cudaStream_t s);
cudaError_t launch_finalise_f64(const Geo& g, const Bufs<double>& b, cudaStream_t s);
// rho,u,T (or W) per cell into out[Nc][2+D].
cudaError_t launch_moments(const Geo& g, const double* W, double* out, int conserved, cudaStream_t s);

}  // namespace cdg
