// sweeps_f32.cu -- FP32-storage instantiations of the CDUGKS step.
#include "sweeps_impl.cuh"

namespace cdg {

cudaError_t launch_step_f32(const Geo& g, const Bufs<float>& b, cudaStream_t s, cudaEvent_t* ev) {
    switch (g.D) {
        case 1: return run_step<float, 1, 256, 1, 1>(g, b, s, ev);
        case 2: return run_step<float, 2, 32, 8, 1>(g, b, s, ev);
        default: return run_step<float, 3, 8, 4, 4>(g, b, s, ev);
    }
}
cudaError_t launch_init_f32(const Geo& g, const Bufs<float>& b, const double* f, cudaStream_t s) {
    return run_init<float>(g, b, f, s);
}
cudaError_t launch_cellc_f32(const Geo& g, const Bufs<float>& b, cudaStream_t s) { return run_cellc<float>(g, b, s); }
cudaError_t launch_finalise_f32(const Geo& g, const Bufs<float>& b, cudaStream_t s) {
    return run_finalise<float>(g, b, s);
}

}  // namespace cdg
