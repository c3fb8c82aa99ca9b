// sweeps_f64.cu -- FP64 instantiations of the CDUGKS step (the plain method),
// plus the precision-independent moment kernel.
#include "sweeps_impl.cuh"

namespace cdg {

namespace {
constexpr int FF = MODE_FUSED | MODE_FACES, SF = MODE_STORED | MODE_FACES, FG = MODE_FUSED | MODE_FACES | MODE_R2;
constexpr int FFS = FF | MODE_SK, SFS = SF | MODE_SK;   // Shakhov collision
constexpr int PFA = MODE_PREP | MODE_FACES | MODE_ACC;   // external acceleration
using Table64 = ShapeTable<
    double,
    ShapeList<Shape<double, 1, 256, 1, 1>, Shape<double, 1, 128, 1, 1>, Shape<double, 1, 64, 1, 1>,
              Shape<double, 1, 128, 1, 1, FF>, Shape<double, 1, 128, 1, 1, FG>, Shape<double, 1, 128, 1, 1, FFS>,
              Shape<double, 1, 128, 1, 1, PFA>, Shape<double, 1, 64, 1, 1, FF, true>, Shape<double, 1, 32, 1, 1, FF>>,
    ShapeList<Shape<double, 2, 16, 8, 1>, Shape<double, 2, 8, 8, 1>, Shape<double, 2, 16, 8, 1, MODE_STORED>,
              Shape<double, 2, 16, 8, 1, FF>, Shape<double, 2, 8, 8, 1, FG>, Shape<double, 2, 16, 8, 1, FFS>,
              Shape<double, 2, 16, 8, 1, PFA>, LeanShape<double, 2, 16, 8, 1>>,
    ShapeList<Shape<double, 3, 4, 4, 4>, Shape<double, 3, 8, 4, 4, MODE_PREP>, Shape<double, 3, 8, 4, 4, MODE_STORED>,
              Shape<double, 3, 8, 4, 4, SF>, Shape<double, 3, 8, 4, 4, SFS>, Shape<double, 3, 8, 4, 4, PFA>>>;
}

int tile_count_f64(int D) { return Table64::count(D); }
TileShape tile_shape_f64(int D, int id) { return Table64::shape(D, id); }
size_t sweep_smem_f64(int D, int id) { return Table64::smem(D, id); }
int tile_mode_f64(int D, int id) { return Table64::mode(D, id); }

cudaError_t launch_step_f64(const Geo& g, const Inst<double>* in, int cur, cudaStream_t s, cudaEvent_t* ev,
                            const void* phi_in) {
    return Table64::step(g, in, cur, s, ev, phi_in);
}
bool batch_persistent_f64(int D, int id) { return Table64::persistent(D, id); }
cudaError_t launch_batch_persist_f64(int D, int id, const PHead* h, const PItem* it, const Inst<double>* in, int* cur,
                                     PState* st, int nsteps, int wait_log2, int test_hook, cudaStream_t s) {
    return Table64::persist(D, id, h, it, in, cur, st, nsteps, wait_log2, test_hook, s);
}
cudaError_t launch_batch_step_f64(const BatchPlan& p, const Inst<double>* insts, int* cur, cudaStream_t s) {
    return run_batch_step<Table64, double>(p, insts, cur, s);
}
cudaError_t launch_init_f64(const Geo& g, const Inst<double>* in, int cur, const double* f, cudaStream_t s) {
    return run_init<double>(g, in, cur, f, s);
}
cudaError_t launch_cellc_f64(const Geo& g, const Inst<double>* in, int cur, cudaStream_t s) {
    return run_cellc<double>(g, in, cur, s);
}
cudaError_t launch_stress_f64(const Geo& g, const Inst<double>* in, int cur, double* out, cudaStream_t s) {
    return run_stress<double>(g, in, cur, out, s);
}
cudaError_t launch_finalise_f64(const Geo& g, const Inst<double>* in, int cur, cudaStream_t s) {
    return run_finalise<double>(g, in, cur, s);
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
