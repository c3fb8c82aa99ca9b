// sweeps_f32.cu -- FP32-storage instantiations of the CDUGKS step.
#include "sweeps_impl.cuh"

namespace cdg {

namespace {
constexpr int FF = MODE_FUSED | MODE_FACES, SF = MODE_STORED | MODE_FACES, FG = MODE_FUSED | MODE_FACES | MODE_R2;
constexpr int FFS = FF | MODE_SK, SFS = SF | MODE_SK;   // Shakhov collision
constexpr int PFA = MODE_PREP | MODE_FACES | MODE_ACC;   // external acceleration
using Table32 = ShapeTable<
    float,
    ShapeList<Shape<float, 1, 256, 1, 1>, Shape<float, 1, 128, 1, 1>, Shape<float, 1, 64, 1, 1>,
              Shape<float, 1, 256, 1, 1, FF, true>, Shape<float, 1, 256, 1, 1, FG>, Shape<float, 1, 256, 1, 1, FFS>,
              Shape<float, 1, 256, 1, 1, PFA>, Shape<float, 1, 128, 1, 1, FF, true>, Shape<float, 1, 64, 1, 1, FF, true>>,
    ShapeList<Shape<float, 2, 32, 8, 1>, Shape<float, 2, 16, 8, 1>, Shape<float, 2, 32, 16, 1, MODE_PREP>,
              Shape<float, 2, 32, 8, 1, MODE_STORED>, Shape<float, 2, 32, 16, 1, MODE_STORED>,
              Shape<float, 2, 32, 16, 1>, Shape<float, 2, 32, 8, 1, FF, true>, Shape<float, 2, 32, 16, 1, FF>,
              Shape<float, 2, 32, 8, 1, SF>, Shape<float, 2, 16, 8, 1, FG>, Shape<float, 2, 32, 8, 1, FFS>,
              Shape<float, 2, 32, 8, 1, PFA>, LeanShape<float, 2, 32, 8, 1>, LeanShape<float, 2, 32, 16, 1>,
              LeanShape<float, 2, 32, 8, 1, false>>,
    ShapeList<Shape<float, 3, 8, 4, 4>, Shape<float, 3, 8, 8, 4, MODE_PREP>, Shape<float, 3, 8, 8, 4, MODE_STORED>,
              Shape<float, 3, 8, 4, 4, MODE_STORED>, Shape<float, 3, 8, 8, 4, SF>, Shape<float, 3, 8, 4, 4, SF>,
              Shape<float, 3, 8, 8, 4, SFS>, Shape<float, 3, 8, 4, 4, PFA>, LeanShape<float, 3, 8, 8, 4>,
              LeanShape<float, 3, 8, 4, 4>, LeanShape<float, 3, 8, 8, 4, false>>>;
}

int tile_count_f32(int D) { return Table32::count(D); }
TileShape tile_shape_f32(int D, int id) { return Table32::shape(D, id); }
size_t sweep_smem_f32(int D, int id) { return Table32::smem(D, id); }
int tile_mode_f32(int D, int id) { return Table32::mode(D, id); }

cudaError_t launch_step_f32(const Geo& g, const Inst<float>* in, int cur, cudaStream_t s, cudaEvent_t* ev,
                            const void* phi_in) {
    return Table32::step(g, in, cur, s, ev, phi_in);
}
bool batch_persistent_f32(int D, int id) { return Table32::persistent(D, id); }
cudaError_t launch_batch_persist_f32(int D, int id, const PHead* h, const PItem* it, const Inst<float>* in, int* cur,
                                     PState* st, int nsteps, int wait_log2, int test_hook, cudaStream_t s) {
    return Table32::persist(D, id, h, it, in, cur, st, nsteps, wait_log2, test_hook, s);
}
cudaError_t launch_batch_step_f32(const BatchPlan& p, const Inst<float>* insts, int* cur, cudaStream_t s) {
    return run_batch_step<Table32, float>(p, insts, cur, s);
}
cudaError_t launch_init_f32(const Geo& g, const Inst<float>* in, int cur, const double* f, cudaStream_t s) {
    return run_init<float>(g, in, cur, f, s);
}
cudaError_t launch_cellc_f32(const Geo& g, const Inst<float>* in, int cur, cudaStream_t s) {
    return run_cellc<float>(g, in, cur, s);
}
cudaError_t launch_stress_f32(const Geo& g, const Inst<float>* in, int cur, double* out, cudaStream_t s) {
    return run_stress<float>(g, in, cur, out, s);
}
cudaError_t launch_finalise_f32(const Geo& g, const Inst<float>* in, int cur, cudaStream_t s) {
    return run_finalise<float>(g, in, cur, s);
}

}  // namespace cdg
