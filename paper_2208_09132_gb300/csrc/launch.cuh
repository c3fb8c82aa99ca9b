// launch.cuh -- host-side launch interface between the C ABI (api.cu) and the
// per-precision translation units that instantiate the kernels.
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"

namespace cdg {

struct TileShape {
    int t[3];
};

// Work of one batched step: sweep items grouped by tile shape, face and cell ranges.
constexpr int kMaxBatchShapes = 8;
struct BatchPlan {
    int D;
    int ntile;
    int tile_id[kMaxBatchShapes];
    const Item* sweep_items[kMaxBatchShapes];
    int n_sweep[kMaxBatchShapes];
    const RItem* face_items;
    int n_face;
    const RItem* cell_items;
    int n_cell;
    const RItem* prep_items;     // acceleration members: cells x runs of kPrepChunks chunks
    int n_prep;
    const QItem* faceq_items;    // Shakhov members: raw face moments
    int n_faceq;
    const QItem* cellq_items;    // Shakhov members: raw cell moments
    int n_cellq;
};

// Instantiated tile shapes of the sweeps per precision (f32 = FP32 storage) and dimension.
int tile_count_f32(int D);
int tile_count_f64(int D);
TileShape tile_shape_f32(int D, int id);
TileShape tile_shape_f64(int D, int id);
size_t sweep_smem_f32(int D, int id);
size_t sweep_smem_f64(int D, int id);
// Sweep mode of a shape (MODE_FUSED / MODE_PREP / MODE_STORED): prepared and
// stored shapes need a phibar+ buffer, stored shapes also a slope buffer.
int tile_mode_f32(int D, int id);
int tile_mode_f64(int D, int id);

// The single-instance launches read the instance from the device table `in`
// and use orientation `cur` (read state buffer cur, write the other).
// One time step: sweep A, face constants, sweep B, W update (+ cell constants of W^{n+1}).
// ev: null, or five events recorded before, between and after the four phases.
// phi_in: the device address of the state buffer the step reads (the tensor
// maps of sweep A's TMA staging), or null (per-cell staging only).
cudaError_t launch_step_f32(const Geo& g, const Inst<float>* in, int cur, cudaStream_t s, cudaEvent_t* ev = nullptr,
                            const void* phi_in = nullptr);
cudaError_t launch_step_f64(const Geo& g, const Inst<double>* in, int cur, cudaStream_t s, cudaEvent_t* ev = nullptr,
                            const void* phi_in = nullptr);
// One time step of every instance of a batch.
cudaError_t launch_batch_step_f32(const BatchPlan& p, const Inst<float>* insts, int* cur, cudaStream_t s);
cudaError_t launch_batch_step_f64(const BatchPlan& p, const Inst<double>* insts, int* cur, cudaStream_t s);
// The persistent batched step (persist.cuh): nsteps steps of every member in one
// launch; only shapes that have it (batch_persistent_*) and one shape per batch.
struct PHead;
struct PItem;
struct PState;
bool batch_persistent_f32(int D, int id);
bool batch_persistent_f64(int D, int id);
cudaError_t launch_batch_persist_f32(int D, int id, const PHead* h, const PItem* it, const Inst<float>* in, int* cur,
                                     PState* st, int nsteps, int wait_log2, int test_hook, cudaStream_t s);
cudaError_t launch_batch_persist_f64(int D, int id, const PHead* h, const PItem* it, const Inst<double>* in, int* cur,
                                     PState* st, int nsteps, int wait_log2, int test_hook, cudaStream_t s);
// Maxwellian initial state from device fields [Nc][2+D] (rho, u, T).
cudaError_t launch_init_f32(const Geo& g, const Inst<float>* in, int cur, const double* fields, cudaStream_t s);
cudaError_t launch_init_f64(const Geo& g, const Inst<double>* in, int cur, const double* fields, cudaStream_t s);
// Cell constants from the stored W.
cudaError_t launch_cellc_f32(const Geo& g, const Inst<float>* in, int cur, cudaStream_t s);
cudaError_t launch_cellc_f64(const Geo& g, const Inst<double>* in, int cur, cudaStream_t s);
// Pressure tensor and heat flux per cell into out[Nc][D*D + D] (device).
cudaError_t launch_stress_f32(const Geo& g, const Inst<float>* in, int cur, double* out, cudaStream_t s);
cudaError_t launch_stress_f64(const Geo& g, const Inst<double>* in, int cur, double* out, cudaStream_t s);
// Finalised distributions into phi_out.
cudaError_t launch_finalise_f32(const Geo& g, const Inst<float>* in, int cur, cudaStream_t s);
cudaError_t launch_finalise_f64(const Geo& g, const Inst<double>* in, int cur, cudaStream_t s);
// rho,u,T (or W) per cell into out[Nc][2+D].
cudaError_t launch_moments(const Geo& g, const double* W, double* out, int conserved, cudaStream_t s);

}  // namespace cdg
