// sweeps_impl.cuh -- launch helpers shared by the two precision translation units.
#pragma once

#include <cstring>
#include <utility>

#include "launch.cuh"
#include "lean.cuh"
#include "persist.cuh"

namespace cdg {

// Block size of the per-face and per-cell kernels: small, so that the FP64
// constant computations of a small problem spread over many SMs.
constexpr int kSmallBlock = 64;
// Block size of the raw-moment reductions (one thread per face or cell and group).
constexpr int kMomBlock = 128;

// A launch of a step kernel with programmatic stream serialisation: it may be
// scheduled while the previous kernel on the stream drains, and waits in
// pdl_wait() before it reads that kernel's results.
template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Tensor maps for the TMA staging of sweep A: the g and b halves of the state
// buffer phi_in ([chunk][cell][g|b][VC]) as tensors (VC, n0[, n1], chunks)
// whose boxes are the tile's halo box of one chunk (the kernel uses them for
// 1D and 2D tiles whose box lies inside the domain).  The encoder is the
// driver's, reached through the runtime; without it the launch stages per cell.
using TensorMapEncode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline TensorMapEncode tensor_map_encoder() {
    static const TensorMapEncode enc = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<TensorMapEncode>(fn);
    }();
    return enc;
}
template <typename T, int D, typename TL>
TmaPair make_tma(const Geo& g, const void* phi_in) {
    TmaPair tp;
    std::memset(&tp, 0, sizeof(tp));
    const TensorMapEncode enc = tensor_map_encoder();
    if (!enc || !phi_in || D > 2 || TL::E0 > 256 || TL::E1 > 256) return tp;
    const cuuint64_t cs = 2 * VC * sizeof(T);                  // bytes per cell and chunk
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], es[4] = {1, 1, 1, 1};
    const cuuint32_t rank = D + 2;
    dims[0] = VC;
    box[0] = VC;
    dims[1] = (cuuint64_t)g.n[0];
    box[1] = TL::E0;
    strides[0] = cs;
    if (D == 2) {
        dims[2] = (cuuint64_t)g.n[1];
        box[2] = TL::E1;
        strides[1] = cs * (cuuint64_t)g.n[0];
    }
    dims[rank - 1] = (cuuint64_t)g.NVT;
    box[rank - 1] = 1;
    strides[rank - 2] = cs * (cuuint64_t)g.Nc;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    char* base = static_cast<char*>(const_cast<void*>(phi_in));
    const CUresult rg = enc(&tp.g, dt, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    const CUresult rb = enc(&tp.b, dt, rank, base + VC * sizeof(T), dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    tp.on = rg == CUDA_SUCCESS && rb == CUDA_SUCCESS;
    return tp;
}

// One instantiated tile shape of the sweeps and its launches.  Prepared
// shapes (MODE_PREP) form phibar+ of every point once per step (k_prep);
// stored shapes (MODE_STORED) form phibar+ and the slopes (k_shslope); the
// sweeps of both load what was formed instead of recomputing it on the halo.
// Face-store shapes (MODE_FACES bit) have sweep A keep the reconstructed
// face values and run k_flux as sweep B.  Shakhov shapes (MODE_SK, face-store
// only) add k_faceq before the face constants and k_cellq before the W update.
// Acceleration shapes (MODE_ACC, prepared face-store only) form the force
// terms in k_prep and take them in k_flux.
// The number of CTAs of a persistent launch: every SM at the occupancy the
// kernel reaches (more would only wait for a slot).
template <typename K>
int persistent_grid(K kern, int threads, size_t smem) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    return sms * (occ > 0 ? occ : 1);
}

// PB: the shape also has the persistent batched step (k_batch_persist).
template <typename T, int D, int TX, int TY, int TZ, int MODE = MODE_FUSED, bool PB = false>
struct Shape {
    static constexpr bool SK = mode_sk(MODE);
    using SM = Smem<T, D, TX, TY, TZ, MODE>;
    using FS = FluxSmem<T, D, TX, TY, TZ, SK>;
    using TL = Tile<D, TX, TY, TZ>;
    static constexpr int mode = MODE;
    static constexpr int SRC = mode_source(MODE);
    static constexpr bool FACES = mode_faces(MODE);
    static_assert(!SK || FACES, "Shakhov shapes are face-store shapes");
    static constexpr bool ACC = mode_acc(MODE);
    static_assert(!ACC || (SRC == MODE_PREP && FACES && !SK && !mode_r2(MODE)),
                  "acceleration shapes are prepared face-store shapes");
    static_assert((MODE & MODE_NOSRC) == 0, "the no-b-source bit is chosen at launch");
    // Face-store TEDDF shapes carry a second pair of sweeps for instances with
    // no b-source (Pr = 1), chosen per launch; the Shakhov shapes have none.
    static constexpr bool NS = FACES && !SK;
    static constexpr int MODE_NS = MODE | MODE_NOSRC;
    // batched steps: the fused shapes (incl. Shakhov) and the acceleration
    // shapes (their pre-pass is batched too)
    static constexpr bool BATCH = SRC == MODE_FUSED || ACC;

    // dynamic shared memory of the larger of the two sweeps
    static size_t smem_bytes() {
        const size_t b = FACES ? FS::bytes : SM::bytes(true);
        return SM::bytes(false) > b ? SM::bytes(false) : b;
    }

    static cudaError_t configure() {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_sweep<T, D, TX, TY, TZ, false, MODE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes(false))))
            return e;
        if constexpr (FACES) {
            if ((e = cudaFuncSetAttribute(k_flux<T, D, TX, TY, TZ, SK, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)FS::bytes)))
                return e;
        } else {
            if ((e = cudaFuncSetAttribute(k_sweep<T, D, TX, TY, TZ, true, MODE>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes(true))))
                return e;
        }
        if constexpr (NS) {
            if ((e = cudaFuncSetAttribute(k_sweep<T, D, TX, TY, TZ, false, MODE_NS>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes(false))))
                return e;
            if ((e = cudaFuncSetAttribute(k_flux<T, D, TX, TY, TZ, false, ACC, true>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS::bytes)))
                return e;
        }
        if constexpr (SRC == MODE_STORED) {
            if ((e = cudaFuncSetAttribute(k_shslope<T, D, TX, TY, TZ, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)shslope_smem_bytes<T, D, TX, TY, TZ, SK>())))
                return e;
        }
        if constexpr (BATCH) {
            if ((e = cudaFuncSetAttribute(k_sweep_batch<T, D, TX, TY, TZ, false, MODE>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes(false))))
                return e;
            if constexpr (FACES) {
                if ((e = cudaFuncSetAttribute(k_flux_batch<T, D, TX, TY, TZ, SK, ACC>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS::bytes)))
                    return e;
            } else {
                if ((e = cudaFuncSetAttribute(k_sweep_batch<T, D, TX, TY, TZ, true, MODE>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes(true))))
                    return e;
            }
        }
        done = true;
        return cudaSuccess;
    }

    static cudaError_t step(const Geo& g, const Inst<T>* in, int cur, cudaStream_t s, cudaEvent_t* ev,
                            const void* phi_in) {
        cudaError_t e = configure();
        if (e) return e;
        const dim3 grid(g.tiles[0] * g.tiles[1] * g.tiles[2], g.G);
        if (ev) cudaEventRecord(ev[0], s);
        if constexpr (SRC == MODE_PREP) {
            const dim3 pg((unsigned)((g.Nc + kPrepCells - 1) / kPrepCells),
                          (unsigned)((g.NVT + kPrepChunks - 1) / kPrepChunks));
            if ((e = launch_pdl(k_prep<T, D, ACC>, pg, dim3(kPrepCells), 0, s, in, cur, kPrepChunks))) return e;
        } else if constexpr (SRC == MODE_STORED) {
            if ((e = launch_pdl(k_shslope<T, D, TX, TY, TZ, SK>, grid, dim3(TL::NT),
                                shslope_smem_bytes<T, D, TX, TY, TZ, SK>(), s, in, cur)))
                return e;
        }
        const TmaPair tma = make_tma<T, D, typename SM::TL>(g, SM::stage(false) ? phi_in : nullptr);
        const bool ns = NS && g.nosrc;
        if constexpr (NS) {
            if (ns)
                e = launch_pdl(k_sweep<T, D, TX, TY, TZ, false, MODE_NS>, grid, dim3(TL::NT), SM::bytes(false), s, in,
                               cur, tma);
        }
        if (!ns) e = launch_pdl(k_sweep<T, D, TX, TY, TZ, false, MODE>, grid, dim3(TL::NT), SM::bytes(false), s, in, cur, tma);
        if (e) return e;
        if (ev) cudaEventRecord(ev[1], s);
        if constexpr (SK) {
            long long nf = 0;
            for (int a = 0; a < D; ++a) nf = g.nf[a] > nf ? g.nf[a] : nf;
            const dim3 qg((unsigned)((nf + kMomBlock - 1) / kMomBlock), (unsigned)g.G, (unsigned)D);
            if ((e = launch_pdl(k_faceq<T, D>, qg, dim3(kMomBlock), 0, s, in, cur))) return e;
        }
        {
            long long nf = 0;
            for (int a = 0; a < D; ++a) nf = g.nf[a] > nf ? g.nf[a] : nf;
            const dim3 fgrid((unsigned)((nf + kSmallBlock - 1) / kSmallBlock), (unsigned)D);
            if ((e = launch_pdl(k_facec<T, D>, fgrid, dim3(kSmallBlock), 0, s, in, cur))) return e;
        }
        if (ev) cudaEventRecord(ev[2], s);
        if constexpr (NS) {
            if (ns) e = launch_pdl(k_flux<T, D, TX, TY, TZ, false, ACC, true>, grid, dim3(TL::NT), FS::bytes, s, in, cur);
            else e = launch_pdl(k_flux<T, D, TX, TY, TZ, false, ACC>, grid, dim3(TL::NT), FS::bytes, s, in, cur);
        } else if constexpr (FACES)
            e = launch_pdl(k_flux<T, D, TX, TY, TZ, SK, ACC>, grid, dim3(TL::NT), FS::bytes, s, in, cur);
        else e = launch_pdl(k_sweep<T, D, TX, TY, TZ, true, MODE>, grid, dim3(TL::NT), SM::bytes(true), s, in, cur,
                            make_tma<T, D, TL>(g, nullptr));
        if (e) return e;
        if (ev) cudaEventRecord(ev[3], s);
        if constexpr (SK) {
            const dim3 cg((unsigned)((g.Nc + kMomBlock - 1) / kMomBlock), (unsigned)g.G);
            if ((e = launch_pdl(k_cellq<T, D>, cg, dim3(kMomBlock), 0, s, in, cur))) return e;
        }
        if ((e = launch_pdl(k_wupdate<T, D>, dim3((unsigned)((g.Nc + kSmallBlock - 1) / kSmallBlock)), dim3(kSmallBlock),
                            0, s, in, cur)))
            return e;
        if (ev) cudaEventRecord(ev[4], s);
        return cudaGetLastError();
    }

    static cudaError_t sweep_batch(bool B, const Item* items, int n, const Inst<T>* insts, const int* cur,
                                   cudaStream_t s) {
        if constexpr (!BATCH) {
            return cudaErrorNotSupported;
        } else {
            cudaError_t e = configure();
            if (e) return e;
            if (n <= 0) return cudaSuccess;
            if (!B)
                return launch_pdl(k_sweep_batch<T, D, TX, TY, TZ, false, MODE>, dim3(n), dim3(TL::NT), SM::bytes(false),
                                  s, items, insts, cur);
            if constexpr (FACES)
                return launch_pdl(k_flux_batch<T, D, TX, TY, TZ, SK, ACC>, dim3(n), dim3(TL::NT), FS::bytes, s, items,
                                  insts, cur);
            else
                return launch_pdl(k_sweep_batch<T, D, TX, TY, TZ, true, MODE>, dim3(n), dim3(TL::NT), SM::bytes(true), s,
                                  items, insts, cur);
        }
    }

    static TileShape shape() { return {{TL::T0, TL::T1, TL::T2}}; }

    static constexpr bool persistent = PB;
    static cudaError_t persist(const PHead* head, const PItem* items, const Inst<T>* insts, int* cur, PState* st,
                               int nsteps, int wait_log2, int test_hook, cudaStream_t s) {
        if constexpr (!PB || SRC != MODE_FUSED || SK) {
            return cudaErrorNotSupported;
        } else {
            using PS = PersistSmem<T, D, TX, TY, TZ, MODE>;
            static bool done = false;
            cudaError_t e;
            if (!done) {
                if ((e = cudaFuncSetAttribute(k_batch_persist<T, D, TX, TY, TZ, MODE>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PS::bytes)))
                    return e;
                done = true;
            }
            const int grid = persistent_grid(k_batch_persist<T, D, TX, TY, TZ, MODE>, TL::NT, PS::bytes);
            if ((e = cudaMemsetAsync(st, 0, sizeof(PState), s))) return e;
            k_batch_persist<T, D, TX, TY, TZ, MODE><<<grid, TL::NT, PS::bytes, s>>>(head, items, insts, cur, st, nsteps,
                                                                                   wait_log2, test_hook);
            return cudaGetLastError();
        }
    }
};

// A lean shape (lean.cuh): sweep A k_lsweep, face constants (with the face
// factor tables when XF), sweep B k_lflux (XF) or k_flux, W update (with the
// cell factor tables).  Single instances take the sweeps without the b-source
// terms when the instance has none (Pr = 1); batched launches keep the general
// ones.
template <typename T, int D, int TX, int TY, int TZ, bool XF = true>
struct LeanShape {
    using LA = LeanA<T, D, TX, TY, TZ>;
    using LB = LeanB<T, D, TX, TY, TZ>;
    using FS = FluxSmem<T, D, TX, TY, TZ>;
    using TL = Tile<D, TX, TY, TZ>;
    static constexpr int mode = MODE_LEAN | MODE_FACES | (XF ? MODE_XF : 0);
    static constexpr size_t b_bytes = XF ? LB::bytes : FS::bytes;
    static size_t smem_bytes() { return LA::bytes > b_bytes ? LA::bytes : b_bytes; }

    static cudaError_t configure() {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_lsweep<T, D, TX, TY, TZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)LA::bytes)) ||
            (e = cudaFuncSetAttribute(k_lsweep<T, D, TX, TY, TZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)LA::bytes)) ||
            (e = cudaFuncSetAttribute(k_lsweep_batch<T, D, TX, TY, TZ, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LA::bytes)))
            return e;
        if constexpr (XF) {
            if ((e = cudaFuncSetAttribute(k_lflux<T, D, TX, TY, TZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)LB::bytes)) ||
                (e = cudaFuncSetAttribute(k_lflux<T, D, TX, TY, TZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)LB::bytes)) ||
                (e = cudaFuncSetAttribute(k_lflux_batch<T, D, TX, TY, TZ, false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LB::bytes)))
                return e;
        } else {
            if ((e = cudaFuncSetAttribute(k_flux<T, D, TX, TY, TZ, false, false, false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS::bytes)) ||
                (e = cudaFuncSetAttribute(k_flux<T, D, TX, TY, TZ, false, false, true>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS::bytes)) ||
                (e = cudaFuncSetAttribute(k_flux_batch<T, D, TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)FS::bytes)))
                return e;
        }
        done = true;
        return cudaSuccess;
    }

    static cudaError_t step(const Geo& g, const Inst<T>* in, int cur, cudaStream_t s, cudaEvent_t* ev, const void*) {
        cudaError_t e = configure();
        if (e) return e;
        const dim3 grid(g.tiles[0] * g.tiles[1] * g.tiles[2], g.G);
        if (ev) cudaEventRecord(ev[0], s);
        if (g.nosrc) e = launch_pdl(k_lsweep<T, D, TX, TY, TZ, true>, grid, dim3(TL::NT), LA::bytes, s, in, cur);
        else e = launch_pdl(k_lsweep<T, D, TX, TY, TZ, false>, grid, dim3(TL::NT), LA::bytes, s, in, cur);
        if (e) return e;
        if (ev) cudaEventRecord(ev[1], s);
        {
            long long nf = 0;
            for (int a = 0; a < D; ++a) nf = g.nf[a] > nf ? g.nf[a] : nf;
            const dim3 fgrid((unsigned)((nf + kSmallBlock - 1) / kSmallBlock), (unsigned)D);
            if ((e = launch_pdl(k_facec<T, D>, fgrid, dim3(kSmallBlock), 0, s, in, cur))) return e;
        }
        if (ev) cudaEventRecord(ev[2], s);
        if constexpr (XF) {
            if (g.nosrc) e = launch_pdl(k_lflux<T, D, TX, TY, TZ, true>, grid, dim3(TL::NT), LB::bytes, s, in, cur);
            else e = launch_pdl(k_lflux<T, D, TX, TY, TZ, false>, grid, dim3(TL::NT), LB::bytes, s, in, cur);
        } else {
            if (g.nosrc) e = launch_pdl(k_flux<T, D, TX, TY, TZ, false, false, true>, grid, dim3(TL::NT), FS::bytes, s, in, cur);
            else e = launch_pdl(k_flux<T, D, TX, TY, TZ, false, false, false>, grid, dim3(TL::NT), FS::bytes, s, in, cur);
        }
        if (e) return e;
        if (ev) cudaEventRecord(ev[3], s);
        if ((e = launch_pdl(k_wupdate<T, D>, dim3((unsigned)((g.Nc + kSmallBlock - 1) / kSmallBlock)), dim3(kSmallBlock),
                            0, s, in, cur)))
            return e;
        if (ev) cudaEventRecord(ev[4], s);
        return cudaGetLastError();
    }

    static cudaError_t sweep_batch(bool B, const Item* items, int n, const Inst<T>* insts, const int* cur,
                                   cudaStream_t s) {
        cudaError_t e = configure();
        if (e) return e;
        if (n <= 0) return cudaSuccess;
        if (!B)
            return launch_pdl(k_lsweep_batch<T, D, TX, TY, TZ, false>, dim3(n), dim3(TL::NT), LA::bytes, s, items, insts,
                              cur);
        if constexpr (XF)
            return launch_pdl(k_lflux_batch<T, D, TX, TY, TZ, false>, dim3(n), dim3(TL::NT), LB::bytes, s, items, insts,
                              cur);
        else
            return launch_pdl(k_flux_batch<T, D, TX, TY, TZ>, dim3(n), dim3(TL::NT), FS::bytes, s, items, insts, cur);
    }

    static TileShape shape() { return {{TL::T0, TL::T1, TL::T2}}; }

    static constexpr bool persistent = false;
    static cudaError_t persist(const PHead*, const PItem*, const Inst<T>*, int*, PState*, int, int, int, cudaStream_t) {
        return cudaErrorNotSupported;
    }
};

// A list of shapes for one dimension, indexed by tile id.
template <typename... S>
struct ShapeList;
template <>
struct ShapeList<> {
    static constexpr int count = 0;
    template <typename T>
    static cudaError_t step(int, const Geo&, const Inst<T>*, int, cudaStream_t, cudaEvent_t*, const void*) {
        return cudaErrorInvalidValue;
    }
    template <typename T>
    static cudaError_t sweep_batch(int, bool, const Item*, int, const Inst<T>*, const int*, cudaStream_t) {
        return cudaErrorInvalidValue;
    }
    static TileShape shape(int) { return {{0, 0, 0}}; }
    static size_t smem(int) { return 0; }
    static int mode(int) { return 0; }
    static bool persistent(int) { return false; }
    template <typename T>
    static cudaError_t persist(int, const PHead*, const PItem*, const Inst<T>*, int*, PState*, int, int, int,
                               cudaStream_t) {
        return cudaErrorInvalidValue;
    }
};
template <typename H, typename... R>
struct ShapeList<H, R...> {
    using Rest = ShapeList<R...>;
    static constexpr int count = 1 + Rest::count;
    template <typename T>
    static cudaError_t step(int id, const Geo& g, const Inst<T>* in, int cur, cudaStream_t s, cudaEvent_t* ev,
                            const void* phi_in) {
        return id == 0 ? H::step(g, in, cur, s, ev, phi_in)
                       : Rest::template step<T>(id - 1, g, in, cur, s, ev, phi_in);
    }
    template <typename T>
    static cudaError_t sweep_batch(int id, bool B, const Item* it, int n, const Inst<T>* in, const int* cur,
                                   cudaStream_t s) {
        return id == 0 ? H::sweep_batch(B, it, n, in, cur, s) : Rest::template sweep_batch<T>(id - 1, B, it, n, in, cur, s);
    }
    static TileShape shape(int id) { return id == 0 ? H::shape() : Rest::shape(id - 1); }
    static size_t smem(int id) { return id == 0 ? H::smem_bytes() : Rest::smem(id - 1); }
    static int mode(int id) { return id == 0 ? H::mode : Rest::mode(id - 1); }
    static bool persistent(int id) { return id == 0 ? H::persistent : Rest::persistent(id - 1); }
    template <typename T>
    static cudaError_t persist(int id, const PHead* h, const PItem* it, const Inst<T>* in, int* cur, PState* st, int n,
                               int w, int th, cudaStream_t s) {
        return id == 0 ? H::persist(h, it, in, cur, st, n, w, th, s)
                       : Rest::template persist<T>(id - 1, h, it, in, cur, st, n, w, th, s);
    }
};

// The shapes of one precision for D = 1, 2, 3.
template <typename T, typename L1, typename L2, typename L3>
struct ShapeTable {
    static int count(int D) { return D == 1 ? L1::count : (D == 2 ? L2::count : L3::count); }
    static TileShape shape(int D, int id) { return D == 1 ? L1::shape(id) : (D == 2 ? L2::shape(id) : L3::shape(id)); }
    static size_t smem(int D, int id) { return D == 1 ? L1::smem(id) : (D == 2 ? L2::smem(id) : L3::smem(id)); }
    static int mode(int D, int id) { return D == 1 ? L1::mode(id) : (D == 2 ? L2::mode(id) : L3::mode(id)); }
    static cudaError_t step(const Geo& g, const Inst<T>* in, int cur, cudaStream_t s, cudaEvent_t* ev,
                            const void* phi_in) {
        if (g.D == 1) return L1::template step<T>(g.tile_id, g, in, cur, s, ev, phi_in);
        if (g.D == 2) return L2::template step<T>(g.tile_id, g, in, cur, s, ev, phi_in);
        return L3::template step<T>(g.tile_id, g, in, cur, s, ev, phi_in);
    }
    static cudaError_t sweep_batch(int D, int id, bool B, const Item* it, int n, const Inst<T>* in, const int* cur,
                                   cudaStream_t s) {
        if (D == 1) return L1::template sweep_batch<T>(id, B, it, n, in, cur, s);
        if (D == 2) return L2::template sweep_batch<T>(id, B, it, n, in, cur, s);
        return L3::template sweep_batch<T>(id, B, it, n, in, cur, s);
    }
    static bool persistent(int D, int id) {
        return D == 1 ? L1::persistent(id) : (D == 2 ? L2::persistent(id) : L3::persistent(id));
    }
    static cudaError_t persist(int D, int id, const PHead* h, const PItem* it, const Inst<T>* in, int* cur, PState* st,
                               int n, int w, int th, cudaStream_t s) {
        if (D == 1) return L1::template persist<T>(id, h, it, in, cur, st, n, w, th, s);
        if (D == 2) return L2::template persist<T>(id, h, it, in, cur, st, n, w, th, s);
        return L3::template persist<T>(id, h, it, in, cur, st, n, w, th, s);
    }
};

template <typename T>
cudaError_t launch_rawq_batch(int D, const QItem* items, int n, const Inst<T>* insts, const int* cur, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    switch (D) {
        case 1: return launch_pdl(k_rawq_batch<T, 1>, dim3(n), dim3(kMomBlock), 0, s, items, insts, cur);
        case 2: return launch_pdl(k_rawq_batch<T, 2>, dim3(n), dim3(kMomBlock), 0, s, items, insts, cur);
        default: return launch_pdl(k_rawq_batch<T, 3>, dim3(n), dim3(kMomBlock), 0, s, items, insts, cur);
    }
}

// Per batched step: the pre-pass of the acceleration members, sweep A per
// tile shape, the raw face moments of the Shakhov members, the face
// constants, sweep B per tile shape, the raw cell moments of the Shakhov
// members, the W update.
template <typename Table, typename T>
cudaError_t run_batch_step(const BatchPlan& p, const Inst<T>* insts, int* cur, cudaStream_t s) {
    cudaError_t e;
    if (p.n_prep > 0) {
        switch (p.D) {
            case 1: e = launch_pdl(k_prep_batch<T, 1, true>, dim3(p.n_prep), dim3(kPrepCells), 0, s, p.prep_items, insts, cur); break;
            case 2: e = launch_pdl(k_prep_batch<T, 2, true>, dim3(p.n_prep), dim3(kPrepCells), 0, s, p.prep_items, insts, cur); break;
            default: e = launch_pdl(k_prep_batch<T, 3, true>, dim3(p.n_prep), dim3(kPrepCells), 0, s, p.prep_items, insts, cur); break;
        }
        if (e) return e;
    }
    for (int k = 0; k < p.ntile; ++k)
        if ((e = Table::sweep_batch(p.D, p.tile_id[k], false, p.sweep_items[k], p.n_sweep[k], insts, cur, s)))
            return e;
    if ((e = launch_rawq_batch<T>(p.D, p.faceq_items, p.n_faceq, insts, cur, s))) return e;
    if (p.n_face > 0) {
        switch (p.D) {
            case 1: e = launch_pdl(k_facec_batch<T, 1>, dim3(p.n_face), dim3(kSmallBlock), 0, s, p.face_items, insts, cur); break;
            case 2: e = launch_pdl(k_facec_batch<T, 2>, dim3(p.n_face), dim3(kSmallBlock), 0, s, p.face_items, insts, cur); break;
            default: e = launch_pdl(k_facec_batch<T, 3>, dim3(p.n_face), dim3(kSmallBlock), 0, s, p.face_items, insts, cur); break;
        }
        if (e) return e;
    }
    for (int k = 0; k < p.ntile; ++k)
        if ((e = Table::sweep_batch(p.D, p.tile_id[k], true, p.sweep_items[k], p.n_sweep[k], insts, cur, s)))
            return e;
    if ((e = launch_rawq_batch<T>(p.D, p.cellq_items, p.n_cellq, insts, cur, s))) return e;
    if (p.n_cell > 0) {
        switch (p.D) {
            case 1: e = launch_pdl(k_wupdate_batch<T, 1>, dim3(p.n_cell), dim3(kSmallBlock), 0, s, p.cell_items, insts, cur); break;
            case 2: e = launch_pdl(k_wupdate_batch<T, 2>, dim3(p.n_cell), dim3(kSmallBlock), 0, s, p.cell_items, insts, cur); break;
            default: e = launch_pdl(k_wupdate_batch<T, 3>, dim3(p.n_cell), dim3(kSmallBlock), 0, s, p.cell_items, insts, cur); break;
        }
        if (e) return e;
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
cudaError_t run_stress(const Geo& g, const Inst<T>* in, int cur, double* out, cudaStream_t s) {
    const dim3 grid((unsigned)g.Nc);
    switch (g.D) {
        case 1: k_stress<T, 1><<<grid, kStressThreads, 0, s>>>(in, cur, out); break;
        case 2: k_stress<T, 2><<<grid, kStressThreads, 0, s>>>(in, cur, out); break;
        default: k_stress<T, 3><<<grid, kStressThreads, 0, s>>>(in, cur, out); break;
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
