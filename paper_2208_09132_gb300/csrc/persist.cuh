// persist.cuh -- the persistent batched step: every phase of every member of a
// batch, for several time steps, in one launch.
//
// A step of one member is four kinds of work, each a set of items: sweep A
// (per tile and velocity group), the face constants (per range of faces),
// sweep B (per tile and group) and the W update (per range of cells).  Items of
// one member depend on each other in that order, and sweep A of the next step
// on the W update of this one; members are independent.  The launch walks one
// list of all items of all members -- per step the sweep A items of every
// member, then the face items, the sweep B items and the W items -- and each
// CTA takes the next item from a global counter.  Before it starts, the item
// waits (thread 0, bounded spin) until the member's counter of the kind it
// depends on has reached the count its step needs; when done, the CTA
// publishes its writes (fence) and counts itself.  An item waits only for items
// earlier in the list, which running CTAs hold, so the walk cannot deadlock
// whatever the number of CTAs.  A wait that runs out sets ST_TIMEOUT in the
// member's status word and an abort flag that stops every CTA.
//
// The list, the per-member item counts and the instance table live in device
// memory and are read at every launch, so a membership change rewrites them in
// place and a captured graph stays valid.  Items read what other items of the
// same launch wrote, so the bodies load coherently (no read-only path).
#pragma once

#include "kernels.cuh"

namespace cdg {

enum { PK_A = 0, PK_F = 1, PK_B = 2, PK_W = 3 };
constexpr int kPMaxMembers = 1024;

// One work item: sweep A / B: tile a, velocity group b; face constants: axis a,
// faces [start, start + count); W update: cells [start, start + count).
struct PItem {
    int inst, kind, a, b;
    long long start, count;
};
// The plan in device memory: items per step and, per member, the items of each
// kind per step.
struct PHead {
    int nmem, nitems, use_lim, pad;
    int per[kPMaxMembers][4];
    int lim[kPMaxMembers];        // with use_lim: member m runs min(lim[m], nsteps) steps of the launch
};
// Per launch (cleared before it): the next item to take, the abort flag and
// the completed items of each kind per member.
struct PState {
    unsigned next;
    int abort;
    int pad[2];
    unsigned cnt[kPMaxMembers][4];
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename T, int D, int TX, int TY, int TZ, int MODE>
struct PersistSmem {
    static constexpr bool FACES = mode_faces(MODE);
    static constexpr size_t a = Smem<T, D, TX, TY, TZ, MODE>::bytes(false);
    static constexpr size_t b = FACES ? FluxSmem<T, D, TX, TY, TZ>::bytes : Smem<T, D, TX, TY, TZ, MODE>::bytes(true);
    static constexpr size_t bytes = a > b ? a : b;
    static constexpr int occ_a = Occ<T, D, TX, TY, TZ, false, MODE>::value;
    static constexpr int occ_b = FACES ? FluxOcc<T, D, TX, TY, TZ>::value : Occ<T, D, TX, TY, TZ, true, MODE>::value;
    static constexpr int occ = occ_a < occ_b ? occ_a : occ_b;
};

// nsteps steps of every member.  wait_log2: a wait gives up after 2^wait_log2
// polls; test_hook = 1 makes the first face item wait for one item more than
// exists (the failure path of the waits, with nothing faulting).
template <typename T, int D, int TX, int TY, int TZ, int MODE>
__global__ void __launch_bounds__(Tile<D, TX, TY, TZ>::NT, (PersistSmem<T, D, TX, TY, TZ, MODE>::occ))
    k_batch_persist(const PHead* __restrict__ head, const PItem* __restrict__ items, const Inst<T>* __restrict__ insts,
                    int* cur, PState* st, int nsteps, int wait_log2, int test_hook) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned s_item;
    __shared__ int s_ok;
    constexpr int NT = Tile<D, TX, TY, TZ>::NT;
    constexpr bool FACES = mode_faces(MODE);
    const int t = threadIdx.x;
    const int nitems = head->nitems;
    const unsigned total = (unsigned)nitems * (unsigned)nsteps;
    for (;;) {
        if (t == 0) s_item = *(volatile int*)&st->abort ? total : atomicAdd(&st->next, 1u);
        __syncthreads();
        const unsigned gi = s_item;
        if (gi >= total) break;
        const int s = (int)(gi / (unsigned)nitems);
        const PItem it = items[gi % (unsigned)nitems];
        const int m = it.inst;
        // this member's steps in this launch (members may stop early: their later
        // items are no work, and nothing waits for them)
        const int nm = head->use_lim ? min(head->lim[m], nsteps) : nsteps;
        if (s >= nm) {
            __syncthreads();      // every thread has read s_item before thread 0 takes the next
            continue;
        }
        // the kind this item waits for, and how many of it its step needs
        int dk;
        unsigned need;
        switch (it.kind) {
            case PK_A: dk = PK_W; need = (unsigned)s * (unsigned)head->per[m][PK_W]; break;
            case PK_F: dk = PK_A; need = (unsigned)(s + 1) * (unsigned)head->per[m][PK_A]; break;
            case PK_B: dk = PK_F; need = (unsigned)(s + 1) * (unsigned)head->per[m][PK_F]; break;
            default: dk = PK_B; need = (unsigned)(s + 1) * (unsigned)head->per[m][PK_B]; break;
        }
        if (test_hook && it.kind == PK_F && s == 0) need += 1;        // a wait that cannot end
        if (t == 0) {
            bool ok = false;
            const long long lim = 1LL << wait_log2;
            for (long long k = 0; k < lim; ++k) {
                if (ld_acquire_u32(&st->cnt[m][dk]) >= need) {
                    ok = true;
                    break;
                }
                if (*(volatile int*)&st->abort) break;
                __nanosleep(64);
            }
            if (!ok) {
                atomicOr(insts[m].b[0].status, ST_TIMEOUT);
                atomicExch(&st->abort, 1);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        // Every body takes the member's record from the table directly: a copy
        // of the whole record on every thread's stack, made again for every
        // item, cost more than the items' own state traffic (each item's
        // acquire also evicts the stack lines from L1, so they go out to L2).
        const int c = (cur[m] + s) & 1;
        const Inst<T>& in = insts[m];
        if (it.kind == PK_A) {
            sweep_body<T, D, TX, TY, TZ, false, MODE, true>(in.g, in.b[c], it.a, it.b, smem);
        } else if (it.kind == PK_F) {
            for (long long k = t; k < it.count; k += NT) facec_body<T, D>(in.g, in.b[c], it.a, it.start + k);
        } else if (it.kind == PK_B) {
            if constexpr (FACES) flux_body<T, D, TX, TY, TZ, false, false, false, true>(in.g, in.b[c], it.a, it.b, smem);
            else sweep_body<T, D, TX, TY, TZ, true, MODE, true>(in.g, in.b[c], it.a, it.b, smem);
        } else {
            for (long long k = t; k < it.count; k += NT) wupdate_body<T, D>(in.g, in.b[c], it.start + k);
        }
        __syncthreads();
        if (t == 0) {
            __threadfence();          // this item's writes before its count
            const unsigned done = atomicAdd(&st->cnt[m][it.kind], 1u) + 1u;
            // the member's last W item of the launch: the state buffers trade places
            // nsteps times (no item of this member reads cur afterwards)
            if (it.kind == PK_W && done == (unsigned)nm * (unsigned)head->per[m][PK_W] && (nm & 1)) cur[m] ^= 1;
        }
    }
}

}  // namespace cdg
