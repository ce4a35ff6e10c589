// batch_persistent.cuh -- a batch's RK4 substep slots in one cooperative launch: every instance
// of a batch of uneven grids (chfpe_create_batch), each stage a grid-stride pass over the work
// lists of the slot's substep level (4-, 2- and 1-point tiles of (instance, tile) items, the
// instance's geometry and stage coefficient copied into shared memory per item), the stages
// separated by the bounded grid barrier of persistent.cuh instead of kernel boundaries.  For
// batches of small instances, where a stage takes microseconds and launch gaps dominate.
//
// Every item is a fixed tile of one instance in every stage, so the in-place last stage writes
// only points the writing thread itself read; states rewritten inside the launch are read with
// L2-only loads (stage_points<..., NC = false>).
#pragma once

#include "kernels.cuh"
#include "persistent.cuh"

namespace chfpe {

template <typename T>
struct BatchPersistArgs {
    const InstGeo<T> *inst;
    const int2 *const *lists;   // [level * 3 + class] work lists (device array of device pointers)
    const int *counts;          // their lengths
    char *y, *za, *zb;          // the batch arenas
    long long nslots;           // substep slots to advance
    int nsub, top;              // slots per nominal step; the level of slot 0 (all instances)
    unsigned *bar;              // grid barrier: arrivals, generation
    int *err;
};

// FOUR: the 4-point class is compiled (its list is empty otherwise); VEC: the 2-point class's
// points per thread
template <typename T, int D, int DEPTH, int M32, int VEC, bool FOUR>
__global__ void __launch_bounds__(128, 4) batch_persistent_kernel(const BatchPersistArgs<T> p) {
    __shared__ __align__(16) InstGeo<T> sg;
    static_assert(sizeof(InstGeo<T>) % 4 == 0 && sizeof(InstGeo<T>) / 4 <= 4 * 128, "geometry copy");
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire_u32(&p.bar[1]);
    for (long long k = 0; k < p.nslots; ++k) {
        const long long j = k % p.nsub;
        const int l = j == 0 ? p.top : __ffsll(j) - 1;
        for (int st = 0; st < 4; ++st) {
            // Horner-form RK4 (the order of batch_rk4): in y, za, zb, za; out za, zb, za, y
            const char *in = st == 0 ? p.y : (st == 2 ? p.zb : p.za);
            char *out = st == 0 ? p.za : (st == 1 ? p.zb : (st == 2 ? p.za : p.y));
            for (int c = 0; c < 3; ++c) {
                const int2 *list = p.lists[l * 3 + c];
                const int n = p.counts[l * 3 + c];
                for (int it = blockIdx.x; it < n; it += gridDim.x) {
                    const int2 item = list[it];
                    __syncthreads();   // every thread is done with the previous item's geometry
                    {
                        const unsigned *src = reinterpret_cast<const unsigned *>(p.inst + item.x);
                        unsigned *dst = reinterpret_cast<unsigned *>(&sg);
                        for (int w = threadIdx.x; w < (int)(sizeof(InstGeo<T>) / 4); w += 128)
                            dst[w] = __ldg(src + w);
                    }
                    __syncthreads();
                    const long long off = sg.off;
                    const T cc = sg.cst[st];
                    if (c == 0) {
                        if constexpr (FOUR) {
                            const int x0 = (item.y * 128 + threadIdx.x) * 4;
                            if (x0 < sg.g.P)
                                stage_points<T, D, DEPTH, 4, M32, false, false, 0, 1>(
                                    sg.g, in + off, p.y + off, out + off, cc, x0);
                        }
                    } else if (c == 1) {
                        const int x0 = (item.y * 128 + threadIdx.x) * VEC;
                        if (x0 < sg.g.P)
                            stage_points<T, D, DEPTH, VEC, M32, false, false, 0, 1>(
                                sg.g, in + off, p.y + off, out + off, cc, x0);
                    } else {
                        const int x0 = item.y * 128 + threadIdx.x;
                        if (x0 < sg.g.P)
                            stage_points<T, D, DEPTH, 1, M32, false, false, 0, 1>(
                                sg.g, in + off, p.y + off, out + off, cc, x0);
                    }
                }
            }
            if (!grid_barrier(p.bar, p.err, gen)) return;
        }
    }
}

}  // namespace chfpe
