// stage_launch.cuh -- host-side launch of the fused RHS + RK4 stage kernels (kernels.cuh,
// bulk.cuh) in every launch shape the autotuner chooses from.  The launchers are instantiated
// per number of modes in stage_d1.cu, stage_d2.cu and stage_d3.cu (separate translation units,
// compiled in parallel); chfpe.cu calls launch_stage_dim<T, D>.
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "bulk.cuh"

namespace chfpe {

// Vectorised stage kernel shape: two consecutive p_d points per thread (float2 / double2), 128
// threads per block, registers capped so that 8 blocks (32 warps) fit on an SM for hierarchies
// of up to 15 members (4 blocks beyond).  Measured on the 32^4 x 15 workload: occupancy beats
// per-thread reuse here (float4 at 8 warps/SM: 1.6 TB/s; float2 at 32 warps/SM: 2.0 TB/s).
constexpr int kVec = 2;

// Launch shapes the autotuner chooses from (FP32, plain storage, the workload hierarchies
// (d, depth) = (1, 5), (2, 2), (2, 4), (3, 2); every other configuration uses shape 0):
//   0  2 points per thread, 128 threads, registers for 8 blocks per SM (4 beyond 15 members)
//   1  2 points per thread, 256 threads, same registers per thread (more p_1 rows per block)
//   2  2 points per thread, 128 threads, registers for 6 blocks per SM (fewer spills)
//   3  4 points per thread, 128 threads, registers for 4 blocks per SM (needs n_pd % 4 == 0)
//   4  shape 3 with every member's tile staged in shared memory by bulk async copies, double
//      buffered across members (two modes only; bulk.cuh)
//   5  shape 4 with the buffers filled by every thread's 16-byte cp.async copies
//   6  shape 3 with 256 threads (2 blocks per SM)
//   7  shape 3 with 64 threads (8 blocks per SM)
//   8  shape 3 with L1 prefetch hints for the next member's q-neighbours
//   9  shape 3 with the next member's q-neighbours staged by cp.async in thread-private shared
//      memory slots (no block barrier)
//  10  shape 3 with registers for 3 blocks per SM (168)
//  11  shape 3 with registers for 2 blocks per SM (255)
//  12  early stores (ES: each member stored once its last contribution is in) in an order that
//      keeps few accumulators open (MemberTable::order), 4 points, 128 threads, 5 blocks per SM
//  13  ES in storage order, 4 points, 128 threads, 5 blocks per SM (102 registers)
//  14  ES in storage order, 2 points, 128 threads, 8 blocks per SM (64)
//  15  ES in storage order, 4 points, 256 threads, 2 blocks per SM
//  16  ES in storage order, 4 points, 128 threads, 4 blocks per SM (128)
//  17  ES in the open-accumulator order, 4 points, 128 threads, 4 blocks per SM
// Shapes 3-17 need n_pd % 4 == 0 (shape 0 runs otherwise).  (Shapes with a block
// covering a small box of grid rows along (q_{d-1}, q_d, p_{d-1}), meant to turn q-neighbour taps
// into L1 hits, ran 2-20 % slower than shape 3 on the two-mode workload and were removed.)
constexpr int kStageVariants = 18;

constexpr bool tunable(int T_size, int D, int DEPTH) {
    return T_size == 4 && ((D == 1 && DEPTH == 5) || (D == 2 && (DEPTH == 2 || DEPTH == 4)) ||
                           (D == 3 && DEPTH == 2));
}

template <typename T, int D, int DEPTH, int M32, int V, int NT, int MINB, bool PF = false,
          bool QST = false, int ES = 0>
static void launch_vec(const StageArgs<T> &a, int batch, cudaStream_t s) {
    const int nthr = a.g.P / V;
    auto kern = stage_vec_kernel<T, D, DEPTH, V, NT, MINB, M32, PF, QST, ES>;
    size_t smem = 0;
    if constexpr (QST) {   // two slot sets of 6 D float4 per thread
        smem = (size_t)2 * 6 * D * NT * sizeof(float4);
        static bool configured = false;
        if (!configured) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            configured = true;
        }
    }
    kern<<<dim3((nthr + NT - 1) / NT, batch), NT, smem, s>>>(a);
}

constexpr int kBulkNT = 128, kBulkTP = kBulkNT * 4;

inline BulkArgs bulk_args(const Geo<float> &g, int *err) {
    BulkArgs b;
    b.tiles_per_plane = (g.Pp + kBulkTP - 1) / kBulkTP;
    b.H = 3 * g.n[3];
    b.buf_floats = kBulkTP + 2 * b.H + 12 * kBulkTP;
    b.err = err;
    return b;
}

inline bool bulk_ok(const Geo<float> &g) { return g.n[3] % 4 == 0; }

// shapes 4 (bulk async copies) and 5 (16-byte cp.async) of two-mode hierarchies
template <int DEPTH, bool CPASYNC>
static void launch_bulk(const StageArgs<float> &a, int batch, int *err, cudaStream_t s) {
    const BulkArgs b = bulk_args(a.g, err);
    const size_t smem = (size_t)2 * b.buf_floats * sizeof(float);
    auto kern = CPASYNC ? stage_cpasync_kernel<DEPTH, kBulkNT> : stage_bulk_kernel<DEPTH, kBulkNT>;
    static size_t configured = 0;   // largest dynamic shared memory opted into so far
    if (smem > configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    kern<<<dim3(a.g.NQ * b.tiles_per_plane, batch), kBulkNT, smem, s>>>(a, b);
}

template <typename T, int D, int DEPTH, int M32>
static void launch_stage_m(const StageArgs<T> &a, int batch, bool vec, int variant, int *err,
                           cudaStream_t s) {
    constexpr int M = member_count(D, DEPTH);
    constexpr int MINB = (sizeof(T) == 4 && M <= 15) ? 8 : 4;
    if (!vec) {
        stage_vec_kernel<T, D, DEPTH, 1, 128, 4, M32>
            <<<dim3((a.g.P + 127) / 128, batch), 128, 0, s>>>(a);
        return;
    }
    if constexpr (tunable(sizeof(T), D, DEPTH) && M32 == M) {
        switch (variant) {
        case 1: launch_vec<T, D, DEPTH, M32, 2, 256, MINB / 2>(a, batch, s); return;
        case 2: launch_vec<T, D, DEPTH, M32, 2, 128, 6>(a, batch, s); return;
        case 3: launch_vec<T, D, DEPTH, M32, 4, 128, 4>(a, batch, s); return;
        case 6: launch_vec<T, D, DEPTH, M32, 4, 256, 2>(a, batch, s); return;
        case 7: launch_vec<T, D, DEPTH, M32, 4, 64, 8>(a, batch, s); return;
        case 8: launch_vec<T, D, DEPTH, M32, 4, 128, 4, true>(a, batch, s); return;
        case 9: launch_vec<T, D, DEPTH, M32, 4, 128, 4, false, true>(a, batch, s); return;
        case 10: launch_vec<T, D, DEPTH, M32, 4, 128, 3>(a, batch, s); return;
        case 11: launch_vec<T, D, DEPTH, M32, 4, 128, 2>(a, batch, s); return;
        case 12: launch_vec<T, D, DEPTH, M32, 4, 128, 5, false, false, 2>(a, batch, s); return;
        case 13: launch_vec<T, D, DEPTH, M32, 4, 128, 5, false, false, 1>(a, batch, s); return;
        case 14: launch_vec<T, D, DEPTH, M32, 2, 128, 8, false, false, 1>(a, batch, s); return;
        case 15: launch_vec<T, D, DEPTH, M32, 4, 256, 2, false, false, 1>(a, batch, s); return;
        case 16: launch_vec<T, D, DEPTH, M32, 4, 128, 4, false, false, 1>(a, batch, s); return;
        case 17: launch_vec<T, D, DEPTH, M32, 4, 128, 4, false, false, 2>(a, batch, s); return;
        case 4:
        case 5:
            if constexpr (D == 2) {
                if (bulk_ok(a.g)) {
                    if (variant == 4) launch_bulk<DEPTH, false>(a, batch, err, s);
                    else launch_bulk<DEPTH, true>(a, batch, err, s);
                    return;
                }
            }
            break;
        default: break;
        }
    }
    launch_vec<T, D, DEPTH, M32, kVec, 128, MINB>(a, batch, s);
}

template <typename T, int D, int DEPTH>
static bool launch_stage_t(const StageArgs<T> &a, int batch, bool vec, int M32, int variant,
                           int *err, cudaStream_t s) {
    constexpr int M = member_count(D, DEPTH);
    if (M32 == M) {
        launch_stage_m<T, D, DEPTH, M>(a, batch, vec, variant, err, s);
        return true;
    }
    if constexpr (sizeof(T) == 4 && D == 2 && DEPTH == 4) {
        if (M32 == 6) {
            launch_stage_m<T, D, DEPTH, 6>(a, batch, vec, 0, err, s);
            return true;
        }
    }
    if constexpr (sizeof(T) == 4 && D == 3 && DEPTH == 2) {
        if (M32 == 4) {
            launch_stage_m<T, D, DEPTH, 4>(a, batch, vec, 0, err, s);
            return true;
        }
    }
    return false;
}

// One RK4 stage of `batch` states of a D-mode hierarchy of the given depth in launch shape
// `variant`; false for a (D, depth, storage) combination that is not compiled.  Specialised for
// T = float, double in stage_d<D>.cu.
template <typename T, int D>
bool launch_stage_dim(int depth, const StageArgs<T> &a, int batch, bool vec, int M32, int variant,
                      int *err, cudaStream_t s);
template <>
bool launch_stage_dim<float, 1>(int depth, const StageArgs<float> &a, int batch, bool vec, int M32,
                                 int variant, int *err, cudaStream_t s);
template <>
bool launch_stage_dim<double, 1>(int depth, const StageArgs<double> &a, int batch, bool vec, int M32,
                                 int variant, int *err, cudaStream_t s);
template <>
bool launch_stage_dim<float, 2>(int depth, const StageArgs<float> &a, int batch, bool vec, int M32,
                                 int variant, int *err, cudaStream_t s);
template <>
bool launch_stage_dim<double, 2>(int depth, const StageArgs<double> &a, int batch, bool vec, int M32,
                                 int variant, int *err, cudaStream_t s);
template <>
bool launch_stage_dim<float, 3>(int depth, const StageArgs<float> &a, int batch, bool vec, int M32,
                                 int variant, int *err, cudaStream_t s);
template <>
bool launch_stage_dim<double, 3>(int depth, const StageArgs<double> &a, int batch, bool vec, int M32,
                                 int variant, int *err, cudaStream_t s);

}  // namespace chfpe
