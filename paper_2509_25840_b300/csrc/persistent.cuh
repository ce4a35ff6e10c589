// persistent.cuh -- a whole sampled propagation (nsamples observations, stride RK4 steps between
// them, every state of a batch) in one cooperative launch: the RK4 stages of stage_points and
// the FP64 observable reduction separated by grid-wide barriers instead of kernel boundaries.
// For small states, where a stage takes a few microseconds and launch gaps dominate.
//
// Every block owns the same tiles in every stage, so the in-place last stage (out = y) writes
// only points the writing thread itself reads.  States rewritten inside the launch are read with
// L2-only loads (stage_points<..., NC = false>, __ldcg), never through the non-coherent path.
// The grid barrier is bounded: a block that waits longer than kBarrierNs (or finds the error
// word set) sets *err = 1 and returns; the host reports CHFPE_ETIMEOUT.
#pragma once

#include "kernels.cuh"

namespace chfpe {

struct PersistArgs {
    char *y, *za, *zb;        // batch arenas, state_bytes apart
    long long state_bytes;
    int batch, tiles_per_state;
    double dt;
    int nsamples, stride;
    const double *CWq, *wp;   // observable weights (as ObserveArgs)
    int wp_ld;
    double vol;               // cell volume
    double *partial;          // [batch][ceil(P / kObsChunk)] chunk sums
    double *out;              // out[b * out_stride + k]
    long long out_stride;
    unsigned *bar;            // [0] arrivals, [1] generation
    int *err;
};

constexpr unsigned long long kBarrierNs = 1000ull * 1000 * 1000;   // 1 s per barrier
constexpr int kObsChunk = 1024;                                     // points per partial sum

__device__ __forceinline__ unsigned long long ptimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid-wide barrier of a cooperative launch; gen is thread 0's copy of the generation
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, unsigned &gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = gen + 1;
        __threadfence();                                    // release this block's writes
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {      // last to arrive: open the barrier
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], target);
        } else {
            const unsigned long long t0 = ptimer();
            while (ld_acquire_u32(&bar[1]) != target) {
                if (ld_acquire_u32(reinterpret_cast<const unsigned *>(err)) != 0u ||
                    ptimer() - t0 > kBarrierNs) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();                                    // acquire the other blocks' writes
        gen = target;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T, int D, int DEPTH, int V, int NT>
__global__ void __launch_bounds__(NT) persistent_kernel(const Geo<T> g, const PersistArgs p) {
    constexpr int M = member_count(D, DEPTH);
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire_u32(&p.bar[1]);
    const int ntiles = p.tiles_per_state * p.batch;

    auto stage = [&](const char *in, const char *yb, char *out, T c) {
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int b = t / p.tiles_per_state;
            const int x0 = ((t - b * p.tiles_per_state) * NT + threadIdx.x) * V;
            if (x0 < g.P) {
                const long long off = (long long)b * p.state_bytes;
                stage_points<T, D, DEPTH, V, M, false>(g, in + off, yb + off, out + off, c, x0);
            }
        }
    };

    const int nchunks = (g.P + kObsChunk - 1) / kObsChunk;
    for (int k = 0; k < p.nsamples; ++k) {
        // observable of member 0 of every state (same weights as observe_partial_kernel): partial
        // sums over fixed chunks of kObsChunk points, then one block per state adds the chunk sums
        // in chunk order -- the order of the additions does not depend on the grid size
        for (int wk = blockIdx.x; wk < p.batch * nchunks; wk += gridDim.x) {
            const int b = wk / nchunks, c = wk - b * nchunks;
            const T *g0 = reinterpret_cast<const T *>(p.y + (long long)b * p.state_bytes);
            const int xe = min(g.P, (c + 1) * kObsChunk);
            double sum = 0.0;
            for (int x = c * kObsChunk + threadIdx.x; x < xe; x += NT) {
                const int qlin = x / g.Pp;
                int r = x - qlin * g.Pp;
                double w = p.CWq[qlin];
                for (int s = D - 1; s >= 0; --s) {
                    const int ip = r % g.n[D + s];
                    r /= g.n[D + s];
                    w *= p.wp[s * p.wp_ld + ip];
                }
                sum += w * (double)__ldcg(g0 + x);
            }
            sum = block_sum<NT>(sum);
            if (threadIdx.x == 0) p.partial[wk] = sum;
            __syncthreads();   // block_sum's shared slots are free before the next chunk
        }
        if (!grid_barrier(p.bar, p.err, gen)) return;
        for (int b = blockIdx.x; b < p.batch; b += gridDim.x) {
            if (threadIdx.x < 32) {
                double s = 0.0;
                for (int j = threadIdx.x; j < nchunks; j += 32)
                    s += __ldcg(&p.partial[(long long)b * nchunks + j]);
                s = warp_sum(s);
                if (threadIdx.x == 0) p.out[(long long)b * p.out_stride + k] = p.vol * s;
            }
        }
        if (k == p.nsamples - 1) break;
        if (p.stride == 0 && !grid_barrier(p.bar, p.err, gen)) return;   // partials read before reuse
        // Horner-form RK4 with the host's stage coefficients (formed in FP64, then rounded)
        const T c1 = (T)(p.dt / 4.0), c2 = (T)(p.dt / 3.0), c3 = (T)(p.dt / 2.0), c4 = (T)p.dt;
        for (int st = 0; st < p.stride; ++st) {
            stage(p.y, p.y, p.za, c1);
            if (!grid_barrier(p.bar, p.err, gen)) return;
            stage(p.za, p.y, p.zb, c2);
            if (!grid_barrier(p.bar, p.err, gen)) return;
            stage(p.zb, p.y, p.za, c3);
            if (!grid_barrier(p.bar, p.err, gen)) return;
            stage(p.za, p.y, p.y, c4);
            if (!grid_barrier(p.bar, p.err, gen)) return;
        }
    }
}

}  // namespace chfpe
