// bulk.cuh -- the fused RHS + RK4 stage for two modes with every member's tile staged in shared
// memory, double-buffered across members: while member m is computed from shared memory, the
// copies of member m + 1 are in flight.  Same arithmetic, in the same order, as stage_points in
// kernels.cuh.  Two ways of filling the buffers:
//   stage_bulk_kernel     one thread issues 1D bulk async copies (cp.async.bulk, completion on
//                         an mbarrier; every wait bounded)
//   stage_cpasync_kernel  every thread issues 16-byte asynchronous copies (cp.async, zero-fill
//                         for points outside the grid, cp.async.wait_group on its own copies)
//
// Tile: TP = NT * 4 consecutive points of one p-plane (p_1 x p_2) of one q-point (q_1, q_2);
// each thread owns 4 consecutive p_2 points.  Per member a buffer holds
//   C   the tile with a halo of 3 p_1 rows on each side; the part outside the p-plane is zero,
//       which is the zero-outside-the-grid boundary along p_1: TP + 6 n_p2 values
//   Q   the same TP points at q-offsets k = -3..3 (k != 0) along q_1 and q_2: 12 chunks; a chunk
//       whose q index lies outside the grid reads as zero.
// The p_2 window comes from C with whole-vector masking (n_p2 % 4 == 0), as in kernels.cuh.
//
// Requirements (checked by the host): d = 2, FP32 with plain storage, n_p2 % 4 == 0, 16-byte
// aligned state pointers.  The bulk kernel's mbarrier waits are bounded (kWaitNs of
// %globaltimer); a block whose wait runs out sets *err = 1, lets its copies land (bounded again)
// and returns without storing, later launches skip their work, and the host reports
// CHFPE_ETIMEOUT.
#pragma once

#include "kernels.cuh"

namespace chfpe {

struct BulkArgs {
    int tiles_per_plane;   // ceil(Pp / TP)
    int H;                 // p_1 halo = 3 n_p2
    int buf_floats;        // floats per member buffer: TP + 2H + 12 TP
    int *err;              // device error word (bulk kernel)
};

constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;   // 0.2 s per wait

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity; false if it did not complete in kWaitNs
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :
        : "r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// geometry of one block's tile
struct Tile {
    int qp, tile, ps, t0, TPe, lo, hi, c_off;
    int iq[2];
    bool qvalid[2][6];   // kk = 0..5 <-> k = -3, -2, -1, +1, +2, +3
};

template <int TP>
__device__ __forceinline__ Tile tile_of(const Geo<float> &g, const BulkArgs &b) {
    Tile t;
    t.qp = blockIdx.x / b.tiles_per_plane;
    t.tile = blockIdx.x - t.qp * b.tiles_per_plane;
    t.ps = t.qp * g.Pp;
    t.t0 = t.ps + t.tile * TP;
    t.TPe = min(TP, g.Pp - t.tile * TP);
    t.lo = max(t.t0 - b.H, t.ps);
    t.hi = min(t.t0 + t.TPe + b.H, t.ps + g.Pp);
    t.c_off = t.lo - (t.t0 - b.H);
    t.iq[0] = t.qp / g.n[1];
    t.iq[1] = t.qp % g.n[1];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
            const int k = kk < 3 ? kk - 3 : kk - 2;
            t.qvalid[s][kk] = t.iq[s] + k >= 0 && t.iq[s] + k < g.n[s];
        }
    return t;
}

// per-point coefficients of this thread's 4 points (as in stage_points)
struct Coef {
    float Fs[2], vq[2][4], VpD[2], VpK[2][4];
    int ip[2];
};

__device__ __forceinline__ Coef coef_of(const Geo<float> &g, const Tile &t, int li, int TP) {
    Coef c;
    const int rel = t.tile * TP + li;
    c.ip[0] = rel / g.n[3];
    c.ip[1] = rel % g.n[3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float q = g.qlo[s] + float(t.iq[s]) * g.qh[s];
        const float Vp = g.VLL[s] + g.VSL[s] * q;
        c.Fs[s] = __ldg(g.F + s * g.NQ + t.qp);
        c.VpD[s] = Vp * g.inv60hp[s];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ipj = c.ip[s] + (s == 1 ? j : 0);
            const float p = g.plo[s] + float(ipj) * g.ph[s];
            c.vq[s][j] = p * g.vq[s];
            c.VpK[s][j] = Vp * g.kappa[s] * p;
        }
    }
    return c;
}

// member m's terms at this thread's 4 points from a staged buffer (C = tile centre, Q = the 12
// q-neighbour chunks), scattered into the accumulators of m and its hierarchy neighbours
template <int DEPTH, int TP>
__device__ __forceinline__ void tile_member(const Geo<float> &g, const float *C, const float *Q,
                                            const Tile &t, const Coef &c, int li, int m,
                                            float (&acc)[member_count(2, DEPTH)][4]) {
    constexpr int D = 2, V = 4;
    constexpr MemberTable<D, DEPTH> tab{};
    float w[12];
#pragma unroll
    for (int vb = 0; vb < 3; ++vb) {
        const int off = (vb - 1) * V;
        const bool okv = c.ip[1] + off >= 0 && c.ip[1] + off < g.n[3];
        const float4 u = okv ? *reinterpret_cast<const float4 *>(C + li + off) : make_float4(0.f, 0.f, 0.f, 0.f);
        w[vb * 4 + 0] = u.x;
        w[vb * 4 + 1] = u.y;
        w[vb * 4 + 2] = u.z;
        w[vb * 4 + 3] = u.w;
    }
    float dp[D][V], v[V], k[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int cc = 4 + j;
        dp[1][j] = 45.f * (w[cc + 1] - w[cc - 1]) - 9.f * (w[cc + 2] - w[cc - 2]) + (w[cc + 3] - w[cc - 3]);
        v[j] = w[cc];
    }
    {
        const int r = g.n[3];   // p_1 stride
        const float4 p1 = *reinterpret_cast<const float4 *>(C + li + r);
        const float4 m1 = *reinterpret_cast<const float4 *>(C + li - r);
        const float4 p2 = *reinterpret_cast<const float4 *>(C + li + 2 * r);
        const float4 m2 = *reinterpret_cast<const float4 *>(C + li - 2 * r);
        const float4 p3 = *reinterpret_cast<const float4 *>(C + li + 3 * r);
        const float4 m3 = *reinterpret_cast<const float4 *>(C + li - 3 * r);
        dp[0][0] = 45.f * (p1.x - m1.x) - 9.f * (p2.x - m2.x) + (p3.x - m3.x);
        dp[0][1] = 45.f * (p1.y - m1.y) - 9.f * (p2.y - m2.y) + (p3.y - m3.y);
        dp[0][2] = 45.f * (p1.z - m1.z) - 9.f * (p2.z - m2.z) + (p3.z - m3.z);
        dp[0][3] = 45.f * (p1.w - m1.w) - 9.f * (p2.w - m2.w) + (p3.w - m3.w);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) k[j] = 0.f;
#pragma unroll
    for (int s = 0; s < D; ++s) {
        float4 q[6];
#pragma unroll
        for (int kk = 0; kk < 6; ++kk)
            q[kk] = t.qvalid[s][kk] ? *reinterpret_cast<const float4 *>(Q + (s * 6 + kk) * TP + li)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
        float dq[V];
        dq[0] = 45.f * (q[3].x - q[2].x) - 9.f * (q[4].x - q[1].x) + (q[5].x - q[0].x);
        dq[1] = 45.f * (q[3].y - q[2].y) - 9.f * (q[4].y - q[1].y) + (q[5].y - q[0].y);
        dq[2] = 45.f * (q[3].z - q[2].z) - 9.f * (q[4].z - q[1].z) + (q[5].z - q[0].z);
        dq[3] = 45.f * (q[3].w - q[2].w) - 9.f * (q[4].w - q[1].w) + (q[5].w - q[0].w);
#pragma unroll
        for (int j = 0; j < V; ++j) k[j] += c.Fs[s] * dp[s][j] - c.vq[s][j] * dq[j];
    }
    float gm = 0.f;
#pragma unroll
    for (int s = 0; s < D; ++s) gm += float(tab.n[m][s]) * g.gam[s];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        acc[m][j] += k[j] - gm * v[j];
#pragma unroll
        for (int s = 0; s < D; ++s) {
            if (tab.dn[m][s] >= 0) {
                const float wl = g.link[s][tab.n[m][s]];
                acc[tab.dn[m][s]][j] += wl * (c.VpD[s] * dp[s][j] - c.VpK[s][j] * v[j]);
            }
            if (tab.up[m][s] >= 0) {
                const float wl = g.link[s][tab.n[m][s] + 1];
                acc[tab.up[m][s]][j] += wl * (c.VpD[s] * dp[s][j] + c.VpK[s][j] * v[j]);
            }
        }
    }
}

// out = y + c acc (y == nullptr: out = c acc) for every member at this thread's 4 points
template <int M>
__device__ __forceinline__ void tile_store(const StageArgs<float> &a, long long boff, int x0,
                                           const float (&acc)[M][4]) {
    const float *yb = a.y ? reinterpret_cast<const float *>(a.y + boff) : nullptr;
    float *ob = reinterpret_cast<float *>(a.out + boff);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        float rr[4];
        if (yb) {
            const float4 yv = *reinterpret_cast<const float4 *>(yb + (long long)m * a.g.P + x0);
            rr[0] = yv.x + a.c * acc[m][0];
            rr[1] = yv.y + a.c * acc[m][1];
            rr[2] = yv.z + a.c * acc[m][2];
            rr[3] = yv.w + a.c * acc[m][3];
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) rr[j] = a.c * acc[m][j];
        }
        *reinterpret_cast<float4 *>(ob + (long long)m * a.g.P + x0) = make_float4(rr[0], rr[1], rr[2], rr[3]);
    }
}

template <int DEPTH, int NT>
__global__ void __launch_bounds__(NT, 4) stage_bulk_kernel(const StageArgs<float> a, const BulkArgs b) {
    constexpr int TP = NT * 4;
    constexpr int M = member_count(2, DEPTH);
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ int failed_before;

    // after a wait gave up in an earlier launch, skip the work (block-uniform decision)
    if (threadIdx.x == 0) failed_before = *reinterpret_cast<volatile int *>(b.err);
    __syncthreads();
    if (failed_before) return;

    const Geo<float> &g = a.g;
    const int tid = threadIdx.x;
    const Tile t = tile_of<TP>(g, b);
    const int H = b.H;
    const long long boff = (long long)blockIdx.y * a.state_bytes;
    const float *in = reinterpret_cast<const float *>(a.in + boff);
    uint32_t bytes = (uint32_t)(t.hi - t.lo) * 4u;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int kk = 0; kk < 6; ++kk)
            if (t.qvalid[s][kk]) bytes += (uint32_t)t.TPe * 4u;

    // zero the never-copied part of C in both buffers (rows beyond the p-plane)
    for (int bi = 0; bi < 2; ++bi) {
        float *C = smem + bi * b.buf_floats;
        for (int j = tid; j < t.c_off; j += NT) C[j] = 0.f;
        for (int j = t.c_off + (t.hi - t.lo) + tid; j < TP + 2 * H; j += NT) C[j] = 0.f;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int m, int bi) {   // thread 0: all copies of member m into buffer bi
        float *buf = smem + bi * b.buf_floats;
        const float *src = in + (long long)m * g.P;
        const uint32_t bar = smem_u32(&mbar[bi]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        bulk_copy(smem_u32(buf + t.c_off), src + t.lo, (uint32_t)(t.hi - t.lo) * 4u, bar);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) {
                const int k = kk < 3 ? kk - 3 : kk - 2;
                if (t.qvalid[s][kk])
                    bulk_copy(smem_u32(buf + TP + 2 * H + (s * 6 + kk) * TP), src + t.t0 + k * g.st[s],
                              (uint32_t)t.TPe * 4u, bar);
            }
    };
    if (tid == 0) issue(0, 0);

    const int li = tid * 4;
    const bool active = li < t.TPe;
    const Coef c = coef_of(g, t, li, TP);
    float acc[M][4];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[m][j] = 0.f;

    bool ok = true;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int bi = m & 1;
        if (m + 1 < M && tid == 0) issue(m + 1, bi ^ 1);
        ok = mbar_wait_bounded(smem_u32(&mbar[bi]), (uint32_t)((m >> 1) & 1)) && ok;
        const float *buf = smem + bi * b.buf_floats;
        if (active) tile_member<DEPTH, TP>(g, buf + H, buf + TP + 2 * H, t, c, li, m, acc);
        // every thread is done with buffer bi before it is refilled (member m + 2); the vote
        // makes a timed-out wait a block-uniform decision
        if (!__syncthreads_and(ok ? 1 : 0)) {
            if (tid == 0) {
                atomicExch(b.err, 1);
                // let copies still in flight (members m and m + 1) land, bounded again, before
                // the block's shared memory goes away
                mbar_wait_bounded(smem_u32(&mbar[bi]), (uint32_t)((m >> 1) & 1));
                if (m + 1 < M) mbar_wait_bounded(smem_u32(&mbar[bi ^ 1]), (uint32_t)(((m + 1) >> 1) & 1));
            }
            return;
        }
    }
    if (active) tile_store<M>(a, boff, t.t0 + li, acc);
}

template <int DEPTH, int NT>
__global__ void __launch_bounds__(NT, 4) stage_cpasync_kernel(const StageArgs<float> a, const BulkArgs b) {
    constexpr int TP = NT * 4;
    constexpr int M = member_count(2, DEPTH);
    extern __shared__ __align__(128) float smem[];

    const Geo<float> &g = a.g;
    const int tid = threadIdx.x;
    const Tile t = tile_of<TP>(g, b);
    const int H = b.H;
    const long long boff = (long long)blockIdx.y * a.state_bytes;
    const float *in = reinterpret_cast<const float *>(a.in + boff);
    const int li = tid * 4;
    const bool active = li < t.TPe;
    const int cpieces = (TP + 2 * H) / 4;

    // all threads: the copies of member m into buffer bi, one commit group
    auto issue = [&](int m, int bi) {
        float *buf = smem + bi * b.buf_floats;
        const float *src = in + (long long)m * g.P;
        for (int j = tid; j < cpieces; j += NT) {
            const int gp = t.t0 - H + 4 * j;                 // first point of the piece
            const bool inside = gp >= t.lo && gp + 4 <= t.hi;
            cp_async16(buf + 4 * j, inside ? src + gp : src, inside ? 16 : 0);
        }
        if (active) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int kk = 0; kk < 6; ++kk) {
                    const int k = kk < 3 ? kk - 3 : kk - 2;
                    const bool v = t.qvalid[s][kk];
                    cp_async16(buf + TP + 2 * H + (s * 6 + kk) * TP + li,
                               v ? src + t.t0 + k * g.st[s] + li : src, v ? 16 : 0);
                }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(0, 0);

    const Coef c = coef_of(g, t, li, TP);
    float acc[M][4];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[m][j] = 0.f;

#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int bi = m & 1;
        if (m + 1 < M) {
            issue(m + 1, bi ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");   // member m's group is done
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();                                           // everyone's copies visible
        const float *buf = smem + bi * b.buf_floats;
        if (active) tile_member<DEPTH, TP>(g, buf + H, buf + TP + 2 * H, t, c, li, m, acc);
        __syncthreads();                                           // buffer bi free for m + 2
    }
    if (active) tile_store<M>(a, boff, t.t0 + li, acc);
}

}  // namespace chfpe
