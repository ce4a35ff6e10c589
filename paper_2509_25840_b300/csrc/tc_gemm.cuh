// tc_gemm.cuh -- BF16 GEMM on the fifth-generation tensor cores (tcgen05) of sm_100-class GPUs,
// for the surrogate's contractions:
//
//   C[m][n] (=, or += with FP32 atomics under split-K) sum_k A(m, k) B(n, k)  (+ bias[n])
//   A(m, k) = TA ? A[k * lda + m] : A[m * lda + k];   B(n, k) = TB ? B[k * ldb + n] : B[n * ldb + k]
//
// One CTA of 128 threads computes a 128 x BN tile of C (BN a multiple of 16 up to 128).  K is
// walked in tiles of 32 through a ring of kStages shared-memory buffers.  Each tile is laid out as
// the tensor core's canonical K-major arrangement without swizzling: 8 x 8 "core matrices" of 128
// contiguous bytes (8 rows of 8 BF16 along k); the core matrices of one 8-row group lie rows / 8 *
// 128 B apart along k (the descriptor's leading-dimension offset) and consecutive 8-row groups
// 128 B apart (its stride offset).  Operands stored row by row (k contiguous) are copied with
// 16-byte cp.async (zero-filled outside the matrix), kStages - 1 tiles ahead of the MMAs, into
// K-major core matrices; operands stored k-major go the same way into MN-major core matrices,
// which the MMA reads transposed (the operand's major bit of the instruction descriptor), so no
// operand is ever transposed by the threads.  One thread issues two
// tcgen05.mma (M = 128, N = BN, K = 16, BF16 x BF16 -> FP32) per tile, accumulating in tensor
// memory (TMEM: 128 lanes = rows, BN columns), and tcgen05.commit arrives on the tile's buffer
// mbarrier once they have completed, which frees the buffer for the copy kStages - 1 tiles later.
// The epilogue waits for the last commit; each warp reads its 32 rows of the accumulator from
// TMEM (tcgen05.ld, 16 columns at a time), adds the bias and stores (or atomically adds) FP32.
//
// Every wait on an mbarrier is bounded and decided for the whole block; a wait that runs out sets
// *err (the caller turns it into an error status), and the CTA still waits (bounded) for its own
// MMAs before it frees TMEM.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace chfpe {
namespace tc {

typedef __nv_bfloat16 bf16;

constexpr int kBM = 128;            // rows of a C tile (TMEM lanes)
constexpr int kBK = 32;             // k per shared-memory tile (two MMAs of K = 16)
constexpr int kStages = 4;          // shared-memory tiles in flight
constexpr int kThreads = 128;
constexpr int kTileA = kBM * kBK * 2, kTileB = 128 * kBK * 2;   // bytes (B tile for BN = 128)
constexpr int kStageBytes = kTileA + kTileB;
constexpr int kSmemTiles = kStages * kStageBytes;
constexpr int kSmemBytes = kSmemTiles + 128;                       // + mbarriers, TMEM address
// TMEM columns a CTA allocates (FP32 accumulator columns, BN <= 128); three CTAs per SM (3 x 64 KB
// of shared memory) hold 384 of the SM's 512
constexpr int kTmemCols = 128;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor of a K-major tile without swizzling: start address, leading
// dimension byte offset (between core matrices adjacent along k), stride dimension byte offset
// (between adjacent 8-row groups), descriptor version 1 (bits 46-48), no base offset, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A (bits 7-9 = 1) and
// B (bits 10-12 = 1), A MN-major if ta (bit 15), B MN-major if tb (bit 16), N >> 3 in bits 17-22,
// M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, bool ta, bool tb) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((ta ? 1u : 0u) << 15) | ((tb ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// true once the phase of the given parity has completed; gives up after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    const uint32_t a = smem_addr(bar);
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 bytes global -> shared, asynchronous; src_bytes = 0 writes zeros and reads nothing
__device__ __forceinline__ void cp16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

// tile rows r0.. (rows_tile of them) of operand X, k in [k0, k0 + 32), into shared memory: core
// matrix (row group g, k group j) at byte (j * rows_tile / 8 + g) * 128 (so the descriptor's
// leading-dimension offset, along k, is rows_tile / 8 * 128 B and its stride offset, along the
// rows, 128 B, in both orientations); zeros outside (rows, kend).  Whole aligned 16-byte chunks go
// by cp.async, the rest element by element.
// T = false: X row by row (element (r, k) at X[r * ld + k]); K-major core matrices (8 rows of 8 k)
// T = true: X k-major (element (r, k) at X[k * ld + r]); MN-major core matrices (8 k of 8 rows),
//           which the MMA reads with the operand's transpose bit set
template <bool T>
__device__ __forceinline__ void load_tile(unsigned char *S, int rows_tile, const bf16 *__restrict__ X,
                                          int ld, int rows, int kend, int r0, int k0) {
    const int groups = rows_tile / 8;
    if (!T) {
        for (int c = threadIdx.x; c < rows_tile * (kBK / 8); c += kThreads) {
            const int r = c / (kBK / 8), j = c % (kBK / 8);
            const int gr = r0 + r, gk = k0 + j * 8;
            unsigned char *dst = S + (j * groups + (r >> 3)) * 128 + (r & 7) * 16;
            const bool in = gr < rows && gk < kend;
            const bf16 *src = X + (long long)(in ? gr : 0) * ld + (in ? gk : 0);
            if (!in || (gk + 8 <= kend && (reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
                cp16(dst, src, in ? 16 : 0);
            } else {
                bf16 t[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) t[e] = (gk + e < kend) ? src[e] : __float2bfloat16(0.f);
                uint4 v;
                memcpy(&v, t, 16);
                *reinterpret_cast<uint4 *>(dst) = v;
            }
        }
    } else {
        // MN-major core matrices: (row group g, k group j) holds 8 k-rows of 8 consecutive
        // matrix rows, so a 16-byte global chunk (8 rows at one k) is one core-matrix row
        for (int c = threadIdx.x; c < kBK * groups; c += kThreads) {
            const int k = c / groups, g = c - k * groups;
            const int gk = k0 + k, gr = r0 + g * 8;
            unsigned char *dst = S + ((k >> 3) * groups + g) * 128 + (k & 7) * 16;
            const bool in = gk < kend && gr < rows;
            const bf16 *src = X + (long long)(in ? gk : 0) * ld + (in ? gr : 0);
            if (!in || (gr + 8 <= rows && (reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
                cp16(dst, src, in ? 16 : 0);
            } else {
                bf16 t[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) t[e] = (gr + e < rows) ? src[e] : __float2bfloat16(0.f);
                uint4 v;
                memcpy(&v, t, 16);
                *reinterpret_cast<uint4 *>(dst) = v;
            }
        }
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// grid (ceil(N / BN), ceil(M / 128), splits); split z covers k in [z klen, min(K, (z + 1) klen))
template <bool TA, bool TB>
__global__ void __launch_bounds__(kThreads, 1) gemm_tc_kernel(
    const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb, float *__restrict__ C,
    const float *__restrict__ bias, int M, int N, int K, int klen, int accumulate, int BN, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kSmemTiles);                 // [kStages]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kSmemTiles + 8 * kStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * klen, ke = min(K, kb + klen);
    const int nk = (ke - kb + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(kBM, BN, TA, TB);   // BN a multiple of 16 in [16, 128]
    const long long limit = 1ll << 24;
    bool ok = true;
    int last = -1;   // the last k tile whose MMAs were committed

    auto buf = [&](int t) { return smem + (t % kStages) * kStageBytes; };
    auto copy_tile = [&](int t) {
        unsigned char *Sa = buf(t);
        load_tile<TA>(Sa, kBM, A, lda, M, ke, m0, kb + t * kBK);
        load_tile<TB>(Sa + kTileA, BN, B, ldb, N, ke, n0, kb + t * kBK);
    };
    // prologue: tiles 0 .. kStages - 2, one cp.async group each (empty groups keep the count)
    for (int t = 0; t < kStages - 1; ++t) {
        if (t < nk) copy_tile(t);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int kt = 0; kt < nk; ++kt) {
        // tile kt is group kt: at most the kStages - 2 newest groups may still be in flight
        asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_addr(buf(kt)), b0 = a0 + kTileA;
            const uint32_t lbo_a = (kBM / 8) * 128, lbo_b = (BN / 8) * 128;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 2 * lbo_a, lbo_a, 128);
                const uint64_t bd = smem_desc(b0 + kk * 2 * lbo_b, lbo_b, 128);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_addr(&bar[kt % kStages])) : "memory");
        }
        last = kt;
        // refill: tile kt + kStages - 1 takes the buffer of tile kt - 1 once its MMAs completed
        const int nt = kt + kStages - 1;
        if (nt < nk) {
            if (kt >= 1) {
                const int t = kt - 1;
                if (!__syncthreads_and(mbar_wait(&bar[t % kStages], (t / kStages) & 1, limit) ? 1 : 0)) {
                    ok = false;
                    break;
                }
            }
            copy_tile(nt);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // the last commit covers every MMA issued before it
    if (ok && nk > 0)
        ok = __syncthreads_and(mbar_wait(&bar[(nk - 1) % kStages], ((nk - 1) / kStages) & 1, limit) ? 1 : 0) != 0;
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        // own MMAs may still run: wait (bounded) for the last commit before TMEM is freed
        if (last >= 0) mbar_wait(&bar[last % kStages], (last / kStages) & 1, limit);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + warp * 32 + lane;
        const bool add_bias = bias != nullptr && blockIdx.z == 0;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
                const int col0 = n0 + c0;
                float *dst = C + (long long)row * N + col0;
                if (add_bias) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += (col0 + i < N) ? __ldg(bias + col0 + i) : 0.f;
                }
                if (col0 + 16 <= N && (N & 3) == 0) {   // 16-byte aligned: four vector stores
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 x = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        float4 *d4 = reinterpret_cast<float4 *>(dst) + q;
                        if (accumulate) atomicAdd(d4, x); else *d4 = x;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (col0 + i < N) {
                            if (accumulate) atomicAdd(dst + i, v[i]); else dst[i] = v[i];
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace chfpe
