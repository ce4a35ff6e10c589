// tc_gemm.cuh -- BF16 GEMM on the fifth-generation tensor cores (tcgen05) of sm_100-class GPUs,
// for the surrogate's contractions:
//
//   C[m][n] (=, or += with FP32 atomics under split-K) sum_k A(m, k) B(n, k)  (+ bias[n])
//   A(m, k) = TA ? A[k * lda + m] : A[m * lda + k];   B(n, k) = TB ? B[k * ldb + n] : B[n * ldb + k]
//
// One CTA of 128 threads computes a 128 x BN tile of C.  K is walked in tiles of 64: all threads
// copy the A and B tiles from global memory into shared memory (two buffers), laid out as the
// tensor core's canonical K-major arrangement without swizzling -- 8 x 8 "core matrices" of 128
// contiguous bytes (8 rows of 8 BF16 along k), the core matrices of one 8-row group rows / 8 *
// 128 B apart along k (the leading-dimension offset) and consecutive 8-row groups 128 B apart
// (the stride offset).  Either storage order of either operand is transposed during that copy, so the MMA
// only ever reads K-major tiles.  One elected thread then issues four tcgen05.mma (M = 128,
// N = BN, K = 16, BF16 x BF16 -> FP32) that accumulate into tensor memory (TMEM: 128 lanes = rows,
// BN columns), and tcgen05.commit arrives on the buffer's mbarrier once they have completed, which
// tells the copy two tiles later that the buffer is free.  The epilogue waits for the last
// commit, and each warp reads its 32 rows of the accumulator from TMEM (tcgen05.ld, 16 columns at
// a time), adds the bias and stores (or atomically adds) FP32 results.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets *err (the caller turns it into
// an error status), and the CTA still waits (bounded) for its own MMAs before it frees TMEM.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace chfpe {
namespace tc {

typedef __nv_bfloat16 bf16;

constexpr int kBM = 128;            // rows of a C tile (TMEM lanes)
constexpr int kBK = 64;             // k per shared-memory tile (four MMAs of K = 16)
constexpr int kThreads = 128;

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
// B (bits 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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

// tile rows r0.. of operand X into the canonical K-major layout of shared memory:
// core matrix (row group g, k group j) at byte (j * rows / 8 + g) * 128, row r % 8 at +16 (r % 8)
// T = true: X is stored k-major in global memory (element (r, k) at X[k * ld + r])
template <bool T>
__device__ __forceinline__ void load_tile(unsigned char *S, int rows_tile, const bf16 *__restrict__ X,
                                          int ld, int rows, int kend, int r0, int k0) {
    const int groups = rows_tile / 8;
    if (!T) {
        // 16-byte chunks (row r, k group j): rows_tile * 8 chunks
        for (int c = threadIdx.x; c < rows_tile * 8; c += kThreads) {
            const int r = c >> 3, j = c & 7;
            const int gr = r0 + r, gk = k0 + j * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gr < rows && gk < kend) {
                const bf16 *src = X + (long long)gr * ld + gk;
                if (gk + 8 <= kend && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                    v = __ldg(reinterpret_cast<const uint4 *>(src));
                } else {
                    bf16 t[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) t[e] = (gk + e < kend) ? src[e] : __float2bfloat16(0.f);
                    memcpy(&v, t, 16);
                }
            }
            *reinterpret_cast<uint4 *>(S + (j * groups + (r >> 3)) * 128 + (r & 7) * 16) = v;
        }
    } else {
        // 16-byte chunks (k, row group g) of 8 consecutive rows at one k, scattered to 8 rows
        for (int c = threadIdx.x; c < kBK * groups; c += kThreads) {
            const int k = c / groups, g = c - k * groups;
            const int gk = k0 + k, gr = r0 + g * 8;
            bf16 t[8];
            if (gk < kend && gr < rows) {
                const bf16 *src = X + (long long)gk * ld + gr;
                if (gr + 8 <= rows && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                    uint4 v = __ldg(reinterpret_cast<const uint4 *>(src));
                    memcpy(t, &v, 16);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) t[e] = (gr + e < rows) ? src[e] : __float2bfloat16(0.f);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) t[e] = __float2bfloat16(0.f);
            }
            bf16 *base = reinterpret_cast<bf16 *>(S + ((k >> 3) * groups + g) * 128) + (k & 7);
#pragma unroll
            for (int e = 0; e < 8; ++e) base[e * 8] = t[e];
        }
    }
}


// shared memory of one CTA: two buffers of (A tile 16 KB, B tile BN x 128 B) with BN <= 128, then
// 32 KB that no tile uses (every descriptor's reach, read either way round, stays inside the
// allocation), then the mbarriers and the TMEM address
constexpr int kTileA = kBM * kBK * 2, kTileB = 128 * kBK * 2;
constexpr int kSmemTiles = 2 * (kTileA + kTileB) + 32 * 1024;
constexpr int kSmemBytes = kSmemTiles + 64;
// TMEM columns a CTA allocates (FP32 accumulator columns; BN <= 128 are used): twice the widest
// tile, and two CTAs (2 x 96 KB of shared memory) per SM hold at most the SM's 512
constexpr int kTmemCols = 256;

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
    const float *__restrict__ bias, int M, int N, int K, int klen, int accumulate, int BN,
    int *err) {
    constexpr int tmem_cols = kTmemCols;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kSmemTiles);      // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kSmemTiles + 16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * klen, ke = min(K, kb + klen);
    const int nk = (ke - kb + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(tmem_slot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(kBM, BN);   // BN a multiple of 16 in [16, 128]
    const long long limit = 1ll << 24;
    bool ok = true;
    int last = -1;   // the last k tile whose MMAs were committed

    for (int kt = 0; kt < nk; ++kt) {
        const int b = kt & 1;
        unsigned char *Sa = smem + b * (kTileA + kTileB);
        unsigned char *Sb = Sa + kTileA;
        if (kt >= 2) {   // buffer free: the MMAs of tile kt - 2 have completed (a block-wide decision)
            if (!__syncthreads_and(mbar_wait(&bar[b], ((kt >> 1) - 1) & 1, limit) ? 1 : 0)) {
                ok = false;
                break;
            }
        }
        const int k0 = kb + kt * kBK;
        load_tile<TA>(Sa, kBM, A, lda, M, ke, m0, k0);
        load_tile<TB>(Sb, BN, B, ldb, N, ke, n0, k0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_addr(Sa), b0 = smem_addr(Sb);
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
                         ::"r"(smem_addr(&bar[b])) : "memory");
        }
        last = kt;
    }
    // the last commit covers every MMA issued before it
    if (ok && nk > 0)
        ok = __syncthreads_and(mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1, limit) ? 1 : 0) != 0;
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        // own MMAs may still run: wait (bounded) for the last commit before TMEM is freed
        if (last >= 0) mbar_wait(&bar[last & 1], (last >> 1) & 1, limit);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + warp * 32 + lane;
        const bool add_bias = bias != nullptr && blockIdx.z == 0;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = n0 + c0 + i;
                    if (col < N) {
                        const float x = v[i] + (add_bias ? bias[col] : 0.f);
                        float *dst = C + (long long)row * N + col;
                        if (accumulate) atomicAdd(dst, x); else *dst = x;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace chfpe
