// surrogate.cu -- learned surrogate of the 2D response: 12 model parameters -> a normalised
// R2(t1, t2) on a 64 x 64 grid plus log10 of its scale.
//
// Network (all sizes fixed):
//   x [12] -> 4 x [Linear(512) + SiLU] -> h4 [512]
//   head:    s = h4 . w_h + b_h                                   (log10 of max |R2|)
//   decoder: h4 viewed as an NHWC image 4 x 4 x 32 (feature f -> y = f / 128, x = f / 32 % 4,
//            c = f % 32), then 4 x [nearest upsample x2, conv 3x3 with zero padding 1] with
//            32 -> 32 -> 16 -> 8 -> 1 channels and SiLU after all but the last -> y [64 x 64]
// Loss: mean over pixels of (y - t)^2 + w_s * mean over the batch of (s - t_s)^2.
//
// Every contraction -- the linear layers, the convolutions as im2col GEMMs, their data gradients
// and their weight gradients -- runs in one hand-written kernel: BF16 on the tcgen05 tensor cores
// with FP32 accumulation in tensor memory (tc_gemm.cuh), operands read in either storage order so
// that no transposed copy is ever made.  The earlier warp-level mma.sync.m16n8k16 kernel stays
// selectable (CHFPE_SURROGATE_GEMM=mma) for comparison.  Training keeps FP32 master weights, FP32 gradients and FP32
// AdamW moments; the BF16 weight copy the GEMMs read is refreshed after every update.
#include "../../include/chfpe.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tc_gemm.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace chfpe {
void set_last_error(const std::string &msg);   // chfpe.cu
}

typedef __nv_bfloat16 bf16;

namespace {

chfpe_status sfail(chfpe_status s, const std::string &m) {
    chfpe::set_last_error(m);
    return s;
}

#define SCK(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return sfail(CHFPE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

#define SLAUNCH() SCK(cudaGetLastError())

// ------------------------------------------------------------------------------------------
// BF16 tensor-core GEMM
//   C[m][n] (=, or += with atomics) sum_{k in split} A(m, k) B(n, k)  (+ bias[n] on split 0)
//   A(m, k) = TA ? A[k * lda + m] : A[m * lda + k];  B(n, k) = TB ? B[k * ldb + n] : B[n * ldb + k]
// 64 x 64 output tile per block of 4 warps (32 x 32 each); k-steps of 16 staged in shared memory
// as [row][k] with rows padded to 24 bf16 (48 B), which makes the fragment reads conflict free.
// Split-K over gridDim.z: split z covers k in [z * klen, min(K, (z + 1) * klen)), klen a multiple
// of 16, and adds its partial sums to C.
// ------------------------------------------------------------------------------------------

constexpr int GT = 64, GK = 16, GPAD = 24;

// tile rows r0..r0+63 of a row-major [rows x ld] operand, k in [k0, k0 + 16), zero outside
// (rows, kend)
__device__ __forceinline__ void load_tile_n(bf16 (*S)[GPAD], const bf16 *X, int ld, int rows,
                                            int kend, int r0, int k0) {
    const int t = threadIdx.x;   // 128 threads: 64 rows x 2 chunks of 8 k
    const int r = t >> 1, c = (t & 1) * 8;
    const int gr = r0 + r, gk = k0 + c;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (gr < rows) {
        const bf16 *src = X + (long long)gr * ld + gk;
        if (gk + 8 <= kend && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            v = *reinterpret_cast<const uint4 *>(src);
        } else {
            bf16 tmp[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) tmp[j] = (gk + j < kend) ? src[j] : __float2bfloat16(0.f);
            memcpy(&v, tmp, 16);
        }
    }
    *reinterpret_cast<uint2 *>(&S[r][c]) = make_uint2(v.x, v.y);
    *reinterpret_cast<uint2 *>(&S[r][c + 4]) = make_uint2(v.z, v.w);
}

// the same tile from a k-major [K x ld] operand (element (row, k) at X[k * ld + row])
__device__ __forceinline__ void load_tile_t(bf16 (*S)[GPAD], const bf16 *X, int ld, int rows,
                                            int kend, int r0, int k0) {
    const int t = threadIdx.x;   // 128 threads: 16 k x 8 chunks of 8 rows
    const int kk = t >> 3, r = (t & 7) * 8;
    const int gk = k0 + kk, gr = r0 + r;
    bf16 tmp[8];
    if (gk < kend) {
        const bf16 *src = X + (long long)gk * ld + gr;
        if (gr + 8 <= rows && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            uint4 v = *reinterpret_cast<const uint4 *>(src);
            memcpy(tmp, &v, 16);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) tmp[j] = (gr + j < rows) ? src[j] : __float2bfloat16(0.f);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) tmp[j] = __float2bfloat16(0.f);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) S[r + j][kk] = tmp[j];
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const bf16 *__restrict__ A, int lda,
                                                        const bf16 *__restrict__ B, int ldb,
                                                        float *__restrict__ C,
                                                        const float *__restrict__ bias, int M,
                                                        int N, int K, int klen, int accumulate) {
    __shared__ __align__(16) bf16 As[GT][GPAD];
    __shared__ __align__(16) bf16 Bs[GT][GPAD];
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int kb = blockIdx.z * klen;
    const int ke = min(K, kb + klen);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, tg = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    for (int k0 = kb; k0 < ke; k0 += GK) {
        if (TA) load_tile_t(As, A, lda, M, ke, m0, k0); else load_tile_n(As, A, lda, M, ke, m0, k0);
        if (TB) load_tile_t(Bs, B, ldb, N, ke, n0, k0); else load_tile_n(Bs, B, ldb, N, ke, n0, k0);
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int rb = wm + i * 16;
            af[i][0] = *reinterpret_cast<const uint32_t *>(&As[rb + g][tg * 2]);
            af[i][1] = *reinterpret_cast<const uint32_t *>(&As[rb + g + 8][tg * 2]);
            af[i][2] = *reinterpret_cast<const uint32_t *>(&As[rb + g][tg * 2 + 8]);
            af[i][3] = *reinterpret_cast<const uint32_t *>(&As[rb + g + 8][tg * 2 + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cb = wn + j * 8;
            bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[cb + g][tg * 2]);
            bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[cb + g][tg * 2 + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]),
                      "r"(bfr[j][0]), "r"(bfr[j][1]));
        __syncthreads();
    }
    const bool add_bias = bias != nullptr && blockIdx.z == 0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn + j * 8 + tg * 2 + (r & 1);
                if (row < M && col < N) {
                    const float v = acc[i][j][r] + (add_bias ? bias[col] : 0.f);
                    float *dst = C + (long long)row * N + col;
                    if (accumulate) atomicAdd(dst, v); else *dst = v;
                }
            }
}

// ------------------------------------------------------------------------------------------
// element-wise and reduction kernels
// ------------------------------------------------------------------------------------------

#define GRID_STRIDE(i, n)                                                                   \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n);           \
         i += (long long)gridDim.x * blockDim.x)

__global__ void to_bf16_kernel(const float *__restrict__ x, bf16 *__restrict__ y, long long n) {
    GRID_STRIDE(i, n) y[i] = __float2bfloat16_rn(x[i]);
}

// [B x nin] FP32 -> [B x kin] BF16, zero padded
__global__ void pad_input_kernel(const float *__restrict__ X, bf16 *__restrict__ H, int B, int nin,
                                 int kin) {
    GRID_STRIDE(i, (long long)B * kin) {
        const int c = (int)(i % kin);
        const long long b = i / kin;
        H[i] = __float2bfloat16_rn(c < nin ? X[b * nin + c] : 0.f);
    }
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.f / (1.f + expf(-z)); }

// h = silu(z) = z sigma(z), stored as BF16
__global__ void silu_fwd_kernel(const float *__restrict__ z, bf16 *__restrict__ h, long long n) {
    GRID_STRIDE(i, n) h[i] = __float2bfloat16_rn(z[i] * sigmoidf(z[i]));
}

// dz = dh silu'(z),  silu'(z) = sigma(z) (1 + z (1 - sigma(z))); FP32 and BF16 copies
__global__ void silu_bwd_kernel(const float *__restrict__ z, const float *__restrict__ dh,
                                float *__restrict__ dz, bf16 *__restrict__ dzb, long long n) {
    GRID_STRIDE(i, n) {
        const float s = sigmoidf(z[i]);
        const float v = dh[i] * s * (1.f + z[i] * (1.f - s));
        dz[i] = v;
        dzb[i] = __float2bfloat16_rn(v);
    }
}

// im2col of the nearest-upsampled (x2) NHWC activation A [B, Hin, Hin, Cin] for a 3x3
// convolution with zero padding 1: row (b, y, x) of the H = 2 Hin output image, column
// ci * 9 + ky * 3 + kx holds A[b, (y + ky - 1) / 2, (x + kx - 1) / 2, ci] (0 outside the image);
// columns Cin * 9 .. Kp - 1 are 0.  One thread per (row, ci) writes its 9 taps; one extra thread
// per row writes the padding columns.
__global__ void im2col_up_kernel(const bf16 *__restrict__ A, bf16 *__restrict__ X, int B, int Hin,
                                 int Cin, int Kp) {
    const int H = 2 * Hin;
    const long long rows = (long long)B * H * H;
    const int per_row = Cin + (Kp > Cin * 9 ? 1 : 0);
    GRID_STRIDE(i, rows * per_row) {
        const int ci = (int)(i % per_row);
        const long long r = i / per_row;
        bf16 *dst = X + r * Kp;
        if (ci == Cin) {
            for (int c = Cin * 9; c < Kp; ++c) dst[c] = __float2bfloat16(0.f);
            continue;
        }
        const int x = (int)(r % H), y = (int)((r / H) % H);
        const long long b = r / ((long long)H * H);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int yy = y + ky - 1, xx = x + kx - 1;
                bf16 v = __float2bfloat16(0.f);
                if (yy >= 0 && yy < H && xx >= 0 && xx < H)
                    v = A[((b * Hin + yy / 2) * Hin + xx / 2) * Cin + ci];
                dst[ci * 9 + ky * 3 + kx] = v;
            }
    }
}

// adjoint of the above: dA[b, yi, xi, ci] = sum over the four upsampled pixels (Y, X) of
// (yi, xi) and the taps (ky, kx) whose output pixel (Y - ky + 1, X - kx + 1) lies in the image of
// dX[(b, Y - ky + 1, X - kx + 1)][ci * 9 + ky * 3 + kx]
__global__ void col2im_up_kernel(const float *__restrict__ dX, float *__restrict__ dA, int B,
                                 int Hin, int Cin, int Kp) {
    const int H = 2 * Hin;
    GRID_STRIDE(i, (long long)B * Hin * Hin * Cin) {
        const int ci = (int)(i % Cin);
        const long long p = i / Cin;
        const int xi = (int)(p % Hin), yi = (int)((p / Hin) % Hin);
        const long long b = p / ((long long)Hin * Hin);
        float s = 0.f;
        for (int uy = 0; uy < 2; ++uy)
            for (int ux = 0; ux < 2; ++ux) {
                const int Y = 2 * yi + uy, X = 2 * xi + ux;
#pragma unroll
                for (int ky = 0; ky < 3; ++ky) {
                    const int y = Y - ky + 1;
                    if (y < 0 || y >= H) continue;
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
                        const int x = X - kx + 1;
                        if (x < 0 || x >= H) continue;
                        s += dX[((b * H + y) * H + x) * Kp + ci * 9 + ky * 3 + kx];
                    }
                }
            }
        dA[i] = s;
    }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// db[n] += sum over rows of dZ[row][n]; grid (N, chunks), each block one contiguous row chunk
__global__ void colsum_kernel(const float *__restrict__ dZ, float *__restrict__ db, long long rows,
                              int N, long long chunk) {
    const int n = blockIdx.x;
    const long long r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    float s = 0.f;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += dZ[r * N + n];
    s = warp_sum_f(s);
    __shared__ float sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.f;
        s = warp_sum_f(s);
        if (threadIdx.x == 0) atomicAdd(db + n, s);
    }
}

// squared-error term w * mean((y - t)^2) over n values: gradient 2 w (y - t) / n in FP32 and
// BF16, loss added to *loss in FP64
__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ t,
                           float *__restrict__ dy, bf16 *__restrict__ dyb, long long n, float w,
                           double *__restrict__ loss) {
    double s = 0.0;
    const float scale = 2.f * w / (float)n;
    GRID_STRIDE(i, n) {
        const float e = y[i] - t[i];
        dy[i] = scale * e;
        dyb[i] = __float2bfloat16_rn(scale * e);
        s += (double)e * (double)e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(loss, (double)w * s / (double)n);
}

// dH[b][f] += dS[b] * w_h[f]   (the scale head's part of the gradient of h4; FP32)
__global__ void add_outer_kernel(float *__restrict__ dH, const float *__restrict__ dS,
                                 const float *__restrict__ wh, int B, int F) {
    GRID_STRIDE(i, (long long)B * F) dH[i] += dS[i / F] * wh[i % F];
}

// AdamW (decoupled weight decay) with bias-corrected moments; c1 = 1 - b1^t, c2 = 1 - b2^t
__global__ void adamw_kernel(float *__restrict__ p, const float *__restrict__ g,
                             float *__restrict__ m, float *__restrict__ v, long long n, float lr,
                             float b1, float b2, float eps, float wd, float c1, float c2) {
    GRID_STRIDE(i, n) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
    }
}

// rows perm[0..B) of the dataset into the contiguous batch buffers
__global__ void gather_kernel(const int *__restrict__ perm, const float *__restrict__ X,
                              const float *__restrict__ T, const float *__restrict__ TS,
                              float *__restrict__ Xb, float *__restrict__ Tb,
                              float *__restrict__ TSb, int nin, int nout) {
    const int b = blockIdx.x;
    const long long src = perm[b];
    for (int j = threadIdx.x; j < nout; j += blockDim.x) Tb[(long long)b * nout + j] = T[src * nout + j];
    for (int j = threadIdx.x; j < nin; j += blockDim.x) Xb[b * nin + j] = X[src * nin + j];
    if (threadIdx.x == 0) TSb[b] = TS[src];
}

// ------------------------------------------------------------------------------------------
// network description
// ------------------------------------------------------------------------------------------

constexpr int NIN = CHFPE_SURROGATE_NIN, KIN = 16, WID = 512, NPIX = CHFPE_SURROGATE_NOUT;
constexpr int NCONV = 4;
constexpr int CIN[NCONV] = {32, 32, 16, 8}, COUT[NCONV] = {32, 16, 8, 1}, HIN[NCONV] = {4, 8, 16, 32};
constexpr int NLAYERS = 9;   // 4 linear, the scale head, 4 convolutions

constexpr int kpad(int c) { return (c * 9 + 15) / 16 * 16; }

struct Layer {        // weight [N x Kp] row-major (columns >= K are zero), bias [N]
    int N, K, Kp;     // K = fan-in (natural row length), Kp = stored row length
    long long w, b;   // offsets (elements) in the padded parameter buffer
};

int nblk(long long n) {
    const long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 148 * 16));
}

long long conv_rows(int c, int B) { return (long long)B * (2 * HIN[c]) * (2 * HIN[c]); }

}  // namespace

struct chfpe_surrogate {
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    Layer L[NLAYERS];           // natural order: linear 0-3, head, conv 0-3
    long long nparam = 0;       // padded buffer length
    long long nnatural = 0;     // parameters in the natural layout
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16 *pb = nullptr;
    long long step = 0;
    // activations, sized for max_batch rows
    bf16 *H[5] = {};            // H[0] padded input; H[l + 1] = silu(Z[l])
    float *Z[4] = {};
    float *S = nullptr;         // scale head [B]
    bf16 *Xc[NCONV] = {};       // im2col matrices
    float *Zc[NCONV] = {};      // conv outputs (the last one is the image y)
    bf16 *Ac[NCONV - 1] = {};   // silu(Zc) for the next conv
    // backward scratch
    float *dZ = nullptr; bf16 *dZb = nullptr;
    float *dA = nullptr;        // gradient of a conv input; after conv 0 the gradient of h4
    float *dXcol = nullptr;
    float *dS = nullptr; bf16 *dSb = nullptr;
    // training batch buffers and loss
    float *Xb = nullptr, *Tb = nullptr, *TSb = nullptr;
    double *loss = nullptr;
    std::vector<void *> allocs;

    Layer &mlp(int l) { return L[l]; }
    Layer &head() { return L[4]; }
    Layer &conv(int c) { return L[5 + c]; }
};

namespace {

template <typename T>
chfpe_status dalloc(chfpe_surrogate *h, T **ptr, long long n) {
    void *q = nullptr;
    const size_t bytes = (size_t)std::max<long long>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, (bytes + 255) / 256 * 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(CHFPE_ENOMEM, std::string("surrogate: cudaMalloc of ") + std::to_string(bytes) +
                                       " bytes failed: " + cudaGetErrorString(e));
    }
    h->allocs.push_back(q);
    *ptr = static_cast<T *>(q);
    return CHFPE_OK;
}

// error word of the tensor-core GEMM's bounded waits (set on the device, read after a stream
// synchronisation by tc_check)
__device__ int g_tc_err;

int *tc_err_ptr() {
    static int *p = nullptr;
    if (!p && cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_tc_err) != cudaSuccess) p = nullptr;
    return p;
}

// the tcgen05 kernels need more than 48 KB of dynamic shared memory: opt in once per instantiation
cudaError_t tc_configure() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(chfpe::tc::gemm_tc_kernel<false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, chfpe::tc::kSmemBytes);
    if (!e) e = cudaFuncSetAttribute(chfpe::tc::gemm_tc_kernel<false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, chfpe::tc::kSmemBytes);
    if (!e) e = cudaFuncSetAttribute(chfpe::tc::gemm_tc_kernel<true, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, chfpe::tc::kSmemBytes);
    if (!e) e = cudaFuncSetAttribute(chfpe::tc::gemm_tc_kernel<true, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, chfpe::tc::kSmemBytes);
    if (!e) e = tc_err_ptr() ? cudaSuccess : cudaErrorInvalidSymbol;
    if (!e) e = cudaMemset(tc_err_ptr(), 0, sizeof(int));
    done = e == cudaSuccess;
    return e;
}

// after a synchronisation of the stream: CHFPE_ETIMEOUT if a tensor-core GEMM's wait ran out
chfpe_status tc_check(cudaStream_t s) {
    int *p = tc_err_ptr();
    if (!p) return CHFPE_OK;
    int v = 0;
    SCK(cudaMemcpyAsync(&v, p, sizeof v, cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (v) {
        SCK(cudaMemsetAsync(p, 0, sizeof(int), s));
        return sfail(CHFPE_ETIMEOUT, "surrogate: a tensor-core GEMM wait timed out");
    }
    return CHFPE_OK;
}

// CHFPE_SURROGATE_GEMM=mma selects the mma.sync kernel (kept for comparison); the default is the
// tcgen05 kernel
bool use_tc() {
    const char *e = getenv("CHFPE_SURROGATE_GEMM");
    return !(e && e[0] == 'm');
}

template <bool TA, bool TB>
chfpe_status gemm_t(cudaStream_t s, const bf16 *A, int lda, const bf16 *B, int ldb, float *C,
                    const float *bias, int M, int N, int K, int splits) {
    const int accumulate = splits > 1 ? 1 : 0;
    if (M <= 0 || N <= 0) return CHFPE_OK;
    if (K <= 0) {
        if (!accumulate) SCK(cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), s));
        return CHFPE_OK;
    }
    if (use_tc() && (M + chfpe::tc::kBM - 1) / chfpe::tc::kBM <= 65535) {
        using namespace chfpe::tc;
        SCK(tc_configure());
        splits = std::max(1, std::min(splits, (K + kBK - 1) / kBK));
        int klen = (K + splits - 1) / splits;
        klen = (klen + kBK - 1) / kBK * kBK;
        const int nz = (K + klen - 1) / klen;
        // 128-wide tiles when they fill the GPU twice over, else at most 64 (more CTAs)
        const long long t128 = (long long)((N + 127) / 128) * ((M + kBM - 1) / kBM) * nz;
        const int BN = (N >= 128 && t128 >= 2 * 148) ? 128 : std::min(64, (N + 15) / 16 * 16);
        dim3 grid((N + BN - 1) / BN, (M + kBM - 1) / kBM, nz);
        gemm_tc_kernel<TA, TB><<<grid, kThreads, kSmemBytes, s>>>(A, lda, B, ldb, C, bias, M, N, K,
                                                                  klen, accumulate, BN, tc_err_ptr());
        SLAUNCH();
        return CHFPE_OK;
    }
    splits = std::max(1, std::min(splits, (K + GK - 1) / GK));
    int klen = (K + splits - 1) / splits;
    klen = (klen + GK - 1) / GK * GK;
    const int nz = (K + klen - 1) / klen;
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, nz);
    gemm_bf16_kernel<TA, TB><<<grid, 128, 0, s>>>(A, lda, B, ldb, C, bias, M, N, K, klen, accumulate);
    SLAUNCH();
    return CHFPE_OK;
}

// dispatch on the storage orders; splits > 1 adds into C, splits == 1 overwrites it
chfpe_status gemm(cudaStream_t s, bool ta, const bf16 *A, int lda, bool tb, const bf16 *B, int ldb,
                  float *C, const float *bias, int M, int N, int K, int splits) {
    if (!ta && !tb) return gemm_t<false, false>(s, A, lda, B, ldb, C, bias, M, N, K, splits);
    if (!ta && tb) return gemm_t<false, true>(s, A, lda, B, ldb, C, bias, M, N, K, splits);
    if (ta && !tb) return gemm_t<true, false>(s, A, lda, B, ldb, C, bias, M, N, K, splits);
    return gemm_t<true, true>(s, A, lda, B, ldb, C, bias, M, N, K, splits);
}

// split count for a weight-gradient GEMM (reduction over the batch rows): about two blocks per
// SM, each split at least 256 rows long, and never fewer than 2 (the result adds into the zeroed
// gradient)
int wgrad_splits(int M, int N, long long K) {
    const long long tiles = (long long)((M + GT - 1) / GT) * ((N + GT - 1) / GT);
    long long s = (2 * 148 + tiles - 1) / tiles;
    s = std::min<long long>(s, std::max<long long>(1, K / 256));
    return (int)std::max<long long>(2, s);
}

void layout(chfpe_surrogate *h) {
    long long off = 0;
    auto add = [&](Layer &L, int N, int K, int Kp) {
        L.N = N; L.K = K; L.Kp = Kp;
        L.w = off; off += ((long long)N * Kp + 63) / 64 * 64;   // 256-B aligned blocks
        L.b = off; off += (N + 63) / 64 * 64;
    };
    add(h->mlp(0), WID, NIN, KIN);
    for (int l = 1; l < 4; ++l) add(h->mlp(l), WID, WID, WID);
    add(h->head(), 1, WID, WID);
    for (int c = 0; c < NCONV; ++c) add(h->conv(c), COUT[c], CIN[c] * 9, kpad(CIN[c]));
    h->nparam = off;
    long long nat = 0;
    for (int i = 0; i < NLAYERS; ++i) nat += (long long)h->L[i].N * h->L[i].K + h->L[i].N;
    h->nnatural = nat;
}

// natural layout <-> padded buffer (host side); to_padded copies natural into padded
void repack(const chfpe_surrogate *h, float *padded, float *natural, bool to_padded) {
    long long q = 0;
    for (int i = 0; i < NLAYERS; ++i) {
        const Layer &L = h->L[i];
        for (int r = 0; r < L.N; ++r)
            for (int k = 0; k < L.K; ++k, ++q) {
                float &pv = padded[L.w + (long long)r * L.Kp + k];
                if (to_padded) pv = natural[q]; else natural[q] = pv;
            }
        for (int r = 0; r < L.N; ++r, ++q) {
            float &pv = padded[L.b + r];
            if (to_padded) pv = natural[q]; else natural[q] = pv;
        }
    }
}

chfpe_status refresh_bf16(chfpe_surrogate *h) {
    to_bf16_kernel<<<nblk(h->nparam), 256, 0, h->stream>>>(h->p, h->pb, h->nparam);
    SLAUNCH();
    return CHFPE_OK;
}

// forward pass of B <= max_batch rows of X [B x 12] (device FP32); the image lands in h->Zc[3],
// the scale in h->S
chfpe_status forward(chfpe_surrogate *h, const float *X, int B) {
    cudaStream_t s = h->stream;
    chfpe_status st;
    pad_input_kernel<<<nblk((long long)B * KIN), 256, 0, s>>>(X, h->H[0], B, NIN, KIN);
    SLAUNCH();
    for (int l = 0; l < 4; ++l) {
        const Layer &L = h->mlp(l);
        if ((st = gemm(s, false, h->H[l], L.Kp, false, h->pb + L.w, L.Kp, h->Z[l], h->p + L.b, B,
                       L.N, L.Kp, 1)))
            return st;
        silu_fwd_kernel<<<nblk((long long)B * WID), 256, 0, s>>>(h->Z[l], h->H[l + 1], (long long)B * WID);
        SLAUNCH();
    }
    const Layer &Lh = h->head();
    if ((st = gemm(s, false, h->H[4], WID, false, h->pb + Lh.w, WID, h->S, h->p + Lh.b, B, 1, WID, 1)))
        return st;
    const bf16 *A = h->H[4];
    for (int c = 0; c < NCONV; ++c) {
        const Layer &L = h->conv(c);
        const long long rows = conv_rows(c, B);
        const int per_row = CIN[c] + (L.Kp > L.K ? 1 : 0);
        im2col_up_kernel<<<nblk(rows * per_row), 256, 0, s>>>(A, h->Xc[c], B, HIN[c], CIN[c], L.Kp);
        SLAUNCH();
        if ((st = gemm(s, false, h->Xc[c], L.Kp, false, h->pb + L.w, L.Kp, h->Zc[c], h->p + L.b,
                       (int)rows, L.N, L.Kp, 1)))
            return st;
        if (c < NCONV - 1) {
            silu_fwd_kernel<<<nblk(rows * L.N), 256, 0, s>>>(h->Zc[c], h->Ac[c], rows * L.N);
            SLAUNCH();
            A = h->Ac[c];
        }
    }
    return CHFPE_OK;
}

chfpe_status colsum(cudaStream_t s, const float *dZ, float *db, long long rows, int N) {
    const long long chunk = 8192;
    const long long nch = (rows + chunk - 1) / chunk;
    colsum_kernel<<<dim3(N, (unsigned)nch), 256, 0, s>>>(dZ, db, rows, N, chunk);
    SLAUNCH();
    return CHFPE_OK;
}

// gradients of the loss for the batch whose forward pass is in the buffers, targets T [B x 4096]
// and TS [B]: h->g is overwritten and the loss added to *h->loss
chfpe_status backward(chfpe_surrogate *h, const float *T, const float *TS, int B, float w_scale) {
    cudaStream_t s = h->stream;
    chfpe_status st;
    SCK(cudaMemsetAsync(h->g, 0, (size_t)h->nparam * sizeof(float), s));
    const long long rows3 = conv_rows(NCONV - 1, B);
    mse_kernel<<<nblk(rows3), 256, 0, s>>>(h->Zc[NCONV - 1], T, h->dZ, h->dZb, rows3, 1.f, h->loss);
    SLAUNCH();
    mse_kernel<<<1, 256, 0, s>>>(h->S, TS, h->dS, h->dSb, B, w_scale, h->loss);
    SLAUNCH();
    for (int c = NCONV - 1; c >= 0; --c) {
        const Layer &L = h->conv(c);
        const long long rows = conv_rows(c, B);
        // bias: column sums of dZ [rows x Cout]
        if ((st = colsum(s, h->dZ, h->g + L.b, rows, L.N))) return st;
        // weight: dW[co][k] = sum_rows dZ[row][co] Xc[row][k]
        if ((st = gemm(s, true, h->dZb, L.N, true, h->Xc[c], L.Kp, h->g + L.w, nullptr, L.N, L.Kp,
                       (int)rows, wgrad_splits(L.N, L.Kp, rows))))
            return st;
        // data: dXc[row][k] = sum_co dZ[row][co] W[co][k]
        if ((st = gemm(s, false, h->dZb, L.N, true, h->pb + L.w, L.Kp, h->dXcol, nullptr, (int)rows,
                       L.Kp, L.N, 1)))
            return st;
        const long long nin = (long long)B * HIN[c] * HIN[c] * CIN[c];
        col2im_up_kernel<<<nblk(nin), 256, 0, s>>>(h->dXcol, h->dA, B, HIN[c], CIN[c], L.Kp);
        SLAUNCH();
        if (c > 0) {
            silu_bwd_kernel<<<nblk(nin), 256, 0, s>>>(h->Zc[c - 1], h->dA, h->dZ, h->dZb, nin);
            SLAUNCH();
        }
    }
    // h->dA now holds the gradient of h4 [B x 512] through the decoder; add the scale head's part
    {
        const Layer &L = h->head();
        if ((st = colsum(s, h->dS, h->g + L.b, B, 1))) return st;
        if ((st = gemm(s, true, h->dSb, 1, true, h->H[4], WID, h->g + L.w, nullptr, 1, WID, B,
                       wgrad_splits(1, WID, B))))
            return st;
        add_outer_kernel<<<nblk((long long)B * WID), 256, 0, s>>>(h->dA, h->dS, h->p + L.w, B, WID);
        SLAUNCH();
    }
    for (int l = 3; l >= 0; --l) {
        const Layer &L = h->mlp(l);
        silu_bwd_kernel<<<nblk((long long)B * WID), 256, 0, s>>>(h->Z[l], h->dA, h->dZ, h->dZb,
                                                                 (long long)B * WID);
        SLAUNCH();
        if ((st = colsum(s, h->dZ, h->g + L.b, B, WID))) return st;
        if ((st = gemm(s, true, h->dZb, WID, true, h->H[l], L.Kp, h->g + L.w, nullptr, WID, L.Kp, B,
                       wgrad_splits(WID, L.Kp, B))))
            return st;
        if (l > 0) {   // dH[b][i] = sum_o dZ[b][o] W[o][i]
            if ((st = gemm(s, false, h->dZb, WID, true, h->pb + L.w, L.Kp, h->dA, nullptr, B, L.Kp,
                           WID, 1)))
                return st;
        }
    }
    return CHFPE_OK;
}

constexpr float kB1 = 0.9f, kB2 = 0.999f, kEps = 1e-8f;

chfpe_status adamw_step(chfpe_surrogate *h, float lr, float wd) {
    h->step += 1;
    const float c1 = (float)(1.0 - std::pow((double)kB1, (double)h->step));
    const float c2 = (float)(1.0 - std::pow((double)kB2, (double)h->step));
    adamw_kernel<<<nblk(h->nparam), 256, 0, h->stream>>>(h->p, h->g, h->m, h->v, h->nparam, lr,
                                                         kB1, kB2, kEps, wd, c1, c2);
    SLAUNCH();
    return refresh_bf16(h);
}

// SplitMix64 (Steele, Lea and Flood, 2014) for the initial weights and the epoch shuffles
uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unit(uint64_t &x) { return (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

extern "C" {

long long chfpe_surrogate_param_count(void) {
    chfpe_surrogate tmp;
    layout(&tmp);
    return tmp.nnatural;
}

void chfpe_surrogate_destroy(chfpe_surrogate *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *q : h->allocs) cudaFree(q);
    if (h->owns_stream) cudaStreamDestroy(h->stream);
    delete h;
}

chfpe_status chfpe_surrogate_create(int max_batch, unsigned long long seed, void *stream,
                                    chfpe_surrogate **out) {
    if (!out) return sfail(CHFPE_EINVAL, "surrogate_create: out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > 4096)
        return sfail(CHFPE_EINVAL, "surrogate_create: max_batch must be in [1, 4096]");
    chfpe_surrogate *h = new (std::nothrow) chfpe_surrogate;
    if (!h) return sfail(CHFPE_ENOMEM, "surrogate_create: host allocation failed");
    h->max_batch = max_batch;
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return sfail(CHFPE_ECUDA, std::string("surrogate_create: ") + cudaGetErrorString(e));
        }
        h->owns_stream = true;
    }
    layout(h);
    const long long Bm = max_batch;
    chfpe_status st = CHFPE_OK;
    auto fail = [&](chfpe_status s) { chfpe_surrogate_destroy(h); return s; };
    if ((st = dalloc(h, &h->p, h->nparam)) || (st = dalloc(h, &h->g, h->nparam)) ||
        (st = dalloc(h, &h->m, h->nparam)) || (st = dalloc(h, &h->v, h->nparam)) ||
        (st = dalloc(h, &h->pb, h->nparam)))
        return fail(st);
    if ((st = dalloc(h, &h->H[0], Bm * KIN))) return fail(st);
    for (int l = 0; l < 4; ++l)
        if ((st = dalloc(h, &h->H[l + 1], Bm * WID)) || (st = dalloc(h, &h->Z[l], Bm * WID)))
            return fail(st);
    long long dz = Bm * WID, dx = 0, da = Bm * WID;
    for (int c = 0; c < NCONV; ++c) {
        const long long rows = conv_rows(c, (int)Bm);
        if ((st = dalloc(h, &h->Xc[c], rows * h->conv(c).Kp)) || (st = dalloc(h, &h->Zc[c], rows * COUT[c])))
            return fail(st);
        if (c < NCONV - 1 && (st = dalloc(h, &h->Ac[c], rows * COUT[c]))) return fail(st);
        dz = std::max(dz, rows * COUT[c]);
        dx = std::max(dx, rows * h->conv(c).Kp);
        da = std::max(da, Bm * HIN[c] * HIN[c] * CIN[c]);
    }
    if ((st = dalloc(h, &h->S, Bm)) || (st = dalloc(h, &h->dZ, dz)) || (st = dalloc(h, &h->dZb, dz)) ||
        (st = dalloc(h, &h->dA, da)) || (st = dalloc(h, &h->dXcol, dx)) || (st = dalloc(h, &h->dS, Bm)) ||
        (st = dalloc(h, &h->dSb, Bm)) || (st = dalloc(h, &h->Xb, Bm * NIN)) ||
        (st = dalloc(h, &h->Tb, Bm * NPIX)) || (st = dalloc(h, &h->TSb, Bm)) || (st = dalloc(h, &h->loss, 1)))
        return fail(st);
    // initial weights: uniform in +-sqrt(6 / fan_in) (+-sqrt(1.5 / fan_in) for the two output
    // layers), biases 0, padding columns 0
    std::vector<float> w(h->nparam, 0.f);
    uint64_t x = seed;
    for (int i = 0; i < NLAYERS; ++i) {
        const Layer &L = h->L[i];
        const bool out_layer = (i == 4) || (i == NLAYERS - 1);
        const double a = std::sqrt((out_layer ? 1.5 : 6.0) / L.K);
        for (int r = 0; r < L.N; ++r)
            for (int k = 0; k < L.K; ++k)
                w[L.w + (long long)r * L.Kp + k] = (float)(a * (2.0 * unit(x) - 1.0));
    }
    cudaError_t e = cudaMemcpyAsync(h->p, w.data(), h->nparam * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->m, 0, h->nparam * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->v, 0, h->nparam * sizeof(float), h->stream);
    if (e == cudaSuccess && (st = refresh_bf16(h))) return fail(st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        chfpe_surrogate_destroy(h);
        return sfail(CHFPE_ECUDA, std::string("surrogate_create: ") + cudaGetErrorString(e));
    }
    *out = h;
    return CHFPE_OK;
}

chfpe_status chfpe_surrogate_get_params(chfpe_surrogate *h, float *host) {
    if (!h || !host) return sfail(CHFPE_EINVAL, "surrogate_get_params: NULL argument");
    std::vector<float> w(h->nparam);
    SCK(cudaMemcpyAsync(w.data(), h->p, h->nparam * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    SCK(cudaStreamSynchronize(h->stream));
    repack(h, w.data(), host, false);
    return CHFPE_OK;
}

chfpe_status chfpe_surrogate_set_params(chfpe_surrogate *h, const float *host) {
    if (!h || !host) return sfail(CHFPE_EINVAL, "surrogate_set_params: NULL argument");
    std::vector<float> w(h->nparam, 0.f);
    repack(h, w.data(), const_cast<float *>(host), true);
    SCK(cudaMemcpyAsync(h->p, w.data(), h->nparam * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    SCK(cudaMemsetAsync(h->m, 0, h->nparam * sizeof(float), h->stream));
    SCK(cudaMemsetAsync(h->v, 0, h->nparam * sizeof(float), h->stream));
    h->step = 0;
    chfpe_status st = refresh_bf16(h);
    if (st) return st;
    SCK(cudaStreamSynchronize(h->stream));
    return CHFPE_OK;
}

chfpe_status chfpe_surrogate_infer(chfpe_surrogate *h, const float *X, int n, float *Y, float *S) {
    if (!h || n < 0 || (n > 0 && (!X || !Y || !S)))
        return sfail(CHFPE_EINVAL, "surrogate_infer: need a handle, n >= 0 and non-NULL buffers");
    chfpe_status st;
    for (int i0 = 0; i0 < n; i0 += h->max_batch) {
        const int B = std::min(h->max_batch, n - i0);
        if ((st = forward(h, X + (long long)i0 * NIN, B))) return st;
        SCK(cudaMemcpyAsync(Y + (long long)i0 * NPIX, h->Zc[NCONV - 1], (size_t)B * NPIX * sizeof(float),
                            cudaMemcpyDeviceToDevice, h->stream));
        SCK(cudaMemcpyAsync(S + i0, h->S, (size_t)B * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    }
    return CHFPE_OK;
}

chfpe_status chfpe_surrogate_gradients(chfpe_surrogate *h, const float *X, const float *T,
                                       const float *TS, int n, float w_scale, double *loss,
                                       float *grad_host) {
    if (!h || n < 1 || n > h->max_batch || !X || !T || !TS || !loss)
        return sfail(CHFPE_EINVAL, "surrogate_gradients: need 1 <= n <= max_batch and non-NULL pointers");
    chfpe_status st;
    SCK(cudaMemsetAsync(h->loss, 0, sizeof(double), h->stream));
    if ((st = forward(h, X, n)) || (st = backward(h, T, TS, n, w_scale))) return st;
    SCK(cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    std::vector<float> gp;
    if (grad_host) {
        gp.resize(h->nparam);
        SCK(cudaMemcpyAsync(gp.data(), h->g, h->nparam * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    }
    SCK(cudaStreamSynchronize(h->stream));
    if ((st = tc_check(h->stream))) return st;
    if (grad_host) repack(h, gp.data(), grad_host, false);
    return CHFPE_OK;
}

chfpe_status chfpe_surrogate_train(chfpe_surrogate *h, const float *X, const float *T,
                                   const float *TS, int n, int batch, int epochs, float lr,
                                   float weight_decay, float w_scale, unsigned long long seed,
                                   double *epoch_loss) {
    if (!h || n < 1 || batch < 1 || batch > h->max_batch || epochs < 0 || !X || !T || !TS ||
        !(lr >= 0.f) || !(weight_decay >= 0.f) || !(w_scale >= 0.f))
        return sfail(CHFPE_EINVAL, "surrogate_train: need n >= 1, 1 <= batch <= max_batch, epochs >= 0, "
                                   "lr, weight_decay, w_scale >= 0 and non-NULL pointers");
    chfpe_status st;
    int *dperm = nullptr;
    SCK(cudaMalloc(&dperm, (size_t)n * sizeof(int)));
    std::vector<int> perm(n);
    uint64_t x = seed;
    const int B = std::min(batch, n);
    const int steps = std::max(1, n / B);   // whole batches per epoch; the rest waits for a reshuffle
    cudaError_t e = cudaSuccess;
    st = CHFPE_OK;
    for (int ep = 0; ep < epochs && st == CHFPE_OK && e == cudaSuccess; ++ep) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) {   // Fisher-Yates
            const int j = std::min(i, (int)(unit(x) * (i + 1)));
            std::swap(perm[i], perm[j]);
        }
        // perm is reused next epoch: the synchronous copy keeps the host buffer free
        if ((e = cudaMemcpy(dperm, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(h->loss, 0, sizeof(double), h->stream)) != cudaSuccess) break;
        for (int b = 0; b < steps && st == CHFPE_OK; ++b) {
            gather_kernel<<<B, 256, 0, h->stream>>>(dperm + (long long)b * B, X, T, TS, h->Xb, h->Tb,
                                                    h->TSb, NIN, NPIX);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((st = forward(h, h->Xb, B)) || (st = backward(h, h->Tb, h->TSb, B, w_scale)) ||
                (st = adamw_step(h, lr, weight_decay)))
                break;
        }
        if (st != CHFPE_OK || e != cudaSuccess) break;
        double l = 0.0;
        if ((e = cudaMemcpyAsync(&l, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) break;
        if (epoch_loss) epoch_loss[ep] = l / steps;
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(dperm);
    if (st != CHFPE_OK) return st;
    if (e != cudaSuccess) return sfail(CHFPE_ECUDA, std::string("surrogate_train: ") + cudaGetErrorString(e));
    return tc_check(h->stream);
}

chfpe_status chfpe_surrogate_gemm(const void *A, int ta, int lda, const void *B, int tb, int ldb,
                                  float *C, const float *bias, int M, int N, int K, int splits,
                                  void *stream) {
    if (!A || !B || !C || M < 0 || N < 0 || K < 0 || splits < 1 || lda < 1 || ldb < 1)
        return sfail(CHFPE_EINVAL, "surrogate_gemm: bad arguments");
    const chfpe_status st = gemm(static_cast<cudaStream_t>(stream), ta != 0, static_cast<const bf16 *>(A),
                                 lda, tb != 0, static_cast<const bf16 *>(B), ldb, C, bias, M, N, K, splits);
    if (st) return st;
    return tc_check(static_cast<cudaStream_t>(stream));
}

}  // extern "C"
