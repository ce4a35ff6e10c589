// hermite.cuh -- the CHFPE hot path with the momenta in Hermite functions (Sec. III A, Appendix A,
// Eq. HEOM2FP-H): every member is g^(n)(q,p) = sum_k c^(n)_k(q) prod_s psi_{k_s}(p_s), psi_j the
// orthonormal Hermite functions of width a_s = sqrt(2 m_s kT) (the paper's expansion, whose
// prefactor psi_0(p) exp(-U/2kT) is the exp(-H/2kT) of the symmetrised members), stored
// [batch][member][q_1..q_d][k_1..k_d], k_d fastest.  The momentum derivatives of the grid kernels
// become ladder couplings; only the q axes carry a stencil:
//   dc^(n)_k/dt = sum_s [ sqrt(k_s+1) D+_s c^(n)_{k+e_s} - sqrt(k_s) D-_s c^(n)_{k-e_s} ]
//               - sum_s n_s gamma_s c^(n)_k
//               - sum_s sqrt((n_s+1) c_s) V_s' sqrt(k_s) / sqrt(m_s kT) c^(n+e_s)_{k-e_s}
//               + sum_s sqrt(n_s c_s)     V_s' sqrt(k_s+1) / sqrt(m_s kT) c^(n-e_s)_{k+e_s}
//   D+-_s = dU/dq_s / (2 sqrt(m_s kT)) -+ (sqrt(m_s kT) / m_s) d/dq_s
// (c_s = zeta_s gamma_s m_s kT; coefficients with k_s outside [0, K_s) are zero; d/dq_s the
// 6th-order central difference with zero values outside the q-grid, or the compact scheme of
// Sec. III B).  The insertion X^x raises k:  (X^x c)_k = -sum_s dX/dq_s sqrt(k_s) / sqrt(m_s kT)
// c_{k-e_s};  only c^(0)_0 reaches the observable.
//
// Compact q-derivatives (Sec. III B, Eqs. for A_i and B_i): along every q line,
//   A f' = B f / h,  A = tridiag(1/3, 1, 1/3),  (B f)_i = a (f_{i+1} - f_{i-1}) + b (f_{i+2} - f_{i-2}),
// zero values outside the line, a = 7/9, b = 1/36 (the sixth-order Pade scheme; the printed
// a = 7/18 is inconsistent with alpha = 1/3 and is read as 7/9).  hderiv_pcr_kernel forms B f and
// solves the tridiagonal systems of a tile of lines by parallel cyclic reduction (Sec. III C) in
// shared memory: ceil(log2 n) levels, at level l every row i eliminates its couplings to rows
// i -+ 2^l with those rows' equations, after which every row stands alone.  A is the same for
// every line, so the row multipliers of every level (and the final 1/(b_i h)) are computed once
// on the host in FP64; the device updates only the right-hand sides.  The stage kernel then
// reads the derivative arrays instead of forming stencils.
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"

namespace chfpe {

template <typename T>
struct HGeo {
    int P, NQ, Pk;              // points per member (q x k), q points, k points per q point
    int n[6], st[6];            // axis sizes and strides: q_1..q_d, k_1..k_d
    const T *Fh;                // [D][NQ]: dU/dq_s / (2 sqrt(m_s kT))
    T cq[3];                    // sqrt(m_s kT) / m_s / (60 h_qs)
    T qlo[3], qh[3];
    T VLL[3], VSL[3], gam[3];
    T lk[3];                    // 1 / sqrt(m_s kT)
    T link[3][kMaxDepth + 2];   // sqrt(k c_s)
};

template <typename T>
struct HStageArgs {
    const char *in;             // stencil input, batch of states
    const char *y;              // base states or nullptr: out = c * M in
    char *out;
    long long state_bytes;
    T c;
    const T *dq;                // compact scheme: d/dq_s of state b at dq + (b D + s) dq_state
    long long dq_state;         // (elements; nullptr: explicit stencils, cq holds 1/(60 h) then)
    const T *c2;                // compact scheme, two modes, n_2 <= 32: the q_2 axis' PCR table
    int lv2, skew2;             // ([lv2][2][n_2], then 1 / (b h)) for a row kernel that solves the
                                // q_2 lines itself (hstage_solves_q2); skew2: the skew part
    HGeo<T> g;
};

// Tile of 32 q lines along one axis: every line is n values `st` elements apart; line l of a
// state starts at (l / st) n st + l % st (the member index is the outermost part of l / st)
template <typename T>
struct HDerivArgs {
    const char *in;             // batch of states, in_state bytes apart
    long long in_state;
    T *out;                     // derivatives: out + b out_state + (same offset as the input)
    long long out_state;        // elements
    int n, st, lines;           // line length, axis stride, lines per state (M P / n)
    int levels;                 // PCR levels, 2^levels >= n
    const T *coef;              // [levels][2][n] row multipliers (rows i - 2^l, i + 2^l), then
                                // [n] 1 / (b_i h) of the reduced diagonal
    int skew;                   // 1: the skew-symmetric part of the compact derivative
};

constexpr int kPcrCols = 32, kPcrRows = 8;

// (B f)_i = a (f_{i+1} - f_{i-1}) + b (f_{i+2} - f_{i-2}) of column tx of a shared tile, zero
// values outside the line
template <typename T>
__device__ __forceinline__ T pcr_bf(const T *F, int i, int n, int tx) {
    const T ca = T(7) / T(9), cb = T(1) / T(36);
    const T f1 = (i + 1 < n ? F[(i + 1) * kPcrCols + tx] : T(0)) - (i >= 1 ? F[(i - 1) * kPcrCols + tx] : T(0));
    const T f2 = (i + 2 < n ? F[(i + 2) * kPcrCols + tx] : T(0)) - (i >= 2 ? F[(i - 2) * kPcrCols + tx] : T(0));
    return ca * f1 + cb * f2;
}

// PCR on the columns of the shared tile `cur` (right-hand sides), `nxt` as scratch; returns the
// buffer that holds the reduced right-hand sides d_i (x_i = d_i / b_i)
template <typename T>
__device__ __forceinline__ T *pcr_solve(T *cur, T *nxt, const HDerivArgs<T> &a, int tx, int ty) {
    const int n = a.n;
    for (int l = 0; l < a.levels; ++l) {
        const int o = 1 << l;
        const T *k1 = a.coef + (long long)2 * l * n, *k2 = k1 + n;
        for (int i = ty; i < n; i += kPcrRows) {
            T v = cur[i * kPcrCols + tx];
            if (i - o >= 0) v -= k1[i] * cur[(i - o) * kPcrCols + tx];
            if (i + o < n) v -= k2[i] * cur[(i + o) * kPcrCols + tx];
            nxt[i * kPcrCols + tx] = v;
        }
        __syncthreads();
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
    return cur;
}

// compact first derivative along one q axis of a tile of 32 lines of every state in the batch
// (blockIdx.y): load, B f, PCR, scale, store; 2 n 32 values of shared memory.
// SKEW: the skew-symmetric part (A^{-1} B f + B A^{-1} f) / 2h instead (3 n 32 values): the first
// term as above, then a second PCR on f itself and B applied to its solution
template <typename T, bool SKEW>
__global__ void __launch_bounds__(kPcrCols * kPcrRows) hderiv_pcr_kernel(const HDerivArgs<T> a) {
    extern __shared__ __align__(16) unsigned char pcr_smem[];
    T *buf0 = reinterpret_cast<T *>(pcr_smem);
    T *buf1 = buf0 + a.n * kPcrCols;
    T *buf2 = buf1 + a.n * kPcrCols;          // SKEW only
    const int tx = threadIdx.x, ty = threadIdx.y, n = a.n;
    const int line = blockIdx.x * kPcrCols + tx;
    const bool ok = line < a.lines;
    const int outer = ok ? line / a.st : 0;
    const long long base = (long long)outer * n * a.st + (ok ? line - outer * a.st : 0);
    const T *f = reinterpret_cast<const T *>(a.in + (long long)blockIdx.y * a.in_state) + base;
    T *F = SKEW ? buf2 : buf1;                // f, kept while the first solve runs (SKEW)
    for (int i = ty; i < n; i += kPcrRows) F[i * kPcrCols + tx] = ok ? __ldg(f + (long long)i * a.st) : T(0);
    __syncthreads();
    for (int i = ty; i < n; i += kPcrRows) buf0[i * kPcrCols + tx] = pcr_bf(F, i, n, tx);
    __syncthreads();
    const T *binv = a.coef + (long long)2 * a.levels * n;   // 1 / (b_i h)
    T *x1 = pcr_solve(buf0, buf1, a, tx, ty);               // A^{-1} B f, unscaled
    if constexpr (SKEW) {
        // x1 lies in buf0 or buf1; the other one is scratch for the solve A y = f (f in buf2)
        T *scratch = x1 == buf0 ? buf1 : buf0;
        T *y = pcr_solve(buf2, scratch, a, tx, ty);         // A y = f: d_i, y_i = d_i / b_i
        // y / h = d_i binv_i, in place; then out = (x1 binv + B (y / h)) / 2
        for (int i = ty; i < n; i += kPcrRows) y[i * kPcrCols + tx] *= binv[i];
        __syncthreads();
        if (ok) {
            T *o = a.out + (long long)blockIdx.y * a.out_state + base;
            for (int i = ty; i < n; i += kPcrRows)
                o[(long long)i * a.st] = T(0.5) * (x1[i * kPcrCols + tx] * binv[i] + pcr_bf(y, i, n, tx));
        }
    } else if (ok) {
        T *o = a.out + (long long)blockIdx.y * a.out_state + base;
        for (int i = ty; i < n; i += kPcrRows) o[(long long)i * a.st] = x1[i * kPcrCols + tx] * binv[i];
    }
}

// The same compact derivative for lines of at most 32 points, a line per warp: lane r holds row
// r, (B f)_r and every PCR level take register shuffles (the level's row multipliers are the
// lane's registers), no block barrier between levels.  A block loads a tile of 32 lines into
// shared memory with coalesced loads (row-padded to 33 columns), its 8 warps solve 4 lines each,
// and the tile is stored back coalesced.
template <typename T>
__device__ __forceinline__ T warp_bf(T v, int r, int n) {
    const T ca = T(7) / T(9), cb = T(1) / T(36);
    const T p1 = __shfl_down_sync(0xffffffffu, v, 1), m1 = __shfl_up_sync(0xffffffffu, v, 1);
    const T p2 = __shfl_down_sync(0xffffffffu, v, 2), m2 = __shfl_up_sync(0xffffffffu, v, 2);
    return ca * ((r + 1 < n ? p1 : T(0)) - (r >= 1 ? m1 : T(0))) +
           cb * ((r + 2 < n ? p2 : T(0)) - (r >= 2 ? m2 : T(0)));
}

template <typename T>
__device__ __forceinline__ T warp_pcr(T d, const T *k1, const T *k2, int levels) {
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        if (l >= levels) break;
        const int o = 1 << l;
        const T dm = __shfl_up_sync(0xffffffffu, d, o), dp = __shfl_down_sync(0xffffffffu, d, o);
        d -= k1[l] * dm + k2[l] * dp;   // the multipliers are zero where r -+ 2^l leaves the line
    }
    return d;
}

template <typename T, bool SKEW>
__global__ void __launch_bounds__(kPcrCols * kPcrRows) hderiv_warp_kernel(const HDerivArgs<T> a) {
    __shared__ T tile[32][kPcrCols + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, n = a.n;
    const int line = blockIdx.x * kPcrCols + tx;
    const bool ok = line < a.lines;
    const int outer = ok ? line / a.st : 0;
    const long long base = (long long)outer * n * a.st + (ok ? line - outer * a.st : 0);
    const T *f = reinterpret_cast<const T *>(a.in + (long long)blockIdx.y * a.in_state) + base;
    {
        T v[32 / kPcrRows];   // every load of the tile in flight before the first store
#pragma unroll
        for (int j = 0; j < 32 / kPcrRows; ++j) {
            const int i = ty + j * kPcrRows;
            v[j] = (ok && i < n) ? __ldg(f + (long long)i * a.st) : T(0);
        }
#pragma unroll
        for (int j = 0; j < 32 / kPcrRows; ++j) tile[ty + j * kPcrRows][tx] = v[j];
    }
    // lane tx is row tx of the warp's lines: its multipliers of every level and 1 / (b h)
    T k1[5], k2[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        k1[l] = (l < a.levels && tx < n) ? a.coef[(long long)2 * l * n + tx] : T(0);
        k2[l] = (l < a.levels && tx < n) ? a.coef[(long long)(2 * l + 1) * n + tx] : T(0);
    }
    const T binv = tx < n ? a.coef[(long long)2 * a.levels * n + tx] : T(0);
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < kPcrCols / kPcrRows; ++cc) {   // 4 independent lines per warp, interleaved
        const int c = ty + cc * kPcrRows;
        const T v = tx < n ? tile[tx][c] : T(0);
        T r = warp_pcr(warp_bf(v, tx, n), k1, k2, a.levels) * binv;    // A^{-1} B f / h
        if constexpr (SKEW) {
            const T yv = warp_pcr(v, k1, k2, a.levels) * binv;             // A^{-1} f / h
            r = T(0.5) * (r + warp_bf(yv, tx, n));
        }
        __syncwarp();
        if (tx < n) tile[tx][c] = r;
    }
    __syncthreads();
    if (ok) {
        T *o = a.out + (long long)blockIdx.y * a.out_state + base;
#pragma unroll
        for (int j = 0; j < 32 / kPcrRows; ++j) {
            const int i = ty + j * kPcrRows;
            if (i < n) o[(long long)i * a.st] = tile[i][tx];
        }
    }
}

// 45 (f+1 - f-1) - 9 (f+2 - f-2) + (f+3 - f-3) along q axis `s` of the point x (q index i)
template <typename T>
__device__ __forceinline__ T hstencil(const T *__restrict__ f, int x, int i, int N, int st) {
    const T p1 = (i + 1 < N) ? __ldg(f + x + st) : T(0);
    const T m1 = (i >= 1) ? __ldg(f + x - st) : T(0);
    const T p2 = (i + 2 < N) ? __ldg(f + x + 2 * st) : T(0);
    const T m2 = (i >= 2) ? __ldg(f + x - 2 * st) : T(0);
    const T p3 = (i + 3 < N) ? __ldg(f + x + 3 * st) : T(0);
    const T m3 = (i >= 3) ? __ldg(f + x - 3 * st) : T(0);
    return T(45) * (p1 - m1) - T(9) * (p2 - m2) + (p3 - m3);
}

// Explicit q-stencil sums of every value along every q axis into the derivative arrays:
//   out[b][s][x] = 45 (c_{+1} - c_{-1}) - 9 (c_{+2} - c_{-2}) + (c_{+3} - c_{-3})   along q_s,
// zero values outside the q-grid (the stage kernel scales them by cq_s, which carries 1 / 60 h).
// For three modes, where the stage's gather form would re-form the stencils of both ladder
// neighbours of every value; one thread per V consecutive values of every member (V > 1 where a
// q point's K_1..K_D values are a multiple of V: the V values share their q indices, every tap is
// one vector load).
template <typename T, int D, int V>
__global__ void __launch_bounds__(256) hstencil_sums_kernel(const HGeo<T> g, const char *in, long long in_state,
                                                            T *out, long long out_state, long long total) {
    typedef typename VecOf<T, V>::type VT;
    const long long x = ((long long)blockIdx.x * 256 + threadIdx.x) * V;
    if (x >= total) return;
    const T *c = reinterpret_cast<const T *>(in + (long long)blockIdx.y * in_state) + x;
    T *o = out + (long long)blockIdx.y * D * out_state + x;
    const int r = (int)(x % g.P);                       // index inside the member
#pragma unroll
    for (int s = 0; s < D; ++s) {
        const int i = (r / g.st[s]) % g.n[s], st = g.st[s], n = g.n[s];
        T acc[V];
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = T(0);
#pragma unroll
        for (int t = 1; t <= 3; ++t) {
            const T w = t == 1 ? T(45) : (t == 2 ? T(-9) : T(1));
            VT p, m;
            if (i + t < n) p = __ldg(reinterpret_cast<const VT *>(c + (long long)t * st));
            if (i - t >= 0) m = __ldg(reinterpret_cast<const VT *>(c - (long long)t * st));
            const T *pe = reinterpret_cast<const T *>(&p), *me = reinterpret_cast<const T *>(&m);
#pragma unroll
            for (int e = 0; e < V; ++e)
                acc[e] += w * ((i + t < n ? pe[e] : T(0)) - (i - t >= 0 ? me[e] : T(0)));
        }
        *reinterpret_cast<VT *>(o + (long long)s * out_state) = *reinterpret_cast<const VT *>(acc);
    }
}

// one RK4 stage, one thread per (q, k) point for every member (gather form: each output reads the
// q-stencils of its k +- e_s neighbours and the link values of its member neighbours)
template <typename T, int D, int DEPTH, int NT, bool PRE = false>
__global__ void __launch_bounds__(NT) hstage_kernel(const HStageArgs<T> a) {
    constexpr MemberTable<D, DEPTH> tab{};
    constexpr int M = MemberTable<D, DEPTH>::M;
    const HGeo<T> &g = a.g;
    const int x = blockIdx.x * NT + threadIdx.x;
    if (x >= g.P) return;
    const long long boff = (long long)blockIdx.y * a.state_bytes;
    const T *in = reinterpret_cast<const T *>(a.in + boff);
    T *out = reinterpret_cast<T *>(a.out + boff);
    const T *y = a.y ? reinterpret_cast<const T *>(a.y + boff) : nullptr;
    const T *dqb = PRE ? a.dq + (long long)blockIdx.y * D * a.dq_state : nullptr;

    int idx[2 * D];
    {
        int r = x;
#pragma unroll
        for (int ax = 2 * D - 1; ax >= 0; --ax) {
            idx[ax] = r % g.n[ax];
            r /= g.n[ax];
        }
    }
    const int qlin = x / g.Pk;
    T F[D], Vl[D], sk[D], sk1[D];
    bool hp[D], hm[D];
#pragma unroll
    for (int s = 0; s < D; ++s) {
        F[s] = __ldg(g.Fh + s * g.NQ + qlin);
        const T q = g.qlo[s] + T(idx[s]) * g.qh[s];
        Vl[s] = (g.VLL[s] + g.VSL[s] * q) * g.lk[s];
        const int k = idx[D + s];
        sk[s] = sqrt(T(k));
        sk1[s] = sqrt(T(k + 1));
        hp[s] = k + 1 < g.n[D + s];
        hm[s] = k >= 1;
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const T *c = in + (long long)m * g.P;
        T gm = T(0);
#pragma unroll
        for (int s = 0; s < D; ++s) gm += T(tab.n[m][s]) * g.gam[s];
        T acc = -gm * __ldg(c + x);
#pragma unroll
        for (int s = 0; s < D; ++s) {
            const int sk_st = g.st[D + s];
            if (hp[s]) {             // sqrt(k+1) D+ c_{k+e_s}
                const int xp = x + sk_st;
                const T dq = PRE ? __ldg(dqb + s * a.dq_state + (long long)m * g.P + xp)
                                 : hstencil<T>(c, xp, idx[s], g.n[s], g.st[s]);
                acc += sk1[s] * (F[s] * __ldg(c + xp) - g.cq[s] * dq);
            }
            if (hm[s]) {             // - sqrt(k) D- c_{k-e_s}
                const int xm = x - sk_st;
                const T dq = PRE ? __ldg(dqb + s * a.dq_state + (long long)m * g.P + xm)
                                 : hstencil<T>(c, xm, idx[s], g.n[s], g.st[s]);
                acc -= sk[s] * (F[s] * __ldg(c + xm) + g.cq[s] * dq);
            }
            if (tab.up[m][s] >= 0 && hm[s]) {
                const T *cu = in + (long long)tab.up[m][s] * g.P;
                acc -= g.link[s][tab.n[m][s] + 1] * Vl[s] * sk[s] * __ldg(cu + x - sk_st);
            }
            if (tab.dn[m][s] >= 0 && hp[s]) {
                const T *cd = in + (long long)tab.dn[m][s] * g.P;
                acc += g.link[s][tab.n[m][s]] * Vl[s] * sk1[s] * __ldg(cd + x + sk_st);
            }
        }
        const long long o = (long long)m * g.P + x;
        out[o] = y ? y[o] + a.c * acc : a.c * acc;
    }
}

// The same stage for two modes with explicit q stencils, one block per (state, member, chunk of
// q_1 rows), marching along q_1.  A q_1 row (every q_2 and k of one q_1 value, L = n_2 K_1 K_2
// contiguous values) is the unit: a ring of 7 rows in shared memory holds the q_1 stencil's
// window, filled by asynchronous copies one row ahead (rows outside the grid are zeros), so each
// row is read from global memory once per chunk plus the chunk's 6 halo rows.  Every ring row is
// padded with zeros along q_2 (3 K_1 K_2 values each side), so the q_2 taps need no test.  Per
// row, phase 1 forms every element's q-derivative sums D_1 c, D_2 c into shared memory while the
// row's base values y and the four hierarchy-link rows (the neighbour members, same row) arrive
// by asynchronous copies; phase 2 forms, with F_s and the centre values of the same q point,
//   dc_k/dt = -gamma c_k + sum_s [ sqrt(k_s+1) A_s(k+e_s) - sqrt(k_s) B_s(k-e_s) ] + links,
//   A_s = F_s c - cq_s D_s c,   B_s = F_s c + cq_s D_s c,
// and stores y + c * (dc/dt).  Thread t owns the row positions t + j kRowThreads (j < E) in
// every row, their ladder factors (zero where k -+ e_s leaves the basis) kept in registers.
// Equal to hstage_kernel up to the order of the additions.
constexpr int kRowThreads = 256, kRowMaxM = 21;

template <typename T>
struct HRowArgs {
    HStageArgs<T> s;
    int rows;                    // q_1 rows per chunk
    int vec;                     // 1: rows start on 16-byte boundaries (16-byte copies)
    int pad;                     // zeros on each side of a ring row (>= 3 K_1 K_2, 16-byte multiple)
    int lpad;                    // zeros on each side of a link row (pair kernel: >= K_2, 16-byte multiple)
    int mt[kRowMaxM][6];         // per member: n_1, n_2, up_1, up_2, dn_1, dn_2 (-1: none)
};

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// n values global -> shared, asynchronous, by the whole block (vec: 16-byte copies)
template <typename T>
__device__ __forceinline__ void hrow_copy(T *dst, const T *src, int n, bool vec) {
    if (vec) {
        constexpr int W = 16 / sizeof(T);
        for (int x = threadIdx.x * W; x < n; x += kRowThreads * W) cp_async16(dst + x, src + x, 16);
    } else {
        for (int x = threadIdx.x; x < n; x += kRowThreads) cp_async_elem(dst + x, src + x);
    }
}

template <typename T, int E>
__global__ void __launch_bounds__(kRowThreads, 3) hstage_row_kernel(const HRowArgs<T> ra) {
    const HStageArgs<T> &a = ra.s;
    const HGeo<T> &g = a.g;
    extern __shared__ __align__(16) unsigned char hrow_smem[];
    const int n1 = g.n[0], n2 = g.n[1], K1 = g.n[2], K2 = g.n[3];
    const int KK = K1 * K2, L = n2 * KK, S = L + 2 * ra.pad;   // row, padded row
    T *ring = reinterpret_cast<T *>(hrow_smem) + ra.pad;      // 7 padded rows (interiors)
    T *dd = ring + 7 * S;                                      // D_1 c, D_2 c (padded rows)
    T *lrow = dd + 2 * S - ra.pad;                             // y, up_1, up_2, dn_1, dn_2 of row i
    T *fr = lrow + 5 * L;                                      // 7 rows of (F_1, F_2)
    const int m = blockIdx.x;
    int mt[6];
#pragma unroll
    for (int i = 0; i < kRowMaxM; ++i)
        if (i == m) {
#pragma unroll
            for (int f = 0; f < 6; ++f) mt[f] = ra.mt[i][f];
        }
    const int r0 = blockIdx.y * ra.rows, r1 = min(n1, r0 + ra.rows);
    const long long boff = (long long)blockIdx.z * a.state_bytes;
    const T *in = reinterpret_cast<const T *>(a.in + boff);
    const T *cm = in + (long long)m * g.P;
    T *out = reinterpret_cast<T *>(a.out + boff) + (long long)m * g.P;
    const T *y = a.y ? reinterpret_cast<const T *>(a.y + boff) + (long long)m * g.P : nullptr;
    const bool vec = ra.vec != 0;
    // the members of the links (nullptr: none) and their factors
    const T *lsrc[5] = {y, mt[2] >= 0 ? in + (long long)mt[2] * g.P : nullptr,
                        mt[3] >= 0 ? in + (long long)mt[3] * g.P : nullptr,
                        mt[4] >= 0 ? in + (long long)mt[4] * g.P : nullptr,
                        mt[5] >= 0 ? in + (long long)mt[5] * g.P : nullptr};
    const T wup0 = mt[2] >= 0 ? g.link[0][mt[0] + 1] * g.lk[0] : T(0);
    const T wup1 = mt[3] >= 0 ? g.link[1][mt[1] + 1] * g.lk[1] : T(0);
    const T wdn0 = mt[4] >= 0 ? g.link[0][mt[0]] * g.lk[0] : T(0);
    const T wdn1 = mt[5] >= 0 ? g.link[1][mt[1]] * g.lk[1] : T(0);
    // zero padding of the 9 padded rows (never written again); link rows of absent members
    for (int j = threadIdx.x; j < 9 * 2 * ra.pad; j += kRowThreads) {
        const int r = j / (2 * ra.pad), o = j - r * 2 * ra.pad;
        ring[r * S + (o < ra.pad ? o - ra.pad : L + o - ra.pad)] = T(0);
    }
#pragma unroll
    for (int l = 1; l < 5; ++l)
        if (!lsrc[l])
            for (int x = threadIdx.x; x < L; x += kRowThreads) lrow[l * L + x] = T(0);
    // row i of the window into its slot: copied, or zeros outside the grid
    auto load_row = [&](int i) {
        const int sl = (i + 7) % 7;
        T *dst = ring + sl * S;
        if (i >= 0 && i < n1) {
            hrow_copy(dst, cm + (long long)i * L, L, vec);
            for (int x = threadIdx.x; x < n2; x += kRowThreads) {
                cp_async_elem(fr + sl * 2 * n2 + x, g.Fh + (long long)i * n2 + x);
                cp_async_elem(fr + sl * 2 * n2 + n2 + x, g.Fh + g.NQ + (long long)i * n2 + x);
            }
        } else {
            for (int x = threadIdx.x; x < L; x += kRowThreads) dst[x] = T(0);
        }
    };
    for (int i = r0 - 3; i <= r0 + 3; ++i) load_row(i);
    asm volatile("cp.async.commit_group;" ::: "memory");
    // this thread's positions and their ladder factors
    int xs[E], q2s[E];
    T s1a[E], s0a[E], s1b[E], s0b[E], V2[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int x = threadIdx.x + j * kRowThreads;
        const int xr = x < L ? x : L - 1;
        const int q2 = xr / KK, kk = xr - q2 * KK, k1 = kk / K2, k2 = kk - k1 * K2;
        xs[j] = x;
        q2s[j] = q2;
        s1a[j] = k1 + 1 < K1 ? sqrt(T(k1 + 1)) : T(0);
        s0a[j] = sqrt(T(k1));
        s1b[j] = k2 + 1 < K2 ? sqrt(T(k2 + 1)) : T(0);
        s0b[j] = sqrt(T(k2));
        V2[j] = g.VLL[1] + g.VSL[1] * (g.qlo[1] + T(q2) * g.qh[1]);
    }
    const T gm = T(mt[0]) * g.gam[0] + T(mt[1]) * g.gam[1];
    const T cq1 = g.cq[0], cq2 = g.cq[1];
    for (int i = r0; i < r1; ++i) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        // the row's base values and link rows, in flight during phase 1
        const long long ro = (long long)i * L;
#pragma unroll
        for (int l = 0; l < 5; ++l)
            if (lsrc[l]) hrow_copy(lrow + l * L, lsrc[l] + ro, L, vec);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // phase 1: D_1 c, D_2 c of every element of row i
        const T *R0 = ring + (i % 7) * S;
        {
            const T *Rp1 = ring + ((i + 1) % 7) * S, *Rp2 = ring + ((i + 2) % 7) * S, *Rp3 = ring + ((i + 3) % 7) * S;
            const T *Rm1 = ring + ((i + 6) % 7) * S, *Rm2 = ring + ((i + 5) % 7) * S, *Rm3 = ring + ((i + 4) % 7) * S;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int x = xs[j];
                if (j == E - 1 && x >= L) break;
                dd[x] = T(45) * (Rp1[x] - Rm1[x]) - T(9) * (Rp2[x] - Rm2[x]) + (Rp3[x] - Rm3[x]);
                dd[S + x] = T(45) * (R0[x + KK] - R0[x - KK]) - T(9) * (R0[x + 2 * KK] - R0[x - 2 * KK]) +
                            (R0[x + 3 * KK] - R0[x - 3 * KK]);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        // the next row of the window (its slot held row i - 3), in flight during phase 2
        if (i + 1 < r1) load_row(i + 4);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // phase 2
        const T V1 = g.VLL[0] + g.VSL[0] * (g.qlo[0] + T(i) * g.qh[0]);
        const T ldn0 = wdn0 * V1, lup0 = wup0 * V1;
        const T *F = fr + (i % 7) * 2 * n2;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int x = xs[j];
            if (j == E - 1 && x >= L) break;
            const T F1 = F[q2s[j]], F2 = F[n2 + q2s[j]];
            T acc = -gm * R0[x];
            acc += s1a[j] * (F1 * R0[x + K2] - cq1 * dd[x + K2] + ldn0 * lrow[3 * L + min(x + K2, L - 1)]);
            acc -= s0a[j] * (F1 * R0[x - K2] + cq1 * dd[x - K2] + lup0 * lrow[L + max(x - K2, 0)]);
            acc += s1b[j] * (F2 * R0[x + 1] - cq2 * dd[S + x + 1] + wdn1 * V2[j] * lrow[4 * L + min(x + 1, L - 1)]);
            acc -= s0b[j] * (F2 * R0[x - 1] + cq2 * dd[S + x - 1] + wup1 * V2[j] * lrow[2 * L + max(x - 1, 0)]);
            out[ro + x] = y ? lrow[x] + a.c * acc : a.c * acc;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// The row-marching stage for even K_2 with element pairs: thread t owns the pairs (x, x + 1),
// x = 2 (t + j kRowThreads), of every row (both of one k_1 row and one q point), read and written
// as 2-vectors; the link and base rows carry zero pads of >= K_2 values each side, so no
// neighbour index needs a clamp.  Same phases and shared memory as hstage_row_kernel.
template <typename T>
__device__ __forceinline__ typename VecOf<T, 2>::type ld2(const T *p) {
    return *reinterpret_cast<const typename VecOf<T, 2>::type *>(p);
}

template <typename T, int E>
__global__ void __launch_bounds__(kRowThreads, 3) hstage_row2_kernel(const HRowArgs<T> ra) {
    typedef typename VecOf<T, 2>::type T2;
    const HStageArgs<T> &a = ra.s;
    const HGeo<T> &g = a.g;
    extern __shared__ __align__(16) unsigned char hrow_smem[];
    const int n1 = g.n[0], n2 = g.n[1], K1 = g.n[2], K2 = g.n[3];
    const int KK = K1 * K2, L = n2 * KK, S = L + 2 * ra.pad, SL = L + 2 * ra.lpad;
    T *ring = reinterpret_cast<T *>(hrow_smem) + ra.pad;      // 7 padded rows (interiors)
    T *dd = ring + 7 * S;                                      // D_1 c, D_2 c (padded rows)
    T *lrow = dd + 2 * S - ra.pad + ra.lpad;                   // y, up_1, up_2, dn_1, dn_2 (padded)
    T *fr = lrow + 5 * SL - ra.lpad;                           // 7 rows of (F_1, F_2)
    const int m = blockIdx.x;
    int mt[6];
#pragma unroll
    for (int i = 0; i < kRowMaxM; ++i)
        if (i == m) {
#pragma unroll
            for (int f = 0; f < 6; ++f) mt[f] = ra.mt[i][f];
        }
    const int r0 = blockIdx.y * ra.rows, r1 = min(n1, r0 + ra.rows);
    const long long boff = (long long)blockIdx.z * a.state_bytes;
    const T *in = reinterpret_cast<const T *>(a.in + boff);
    const T *cm = in + (long long)m * g.P;
    T *out = reinterpret_cast<T *>(a.out + boff) + (long long)m * g.P;
    const T *y = a.y ? reinterpret_cast<const T *>(a.y + boff) + (long long)m * g.P : nullptr;
    const bool vec = ra.vec != 0;
    const T *lsrc[5] = {y, mt[2] >= 0 ? in + (long long)mt[2] * g.P : nullptr,
                        mt[3] >= 0 ? in + (long long)mt[3] * g.P : nullptr,
                        mt[4] >= 0 ? in + (long long)mt[4] * g.P : nullptr,
                        mt[5] >= 0 ? in + (long long)mt[5] * g.P : nullptr};
    const T wup0 = mt[2] >= 0 ? g.link[0][mt[0] + 1] * g.lk[0] : T(0);
    const T wup1 = mt[3] >= 0 ? g.link[1][mt[1] + 1] * g.lk[1] : T(0);
    const T wdn0 = mt[4] >= 0 ? g.link[0][mt[0]] * g.lk[0] : T(0);
    const T wdn1 = mt[5] >= 0 ? g.link[1][mt[1]] * g.lk[1] : T(0);
    // zero pads (never written again); the link rows of absent members
    for (int j = threadIdx.x; j < 9 * 2 * ra.pad; j += kRowThreads) {
        const int r = j / (2 * ra.pad), o = j - r * 2 * ra.pad;
        ring[r * S + (o < ra.pad ? o - ra.pad : L + o - ra.pad)] = T(0);
    }
    for (int j = threadIdx.x; j < 5 * 2 * ra.lpad; j += kRowThreads) {
        const int r = j / (2 * ra.lpad), o = j - r * 2 * ra.lpad;
        lrow[r * SL + (o < ra.lpad ? o - ra.lpad : L + o - ra.lpad)] = T(0);
    }
#pragma unroll
    for (int l = 1; l < 5; ++l)
        if (!lsrc[l])
            for (int x = threadIdx.x; x < L; x += kRowThreads) lrow[l * SL + x] = T(0);
    auto load_row = [&](int i) {
        const int sl = (i + 7) % 7;
        T *dst = ring + sl * S;
        if (i >= 0 && i < n1) {
            hrow_copy(dst, cm + (long long)i * L, L, vec);
            for (int x = threadIdx.x; x < n2; x += kRowThreads) {
                cp_async_elem(fr + sl * 2 * n2 + x, g.Fh + (long long)i * n2 + x);
                cp_async_elem(fr + sl * 2 * n2 + n2 + x, g.Fh + g.NQ + (long long)i * n2 + x);
            }
        } else {
            for (int x = threadIdx.x; x < L; x += kRowThreads) dst[x] = T(0);
        }
    };
    for (int i = r0 - 3; i <= r0 + 3; ++i) load_row(i);
    asm volatile("cp.async.commit_group;" ::: "memory");
    // this thread's pairs: k_1 and q_2 shared, k_2 = kb and kb + 1 (kb even)
    int xs[E], q2s[E];
    T s1a[E], s0a[E], s1b0[E], s0b0[E], s1b1[E], s0b1[E], V2[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int x = 2 * (threadIdx.x + j * kRowThreads);
        const int xr = x < L ? x : L - 2;
        const int q2 = xr / KK, kk = xr - q2 * KK, k1 = kk / K2, kb = kk - k1 * K2;
        xs[j] = x;
        q2s[j] = q2;
        s1a[j] = k1 + 1 < K1 ? sqrt(T(k1 + 1)) : T(0);
        s0a[j] = sqrt(T(k1));
        s1b0[j] = sqrt(T(kb + 1));
        s0b0[j] = sqrt(T(kb));
        s1b1[j] = kb + 2 < K2 ? sqrt(T(kb + 2)) : T(0);
        s0b1[j] = sqrt(T(kb + 1));
        V2[j] = g.VLL[1] + g.VSL[1] * (g.qlo[1] + T(q2) * g.qh[1]);
    }
    const T gm = T(mt[0]) * g.gam[0] + T(mt[1]) * g.gam[1];
    const T cq1 = g.cq[0], cq2 = g.cq[1];
    for (int i = r0; i < r1; ++i) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const long long ro = (long long)i * L;
#pragma unroll
        for (int l = 0; l < 5; ++l)
            if (lsrc[l]) hrow_copy(lrow + l * SL, lsrc[l] + ro, L, vec);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // phase 1: D_1 c, D_2 c of every pair of row i
        const T *R0 = ring + (i % 7) * S;
        {
            const T *Rp1 = ring + ((i + 1) % 7) * S, *Rp2 = ring + ((i + 2) % 7) * S, *Rp3 = ring + ((i + 3) % 7) * S;
            const T *Rm1 = ring + ((i + 6) % 7) * S, *Rm2 = ring + ((i + 5) % 7) * S, *Rm3 = ring + ((i + 4) % 7) * S;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int x = xs[j];
                if (j == E - 1 && x >= L) break;
                const T2 p1 = ld2(Rp1 + x), m1 = ld2(Rm1 + x), p2 = ld2(Rp2 + x), m2 = ld2(Rm2 + x);
                const T2 p3 = ld2(Rp3 + x), m3 = ld2(Rm3 + x);
                const T2 u1 = ld2(R0 + x + KK), v1 = ld2(R0 + x - KK), u2 = ld2(R0 + x + 2 * KK);
                const T2 v2 = ld2(R0 + x - 2 * KK), u3 = ld2(R0 + x + 3 * KK), v3 = ld2(R0 + x - 3 * KK);
                T2 d1, d2;
                d1.x = T(45) * (p1.x - m1.x) - T(9) * (p2.x - m2.x) + (p3.x - m3.x);
                d1.y = T(45) * (p1.y - m1.y) - T(9) * (p2.y - m2.y) + (p3.y - m3.y);
                d2.x = T(45) * (u1.x - v1.x) - T(9) * (u2.x - v2.x) + (u3.x - v3.x);
                d2.y = T(45) * (u1.y - v1.y) - T(9) * (u2.y - v2.y) + (u3.y - v3.y);
                *reinterpret_cast<T2 *>(dd + x) = d1;
                *reinterpret_cast<T2 *>(dd + S + x) = d2;
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (i + 1 < r1) load_row(i + 4);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // phase 2
        const T V1 = g.VLL[0] + g.VSL[0] * (g.qlo[0] + T(i) * g.qh[0]);
        const T ldn0 = wdn0 * V1, lup0 = wup0 * V1;
        const T *F = fr + (i % 7) * 2 * n2;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int x = xs[j];
            if (j == E - 1 && x >= L) break;
            const T F1 = F[q2s[j]], F2 = F[n2 + q2s[j]];
            const T ldn1 = wdn1 * V2[j], lup1 = wup1 * V2[j];
            const T2 c = ld2(R0 + x), cL = ld2(R0 + x - 2), cR = ld2(R0 + x + 2);
            const T2 cU = ld2(R0 + x + K2), cD = ld2(R0 + x - K2);
            const T2 e1U = ld2(dd + x + K2), e1D = ld2(dd + x - K2);
            const T2 e2L = ld2(dd + S + x - 2), e2C = ld2(dd + S + x), e2R = ld2(dd + S + x + 2);
            const T2 up0 = ld2(lrow + SL + x - K2), dn0 = ld2(lrow + 3 * SL + x + K2);
            const T2 up1L = ld2(lrow + 2 * SL + x - 2), up1C = ld2(lrow + 2 * SL + x);
            const T2 dn1C = ld2(lrow + 4 * SL + x), dn1R = ld2(lrow + 4 * SL + x + 2);
            T acc0 = -gm * c.x, acc1 = -gm * c.y;
            acc0 += s1a[j] * (F1 * cU.x - cq1 * e1U.x + ldn0 * dn0.x) - s0a[j] * (F1 * cD.x + cq1 * e1D.x + lup0 * up0.x);
            acc1 += s1a[j] * (F1 * cU.y - cq1 * e1U.y + ldn0 * dn0.y) - s0a[j] * (F1 * cD.y + cq1 * e1D.y + lup0 * up0.y);
            acc0 += s1b0[j] * (F2 * c.y - cq2 * e2C.y + ldn1 * dn1C.y) - s0b0[j] * (F2 * cL.y + cq2 * e2L.y + lup1 * up1L.y);
            acc1 += s1b1[j] * (F2 * cR.x - cq2 * e2R.x + ldn1 * dn1R.x) - s0b1[j] * (F2 * c.x + cq2 * e2C.x + lup1 * up1C.x);
            T2 r;
            if (y) {
                const T2 yv = ld2(lrow + x);
                r.x = yv.x + a.c * acc0;
                r.y = yv.y + a.c * acc1;
            } else {
                r.x = a.c * acc0;
                r.y = a.c * acc1;
            }
            *reinterpret_cast<T2 *>(out + ro + x) = r;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// The row-marching stage for the compact q-derivatives (even K_2, element pairs): D_1 c and D_2 c
// come from the derivative arrays, so no stencil window is needed.  Per row, the centre values,
// both derivative rows, the base values and the four link rows (8 zero-padded rows) and F are
// copied by cp.async into one of two buffers while the other buffer's row is computed as in
// phase 2 of hstage_row2_kernel; one block barrier per row.
template <typename T, int E>
__global__ void __launch_bounds__(kRowThreads, 3) hstage_rowpre_kernel(const HRowArgs<T> ra) {
    typedef typename VecOf<T, 2>::type T2;
    const HStageArgs<T> &a = ra.s;
    const HGeo<T> &g = a.g;
    extern __shared__ __align__(16) unsigned char hrow_smem[];
    const int n1 = g.n[0], n2 = g.n[1], K1 = g.n[2], K2 = g.n[3];
    const int KK = K1 * K2, L = n2 * KK, SL = L + 2 * ra.lpad;
    // two buffers of 8 padded rows: c, D_1 c, D_2 c, y, up_1, up_2, dn_1, dn_2; then 2 x (F_1, F_2)
    T *buf = reinterpret_cast<T *>(hrow_smem) + ra.lpad;
    T *fr = buf + 16 * SL - ra.lpad;
    const int m = blockIdx.x;
    int mt[6];
#pragma unroll
    for (int i = 0; i < kRowMaxM; ++i)
        if (i == m) {
#pragma unroll
            for (int f = 0; f < 6; ++f) mt[f] = ra.mt[i][f];
        }
    const int r0 = blockIdx.y * ra.rows, r1 = min(n1, r0 + ra.rows);
    const long long boff = (long long)blockIdx.z * a.state_bytes;
    const T *in = reinterpret_cast<const T *>(a.in + boff);
    T *out = reinterpret_cast<T *>(a.out + boff) + (long long)m * g.P;
    const T *y = a.y ? reinterpret_cast<const T *>(a.y + boff) + (long long)m * g.P : nullptr;
    const T *dq = a.dq + (long long)blockIdx.z * 2 * a.dq_state + (long long)m * g.P;
    const bool vec = ra.vec != 0;
    const bool own2 = a.c2 != nullptr;   // D_2 c solved here from the centre row
    const T *src[8] = {in + (long long)m * g.P, dq, own2 ? nullptr : dq + a.dq_state, y,
                       mt[2] >= 0 ? in + (long long)mt[2] * g.P : nullptr,
                       mt[3] >= 0 ? in + (long long)mt[3] * g.P : nullptr,
                       mt[4] >= 0 ? in + (long long)mt[4] * g.P : nullptr,
                       mt[5] >= 0 ? in + (long long)mt[5] * g.P : nullptr};
    const T wup0 = mt[2] >= 0 ? g.link[0][mt[0] + 1] * g.lk[0] : T(0);
    const T wup1 = mt[3] >= 0 ? g.link[1][mt[1] + 1] * g.lk[1] : T(0);
    const T wdn0 = mt[4] >= 0 ? g.link[0][mt[0]] * g.lk[0] : T(0);
    const T wdn1 = mt[5] >= 0 ? g.link[1][mt[1]] * g.lk[1] : T(0);
    // zero pads (never written again); the rows of absent sources in both buffers
    for (int j = threadIdx.x; j < 16 * 2 * ra.lpad; j += kRowThreads) {
        const int r = j / (2 * ra.lpad), o = j - r * 2 * ra.lpad;
        buf[r * SL + (o < ra.lpad ? o - ra.lpad : L + o - ra.lpad)] = T(0);
    }
#pragma unroll
    for (int l = 3; l < 8; ++l)
        if (!src[l])
            for (int x = threadIdx.x; x < 2 * L; x += kRowThreads) {
                const int b = x >= L ? 1 : 0;
                buf[(b * 8 + l) * SL + x - b * L] = T(0);
            }
    auto issue = [&](int i) {
        const int b = i & 1;
        const long long ro = (long long)i * L;
#pragma unroll
        for (int l = 0; l < 8; ++l)
            if (src[l]) hrow_copy(buf + (b * 8 + l) * SL, src[l] + ro, L, vec);
        for (int x = threadIdx.x; x < n2; x += kRowThreads) {
            cp_async_elem(fr + b * 2 * n2 + x, g.Fh + (long long)i * n2 + x);
            cp_async_elem(fr + b * 2 * n2 + n2 + x, g.Fh + g.NQ + (long long)i * n2 + x);
        }
    };
    if (r0 < r1) issue(r0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    // q_2 lines: lane r is row r (q_2 = r) of a line; the PCR multipliers of every level, 1 / (b h)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T pk1[5], pk2[5], pbinv = T(0);
    if (own2) {
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            pk1[l] = (l < a.lv2 && lane < n2) ? a.c2[(long long)2 * l * n2 + lane] : T(0);
            pk2[l] = (l < a.lv2 && lane < n2) ? a.c2[(long long)(2 * l + 1) * n2 + lane] : T(0);
        }
        pbinv = lane < n2 ? a.c2[(long long)2 * a.lv2 * n2 + lane] : T(0);
    }
    int xs[E], q2s[E];
    T s1a[E], s0a[E], s1b0[E], s0b0[E], s1b1[E], s0b1[E], V2[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int x = 2 * (threadIdx.x + j * kRowThreads);
        const int xr = x < L ? x : L - 2;
        const int q2 = xr / KK, kk = xr - q2 * KK, k1 = kk / K2, kb = kk - k1 * K2;
        xs[j] = x;
        q2s[j] = q2;
        s1a[j] = k1 + 1 < K1 ? sqrt(T(k1 + 1)) : T(0);
        s0a[j] = sqrt(T(k1));
        s1b0[j] = sqrt(T(kb + 1));
        s0b0[j] = sqrt(T(kb));
        s1b1[j] = kb + 2 < K2 ? sqrt(T(kb + 2)) : T(0);
        s0b1[j] = sqrt(T(kb + 1));
        V2[j] = g.VLL[1] + g.VSL[1] * (g.qlo[1] + T(q2) * g.qh[1]);
    }
    const T gm = T(mt[0]) * g.gam[0] + T(mt[1]) * g.gam[1];
    const T cq1 = g.cq[0], cq2 = g.cq[1];
    for (int i = r0; i < r1; ++i) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (i + 1 < r1) issue(i + 1);   // into the buffer the previous row used
        asm volatile("cp.async.commit_group;" ::: "memory");
        const int b = i & 1;
        if (own2) {
            // D_2 c of the row: the compact derivative along q_2 of each of the K_1 K_2 lines
            // (values KK apart), a line per warp, by register shuffles (as hderiv_warp_kernel)
            const T *cr = buf + (b * 8) * SL;
            T *d2w = buf + (b * 8 + 2) * SL;
            for (int kk = warp; kk < KK; kk += kRowThreads / 32) {
                const T v = lane < n2 ? cr[lane * KK + kk] : T(0);
                T r = warp_pcr(warp_bf(v, lane, n2), pk1, pk2, a.lv2) * pbinv;
                if (a.skew2) r = T(0.5) * (r + warp_bf(warp_pcr(v, pk1, pk2, a.lv2) * pbinv, lane, n2));
                if (lane < n2) d2w[lane * KK + kk] = r;
            }
            __syncthreads();
        }
        const T *R0 = buf + (b * 8) * SL, *d1 = R0 + SL, *d2 = R0 + 2 * SL, *yr = R0 + 3 * SL;
        const T *u0 = R0 + 4 * SL, *u1 = R0 + 5 * SL, *w0 = R0 + 6 * SL, *w1 = R0 + 7 * SL;
        const T *F = fr + b * 2 * n2;
        const T V1 = g.VLL[0] + g.VSL[0] * (g.qlo[0] + T(i) * g.qh[0]);
        const T ldn0 = wdn0 * V1, lup0 = wup0 * V1;
        const long long ro = (long long)i * L;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int x = xs[j];
            if (j == E - 1 && x >= L) break;
            const T F1 = F[q2s[j]], F2 = F[n2 + q2s[j]];
            const T ldn1 = wdn1 * V2[j], lup1 = wup1 * V2[j];
            const T2 c = ld2(R0 + x), cL = ld2(R0 + x - 2), cR = ld2(R0 + x + 2);
            const T2 cU = ld2(R0 + x + K2), cD = ld2(R0 + x - K2);
            const T2 e1U = ld2(d1 + x + K2), e1D = ld2(d1 + x - K2);
            const T2 e2L = ld2(d2 + x - 2), e2C = ld2(d2 + x), e2R = ld2(d2 + x + 2);
            const T2 up0 = ld2(u0 + x - K2), dn0 = ld2(w0 + x + K2);
            const T2 up1L = ld2(u1 + x - 2), up1C = ld2(u1 + x);
            const T2 dn1C = ld2(w1 + x), dn1R = ld2(w1 + x + 2);
            T acc0 = -gm * c.x, acc1 = -gm * c.y;
            acc0 += s1a[j] * (F1 * cU.x - cq1 * e1U.x + ldn0 * dn0.x) - s0a[j] * (F1 * cD.x + cq1 * e1D.x + lup0 * up0.x);
            acc1 += s1a[j] * (F1 * cU.y - cq1 * e1U.y + ldn0 * dn0.y) - s0a[j] * (F1 * cD.y + cq1 * e1D.y + lup0 * up0.y);
            acc0 += s1b0[j] * (F2 * c.y - cq2 * e2C.y + ldn1 * dn1C.y) - s0b0[j] * (F2 * cL.y + cq2 * e2L.y + lup1 * up1L.y);
            acc1 += s1b1[j] * (F2 * cR.x - cq2 * e2R.x + ldn1 * dn1R.x) - s0b1[j] * (F2 * c.x + cq2 * e2C.x + lup1 * up1C.x);
            T2 r;
            if (y) {
                const T2 yv = ld2(yr + x);
                r.x = yv.x + a.c * acc0;
                r.y = yv.y + a.c * acc1;
            } else {
                r.x = a.c * acc0;
                r.y = a.c * acc1;
            }
            *reinterpret_cast<T2 *>(out + ro + x) = r;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// The gather stage reading the derivative arrays (compact scheme, or the three-mode stencil
// sums) in element pairs: thread t owns the values x, x + 1 (x = 2t) of every member, the same q
// point and k except k_D = kb, kb + 1 (kb even, K_D even); the neighbours along k_1..k_{D-1} are
// 2-vector loads at x -+ stride, those along k_D come from the pairs at x - 2 and x + 2 (read
// only where they lie inside the k_D row).  Equal to hstage_kernel<..., true> up to the order of
// the additions.
template <typename T, int D, int DEPTH, int NT>
__global__ void __launch_bounds__(NT) hstage_pre2_kernel(const HStageArgs<T> a) {
    typedef typename VecOf<T, 2>::type T2;
    constexpr MemberTable<D, DEPTH> tab{};
    constexpr int M = MemberTable<D, DEPTH>::M;
    const HGeo<T> &g = a.g;
    const int x = 2 * (blockIdx.x * NT + threadIdx.x);
    if (x >= g.P) return;
    const long long boff = (long long)blockIdx.y * a.state_bytes;
    const T *in = reinterpret_cast<const T *>(a.in + boff);
    T *out = reinterpret_cast<T *>(a.out + boff);
    const T *y = a.y ? reinterpret_cast<const T *>(a.y + boff) : nullptr;
    const T *dqb = a.dq + (long long)blockIdx.y * D * a.dq_state;
    int idx[2 * D];
    {
        int r = x;
#pragma unroll
        for (int ax = 2 * D - 1; ax >= 0; --ax) {
            idx[ax] = r % g.n[ax];
            r /= g.n[ax];
        }
    }
    const int qlin = x / g.Pk, KD = g.n[2 * D - 1], kb = idx[2 * D - 1];
    const bool hl = kb >= 1, hr = kb + 2 < KD;      // the k_D neighbours x - 1 and x + 2 exist
    T F[D], Vl[D], sk[D], sk1[D];
    bool hp[D], hm[D];
#pragma unroll
    for (int s = 0; s < D; ++s) {
        F[s] = __ldg(g.Fh + s * g.NQ + qlin);
        const T q = g.qlo[s] + T(idx[s]) * g.qh[s];
        Vl[s] = (g.VLL[s] + g.VSL[s] * q) * g.lk[s];
        const int k = idx[D + s];
        sk[s] = sqrt(T(k));
        sk1[s] = sqrt(T(k + 1));
        hp[s] = k + 1 < g.n[D + s];
        hm[s] = k >= 1;
    }
    const T s0 = sqrt(T(kb)), s1 = sqrt(T(kb + 1)), s2 = sqrt(T(kb + 2));   // along k_D
    auto ld = [](const T *p) { return __ldg(reinterpret_cast<const T2 *>(p)); };
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const T *c = in + (long long)m * g.P;
        T gm = T(0);
#pragma unroll
        for (int s = 0; s < D; ++s) gm += T(tab.n[m][s]) * g.gam[s];
        const T2 c0 = ld(c + x);
        T acc0 = -gm * c0.x, acc1 = -gm * c0.y;
#pragma unroll
        for (int s = 0; s < D - 1; ++s) {            // k_s, s < D - 1: both values alike
            const int e = g.st[D + s];
            const T *dq = dqb + (long long)s * a.dq_state + (long long)m * g.P;
            if (hp[s]) {
                const T2 cp = ld(c + x + e), dp = ld(dq + x + e);
                acc0 += sk1[s] * (F[s] * cp.x - g.cq[s] * dp.x);
                acc1 += sk1[s] * (F[s] * cp.y - g.cq[s] * dp.y);
                if (tab.dn[m][s] >= 0) {
                    const T2 v = ld(in + (long long)tab.dn[m][s] * g.P + x + e);
                    const T w = g.link[s][tab.n[m][s]] * Vl[s] * sk1[s];
                    acc0 += w * v.x;
                    acc1 += w * v.y;
                }
            }
            if (hm[s]) {
                const T2 cm = ld(c + x - e), dm = ld(dq + x - e);
                acc0 -= sk[s] * (F[s] * cm.x + g.cq[s] * dm.x);
                acc1 -= sk[s] * (F[s] * cm.y + g.cq[s] * dm.y);
                if (tab.up[m][s] >= 0) {
                    const T2 u = ld(in + (long long)tab.up[m][s] * g.P + x - e);
                    const T w = g.link[s][tab.n[m][s] + 1] * Vl[s] * sk[s];
                    acc0 -= w * u.x;
                    acc1 -= w * u.y;
                }
            }
        }
        {                                            // k_D: values kb (x) and kb + 1 (x + 1)
            constexpr int s = D - 1;
            const T *dq = dqb + (long long)s * a.dq_state + (long long)m * g.P;
            const T2 d0 = ld(dq + x);
            // + sqrt(k+1) (F c - cq D)(k+1): x + 1 for the first value, x + 2 for the second
            acc0 += s1 * (F[s] * c0.y - g.cq[s] * d0.y);
            // - sqrt(k) (F c + cq D)(k-1): x - 1 for the first, x for the second
            acc1 -= s1 * (F[s] * c0.x + g.cq[s] * d0.x);
            if (hr) {
                const T2 cr = ld(c + x + 2), dr = ld(dq + x + 2);
                acc1 += s2 * (F[s] * cr.x - g.cq[s] * dr.x);
            }
            if (hl) {
                const T2 cl = ld(c + x - 2), dl = ld(dq + x - 2);
                acc0 -= s0 * (F[s] * cl.y + g.cq[s] * dl.y);
            }
            if (tab.dn[m][s] >= 0) {                 // + sqrt((n+1)... ) V' sqrt(k+1) c^(n-e)_{k+1}
                const T *cd = in + (long long)tab.dn[m][s] * g.P;
                const T w = g.link[s][tab.n[m][s]] * Vl[s];
                const T2 v0 = ld(cd + x);
                acc0 += w * s1 * v0.y;
                if (hr) acc1 += w * s2 * ld(cd + x + 2).x;
            }
            if (tab.up[m][s] >= 0) {                 // - ... V' sqrt(k) c^(n+e)_{k-1}
                const T *cu = in + (long long)tab.up[m][s] * g.P;
                const T w = g.link[s][tab.n[m][s] + 1] * Vl[s];
                const T2 u0 = ld(cu + x);
                acc1 -= w * s1 * u0.x;
                if (hl) acc0 -= w * s0 * ld(cu + x - 2).y;
            }
        }
        const long long o = (long long)m * g.P + x;
        T2 r;
        if (y) {
            const T2 yv = *reinterpret_cast<const T2 *>(y + o);   // y may be out itself
            r.x = yv.x + a.c * acc0;
            r.y = yv.y + a.c * acc1;
        } else {
            r.x = a.c * acc0;
            r.y = a.c * acc1;
        }
        *reinterpret_cast<T2 *>(out + o) = r;
    }
}

template <typename T>
struct HInsertArgs {
    const char *in;
    char *out;
    long long in_state, out_state;   // batch strides in bytes (in_state may be 0: one input)
    int P, M, d, Pk;
    int n[6], st[6];
    T qlo[3], qh[3];
    T lin[3];
    T quad[3][3];                    // symmetric part
    T lk[3];                         // 1 / sqrt(m_s kT)
};

// X^x on every member: out_k = -sum_s dX/dq_s sqrt(k_s) / sqrt(m_s kT) in_{k-e_s}
template <typename T>
__global__ void __launch_bounds__(256) hinsert_kernel(const HInsertArgs<T> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.P) return;
    const T *in = reinterpret_cast<const T *>(a.in + (long long)blockIdx.y * a.in_state);
    T *out = reinterpret_cast<T *>(a.out + (long long)blockIdx.y * a.out_state);
    const int d = a.d;
    int idx[6];
    int r = x;
    for (int ax = 2 * d - 1; ax >= 0; --ax) {
        idx[ax] = r % a.n[ax];
        r /= a.n[ax];
    }
    T G[3];
    for (int s = 0; s < d; ++s) {
        T gs = a.lin[s];
        for (int b = 0; b < d; ++b) gs += a.quad[s][b] * (a.qlo[b] + T(idx[b]) * a.qh[b]);
        G[s] = gs * a.lk[s] * sqrt(T(idx[d + s]));
    }
    for (int m = 0; m < a.M; ++m) {
        const T *c = in + (long long)m * a.P;
        T v = T(0);
        for (int s = 0; s < d; ++s)
            if (idx[d + s] >= 1) v -= G[s] * __ldg(c + x - a.st[d + s]);
        out[(long long)m * a.P + x] = v;
    }
}

// equilibrium sample: c^(0)_0(q) = cnorm exp(-U(q)/2kT) (the caller divides by the q-volume
// times sum exp(-U/kT), accumulated here in partial[]), every other k and member 0
template <int NT>
__global__ void __launch_bounds__(NT) hboltzmann_kernel(double *c0, int P, int Pk,
                                                        const double *Uq, double inv2kT,
                                                        double cnorm, double *partial, int nblk) {
    double sum = 0.0;
    for (int x = blockIdx.x * NT + threadIdx.x; x < P; x += nblk * NT) {
        const int qlin = x / Pk;
        const bool k0 = (x - qlin * Pk) == 0;
        const double e = exp(-Uq[qlin] * inv2kT);
        c0[x] = k0 ? cnorm * e : 0.0;
        if (k0) sum += e * e;
    }
    sum = block_sum<NT>(sum);
    if (threadIdx.x == 0) partial[blockIdx.x] = sum;
}

// One RK4 stage of `batch` Hermite-representation states of a D-mode hierarchy of the given
// depth; false for a combination that is not compiled.  Specialised in hermite.cu.
template <typename T>
bool launch_hstage(int d, int depth, const HStageArgs<T> &a, int batch, cudaStream_t s);
template <>
bool launch_hstage<float>(int d, int depth, const HStageArgs<float> &a, int batch, cudaStream_t s);
template <>
bool launch_hstage<double>(int d, int depth, const HStageArgs<double> &a, int batch, cudaStream_t s);

// whether the stage of `batch` states with these arguments (a.c2 set) runs the row kernel that
// solves the compact q_2 lines itself, so that the caller leaves out the q_2 PCR pass
template <typename T>
bool hstage_solves_q2(int d, int depth, const HStageArgs<T> &a);
template <>
bool hstage_solves_q2<float>(int d, int depth, const HStageArgs<float> &a);
template <>
bool hstage_solves_q2<double>(int d, int depth, const HStageArgs<double> &a);

// opts the row-marching stage kernels (hstage_row_kernel) into the shared memory they may use;
// once per element type, before any launch or stream capture that uses them
template <typename T>
cudaError_t configure_hstage();
template <>
cudaError_t configure_hstage<float>();
template <>
cudaError_t configure_hstage<double>();

// explicit q-stencil sums of `batch` states (`state` values each) along every q axis into the
// derivative arrays out[b][s][state] (hstencil_sums_kernel), for d = 3
template <typename T>
void launch_hstencil_sums(int d, const HGeo<T> &g, const char *in, long long in_state, T *out,
                          long long state, int members, int batch, cudaStream_t s);
template <>
void launch_hstencil_sums<float>(int d, const HGeo<float> &g, const char *in, long long in_state, float *out,
                                 long long state, int members, int batch, cudaStream_t s);
template <>
void launch_hstencil_sums<double>(int d, const HGeo<double> &g, const char *in, long long in_state, double *out,
                                  long long state, int members, int batch, cudaStream_t s);

// compact derivative along one q axis of `batch` states (hderiv_pcr_kernel); configure_hderiv
// opts the kernels into the shared memory lines of n points need (once, before any launch or
// stream capture that uses them)
template <typename T>
cudaError_t configure_hderiv(int n);
template <>
cudaError_t configure_hderiv<float>(int n);
template <>
cudaError_t configure_hderiv<double>(int n);
template <typename T>
void launch_hderiv(const HDerivArgs<T> &a, int batch, cudaStream_t s);
template <>
void launch_hderiv<float>(const HDerivArgs<float> &a, int batch, cudaStream_t s);
template <>
void launch_hderiv<double>(const HDerivArgs<double> &a, int batch, cudaStream_t s);

}  // namespace chfpe
