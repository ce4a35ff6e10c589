// kernels.cuh -- CUDA kernels of the CHFPE hot path for sm_103a.
//
// All kernels work on the symmetrised members g^(n) = W^(n) exp(H/2kT) / lambda_n (Appendix A's
// exp(-H/2kT) prefactor) stored [batch][member][q_1..q_d][p_1..p_d], p_d fastest.
//
//   stage_vec_kernel, stage_batch_kernel (and persistent.cuh, bulk.cuh)
//                   out = y + c * (M in)   (or out = M in when y == nullptr), where M is the
//                   right-hand side of Eq. HEOM in symmetrised form:
//                     (M g)^(n) = sum_s [dU/dq_s D_ps g^(n) - (p_s/m_s) D_qs g^(n)]
//                               - sum_s n_s gamma_s g^(n)
//                               + sum_s sqrt((n_s+1)c_s) V_s' (D_ps - p_s/2m_skT) g^(n+e_s)
//                               + sum_s sqrt(n_s c_s)     V_s' (D_ps + p_s/2m_skT) g^(n-e_s)
//                   (Eqs. CL_liouville, Phi, Theta; c_s = zeta_s gamma_s m_s kT).  One thread
//                   owns V consecutive p_d points of one row for every member: each member's
//                   p-derivatives are formed once and pushed to the member itself and to its two
//                   neighbours per mode.
//   insert_kernel   out^(n) = sum_s dX/dq_s (D_ps - p_s/2m_skT) g^(n)      (Eq. Opticalexc)
//   observe_*       R = h^2d sum C(q) exp(-H/2kT) g^(0), FP64 accumulation, two passes
//                   (per-block partials, then a fixed-order sum: deterministic)
//   boltzmann_*     g^(0) = exp(-H/2kT) / Z, Z = h^2d sum exp(-H/kT)        (Sec. IV B start)
//   absmax_*        max |x| over a state (equilibration residual)
//
// D_x f = (45 (f+1 - f-1) - 9 (f+2 - f-2) + (f+3 - f-3)) / (60 h), zero outside the grid; the
// 1/(60 h) factors are folded into the coefficients.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cuda_bf16.h>

#include <utility>

namespace chfpe {

constexpr int kMaxD = 3;
constexpr int kMaxDepth = 8;

// ------------------------------------------------------------------------------------------
// compile-time hierarchy member tables: by tier, then lexicographically ascending
// ------------------------------------------------------------------------------------------

constexpr int member_count(int d, int depth) {
    int M = 0;
    for (int t = 0; t <= depth; ++t) {
        long c = 1;
        for (int k = 1; k < d; ++k) c = c * (t + k) / k;
        M += (int)c;
    }
    return M;
}

template <int D, int DEPTH>
struct MemberTable {
    static constexpr int M = member_count(D, DEPTH);
    int n[M][3];
    int up[M][3];   // index of n + e_s, or -1
    int dn[M][3];   // index of n - e_s, or -1
    int order[M];   // a processing order with few right-hand sides open at once (see below)
    int last[M];    // the step of that order after which member i's right-hand side is complete
    int last_st[M]; // the same in storage order: i itself or its highest up-neighbour
    constexpr MemberTable() : n{}, up{}, dn{}, order{}, last{}, last_st{} {
        int c = 0;
        for (int t = 0; t <= DEPTH; ++t) {
            if (D == 1) {
                n[c][0] = t; n[c][1] = 0; n[c][2] = 0; ++c;
            } else if (D == 2) {
                for (int a = 0; a <= t; ++a) { n[c][0] = a; n[c][1] = t - a; n[c][2] = 0; ++c; }
            } else {
                for (int a = 0; a <= t; ++a)
                    for (int b = 0; b <= t - a; ++b) {
                        n[c][0] = a; n[c][1] = b; n[c][2] = t - a - b; ++c;
                    }
            }
        }
        for (int i = 0; i < M; ++i)
            for (int s = 0; s < 3; ++s) {
                up[i][s] = -1;
                dn[i][s] = -1;
                if (s >= D) continue;
                for (int j = 0; j < M; ++j) {
                    bool isup = true, isdn = true;
                    for (int r = 0; r < 3; ++r) {
                        int want_up = n[i][r] + (r == s ? 1 : 0);
                        int want_dn = n[i][r] - (r == s ? 1 : 0);
                        if (n[j][r] != want_up) isup = false;
                        if (n[j][r] != want_dn) isdn = false;
                    }
                    if (isup) up[i][s] = j;
                    if (isdn) dn[i][s] = j;
                }
            }
        // Processing order: member m adds to the accumulators of m and of its neighbours m +- e_s,
        // so accumulator i is open from the first to the last of those members' steps.  A greedy
        // order (each step takes the member that leaves the fewest accumulators open, from the best
        // of all starting members) keeps 7 of the 15 two-mode depth-4 accumulators open at most,
        // against 10 in storage (tier) order.  The contribution relation is symmetric; nb[i] lists
        // member i and its neighbours.
        int nb[M][7] = {}, deg[M] = {};
        for (int i = 0; i < M; ++i) {
            last_st[i] = i;
            for (int s = 0; s < 3; ++s)
                if (up[i][s] > last_st[i]) last_st[i] = up[i][s];
            nb[i][deg[i]++] = i;
            for (int s = 0; s < 3; ++s) {
                if (up[i][s] >= 0) nb[i][deg[i]++] = up[i][s];
                if (dn[i][s] >= 0) nb[i][deg[i]++] = dn[i][s];
            }
        }
        int best_live = M + 1;
        for (int start = 0; start < M; ++start) {
            int ord[M] = {}, cnt[M] = {};
            bool done[M] = {};
            for (int t = 0; t < M; ++t) {
                int pick = -1, pick_delta = M + 1;
                for (int m = 0; m < M; ++m) {
                    if (done[m] || (t == 0 && m != start)) continue;
                    // change in open accumulators when m is processed next
                    int delta = 0;
                    for (int k = 0; k < deg[m]; ++k) {
                        const int i = nb[m][k];
                        const bool was = cnt[i] > 0 && cnt[i] < deg[i];
                        const bool now = cnt[i] + 1 < deg[i];
                        delta += (now ? 1 : 0) - (was ? 1 : 0);
                    }
                    if (delta < pick_delta) { pick_delta = delta; pick = m; }
                }
                done[pick] = true;
                ord[t] = pick;
                for (int k = 0; k < deg[pick]; ++k) ++cnt[nb[pick][k]];
            }
            // the most accumulators live during one step (touched, not yet stored)
            int pos[M] = {}, first[M] = {}, lastt[M] = {};
            for (int t = 0; t < M; ++t) pos[ord[t]] = t;
            for (int i = 0; i < M; ++i) {
                first[i] = M;
                lastt[i] = -1;
                for (int k = 0; k < deg[i]; ++k) {
                    const int u = pos[nb[i][k]];
                    if (u < first[i]) first[i] = u;
                    if (u > lastt[i]) lastt[i] = u;
                }
            }
            int live = 0;
            for (int t = 0; t < M; ++t) {
                int l = 0;
                for (int i = 0; i < M; ++i) l += (first[i] <= t && lastt[i] >= t) ? 1 : 0;
                if (l > live) live = l;
            }
            if (live < best_live) {
                best_live = live;
                for (int t = 0; t < M; ++t) order[t] = ord[t];
                for (int i = 0; i < M; ++i) last[i] = lastt[i];
            }
        }
    }
};

template <int D, int DEPTH>
constexpr MemberTable<D, DEPTH> kMemberTable{};

// f(std::integral_constant<int, S>()) for S = 0, 1, ...: a loop whose index is a compile-time
// constant in the body (member indices, and through them accumulator indices, stay static)
template <typename F, int... S>
__device__ __forceinline__ void static_steps(F &&f, std::integer_sequence<int, S...>) {
    (f(std::integral_constant<int, S>()), ...);
}

// ------------------------------------------------------------------------------------------
// per-instance geometry and coefficients; stage arguments
// ------------------------------------------------------------------------------------------

typedef __nv_bfloat16 bf16;

template <typename T>
struct Geo {
    int P;                // points per member
    int n[6];             // axis sizes: q_1..q_d, p_1..p_d
    int st[6];            // axis strides inside one member
    int Pp;               // points of the p-subgrid (q index = x / Pp)
    int NQ;               // points of the q-subgrid
    const T *F;           // [D][NQ]  dU/dq_s / (60 h_ps)
    T qlo[3], qh[3], plo[3], ph[3];
    T vq[3];              // 1 / (m_s 60 h_qs)
    T inv60hp[3];         // 1 / (60 h_ps)
    T kappa[3];           // 1 / (2 m_s kT)
    T VLL[3], VSL[3];
    T gam[3];
    T link[3][kMaxDepth + 2];   // sqrt(k c_s)
};

// Storage of one state: members [0, M32) as T, members [M32, M) as bf16 (deep tiers, only with
// T = float); M32 = M is the plain layout.  A batch of states is contiguous, state_bytes apart.
template <typename T>
struct StageArgs {
    const char *in;       // stencil input, batch of states
    const char *y;        // base states (same layout) or nullptr: out = c * M in
    char *out;
    long long state_bytes;
    T c;                  // stage coefficient
    Geo<T> g;
};

// ------------------------------------------------------------------------------------------
// vector loads / stores of V consecutive values, stored as T or as bf16
// ------------------------------------------------------------------------------------------

template <typename T, int V> struct VecOf;
template <> struct VecOf<float, 4> { typedef float4 type; };
template <> struct VecOf<float, 2> { typedef float2 type; };
template <> struct VecOf<float, 1> { typedef float type; };
template <> struct VecOf<double, 2> { typedef double2 type; };
template <> struct VecOf<double, 1> { typedef double type; };
template <int V> struct BfVecOf;
template <> struct BfVecOf<1> { typedef unsigned short type; };
template <> struct BfVecOf<2> { typedef unsigned int type; };
template <> struct BfVecOf<4> { typedef uint2 type; };

// NC = true reads through the non-coherent path (data read-only for the kernel's lifetime);
// NC = false reads through L2 only (ld.global.cg, coherent across SMs), for kernels that rewrite
// the state between grid barriers
template <typename T, int V, bool NC = true>
__device__ __forceinline__ void vload(const T *__restrict__ p, bool ok, T (&v)[V]) {
    typedef typename VecOf<T, V>::type VT;
    if (ok) {
        const VT u = NC ? __ldg(reinterpret_cast<const VT *>(p)) : __ldcg(reinterpret_cast<const VT *>(p));
        const T *e = reinterpret_cast<const T *>(&u);
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = e[j];
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = T(0);
    }
}

template <typename T, int V, bool NC = true>
__device__ __forceinline__ void vload(const bf16 *__restrict__ p, bool ok, T (&v)[V]) {
    typedef typename BfVecOf<V>::type VT;
    if (ok) {
        const VT u = NC ? __ldg(reinterpret_cast<const VT *>(p)) : __ldcg(reinterpret_cast<const VT *>(p));
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = (T)__bfloat162float(e[j]);
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = T(0);
    }
}

// plain (coherent) load: used for y, which the last RK4 stage overwrites in place
template <typename T, int V>
__device__ __forceinline__ void vload_rw(const T *p, T (&v)[V]) {
    typedef typename VecOf<T, V>::type VT;
    const VT u = *reinterpret_cast<const VT *>(p);
    const T *e = reinterpret_cast<const T *>(&u);
#pragma unroll
    for (int j = 0; j < V; ++j) v[j] = e[j];
}

template <typename T, int V>
__device__ __forceinline__ void vload_rw(const bf16 *p, T (&v)[V]) {
    typedef typename BfVecOf<V>::type VT;
    const VT u = *reinterpret_cast<const VT *>(p);
    const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
    for (int j = 0; j < V; ++j) v[j] = (T)__bfloat162float(e[j]);
}

template <typename T, int V>
__device__ __forceinline__ void vstore(T *p, const T (&v)[V]) {
    typedef typename VecOf<T, V>::type VT;
    VT u;
    T *e = reinterpret_cast<T *>(&u);
#pragma unroll
    for (int j = 0; j < V; ++j) e[j] = v[j];
    *reinterpret_cast<VT *>(p) = u;
}

template <typename T, int V>
__device__ __forceinline__ void vstore(bf16 *p, const T (&v)[V]) {
    typedef typename BfVecOf<V>::type VT;
    VT u;
    bf16 *e = reinterpret_cast<bf16 *>(&u);
#pragma unroll
    for (int j = 0; j < V; ++j) e[j] = __float2bfloat16_rn((float)v[j]);   // round to nearest even
    *reinterpret_cast<VT *>(p) = u;
}

// (45 (f+1 - f-1) - 9 (f+2 - f-2) + (f+3 - f-3)) along a non-fastest axis, V points at once
template <typename S, typename T, int V, bool NC = true>
__device__ __forceinline__ void vstencil(const S *__restrict__ f, int x0, int i, int N, int st,
                                         T (&out)[V]) {
    T p1[V], m1[V], p2[V], m2[V], p3[V], m3[V];
    vload<T, V, NC>(f + x0 + st, i + 1 < N, p1);
    vload<T, V, NC>(f + x0 - st, i >= 1, m1);
    vload<T, V, NC>(f + x0 + 2 * st, i + 2 < N, p2);
    vload<T, V, NC>(f + x0 - 2 * st, i >= 2, m2);
    vload<T, V, NC>(f + x0 + 3 * st, i + 3 < N, p3);
    vload<T, V, NC>(f + x0 - 3 * st, i >= 3, m3);
#pragma unroll
    for (int j = 0; j < V; ++j)
        out[j] = T(45) * (p1[j] - m1[j]) - T(9) * (p2[j] - m2[j]) + (p3[j] - m3[j]);
}

// member m of a state at `base`: T storage below M32, bf16 from M32 on
template <typename T, int M32>
__device__ __forceinline__ const T *member_t(const char *base, int m, int P) {
    return reinterpret_cast<const T *>(base) + (long long)m * P;
}
template <typename T, int M32>
__device__ __forceinline__ const bf16 *member_h(const char *base, int m, int P) {
    return reinterpret_cast<const bf16 *>(reinterpret_cast<const T *>(base) + (long long)M32 * P) +
           (long long)(m - M32) * P;
}

// one member at V points: its own Liouvillian terms k = sum_s [F_s D_ps g - v_s D_qs g] (the
// q-derivatives are consumed at once), its p-derivatives dp_s (kept for the hierarchy links) and
// its values; the p_d derivative comes from a window of (2 NS + 1) vectors
// qs != nullptr (QS = threads per block): the q-neighbour vectors come from this thread's
// shared-memory slots qs[(s * 6 + kk) * QS], kk = 0..5 <-> offsets -3, -2, -1, +1, +2, +3, which
// hold zeros for neighbours outside the grid (float, V = 4 only)
template <typename S, typename T, int D, int V, bool NC = true, int QS = 0>
__device__ __forceinline__ void member_terms(const S *__restrict__ g, const Geo<T> &a, int x0,
                                             const int (&idx)[2 * D], const T (&Fs)[D],
                                             const T (&vq)[D][V], T (&k)[V], T (&dp)[D][V],
                                             T (&v)[V], const float4 *qs = nullptr) {
    constexpr int NS = (3 + V - 1) / V;          // side vectors of the p_d window
    constexpr int WN = (2 * NS + 1) * V;
    constexpr int L = 2 * D - 1;
    const int iL = idx[L], NL = a.n[L];
    T w[WN];
#pragma unroll
    for (int b = 0; b < 2 * NS + 1; ++b) {
        const int off = (b - NS) * V;
        T tmp[V];
        vload<T, V, NC>(g + x0 + off, iL + off >= 0 && iL + off < NL, tmp);
#pragma unroll
        for (int j = 0; j < V; ++j) w[b * V + j] = tmp[j];
    }
#pragma unroll
    for (int j = 0; j < V; ++j) k[j] = T(0);
#pragma unroll
    for (int s = 0; s < D; ++s) {
        T dq[V];
        if constexpr (QS > 0) {
            static_assert(V == 4, "staged q-neighbours are float4 slots");
            float4 t[6];
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) t[kk] = qs[(s * 6 + kk) * QS];
            const float *p1 = &t[3].x, *m1 = &t[2].x, *p2 = &t[4].x, *m2 = &t[1].x, *p3 = &t[5].x,
                        *m3 = &t[0].x;
#pragma unroll
            for (int j = 0; j < V; ++j)
                dq[j] = T(45) * (p1[j] - m1[j]) - T(9) * (p2[j] - m2[j]) + (p3[j] - m3[j]);
        } else {
            vstencil<S, T, V, NC>(g, x0, idx[s], a.n[s], a.st[s], dq);
        }
        if (s < D - 1) {
            vstencil<S, T, V, NC>(g, x0, idx[D + s], a.n[D + s], a.st[D + s], dp[s]);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int c = NS * V + j;
                dp[s][j] = T(45) * (w[c + 1] - w[c - 1]) - T(9) * (w[c + 2] - w[c - 2]) +
                           (w[c + 3] - w[c - 3]);
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) k[j] += Fs[s] * dp[s][j] - vq[s][j] * dq[j];
    }
#pragma unroll
    for (int j = 0; j < V; ++j) v[j] = w[NS * V + j];
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16 bytes global -> shared, asynchronous; src_bytes = 0 writes 16 zero bytes and reads nothing
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :
                 : "r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// L1 prefetch hint for one member's stencil neighbours along the q axes (in-bounds addresses
// only; the neighbours that miss L1): issued for member m + 1 while member m is computed
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <typename S, typename T, int D>
__device__ __forceinline__ void prefetch_member(const S *g, const Geo<T> &a, int x0,
                                                const int (&idx)[2 * D]) {
#pragma unroll
    for (int ax = 0; ax < D; ++ax)
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            if (idx[ax] + k < a.n[ax]) prefetch_l1(g + x0 + k * a.st[ax]);
            if (idx[ax] >= k) prefetch_l1(g + x0 - k * a.st[ax]);
        }
}

// ------------------------------------------------------------------------------------------
// fused RHS + RK4 stage for V consecutive p_d points of one state
//
// The thread owns the V points x0 .. x0 + V - 1 of one p_d row (n_pd % V == 0, so a row never
// straddles two vectors and every vector access is aligned to V elements) for every member.
// Members are unrolled at compile time: each member's p-derivatives are formed once and pushed
// into register accumulators of the member itself and of its two neighbours per mode.  A
// neighbour along any other axis is one V-wide load for all V points; the p_d stencil reads a
// window of (2 NS + 1) vectors, NS = ceil(3 / V).
// ------------------------------------------------------------------------------------------

// QS > 0 (= threads per block; FP32, V = 4, plain storage): each thread stages the q-neighbour
// vectors of member m + 1 into its own shared-memory slots by cp.async while member m is
// computed (two slot sets, 6 D float4 each; the thread reads only what it copied itself, so
// cp.async.wait_group orders everything and no block barrier is needed)
// ES > 0 (early stores): member i's result is written as soon as the last member adding to it has
// been processed, instead of after the whole hierarchy -- fewer accumulators live at once.  ES = 1
// processes the members in storage order (10 of 15 accumulators open at most for two modes at
// depth 4); ES = 2 in MemberTable::order (7 of 15), which sums the contributions to one member in
// another order than the other shapes (equal up to rounding).
template <typename T, int D, int DEPTH, int V, int M32, bool NC = true, bool PF = false, int QS = 0,
          int ES = 0>
__device__ __forceinline__ void stage_points(const Geo<T> &a, const char *in, const char *y,
                                             char *out, T c, int x0) {
    constexpr MemberTable<D, DEPTH> tab{};
    constexpr int M = MemberTable<D, DEPTH>::M;
    static_assert(QS == 0 || (V == 4 && M32 == M), "q staging: FP32, 4 points, plain storage");
    extern __shared__ float4 qslots[];   // [2][6 D][QS]

    int idx[2 * D];
    {
        int r = x0;
#pragma unroll
        for (int ax = 2 * D - 1; ax >= 0; --ax) {
            idx[ax] = r % a.n[ax];
            r /= a.n[ax];
        }
    }
    const int qlin = x0 / a.Pp;

    // coefficients: everything but p_d is shared by the V points
    T Fs[D], vq[D][V], VpD[D], VpK[D][V];
#pragma unroll
    for (int s = 0; s < D; ++s) {
        const T q = a.qlo[s] + T(idx[s]) * a.qh[s];
        const T Vp = a.VLL[s] + a.VSL[s] * q;
        Fs[s] = __ldg(a.F + s * a.NQ + qlin);
        VpD[s] = Vp * a.inv60hp[s];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int ip = idx[D + s] + (s == D - 1 ? j : 0);
            const T p = a.plo[s] + T(ip) * a.ph[s];
            vq[s][j] = p * a.vq[s];
            VpK[s][j] = Vp * a.kappa[s] * p;
        }
    }

    T acc[M][V];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int j = 0; j < V; ++j) acc[m][j] = T(0);

    // out^(m) = y^(m) + c acc^(m)   (or c acc^(m) without a base state)
    auto store_member = [&](int m) {
        T r[V];
        if (y) {
            T yv[V];
            if (m < M32)
                vload_rw<T, V>(member_t<T, M32>(y, m, a.P) + x0, yv);
            else
                vload_rw<T, V>(member_h<T, M32>(y, m, a.P) + x0, yv);
#pragma unroll
            for (int j = 0; j < V; ++j) r[j] = yv[j] + c * acc[m][j];
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) r[j] = c * acc[m][j];
        }
        if (m < M32)
            vstore<T, V>(const_cast<T *>(member_t<T, M32>(out, m, a.P)) + x0, r);
        else
            vstore<T, V>(const_cast<bf16 *>(member_h<T, M32>(out, m, a.P)) + x0, r);
    };

    auto q_issue = [&](int mm, int buf) {   // member mm's q-neighbours into slot set buf
        const T *g = member_t<T, M32>(in, mm, a.P);
        float4 *slot = qslots + buf * 6 * D * QS + threadIdx.x;
#pragma unroll
        for (int s = 0; s < D; ++s)
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) {
                const int kq = kk < 3 ? kk - 3 : kk - 2;
                const bool ok = idx[s] + kq >= 0 && idx[s] + kq < a.n[s];
                cp_async16(slot + (s * 6 + kk) * QS, ok ? g + x0 + kq * a.st[s] : g, ok ? 16 : 0);
            }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if constexpr (QS > 0) q_issue(0, 0);

    auto member_step = [&](auto stepc) {
        constexpr int step = decltype(stepc)::value;
        constexpr int m = ES == 2 ? kMemberTable<D, DEPTH>.order[step] : step;
        if constexpr (QS > 0) {
            if (m + 1 < M) {
                q_issue(m + 1, (m + 1) & 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");   // member m's slots landed
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
        }
        if constexpr (PF) {
            if (m + 1 < M) {
                if (m + 1 < M32) prefetch_member<T, T, D>(member_t<T, M32>(in, m + 1, a.P), a, x0, idx);
                else prefetch_member<bf16, T, D>(member_h<T, M32>(in, m + 1, a.P), a, x0, idx);
            }
        }
        T k[V], dp[D][V], v[V];
        if constexpr (QS > 0)
            member_terms<T, T, D, V, NC, QS>(member_t<T, M32>(in, m, a.P), a, x0, idx, Fs, vq, k, dp,
                                             v, qslots + (m & 1) * 6 * D * QS + threadIdx.x);
        else if (m < M32)
            member_terms<T, T, D, V, NC>(member_t<T, M32>(in, m, a.P), a, x0, idx, Fs, vq, k, dp, v);
        else
            member_terms<bf16, T, D, V, NC>(member_h<T, M32>(in, m, a.P), a, x0, idx, Fs, vq, k, dp, v);
        T gm = T(0);
#pragma unroll
        for (int s = 0; s < D; ++s) gm += T(tab.n[m][s]) * a.gam[s];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            acc[m][j] += k[j] - gm * v[j];
#pragma unroll
            for (int s = 0; s < D; ++s) {
                if (tab.dn[m][s] >= 0) {
                    const T wl = a.link[s][tab.n[m][s]];
                    acc[tab.dn[m][s]][j] += wl * (VpD[s] * dp[s][j] - VpK[s][j] * v[j]);
                }
                if (tab.up[m][s] >= 0) {
                    const T wl = a.link[s][tab.n[m][s] + 1];
                    acc[tab.up[m][s]][j] += wl * (VpD[s] * dp[s][j] + VpK[s][j] * v[j]);
                }
            }
        }
        if constexpr (ES > 0) {
#pragma unroll
            for (int i = 0; i < M; ++i)
                if ((ES == 2 ? tab.last[i] : tab.last_st[i]) == step) store_member(i);
        }
    };
    static_steps(member_step, std::make_integer_sequence<int, M>());

    if constexpr (ES == 0) {
#pragma unroll
        for (int m = 0; m < M; ++m) store_member(m);
    }
}

template <typename T, int D, int DEPTH, int V, int NT, int MINB, int M32, bool PF = false,
          bool QST = false, int ES = 0>
__global__ void __launch_bounds__(NT, MINB) stage_vec_kernel(const StageArgs<T> a) {
    const int x0 = (blockIdx.x * NT + threadIdx.x) * V;
    if (x0 >= a.g.P) return;
    const long long boff = (long long)blockIdx.y * a.state_bytes;
    stage_points<T, D, DEPTH, V, M32, true, PF, QST ? NT : 0, ES>(
        a.g, a.in + boff, a.y ? a.y + boff : nullptr, a.out + boff, a.c, x0);
}

// ------------------------------------------------------------------------------------------
// the same stage over many instances of different grids in one launch: a work list of
// (instance, tile) items, one tile of NT * V points per block
// ------------------------------------------------------------------------------------------

template <typename T>
struct InstGeo {
    Geo<T> g;
    long long off;        // byte offset of the instance's state inside each batch arena
    T cst[4];             // the instance's RK4 stage coefficients dt_i/4, dt_i/3, dt_i/2, dt_i
};

template <typename T>
struct BatchStageArgs {
    const InstGeo<T> *inst;
    const int2 *work;     // (instance, tile)
    const char *in;
    const char *y;
    char *out;
    int stage;            // 0..3: coefficient cst[stage] of each instance; -1: c for all
    T c;
};

// ES = 1: each member stored as soon as its last contribution is in (storage order), as the
// single-handle launch shapes with early stores
template <typename T, int D, int DEPTH, int V, int NT, int MINB, int M32, int ES = 0>
__global__ void __launch_bounds__(NT, MINB) stage_batch_kernel(const BatchStageArgs<T> b) {
    // the block's instance geometry, copied once into shared memory: every thread reads its
    // sizes, strides and coefficients many times
    __shared__ __align__(16) InstGeo<T> sg;
    static_assert(sizeof(InstGeo<T>) % 4 == 0 && sizeof(InstGeo<T>) / 4 <= 4 * NT, "geometry copy");
    const int2 item = b.work[blockIdx.x];
    {
        const unsigned *src = reinterpret_cast<const unsigned *>(b.inst + item.x);
        unsigned *dst = reinterpret_cast<unsigned *>(&sg);
        for (int w = threadIdx.x; w < (int)(sizeof(InstGeo<T>) / 4); w += NT) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    const int x0 = (item.y * NT + threadIdx.x) * V;
    if (x0 >= sg.g.P) return;
    const long long off = sg.off;
    stage_points<T, D, DEPTH, V, M32, true, false, 0, ES>(sg.g, b.in + off, b.y ? b.y + off : nullptr,
                                                         b.out + off, b.stage >= 0 ? sg.cst[b.stage] : b.c, x0);
}

// ------------------------------------------------------------------------------------------
// optical insertion X^x, every member (Eq. Opticalexc, symmetrised)
// ------------------------------------------------------------------------------------------

template <typename T>
struct InsertArgs {
    const char *in;
    char *out;
    long long in_state, out_state;   // batch strides in bytes (in_state may be 0: one input)
    int P, M, M32, d;                // members >= M32 are stored as bf16
    int n[6], st[6];
    T qlo[3], qh[3], plo[3], ph[3];
    T lin[3];
    T quad[3][3];                    // symmetric part of the quadratic coefficients
    T inv60hp[3], kappa[3];
};

template <typename S, typename T>
__device__ __forceinline__ T ldv(const S *p) { return (T)__ldg(p); }
template <>
__device__ __forceinline__ float ldv<bf16, float>(const bf16 *p) { return __bfloat162float(__ldg(p)); }

template <typename S, typename T>
__device__ __forceinline__ T stencil7s(const S *__restrict__ f, int x, int i, int N, int st) {
    T p1 = (i + 1 < N) ? ldv<S, T>(f + x + st) : T(0);
    T m1 = (i >= 1) ? ldv<S, T>(f + x - st) : T(0);
    T p2 = (i + 2 < N) ? ldv<S, T>(f + x + 2 * st) : T(0);
    T m2 = (i >= 2) ? ldv<S, T>(f + x - 2 * st) : T(0);
    T p3 = (i + 3 < N) ? ldv<S, T>(f + x + 3 * st) : T(0);
    T m3 = (i >= 3) ? ldv<S, T>(f + x - 3 * st) : T(0);
    return T(45) * (p1 - m1) - T(9) * (p2 - m2) + (p3 - m3);
}

template <typename S, typename T>
__device__ __forceinline__ void insert_member(const InsertArgs<T> &a, const S *__restrict__ g,
                                              S *o, int x, const int *idx, const T *G,
                                              const T *Kp) {
    const T v = ldv<S, T>(g + x);
    T acc = T(0);
    for (int s = 0; s < a.d; ++s) {
        const T dp = stencil7s<S, T>(g, x, idx[a.d + s], a.n[a.d + s], a.st[a.d + s]);
        acc += G[s] * dp - Kp[s] * v;
    }
    o[x] = (S)acc;
}

template <typename T>
__global__ void __launch_bounds__(256) insert_kernel(const InsertArgs<T> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.P) return;
    const char *in = a.in + (long long)blockIdx.y * a.in_state;
    char *out = a.out + (long long)blockIdx.y * a.out_state;
    const int d = a.d;
    int idx[6];
    int r = x;
    for (int ax = 2 * d - 1; ax >= 0; --ax) {
        idx[ax] = r % a.n[ax];
        r /= a.n[ax];
    }
    T G[3], Kp[3];
    for (int s = 0; s < d; ++s) {
        T gs = a.lin[s];
        for (int b = 0; b < d; ++b) gs += a.quad[s][b] * (a.qlo[b] + T(idx[b]) * a.qh[b]);
        const T p = a.plo[s] + T(idx[d + s]) * a.ph[s];
        G[s] = gs * a.inv60hp[s];
        Kp[s] = gs * a.kappa[s] * p;
    }
    for (int m = 0; m < a.M; ++m) {
        if (m < a.M32) {
            const T *g = reinterpret_cast<const T *>(in) + (long long)m * a.P;
            T *o = reinterpret_cast<T *>(out) + (long long)m * a.P;
            insert_member<T, T>(a, g, o, x, idx, G, Kp);
        } else {
            const long long hoff = (long long)a.M32 * a.P * sizeof(T);
            const bf16 *g = reinterpret_cast<const bf16 *>(in + hoff) + (long long)(m - a.M32) * a.P;
            bf16 *o = reinterpret_cast<bf16 *>(out + hoff) + (long long)(m - a.M32) * a.P;
            const T v = __bfloat162float(__ldg(g + x));
            T acc = T(0);
            for (int s = 0; s < d; ++s) {
                const T dp = stencil7s<bf16, T>(g, x, idx[d + s], a.n[d + s], a.st[d + s]);
                acc += G[s] * dp - Kp[s] * v;
            }
            o[x] = __float2bfloat16_rn((float)acc);
        }
    }
}

// double <-> mixed storage (members [0, M32) as T, the rest as bf16), one state
template <typename T>
__global__ void to_mixed_kernel(const double *in, char *out, long long n_t, long long n_total) {
    T *o = reinterpret_cast<T *>(out);
    bf16 *oh = reinterpret_cast<bf16 *>(o + n_t);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_total;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < n_t)
            o[i] = (T)in[i];
        else
            oh[i - n_t] = __double2bfloat16(in[i]);
    }
}

template <typename T>
__global__ void from_mixed_kernel(const char *in, double *out, long long n_t, long long n_total) {
    const T *g = reinterpret_cast<const T *>(in);
    const bf16 *gh = reinterpret_cast<const bf16 *>(g + n_t);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_total;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (i < n_t) ? (double)g[i] : (double)__bfloat162float(gh[i - n_t]);
}

// ------------------------------------------------------------------------------------------
// reductions (FP64)
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_down_sync(0xffffffffu, v, o);
        v = (u > v || u != u) ? u : v;      // NaN propagates
    }
    return v;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[NT / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

template <int NT>
__device__ __forceinline__ double block_max(double v) {
    __shared__ double sh[NT / 32];
    v = warp_max(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_max(v);
    return v;
}

struct ObserveArgs {
    const void *in;          // batch of states, member 0 (stored as T) is read
    long long state_bytes;
    int P, Pp, d;
    int np[3];               // p-axis sizes
    const double *CWq;       // [NQ]: C(q) exp(-U(q)/2kT)
    const double *wp;        // [3][maxnp]: exp(-p^2 / 4 m_s kT)
    int wp_ld;
    double *partial;         // [batch][nblk]
    int nblk;
};

// block b of state j sums points b, b + nblk*NT, ... (grid-stride) into partial[j][b]
template <typename T, int NT>
__global__ void __launch_bounds__(NT) observe_partial_kernel(const ObserveArgs a) {
    const T *__restrict__ g =
        reinterpret_cast<const T *>((const char *)a.in + (long long)blockIdx.y * a.state_bytes);
    double sum = 0.0;
    for (int x = blockIdx.x * NT + threadIdx.x; x < a.P; x += a.nblk * NT) {
        const int qlin = x / a.Pp;
        int r = x - qlin * a.Pp;
        double w = a.CWq[qlin];
        for (int s = a.d - 1; s >= 0; --s) {
            const int ip = r % a.np[s];
            r /= a.np[s];
            w *= a.wp[s * a.wp_ld + ip];
        }
        sum += w * (double)g[x];
    }
    sum = block_sum<NT>(sum);
    if (threadIdx.x == 0) a.partial[(long long)blockIdx.y * a.nblk + blockIdx.x] = sum;
}

// out[j * out_stride] = scale * sum_b partial[j][b], fixed order; one warp per state
static __global__ void observe_finish_kernel(const double *partial, int nblk, int batch, double scale,
                                      double *out, long long out_stride) {
    const int j = blockIdx.x;
    if (j >= batch) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(long long)j * nblk + b];
    s = warp_sum(s);
    if (threadIdx.x == 0) out[(long long)j * out_stride] = scale * s;
}

// the same, written to out[j * out_stride + *counter]: the output slot comes from a device
// counter so that a captured graph of one sampling interval can be replayed unchanged
static __global__ void observe_finish_counter_kernel(const double *partial, int nblk, int batch,
                                                     double scale, double *out,
                                                     long long out_stride, const int *counter) {
    const int j = blockIdx.x;
    if (j >= batch) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(long long)j * nblk + b];
    s = warp_sum(s);
    if (threadIdx.x == 0) out[(long long)j * out_stride + *counter] = scale * s;
}

static __global__ void counter_add_kernel(int *counter, int inc) { *counter += inc; }

// Boltzmann: g0[x] = exp(-(U(q) + sum p^2/2m) / 2kT); partial sums of g0^2
template <int NT>
__global__ void __launch_bounds__(NT) boltzmann_kernel(double *g0, int P, int Pp, int d,
                                                       const double *Uq, const int *np,
                                                       const double *plo, const double *ph,
                                                       const double *inv2m, double inv2kT,
                                                       double *partial, int nblk) {
    double sum = 0.0;
    for (int x = blockIdx.x * NT + threadIdx.x; x < P; x += nblk * NT) {
        const int qlin = x / Pp;
        int r = x - qlin * Pp;
        double E = Uq[qlin];
        for (int s = d - 1; s >= 0; --s) {
            const int ip = r % np[s];
            r /= np[s];
            const double p = plo[s] + ip * ph[s];
            E += p * p * inv2m[s];
        }
        const double v = exp(-E * inv2kT);
        g0[x] = v;
        sum += v * v;
    }
    sum = block_sum<NT>(sum);
    if (threadIdx.x == 0) partial[blockIdx.x] = sum;
}

static __global__ void scale_by_sum_kernel(double *g, long long n, const double *partial, int nblk,
                                    double vol) {
    // g *= 1 / (vol * sum partial), the sum taken in fixed order by every thread
    double Z = 0.0;
    for (int b = 0; b < nblk; ++b) Z += partial[b];
    const double s = 1.0 / (vol * Z);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        g[i] *= s;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) absmax_partial_kernel(const T *x, long long n,
                                                            double *partial) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n;
         i += (long long)gridDim.x * NT) {
        const double v = fabs((double)x[i]);
        m = (v > m || v != v) ? v : m;      // NaN propagates
    }
    m = block_max<NT>(m);
    if (threadIdx.x == 0) partial[blockIdx.x] = m;
}

template <typename S, typename D_>
__global__ void convert_kernel(const S *in, D_ *out, long long n) {   // plain element conversion
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (D_)in[i];
}

}  // namespace chfpe
