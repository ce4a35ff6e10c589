// hermite.cu -- launchers of the Hermite-representation stage kernel (hermite.cuh) for every
// compiled (modes, depth), FP32 and FP64, in a translation unit of their own.
#include "hermite.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>

namespace chfpe {

namespace {
constexpr int kHNT = 128;

// row-marching kernel (two modes, explicit stencils): shared memory per block (rows long enough
// that fewer than two blocks fit on an SM run the gather kernel: measured faster there), grid size
constexpr size_t kRowSmemMax = 112 * 1024;
// q_1 chunks per (state, member) fixed by CHFPE_HROW_CHUNKS (a tuning knob like
// CHFPE_STAGE_VARIANT; 0 or unset: from the grid size below)
int row_chunks_forced() {
    static int c = -1;
    if (c < 0) {
        const char *e = std::getenv("CHFPE_HROW_CHUNKS");
        c = e ? std::max(0, std::atoi(e)) : 0;
    }
    return c;
}

// blocks wanted per launch: 8 per SM (about three waves at the kernels' 3 blocks per SM)
int row_target_blocks() {
    static int target = 0;
    if (target == 0) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
        target = 8 * sms;
    }
    return target;
}

template <typename T>
int row_pad(int KK) {
    constexpr int W = 16 / sizeof(T);
    return (3 * KK + W - 1) / W * W;
}

template <typename T>
int row_lpad(int K2) {
    constexpr int W = 16 / sizeof(T);
    return (std::max(K2, 2) + W - 1) / W * W;
}

// shared memory of the scalar (pair = false) and the pair kernel
template <typename T>
size_t row_smem(long long L, int KK, int K2, int n2, bool pair) {
    const long long link = pair ? L + 2 * row_lpad<T>(K2) : L;
    return ((size_t)9 * (size_t)(L + 2 * row_pad<T>(KK)) + (size_t)5 * link + (size_t)14 * n2) * sizeof(T);
}

template <typename T>
bool &row_configured() {
    static bool c = false;
    return c;
}

template <typename K>
cudaError_t configure_kernel(K *k) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmemMax);
    // as much of the unified L1 as shared memory as the blocks need: several blocks per SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

template <typename T, int E>
cudaError_t configure_row_one() {
    cudaError_t e = configure_kernel(hstage_row_kernel<T, E>);
    if (e == cudaSuccess) e = configure_kernel(hstage_row2_kernel<T, E>);
    if (e == cudaSuccess) e = configure_kernel(hstage_rowpre_kernel<T, E>);
    return e;
}

// shared memory of the compact-derivative row kernel: 2 x 8 padded rows, 2 x (F_1, F_2)
template <typename T>
size_t rowpre_smem(long long L, int K2, int n2) {
    return ((size_t)16 * (size_t)(L + 2 * row_lpad<T>(K2)) + (size_t)4 * n2) * sizeof(T);
}

template <typename T>
cudaError_t configure_row() {
    if (row_configured<T>()) return cudaSuccess;
    (void)row_target_blocks();   // the device query before any stream capture
    cudaError_t e = configure_row_one<T, 1>();
    if (e == cudaSuccess) e = configure_row_one<T, 2>();
    if (e == cudaSuccess) e = configure_row_one<T, 3>();
    if (e == cudaSuccess) e = configure_row_one<T, 4>();
    if (e == cudaSuccess) e = configure_row_one<T, 5>();
    if (e == cudaSuccess) e = configure_row_one<T, 6>();
    if (e == cudaSuccess) e = configure_row_one<T, 7>();
    if (e == cudaSuccess) e = configure_row_one<T, 8>();
    if (e == cudaSuccess) row_configured<T>() = true;
    return e;
}

// the row kernel for two modes: element pairs or not, values (pairs) per thread, shared memory;
// false where it does not apply (the gather kernel runs)
template <typename T>
bool row_plan(const HStageArgs<T> &a, bool &pair, int &E, size_t &smem) {
    const int n2 = a.g.n[1], K2 = a.g.n[3], KK = a.g.n[2] * K2;
    const long long L = (long long)n2 * KK;
    // element pairs: even K_2, every pair 2-vector aligned
    const uintptr_t al2 = 2 * sizeof(T) - 1;
    pair = K2 % 2 == 0 && ((uintptr_t)a.in & al2) == 0 && ((uintptr_t)a.out & al2) == 0 &&
           ((uintptr_t)a.y & al2) == 0 && (a.state_bytes & (long long)al2) == 0;
    E = (int)((L + (pair ? 2 : 1) * kRowThreads - 1) / ((pair ? 2 : 1) * kRowThreads));
    // compact derivatives: the pair kernel reading the derivative arrays (aligned like the state);
    // solving the q_2 lines itself needs lines of at most 32 points
    const bool pre = a.dq != nullptr;
    if (pre && (!pair || ((uintptr_t)a.dq & al2) != 0 || (a.dq_state * (long long)sizeof(T)) % (2 * sizeof(T)) != 0))
        return false;
    if (a.c2 && (!pre || n2 > 32 || a.lv2 > 5)) return false;
    smem = pre ? rowpre_smem<T>(L, K2, n2) : row_smem<T>(L, KK, K2, n2, pair);
    return E <= 8 && smem <= kRowSmemMax && row_configured<T>();
}

template <typename T, int K>
bool launch_row(const HStageArgs<T> &a, int batch, cudaStream_t s) {
    constexpr MemberTable<2, K> tab{};
    constexpr int M = MemberTable<2, K>::M;
    static_assert(M <= kRowMaxM, "member table of the row kernel");
    const int n1 = a.g.n[0], n2 = a.g.n[1], K2 = a.g.n[3], KK = a.g.n[2] * K2;
    const long long L = (long long)n2 * KK;
    bool pair = false;
    int E = 0;
    size_t smem = 0;
    if (!row_plan(a, pair, E, smem)) return false;
    const bool pre = a.dq != nullptr;
    const int per = M * batch;
    int chunks = std::max(1, std::min(pre ? n1 : n1 / 4, (row_target_blocks() + per - 1) / per));
    if (row_chunks_forced() > 0) chunks = std::min(row_chunks_forced(), n1);
    HRowArgs<T> ra;
    memset(&ra, 0, sizeof(ra));
    ra.s = a;
    ra.rows = (n1 + chunks - 1) / chunks;
    ra.pad = row_pad<T>(KK);
    ra.lpad = row_lpad<T>(K2);
    ra.vec = ((L * (long long)sizeof(T)) % 16 == 0 && ((uintptr_t)a.in & 15) == 0 &&
              (a.state_bytes & 15) == 0 && ((long long)a.g.P * (long long)sizeof(T)) % 16 == 0 &&
              ((uintptr_t)a.y & 15) == 0 &&
              (!pre || (((uintptr_t)a.dq & 15) == 0 && (a.dq_state * (long long)sizeof(T)) % 16 == 0))) ? 1 : 0;
    for (int m = 0; m < M; ++m)
        for (int f = 0; f < 2; ++f) {
            ra.mt[m][f] = tab.n[m][f];
            ra.mt[m][2 + f] = tab.up[m][f];
            ra.mt[m][4 + f] = tab.dn[m][f];
        }
    const dim3 grid(M, (n1 + ra.rows - 1) / ra.rows, batch);
    if (pre) {
        switch (E) {
#define PCASE(E_) case E_: hstage_rowpre_kernel<T, E_><<<grid, kRowThreads, smem, s>>>(ra); break;
            PCASE(1) PCASE(2) PCASE(3) PCASE(4) PCASE(5) PCASE(6) PCASE(7) PCASE(8)
#undef PCASE
        }
        return true;
    }
    switch (E * 2 + (pair ? 1 : 0)) {
#define RCASE(E_)                                                                    \
    case 2 * E_: hstage_row_kernel<T, E_><<<grid, kRowThreads, smem, s>>>(ra); break; \
    case 2 * E_ + 1: hstage_row2_kernel<T, E_><<<grid, kRowThreads, smem, s>>>(ra); break;
        RCASE(1) RCASE(2) RCASE(3) RCASE(4) RCASE(5) RCASE(6) RCASE(7) RCASE(8)
#undef RCASE
    }
    return true;
}

template <typename T, int D, int K>
void launch_one(const HStageArgs<T> &a, int batch, cudaStream_t s) {
    if constexpr (D == 2 && K <= 5) {
        if (launch_row<T, K>(a, batch, s)) return;
    }
    const dim3 grid((a.g.P + kHNT - 1) / kHNT, batch);
    // derivative arrays in element pairs: even K_D, 2-vector aligned states and arrays
    if constexpr (D >= 2) {
        const uintptr_t al2 = 2 * sizeof(T) - 1;
        if (a.dq && a.g.n[2 * D - 1] % 2 == 0 && ((uintptr_t)a.in & al2) == 0 &&
            ((uintptr_t)a.out & al2) == 0 && ((uintptr_t)a.y & al2) == 0 && ((uintptr_t)a.dq & al2) == 0 &&
            (a.state_bytes & (long long)al2) == 0 && a.dq_state % 2 == 0) {
            const dim3 grid2((a.g.P / 2 + kHNT - 1) / kHNT, batch);
            hstage_pre2_kernel<T, D, K, kHNT><<<grid2, kHNT, 0, s>>>(a);
            return;
        }
    }
    if (a.dq)
        hstage_kernel<T, D, K, kHNT, true><<<grid, kHNT, 0, s>>>(a);
    else
        hstage_kernel<T, D, K, kHNT><<<grid, kHNT, 0, s>>>(a);
}

template <typename T>
size_t deriv_smem(int n, bool skew) { return (size_t)(skew ? 3 : 2) * n * kPcrCols * sizeof(T); }

// largest dynamic shared memory opted into so far, per element type
template <typename T>
size_t &deriv_configured() {
    static size_t c = 48 * 1024;
    return c;
}

template <typename T>
cudaError_t configure_deriv(int n) {
    const size_t smem = deriv_smem<T>(n, true);   // the larger of the two kernels' needs
    if (smem <= deriv_configured<T>()) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(hderiv_pcr_kernel<T, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hderiv_pcr_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e == cudaSuccess) deriv_configured<T>() = smem;
    return e;
}

template <typename T>
void launch_deriv(const HDerivArgs<T> &a, int batch, cudaStream_t s) {
    const dim3 grid((a.lines + kPcrCols - 1) / kPcrCols, batch), block(kPcrCols, kPcrRows);
    if (a.n <= 32 && a.levels <= 5) {   // a line per warp, shuffles
        if (a.skew)
            hderiv_warp_kernel<T, true><<<grid, block, 0, s>>>(a);
        else
            hderiv_warp_kernel<T, false><<<grid, block, 0, s>>>(a);
        return;
    }
    if (a.skew)
        hderiv_pcr_kernel<T, true><<<grid, block, deriv_smem<T>(a.n, true), s>>>(a);
    else
        hderiv_pcr_kernel<T, false><<<grid, block, deriv_smem<T>(a.n, false), s>>>(a);
}

template <typename T>
bool launch_any(int d, int depth, const HStageArgs<T> &a, int batch, cudaStream_t s) {
    switch (d * 16 + depth) {
#define HCASE(D_, K_) case (D_ * 16 + K_): launch_one<T, D_, K_>(a, batch, s); return true;
        HCASE(1, 0) HCASE(1, 1) HCASE(1, 2) HCASE(1, 3) HCASE(1, 4) HCASE(1, 5) HCASE(1, 6)
        HCASE(1, 7) HCASE(1, 8)
        HCASE(2, 0) HCASE(2, 1) HCASE(2, 2) HCASE(2, 3) HCASE(2, 4) HCASE(2, 5)
        HCASE(3, 0) HCASE(3, 1) HCASE(3, 2) HCASE(3, 3)
#undef HCASE
    default: return false;
    }
}
}  // namespace

template <>
bool launch_hstage<float>(int d, int depth, const HStageArgs<float> &a, int batch, cudaStream_t s) {
    return launch_any<float>(d, depth, a, batch, s);
}

template <>
bool launch_hstage<double>(int d, int depth, const HStageArgs<double> &a, int batch, cudaStream_t s) {
    return launch_any<double>(d, depth, a, batch, s);
}

namespace {
template <typename T, int V>
void stencil_sums_v(int d, const HGeo<T> &g, const char *in, long long in_state, T *out, long long state,
                    long long total, int batch, cudaStream_t s) {
    const dim3 grid((unsigned)((total / V + 255) / 256), batch);
    if (d == 3) hstencil_sums_kernel<T, 3, V><<<grid, 256, 0, s>>>(g, in, in_state, out, state, total);
    else if (d == 2) hstencil_sums_kernel<T, 2, V><<<grid, 256, 0, s>>>(g, in, in_state, out, state, total);
    else hstencil_sums_kernel<T, 1, V><<<grid, 256, 0, s>>>(g, in, in_state, out, state, total);
}

template <typename T>
void stencil_sums(int d, const HGeo<T> &g, const char *in, long long in_state, T *out, long long state,
                  int members, int batch, cudaStream_t s) {
    const long long total = (long long)members * g.P;
    constexpr int V = 16 / sizeof(T);
    // vectors: a q point's values (P / NQ of them) a multiple of V, 16-byte aligned states and arrays
    const bool vec = (g.P / g.NQ) % V == 0 && ((uintptr_t)in & 15) == 0 && (in_state & 15) == 0 &&
                     ((uintptr_t)out & 15) == 0 && (state * (long long)sizeof(T)) % 16 == 0;
    if (vec)
        stencil_sums_v<T, V>(d, g, in, in_state, out, state, total, batch, s);
    else
        stencil_sums_v<T, 1>(d, g, in, in_state, out, state, total, batch, s);
}
}  // namespace

template <>
void launch_hstencil_sums<float>(int d, const HGeo<float> &g, const char *in, long long in_state, float *out,
                                 long long state, int members, int batch, cudaStream_t s) {
    stencil_sums<float>(d, g, in, in_state, out, state, members, batch, s);
}

template <>
void launch_hstencil_sums<double>(int d, const HGeo<double> &g, const char *in, long long in_state, double *out,
                                  long long state, int members, int batch, cudaStream_t s) {
    stencil_sums<double>(d, g, in, in_state, out, state, members, batch, s);
}

template <typename T>
bool solves_q2(int d, int depth, const HStageArgs<T> &a) {
    bool pair = false;
    int E = 0;
    size_t smem = 0;
    return d == 2 && depth <= 5 && a.dq && a.c2 && row_plan(a, pair, E, smem);
}

template <>
bool hstage_solves_q2<float>(int d, int depth, const HStageArgs<float> &a) { return solves_q2(d, depth, a); }

template <>
bool hstage_solves_q2<double>(int d, int depth, const HStageArgs<double> &a) { return solves_q2(d, depth, a); }

template <>
cudaError_t configure_hstage<float>() { return configure_row<float>(); }

template <>
cudaError_t configure_hstage<double>() { return configure_row<double>(); }

template <>
cudaError_t configure_hderiv<float>(int n) { return configure_deriv<float>(n); }

template <>
cudaError_t configure_hderiv<double>(int n) { return configure_deriv<double>(n); }

template <>
void launch_hderiv<float>(const HDerivArgs<float> &a, int batch, cudaStream_t s) {
    launch_deriv<float>(a, batch, s);
}

template <>
void launch_hderiv<double>(const HDerivArgs<double> &a, int batch, cudaStream_t s) {
    launch_deriv<double>(a, batch, s);
}

}  // namespace chfpe
