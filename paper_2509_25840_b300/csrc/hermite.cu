// hermite.cu -- launchers of the Hermite-representation stage kernel (hermite.cuh) for every
// compiled (modes, depth), FP32 and FP64, in a translation unit of their own.
#include "hermite.cuh"

namespace chfpe {

namespace {
constexpr int kHNT = 128;

template <typename T, int D, int K>
void launch_one(const HStageArgs<T> &a, int batch, cudaStream_t s) {
    const dim3 grid((a.g.P + kHNT - 1) / kHNT, batch);
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
