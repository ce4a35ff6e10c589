// stage_d3.cu -- the RK4 stage launchers of 3-mode hierarchies (all compiled depths, FP32 and
// FP64), in a translation unit of their own so that the library's objects compile in parallel.
#include "stage_launch.cuh"

namespace chfpe {

namespace {
template <typename T>
bool launch_depth(int depth, const StageArgs<T> &a, int batch, bool vec, int M32, int variant,
                  int *err, cudaStream_t s) {
    switch (depth) {
    case 0: return launch_stage_t<T, 3, 0>(a, batch, vec, M32, variant, err, s);
    case 1: return launch_stage_t<T, 3, 1>(a, batch, vec, M32, variant, err, s);
    case 2: return launch_stage_t<T, 3, 2>(a, batch, vec, M32, variant, err, s);
    case 3: return launch_stage_t<T, 3, 3>(a, batch, vec, M32, variant, err, s);
    default: return false;
    }
}
}  // namespace

template <>
bool launch_stage_dim<float, 3>(int depth, const StageArgs<float> &a, int batch, bool vec, int M32,
                                 int variant, int *err, cudaStream_t s) {
    return launch_depth<float>(depth, a, batch, vec, M32, variant, err, s);
}

template <>
bool launch_stage_dim<double, 3>(int depth, const StageArgs<double> &a, int batch, bool vec, int M32,
                                  int variant, int *err, cudaStream_t s) {
    return launch_depth<double>(depth, a, batch, vec, M32, variant, err, s);
}

}  // namespace chfpe
