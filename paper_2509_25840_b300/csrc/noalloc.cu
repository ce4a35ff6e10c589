// noalloc.cu -- chfpe_observe_noalloc: the observable reduction R = integral C(q) exp(-H/2kT) g^(0)
// for callers that must not allocate device memory.
//
// Who needs it: programs that own every byte of device memory themselves (a process that carves
// a fixed budget out of the GPU at start-up and forbids later allocations, or a host framework
// that hands this library only pre-sized buffers), and latency-critical loops where a
// cudaMalloc -- which can synchronise the device and take milliseconds -- is not acceptable.
// Such callers cannot create a chfpe_handle (it allocates its arenas), so this entry point
// takes the model, grid and optical operator directly and keeps its reduction scratch in a
// file-scope device array instead of an allocation.
//
// The scratch: g_observe_scratch holds one FP64 partial sum per (state, block).  It is a static
// device array of kNoAllocPartials doubles (256 KB) that every GPU loading the library keeps until
// the process exits.  Host code cannot use the array's name as a device address; the address is
// obtained once per device with cudaGetSymbolAddress (on that device's first call, which should
// therefore happen before any stream capture) and passed to the kernels.  Every partial slot a call
// uses is written by that call before it is read, so nothing needs clearing; but all calls share
// the one array, so two calls that overlap on the GPU (e.g. issued on different streams) race.
#include "../../include/chfpe.h"
#include "kernels.cuh"

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

namespace chfpe {
void set_last_error(const std::string &msg);   // chfpe.cu
}

namespace {

constexpr int kNoAllocPartials = 32768;                 // doubles: 256 KB
constexpr int kNoAllocThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_observe_scratch[kNoAllocPartials];

std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

struct NoAllocArgs {
    const void *in;
    long long state;           // values per state (M * P)
    int P, Pp, d;
    int nq[3], np[3];
    double qlo[3], qh[3], plo[3], ph[3];
    double m[3], w2[3], g3[3], g4[3], g2[3][3], gs2s[3][3], gss2[3][3];
    double lin[3], quad[3][3];
    double inv2kT;
    double *partial;           // device address of g_observe_scratch
    int nblk;
};

__device__ double na_weight(const NoAllocArgs &a, int x) {
    // C(q) exp(-U(q)/2kT) prod_s exp(-p_s^2 / (4 m_s kT)), q and p from the grid index of x
    const int qlin = x / a.Pp;
    int r = x - qlin * a.Pp;
    double w = 1.0;
    for (int s = a.d - 1; s >= 0; --s) {
        const int ip = r % a.np[s];
        r /= a.np[s];
        const double p = a.plo[s] + ip * a.ph[s];
        w *= exp(-p * p * (0.5 / a.m[s]) * a.inv2kT);
    }
    double q[3] = {0.0, 0.0, 0.0};
    int rq = qlin;
    for (int s = a.d - 1; s >= 0; --s) {
        q[s] = a.qlo[s] + (rq % a.nq[s]) * a.qh[s];
        rq /= a.nq[s];
    }
    double U = 0.0, C = 0.0;
    for (int s = 0; s < a.d; ++s) {
        const double v = q[s];
        U += 0.5 * a.m[s] * a.w2[s] * v * v + a.g3[s] * v * v * v * (1.0 / 6.0) +
             a.g4[s] * v * v * v * v * (1.0 / 24.0);
        C += a.lin[s] * v;
    }
    for (int i = 0; i < a.d; ++i)
        for (int j = 0; j < a.d; ++j) {
            C += 0.5 * a.quad[i][j] * q[i] * q[j];
            if (j > i)
                U += a.g2[i][j] * q[i] * q[j] +
                     (a.gs2s[i][j] * q[i] * q[i] * q[j] + a.gss2[i][j] * q[i] * q[j] * q[j]) *
                         (1.0 / 6.0);
        }
    return C * exp(-U * a.inv2kT) * w;
}

template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_partial_kernel(const NoAllocArgs a) {
    const T *g = (const T *)a.in + (long long)blockIdx.y * a.state;
    double sum = 0.0;
    for (int x = blockIdx.x * kNoAllocThreads + threadIdx.x; x < a.P; x += a.nblk * kNoAllocThreads)
        sum += na_weight(a, x) * (double)g[x];
    sum = chfpe::block_sum<kNoAllocThreads>(sum);
    if (threadIdx.x == 0) a.partial[(long long)blockIdx.y * a.nblk + blockIdx.x] = sum;
}

chfpe_status na_fail(chfpe_status s, const std::string &m) {
    chfpe::set_last_error(m);      // read back with chfpe_last_error()
    return s;
}

// device address of g_observe_scratch on the current device (looked up once per device)
chfpe_status scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(CHFPE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(CHFPE_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_observe_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(CHFPE_ECUDA, std::string("cudaGetSymbolAddress(g_observe_scratch): ") +
                                            cudaGetErrorString(e));
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return CHFPE_OK;
}

}  // namespace

extern "C" chfpe_status chfpe_observe_noalloc(const chfpe_model *model, const chfpe_grid *grid,
                                              int depth, int precision,
                                              const chfpe_optical *C, const void *states,
                                              int batch, double *R_dev, void *stream) {
    if (!model || !grid || !C || !states || !R_dev) return na_fail(CHFPE_EINVAL, "null argument");
    const int d = model->nmodes;
    if (d < 1 || d > 3) return na_fail(CHFPE_EINVAL, "nmodes must be 1, 2 or 3");
    if (precision != 32 && precision != 64) return na_fail(CHFPE_EINVAL, "precision must be 32 or 64");
    if (depth < 0 || depth > chfpe::kMaxDepth) return na_fail(CHFPE_EINVAL, "depth out of range");
    if (batch < 1 || batch > 65535) return na_fail(CHFPE_EINVAL, "batch must be in 1..65535");
    if (!(model->kT > 0)) return na_fail(CHFPE_EINVAL, "kT must be positive");
    NoAllocArgs a = {};
    a.in = states;
    a.d = d;
    long long P = 1, Pp = 1;
    double vol = 1.0;
    for (int s = 0; s < d; ++s) {
        if (grid->nq[s] < 2 || grid->np[s] < 2) return na_fail(CHFPE_EINVAL, "at least 2 points per axis");
        if (!(model->m[s] > 0)) return na_fail(CHFPE_EINVAL, "masses must be positive");
        a.nq[s] = grid->nq[s];
        a.np[s] = grid->np[s];
        a.qlo[s] = grid->qmin[s];
        a.qh[s] = (grid->qmax[s] - grid->qmin[s]) / (grid->nq[s] - 1);
        a.plo[s] = grid->pmin[s];
        a.ph[s] = (grid->pmax[s] - grid->pmin[s]) / (grid->np[s] - 1);
        vol *= a.qh[s] * a.ph[s];
        P *= (long long)grid->nq[s] * grid->np[s];
        Pp *= grid->np[s];
        a.m[s] = model->m[s];
        a.w2[s] = model->omega[s] * model->omega[s];
        a.g3[s] = model->g3[s];
        a.g4[s] = model->g4[s];
        a.lin[s] = C->lin[s];
        for (int b = 0; b < 3; ++b) {
            a.g2[s][b] = model->g2[s][b];
            a.gs2s[s][b] = model->g_s2s[s][b];
            a.gss2[s][b] = model->g_ss2[s][b];
            a.quad[s][b] = C->quad[s][b];
        }
    }
    const long long M = chfpe::member_count(d, depth);
    if (P * M >= (1LL << 31)) return na_fail(CHFPE_EINVAL, "state too large");
    a.P = (int)P;
    a.Pp = (int)Pp;
    a.state = M * P;
    a.inv2kT = 0.5 / model->kT;
    int nblk = (int)((P + 1023) / 1024);
    if (nblk > 512) nblk = 512;
    if (nblk < 1) nblk = 1;
    if ((long long)nblk * batch > kNoAllocPartials) {
        return na_fail(CHFPE_EINVAL,
                       "batch too large for the fixed reduction scratch: needs " +
                           std::to_string((long long)nblk * batch) + " partial sums, the maximum is " +
                           std::to_string(kNoAllocPartials) + " (batch <= " +
                           std::to_string(kNoAllocPartials / nblk) + " for this grid)");
    }
    a.nblk = nblk;
    chfpe_status st = scratch_address(&a.partial);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 gridDim(nblk, batch);
    if (precision == 64)
        noalloc_partial_kernel<double><<<gridDim, kNoAllocThreads, 0, s>>>(a);
    else
        noalloc_partial_kernel<float><<<gridDim, kNoAllocThreads, 0, s>>>(a);
    chfpe::observe_finish_kernel<<<batch, 32, 0, s>>>(a.partial, nblk, batch, vol, R_dev, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(CHFPE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return CHFPE_OK;
}
