// spectra.cu -- spectra from sampled response functions (Sec. II C):
//   I(w1)          = w1 Im sum_k c_k e^{+i w1 t_k} R1(t_k)                           Eq. 1DIR_Raman
//   I(w1, w2)      = Im sum_{a,b} c_a c_b e^{-i w1 t_a - i w2 t_b} R2(t_b, t_a)      Eq. 2DThz_Raman
//   I(w3, t2, w1)  = Im sum_{a,c} c_a c_c e^{-i w1 t_a + i w3 t_c} R3(t_c, t2, t_a)  Eq. noncorrelation
// with trapezoid weights c_k = dtau (1/2 at both ends) times exp(-eta t_k), t_k = k dtau, on the
// centred frequency grid w_j = 2 pi (j - L/2) / (L dtau), j = 0..L-1.
//
// Each transform is a direct DFT in FP64, one thread per output frequency of one row; the phase
// w_j t_k = 2 pi ((j - L/2) k mod L) / L is reduced in integers before sincospi, so its error does
// not grow with k.  2D transforms are two separable passes (the inner time axis first, into a
// complex intermediate, then the outer axis).  The sizes are a few thousand samples at most, so
// the whole transform takes microseconds.
#include "../../include/chfpe.h"

#include <cuda_runtime.h>

#include <string>

namespace chfpe {
void set_last_error(const std::string &msg);   // chfpe.cu
}

namespace {

chfpe_status sfail(chfpe_status s, const std::string &m) {
    chfpe::set_last_error(m);
    return s;
}

struct Pass {
    const void *in;          // double (real input) or double2 (complex input)
    long long in_row, in_k;  // element strides: row r, sample k
    void *out;               // double2 (complex), or double (imaginary part, or w times it)
    long long out_row, out_j;
    int rows, N, L;
    double dtau, eta;
    int sign;                // +1 or -1: exp(sign i w t)
};

// OUT: 0 complex, 1 Im, 2 w Im
template <bool CIN, int OUT>
__global__ void dft_pass_kernel(const Pass p) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)p.rows * p.L) return;
    const int r = (int)(id / p.L), j = (int)(id - (long long)r * p.L);
    const long long f = j - p.L / 2;                 // frequency index, centred
    double re = 0.0, im = 0.0;
    for (int k = 0; k < p.N; ++k) {
        double c = p.dtau * ((k == 0 || k == p.N - 1) ? 0.5 : 1.0);
        if (p.eta != 0.0) c *= exp(-p.eta * p.dtau * k);
        long long m = (f * k) % p.L;
        if (m < 0) m += p.L;
        double s, co;
        sincospi(2.0 * (double)m / (double)p.L, &s, &co);
        s *= p.sign;
        double xr, xi;
        if (CIN) {
            const double2 x = reinterpret_cast<const double2 *>(p.in)[r * p.in_row + k * p.in_k];
            xr = x.x;
            xi = x.y;
        } else {
            xr = reinterpret_cast<const double *>(p.in)[r * p.in_row + k * p.in_k];
            xi = 0.0;
        }
        re += c * (co * xr - s * xi);
        im += c * (co * xi + s * xr);
    }
    const long long o = r * p.out_row + j * p.out_j;
    if (OUT == 0) {
        reinterpret_cast<double2 *>(p.out)[o] = make_double2(re, im);
    } else if (OUT == 1) {
        reinterpret_cast<double *>(p.out)[o] = im;
    } else {
        const double w = 2.0 * 3.14159265358979323846 * (double)f / ((double)p.L * p.dtau);
        reinterpret_cast<double *>(p.out)[o] = w * im;
    }
}

template <bool CIN, int OUT>
cudaError_t run_pass(const Pass &p, cudaStream_t s) {
    const long long n = (long long)p.rows * p.L;
    dft_pass_kernel<CIN, OUT><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(p);
    return cudaGetLastError();
}

chfpe_status check(int n1, int n2, double dtau, int L1, int L2, double eta) {
    if (n1 < 2 || n2 < 2) return sfail(CHFPE_EINVAL, "spectra need at least 2 samples per axis");
    if (L1 < n1 || L2 < n2) return sfail(CHFPE_EINVAL, "transform length below the sample count");
    if (L1 > (1 << 22) || L2 > (1 << 22)) return sfail(CHFPE_EINVAL, "transform length above 2^22");
    if (!(dtau > 0.0) || !(eta >= 0.0)) return sfail(CHFPE_EINVAL, "dtau > 0 and eta >= 0");
    return CHFPE_OK;
}

// 2D spectrum: R[n1][n2] (outer axis 1, inner axis 2) -> I[L1][L2] with the given signs
chfpe_status spectrum2d(const double *R, int n1, int n2, double dtau, int L1, int L2, double eta,
                        int sign1, int sign2, double *I, void *stream) {
    if (!R || !I) return sfail(CHFPE_EINVAL, "null argument");
    chfpe_status st = check(n1, n2, dtau, L1, L2, eta);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *dR = nullptr, *dI = nullptr;
    double2 *dX = nullptr;
    cudaError_t e = cudaMalloc(&dR, sizeof(double) * n1 * n2);
    if (e == cudaSuccess) e = cudaMalloc(&dX, sizeof(double2) * (size_t)n1 * L2);
    if (e == cudaSuccess) e = cudaMalloc(&dI, sizeof(double) * (size_t)L1 * L2);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dR, R, sizeof(double) * n1 * n2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {   // inner axis: X[a][b] = sum_k c_k e^{sign2 i w_b t_k} R[a][k]
        Pass p{dR, n2, 1, dX, L2, 1, n1, n2, L2, dtau, eta, sign2};
        e = run_pass<false, 0>(p, s);
    }
    if (e == cudaSuccess) {   // outer axis: I[j][b] = Im sum_a c_a e^{sign1 i w_j t_a} X[a][b]
        Pass p{dX, 1, L2, dI, 1, L2, L2, n1, L1, dtau, eta, sign1};
        e = run_pass<true, 1>(p, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(I, dI, sizeof(double) * (size_t)L1 * L2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dR);
    cudaFree(dX);
    cudaFree(dI);
    if (e != cudaSuccess) return sfail(CHFPE_ECUDA, std::string("spectrum: ") + cudaGetErrorString(e));
    return CHFPE_OK;
}

}  // namespace

extern "C" chfpe_status chfpe_spectrum1(const double *R1, int nt, double dtau, int L, double eta,
                                        double *I, void *stream) {
    if (!R1 || !I) return sfail(CHFPE_EINVAL, "null argument");
    chfpe_status st = check(nt, 2, dtau, L, 2, eta);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *dR = nullptr, *dI = nullptr;
    cudaError_t e = cudaMalloc(&dR, sizeof(double) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&dI, sizeof(double) * L);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dR, R1, sizeof(double) * nt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        Pass p{dR, 0, 1, dI, 0, 1, 1, nt, L, dtau, eta, +1};
        e = run_pass<false, 2>(p, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(I, dI, sizeof(double) * L, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dR);
    cudaFree(dI);
    if (e != cudaSuccess) return sfail(CHFPE_ECUDA, std::string("spectrum1: ") + cudaGetErrorString(e));
    return CHFPE_OK;
}

extern "C" chfpe_status chfpe_spectrum2(const double *R2, int nt1, int nt2, double dtau, int L1,
                                        int L2, double eta, double *I, void *stream) {
    return spectrum2d(R2, nt1, nt2, dtau, L1, L2, eta, -1, -1, I, stream);
}

extern "C" chfpe_status chfpe_spectrum3(const double *R3, int nt1, int nt3, double dtau, int L1,
                                        int L3, double eta, double *I, void *stream) {
    return spectrum2d(R3, nt1, nt3, dtau, L1, L3, eta, -1, +1, I, stream);
}
