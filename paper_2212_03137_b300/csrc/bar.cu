// Path-integral Bennett acceptance ratio (Sec. V, Perspective 2, Eqs. (27)-(28)): the self-consistent
// solution for Dlt F_AB = F_B - F_A from dU = U_B - U_A sampled in state A and in state B.
// The sums over samples run on the device (fixed-order block sums, FP64); the host iterates
//     Dlt F = C + ln(<f(-dU + C)>_B / <f(dU - C)>_A) / beta,  C = Dlt F + ln(n_B / n_A) / beta
// from C = ln(n_B / n_A) / beta until C moves by less than tol.
#include <math.h>

#include <vector>

#include "qhp_internal.cuh"

namespace qhp {
namespace {

constexpr int BAR_THREADS = 512;

// f(x) = 1 / (1 + exp(beta x)) without overflow
__device__ __forceinline__ double fermi(double x, double beta) {
    const double y = beta * x;
    if (y > 0.0) {
        const double e = exp(-y);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(y));
}

// block 0: sum_i f(dU_A,i - C); block 1: sum_j f(-dU_B,j + C)
__global__ void __launch_bounds__(BAR_THREADS) k_bar_sums(const double* __restrict__ dA, int nA,
                                                          const double* __restrict__ dB, int nB, double beta,
                                                          double C, double* __restrict__ out) {
    __shared__ double sh[BAR_THREADS];
    const bool a = blockIdx.x == 0;
    const double* d = a ? dA : dB;
    const int n = a ? nA : nB;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += BAR_THREADS) s += a ? fermi(d[i] - C, beta) : fermi(-d[i] + C, beta);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = BAR_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

}  // namespace
}  // namespace qhp

using namespace qhp;

extern "C" int qhp_bar(const double* dU_A, int nA, const double* dU_B, int nB, double beta, double tol,
                       double* dF_out, int* iterations) {
    if (!dU_A || !dU_B || nA < 1 || nB < 1 || !(beta > 0.0) || !(tol > 0.0) || !dF_out) {
        set_error("qhp_bar: need n_A, n_B >= 1 samples, beta > 0, tol > 0");
        return QHP_ERR_ARG;
    }
    double *d = nullptr, *out = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * ((size_t)nA + nB));
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMemcpy(d, dU_A, sizeof(double) * nA, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + nA, dU_B, sizeof(double) * nB, cudaMemcpyHostToDevice);
    int rc = QHP_OK;
    if (e != cudaSuccess) rc = cuda_fail(e, "qhp_bar buffers");
    const double shift = log((double)nB / (double)nA) / beta;
    double C = shift, dF = 0.0;
    int it = 0;
    bool done = false;
    while (rc == QHP_OK && it < 10000 && !done) {
        ++it;
        k_bar_sums<<<2, BAR_THREADS>>>(d, nA, d + nA, nB, beta, C, out);
        double s[2];
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(s, out, sizeof s, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "qhp_bar sums");
            break;
        }
        dF = C + log((s[1] / nB) / (s[0] / nA)) / beta;
        const double Cn = dF + shift;
        done = fabs(Cn - C) < tol;
        C = Cn;
    }
    cudaFree(d);
    cudaFree(out);
    if (rc != QHP_OK) return rc;
    if (!done) {
        set_error("qhp_bar: no convergence in 10000 iterations");
        return QHP_ERR_STATE;
    }
    *dF_out = dF;
    if (iterations) *iterations = it;
    return QHP_OK;
}
