// qhp_estimators_noalloc: the ring-polymer estimators of qhp_get_energy (spring,
// normal-mode kinetic and centroid-virial kinetic energy) on caller-owned device
// arrays, without allocating anything.
//
// Why: some callers cannot allocate device memory at the point where they need
// these numbers - code running while another framework captures a CUDA graph
// (cudaMalloc is not capturable), host threads that must not synchronise with
// the device (cudaMalloc/cudaFree may synchronise implicitly), or applications
// that hand the whole device to their own memory pool.  The per-block partial
// sums therefore live in a file-scope device array of fixed size instead of a
// system's scratch buffer.
#include <math.h>

#include <mutex>

#include "qhp_internal.cuh"

namespace qhp {
namespace {

constexpr int NA_BLOCK = 192;
constexpr int NA_MAX_BLOCKS = 65536;   // partial sums of at most 65536 blocks: 3 x 65536 doubles = 1.5 MiB

// Shared by every call in the process; each GPU that loads the library holds its own
// copy until exit.  Host code must not use this name as an address (it is a host-side
// stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_partials[3 * NA_MAX_BLOCKS];

constexpr int NA_MAX_DEVICES = 64;
double* g_partials_addr[NA_MAX_DEVICES] = {};
std::mutex g_setup_mutex;

struct Omega {
    double w[64];
};

// Per-block sums of spring, kinetic and the centroid-virial sum (x_b - Q_0).F_b; each
// block overwrites its own three partials, so nothing needs clearing between calls.
__global__ void __launch_bounds__(NA_BLOCK) k_est_noalloc(int N, int P, int apb, const double* __restrict__ Q,
                                                          const double* __restrict__ Pm, const double* __restrict__ F,
                                                          const double* __restrict__ mass, Omega om,
                                                          double* __restrict__ partial) {
    __shared__ double qs[NA_BLOCK];
    __shared__ double red[3][NA_BLOCK];
    __shared__ double Tm[64 * 64];
    const int t = threadIdx.x;
    for (int e = t; e < P * P; e += NA_BLOCK) {     // sqrt(P) T[b][k], real DFT basis
        const int b = e / P, k = e % P;
        const double ph = 2.0 * (double)((b * k) % P) / (double)P;
        double v;
        if (k == 0) v = 1.0;
        else if (2 * k < P) v = sqrt(2.0) * cospi(ph);
        else if (2 * k == P) v = (b & 1) ? -1.0 : 1.0;
        else v = sqrt(2.0) * sinpi(ph);
        Tm[e] = v;
    }
    const int la = t / (3 * P), d = (t / P) % 3, n = t % P;
    const int a = blockIdx.x * apb + la;
    const bool valid = a < N;
    const int idx = (a * 3 + d) * P + n;
    const double q = valid ? Q[idx] : 0.0;
    qs[t] = q;
    __syncthreads();
    double spring = 0.0, kin = 0.0, vir = 0.0;
    if (valid) {
        const double m = mass[a];
        const double p = Pm[idx];
        spring = 0.5 * m * om.w[n] * om.w[n] * q * q / ACC;
        kin = p * p / (2.0 * m) / ACC;
        const int base = la * 3 * P + d * P;
        double dev = 0.0;
        for (int k = 1; k < P; ++k) dev = fma(Tm[n * P + k], qs[base + k], dev);
        if (F) vir = dev * F[((size_t)n * N + a) * 3 + d];
    }
    red[0][t] = spring;
    red[1][t] = kin;
    red[2][t] = vir;
    __syncthreads();
    if (t < 3) {
        double s = 0.0;
        for (int k = 0; k < NA_BLOCK; ++k) s += red[t][k];
        partial[(size_t)t * NA_MAX_BLOCKS + blockIdx.x] = s;
    }
}

// One warp per estimator: lane l adds the partials l, l + 32, ... in order, then a fixed
// shuffle tree adds the lanes, so the result is the same bits on every call.
__global__ void k_final_noalloc(int nblocks, int N, int P, double kT, const double* __restrict__ partial,
                                double* __restrict__ out) {
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c >= 3) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)c * NA_MAX_BLOCKS + b];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        if (c == 2) out[2] = 1.5 * N * kT - s / (2.0 * P);
        else out[c] = s;
    }
}

}  // namespace
}  // namespace qhp

using namespace qhp;

extern "C" int qhp_estimators_noalloc(int n_atoms, int P, double temperature, const double* Q, const double* Pm,
                                      const double* F, const double* mass, double* out, void* stream) {
    if (n_atoms <= 0 || P < 1 || P > 64 || (P & (P - 1)) || !(temperature > 0.0) || !Q || !Pm || !mass || !out) {
        set_error("qhp_estimators_noalloc: need n_atoms > 0, P a power of two in [1, 64], T > 0, non-null arrays");
        return QHP_ERR_ARG;
    }
    const int apb = 64 / P;
    const long long blocks = ((long long)n_atoms + apb - 1) / apb;
    if (blocks > NA_MAX_BLOCKS) {
        set_error("qhp_estimators_noalloc: n_atoms = %d exceeds the fixed scratch (at most %lld atoms for P = %d)",
                  n_atoms, (long long)NA_MAX_BLOCKS * apb, P);
        return QHP_ERR_ARG;
    }
    int dev = 0;
    QHP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("qhp_estimators_noalloc: device ordinal %d out of range", dev);
        return QHP_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* partial = nullptr;
    {
        // the device address of the scratch array, with this device current: looked up on every
        // call made outside a stream capture (so a device reset cannot leave a stale address
        // behind) and reused from the last such call while the stream is being captured
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        QHP_CUDA(cudaStreamIsCapturing(st, &cs));
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (cs == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            QHP_CUDA(cudaGetSymbolAddress(&p, g_partials));
            g_partials_addr[dev] = static_cast<double*>(p);
        } else if (!g_partials_addr[dev]) {
            set_error("qhp_estimators_noalloc: the first call on a device must come before any stream capture");
            return QHP_ERR_STATE;
        }
        partial = g_partials_addr[dev];
    }
    Omega om{};
    const double kT = KB * temperature;
    const double pi = 3.141592653589793238462643383279502884;
    for (int k = 0; k < P; ++k) om.w[k] = 2.0 * P * kT / HBAR * sin(pi * k / P);
    k_est_noalloc<<<(unsigned)blocks, NA_BLOCK, 0, st>>>(n_atoms, P, apb, Q, Pm, F, mass, om, partial);
    QHP_CUDA(cudaGetLastError());
    k_final_noalloc<<<1, 96, 0, st>>>((int)blocks, n_atoms, P, kT, partial, out);
    QHP_CUDA(cudaGetLastError());
    return QHP_OK;
}
