// Adaptive quantum thermal bath (Sec. II.B, Sec. III.B): colored-noise segments,
// FDT spectra, gamma(omega) adaptation.
//
// Definitions (the same readings as the oracle, implemented independently):
// * bins j = 0..N (N = n_seg), N_f = 2N, omega_j = 2 pi j / (N_f dt);
// * S_z(omega_j) = Theta(omega_j) gamma_z(omega_j) / gamma0 below omega_cut, else 0;
// * h_l = (1/N_f) sum_{j<N_f} sqrt(S_z(min(j, N_f - j))) cos(2 pi j l / N_f), l in [-N, N);
// * u_n = sum_{l=-N}^{N-1} h_l xi_{n-l}, xi white (FP32 Box-Muller from Philox tag 4,
//   dof element, counter (g + N) >> 1, output (g + N) & 1);
// * records v_n = (p_before + p_after)/(2m), F_n = kick / dt (written by the O step);
// * C_vv = (dt/N) |v~|^2, C_vF = (dt/N) v~ F~*, DFT of the segment zero-padded to N_f;
// * Delta = (m gamma C_vv - Re C_vF)/418.4 averaged per type; SIMPLE gamma -= A Delta,
//   RATIO gamma = <Re C_vF>/(m <C_vv>) with exponential running averages; gamma >= gamma_min.
//
// The convolution is a 4N-point circular FFT convolution that equals the linear one
// on the N outputs kept.  Two real dofs ride in one complex FFT (a + i b): with X the
// transform, A_k = (X_k + X*_{-k})/2 and B_k = (X_k - X*_{-k})/(2i).
#include <math.h>

#include <vector>

#include "qhp_internal.cuh"

namespace qhp {

namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ int brev(int j, int logn) { return (int)(__brev((unsigned)j) >> (32 - logn)); }

// In-place radix-2 decimation-in-time FFT of n points already in bit-reversed order.
// tw[k] = exp(-2 pi i k / n), k < n/2.  sign = -1 forward, +1 inverse (unscaled).
__device__ void fft_dit(float2* buf, int n, const float2* __restrict__ tw, int sign) {
    for (int h = 1; h < n; h <<= 1) {
        __syncthreads();
        const int stride = n / (2 * h);
        for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
            const int pos = t & (h - 1);
            const int i0 = ((t - pos) << 1) + pos, i1 = i0 + h;
            float2 w = __ldg(&tw[pos * stride]);
            if (sign > 0) w.y = -w.y;
            const float2 a = buf[i0], b = cmul(buf[i1], w);
            buf[i0] = cadd(a, b);
            buf[i1] = csub(a, b);
        }
    }
    __syncthreads();
}

__device__ void bitrev_permute(float2* buf, int n, int logn) {
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int r = brev(j, logn);
        if (j < r) {
            const float2 t = buf[j];
            buf[j] = buf[r];
            buf[r] = t;
        }
    }
    __syncthreads();
}

// White normal of dof at global noise index g (g >= -N): one Philox draw covers g pairs.
__device__ __forceinline__ float2 white_pair(uint64_t seed, uint32_t dof, uint64_t gs_even) {
    const uint4 x = philox_draw(seed, dof, gs_even >> 1, TAG_QTB_WHITE);
    return make_float2(normal_f32(x, 0), normal_f32(x, 1));
}

constexpr int GEN_PAIRS = 4;   // dof pairs per block -> 8 dofs = 32-byte output rows

// One colored-noise segment k for all dofs.
__global__ void __launch_bounds__(256) k_qtb_generate(int n_dof, int N, int log4n, int64_t seg, uint64_t seed,
                                                      const int* __restrict__ dof_type,
                                                      const float2* __restrict__ H /*[2][4N]*/,
                                                      const float2* __restrict__ tw4, float* __restrict__ u) {
    extern __shared__ float2 sm[];
    const int n = 4 * N;
    float2* buf = sm;                                  // [4N]
    float* stage = reinterpret_cast<float*>(sm + n);   // [N][8]
    const int pair0 = blockIdx.x * GEN_PAIRS;
    for (int pp = 0; pp < GEN_PAIRS; ++pp) {
        const int da = 2 * (pair0 + pp), db = da + 1;
        const bool va = da < n_dof, vb = db < n_dof;
        // white noise window g in [kN - N, kN + 2N) at t = g - (kN - N), zero pad to 4N
        for (int t2 = threadIdx.x; t2 < n / 2; t2 += blockDim.x) {
            const int t = 2 * t2;
            float2 xa = make_float2(0.f, 0.f), xb = make_float2(0.f, 0.f);
            if (t < 3 * N) {
                const uint64_t gs = (uint64_t)(seg * N) + (uint64_t)t;   // g + N, even
                if (va) xa = white_pair(seed, (uint32_t)da, gs);
                if (vb) xb = white_pair(seed, (uint32_t)db, gs);
            }
            buf[brev(t, log4n)] = make_float2(xa.x, xb.x);
            buf[brev(t + 1, log4n)] = make_float2(xa.y, xb.y);
        }
        fft_dit(buf, n, tw4, -1);
        const int za = va ? dof_type[da] : 0, zb = vb ? dof_type[db] : 0;
        for (int k = threadIdx.x; k <= n / 2; k += blockDim.x) {
            const int km = (n - k) & (n - 1);
            const float2 Xk = buf[k], Xm = buf[km];
            const float2 Ak = make_float2(0.5f * (Xk.x + Xm.x), 0.5f * (Xk.y - Xm.y));   // (X_k + X*_-k)/2
            const float2 Bk = make_float2(0.5f * (Xk.y + Xm.y), -0.5f * (Xk.x - Xm.x));  // (X_k - X*_-k)/(2i)
            const float2 Yk = cadd(cmul(H[za * n + k], Ak), cmul(make_float2(0.f, 1.f), cmul(H[zb * n + k], Bk)));
            if (km != k) {
                const float2 Am = cconj(Ak), Bm = cconj(Bk);                                 // spectra of real signals
                const float2 Ym = cadd(cmul(H[za * n + km], Am), cmul(make_float2(0.f, 1.f), cmul(H[zb * n + km], Bm)));
                buf[km] = Ym;
            }
            buf[k] = Yk;
        }
        bitrev_permute(buf, n, log4n);
        fft_dit(buf, n, tw4, +1);
        const float inv = 1.0f / (float)n;
        for (int m = threadIdx.x; m < N; m += blockDim.x) {
            const float2 y = buf[N + m];
            stage[m * 8 + 2 * pp] = y.x * inv;
            stage[m * 8 + 2 * pp + 1] = y.y * inv;
        }
        __syncthreads();
    }
    // coalesced write of the staged [N][8] block
    const int d0 = pair0 * 2;
    for (int e = threadIdx.x; e < N * 8; e += blockDim.x) {
        const int m = e >> 3, c = e & 7;
        if (d0 + c < n_dof) u[(size_t)m * n_dof + d0 + c] = stage[e];
    }
}

// Per-block sums over dof pairs of: Delta (needs gamma), C_vv, Re C_vF, per type and bin.
__global__ void __launch_bounds__(256) k_qtb_spectra(int n_dof, int N, int log2n, double dt, const int* __restrict__ dof_type,
                                                     const double* __restrict__ m_dof, const double* __restrict__ gamma,
                                                     const float* __restrict__ v, const float* __restrict__ F,
                                                     const float2* __restrict__ tw2, double* __restrict__ part) {
    extern __shared__ float2 sm[];
    const int n = 2 * N, nb = N + 1;
    float2* bv = sm;
    float2* bf = sm + n;
    double* acc = reinterpret_cast<double*>(sm + 2 * n);   // [3][2][nb]
    for (int e = threadIdx.x; e < 6 * nb; e += blockDim.x) acc[e] = 0.0;
    const int n_pairs = (n_dof + 1) / 2;
    const double norm = dt / (double)N;
    for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
        const int da = 2 * p, db = da + 1;
        const bool vb = db < n_dof;
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            float2 xv = make_float2(0.f, 0.f), xf = make_float2(0.f, 0.f);
            if (t < N) {
                xv.x = v[(size_t)t * n_dof + da];
                xf.x = F[(size_t)t * n_dof + da];
                if (vb) {
                    xv.y = v[(size_t)t * n_dof + db];
                    xf.y = F[(size_t)t * n_dof + db];
                }
            }
            const int r = brev(t, log2n);
            bv[r] = xv;
            bf[r] = xf;
        }
        fft_dit(bv, n, tw2, -1);
        fft_dit(bf, n, tw2, -1);
        const int za = dof_type[da], zb = vb ? dof_type[db] : 0;
        const double ma = m_dof[da], mb = vb ? m_dof[db] : 0.0;
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            const int km = (n - k) & (n - 1);
            const float2 Xk = bv[k], Xm = bv[km], Yk = bf[k], Ym = bf[km];
            // a-signal and b-signal spectra at bin k
            const double var = 0.5 * ((double)Xk.x + Xm.x), vai = 0.5 * ((double)Xk.y - Xm.y);
            const double vbr = 0.5 * ((double)Xk.y + Xm.y), vbi = -0.5 * ((double)Xk.x - Xm.x);
            const double far_ = 0.5 * ((double)Yk.x + Ym.x), fai = 0.5 * ((double)Yk.y - Ym.y);
            const double fbr = 0.5 * ((double)Yk.y + Ym.y), fbi = -0.5 * ((double)Yk.x - Ym.x);
            {
                const double cvv = norm * (var * var + vai * vai);
                const double cvf = norm * (var * far_ + vai * fai);    // Re(v F*)
                const double dl = (ma * gamma[za * nb + k] * cvv - cvf) / ACC;
                acc[(0 * 2 + za) * nb + k] += dl;
                acc[(1 * 2 + za) * nb + k] += cvv;
                acc[(2 * 2 + za) * nb + k] += cvf;
            }
            if (vb) {
                const double cvv = norm * (vbr * vbr + vbi * vbi);
                const double cvf = norm * (vbr * fbr + vbi * fbi);
                const double dl = (mb * gamma[zb * nb + k] * cvv - cvf) / ACC;
                acc[(0 * 2 + zb) * nb + k] += dl;
                acc[(1 * 2 + zb) * nb + k] += cvv;
                acc[(2 * 2 + zb) * nb + k] += cvf;
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 6 * nb; e += blockDim.x) part[(size_t)blockIdx.x * 6 * nb + e] = acc[e];
}

// Sum the block partials in fixed order, then adapt gamma per type and bin.
__global__ void k_qtb_adapt(int nblocks, int N, const double* __restrict__ part, double n_O, double n_H,
                            double m_O, double m_H, int adapt, double a_gamma, double gmin, double wavg, int first,
                            double* gamma, double* avg, double* delta_out) {
    const int nb = N + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // (type, bin)
    if (e >= 2 * nb) return;
    const int z = e / nb, k = e % nb;
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nblocks; ++b)
        for (int q = 0; q < 3; ++q) s[q] += part[(size_t)b * 6 * nb + (q * 2 + z) * nb + k];
    const double cnt = z == 0 ? n_O : n_H;
    if (cnt <= 0.0) return;
    const double dbar = s[0] / cnt, cvv = s[1] / cnt, cvf = s[2] / cnt;
    delta_out[z * nb + k] = dbar;
    double g = gamma[z * nb + k];
    if (adapt == QHP_ADAPT_SIMPLE) {
        g = g - a_gamma * dbar;
    } else if (adapt == QHP_ADAPT_RATIO) {
        double* avv = avg + (0 * 2 + z) * nb;
        double* avf = avg + (1 * 2 + z) * nb;
        if (first) {
            avv[k] = cvv;
            avf[k] = cvf;
        } else {
            avv[k] = avv[k] * wavg + cvv * (1.0 - wavg);
            avf[k] = avf[k] * wavg + cvf * (1.0 - wavg);
        }
        g = avf[k] / ((z == 0 ? m_O : m_H) * avv[k]);
    }
    if (adapt != QHP_ADAPT_NONE) gamma[z * nb + k] = fmax(gmin, g);
}

// sqrt(S_z(omega_j)) on bins j = 0..N (Eqs. (13)-(14) with the gamma_z / gamma0 factor).
__global__ void k_qtb_sqrtS(int N, double dt, double kT, double hbar, double gamma0, double wcut,
                            const double* __restrict__ gamma, double* __restrict__ sqrtS /*[2][N+1]*/) {
    const int nb = N + 1, nf = 2 * N;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * nb) return;
    const int bin = e % nb;
    const double w = 2.0 * M_PI * bin / (nf * dt);
    double S = 0.0;
    if (w <= wcut) {
        const double th = (bin == 0) ? kT : 0.5 * hbar * w / tanh(0.5 * hbar * w / kT);
        S = th * gamma[e] / gamma0;
    }
    sqrtS[e] = sqrt(S);
}

// Filter taps of each type for the next segment: h_l, l in [-N, N).
__global__ void k_qtb_taps(int N, const double* __restrict__ sqrtS, double* __restrict__ h /*[2][2N]*/) {
    const int nf = 2 * N, nb = N + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * nf) return;
    const int z = e / nf, li = e % nf;       // l = li - N
    const long long l = li - N;
    double acc = 0.0;
    for (int j = 0; j < nf; ++j) {
        const int bin = j < nf - j ? j : nf - j;
        long long jl = ((long long)j * l) % nf;
        if (jl < 0) jl += nf;
        acc += sqrtS[z * nb + bin] * cospi(2.0 * (double)jl / (double)nf);
    }
    h[e] = acc / nf;
}

__global__ void k_qtb_filter(int N, const double* __restrict__ h, float2* __restrict__ H /*[2][4N]*/) {
    const int n = 4 * N, nf = 2 * N;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * n) return;
    const int z = e / n, k = e % n;
    double re = 0.0, im = 0.0;
    for (int li = 0; li < nf; ++li) {
        const long long l = li - N;                       // tap at circular index l mod 4N
        long long kl = ((long long)k * l) % n;
        if (kl < 0) kl += n;
        double sn, cs;
        sincospi(2.0 * (double)kl / (double)n, &sn, &cs);
        re += h[z * nf + li] * cs;
        im -= h[z * nf + li] * sn;
    }
    H[e] = make_float2((float)re, (float)im);
}

int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

template <typename T>
int qalloc(qhp_system_s* s, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc failed for adQTB buffers: %s", cudaGetErrorString(e));
        return QHP_ERR_NOMEM;
    }
    *p = static_cast<T*>(q);
    s->allocs.push_back({q, count * sizeof(T)});
    return QHP_OK;
}

size_t gen_smem(int N) { return sizeof(float2) * 4 * N + sizeof(float) * 8 * N; }
size_t spec_smem(int N) { return sizeof(float2) * 4 * N + sizeof(double) * 6 * (N + 1); }
constexpr int SPEC_BLOCKS = 592;

int enqueue_filter(qhp_system_s* s) {
    const int N = s->n_seg;
    const double kT = KB * s->temperature;
    const double wcut = s->th.omega_cut_cm > 0.0 ? s->th.omega_cut_cm * CM1 : INFINITY;
    k_qtb_sqrtS<<<(2 * (N + 1) + 127) / 128, 128, 0, s->stream>>>(N, s->th.dt_fs * 1e-3, kT, HBAR, s->th.gamma0,
                                                                  wcut, s->qtb_gamma, s->qtb_sqrtS);
    k_qtb_taps<<<(4 * N + 127) / 128, 128, 0, s->stream>>>(N, s->qtb_sqrtS, s->qtb_h);
    k_qtb_filter<<<(8 * N + 127) / 128, 128, 0, s->stream>>>(N, s->qtb_h, s->qtb_H);
    s->launches += 3;
    QHP_CUDA(cudaGetLastError());
    return QHP_OK;
}

int enqueue_generate(qhp_system_s* s, int64_t seg) {
    const int N = s->n_seg, n_dof = 3 * s->N;
    const int n_pairs = (n_dof + 1) / 2;
    const int grid = (n_pairs + GEN_PAIRS - 1) / GEN_PAIRS;
    k_qtb_generate<<<grid, 256, gen_smem(N), s->stream>>>(n_dof, N, ilog2(4 * N), seg, s->seed, s->qtb_dof_type,
                                                          s->qtb_H, s->qtb_tw4, s->qtb_u);
    s->launches++;
    QHP_CUDA(cudaGetLastError());
    return QHP_OK;
}

}  // namespace

int qtb_setup(qhp_system_s* s) {
    if (s->P != 1) {
        set_error("adQTB runs on a single bead (P = 1)");
        return QHP_ERR_STATE;
    }
    const int N = s->th.n_seg, n_dof = 3 * s->N;
    if (N > 2048) {
        set_error("n_seg above 2048 is not supported");
        return QHP_ERR_ARG;
    }
    if (s->n_seg != N || !s->qtb_u) {
        s->n_seg = N;
        const size_t rows = (size_t)N * n_dof;
        int rc;
        if ((rc = qalloc(s, &s->qtb_u, rows)) || (rc = qalloc(s, &s->qtb_v, rows)) || (rc = qalloc(s, &s->qtb_F, rows)) ||
            (rc = qalloc(s, &s->qtb_gamma, 2 * (size_t)(N + 1))) || (rc = qalloc(s, &s->qtb_h, 4 * (size_t)N)) ||
            (rc = qalloc(s, &s->qtb_sqrtS, 2 * (size_t)(N + 1))) ||
            (rc = qalloc(s, &s->qtb_H, 8 * (size_t)N)) || (rc = qalloc(s, &s->qtb_avg, 4 * (size_t)(N + 1))) ||
            (rc = qalloc(s, &s->qtb_delta, 2 * (size_t)(N + 1))) ||
            (rc = qalloc(s, &s->qtb_part, (size_t)SPEC_BLOCKS * 6 * (N + 1))) ||
            (rc = qalloc(s, &s->qtb_tw4, 2 * (size_t)N)) || (rc = qalloc(s, &s->qtb_tw2, (size_t)N)) ||
            (rc = qalloc(s, &s->qtb_dof_type, n_dof)) || (rc = qalloc(s, &s->qtb_mdof, n_dof)))
            return rc;
        std::vector<float2> tw4(2 * N), tw2(N);
        for (int k = 0; k < 2 * N; ++k) {
            const double a = -2.0 * M_PI * k / (4.0 * N);
            tw4[k] = make_float2((float)cos(a), (float)sin(a));
        }
        for (int k = 0; k < N; ++k) {
            const double a = -2.0 * M_PI * k / (2.0 * N);
            tw2[k] = make_float2((float)cos(a), (float)sin(a));
        }
        std::vector<int> dt_(n_dof);
        std::vector<double> md(n_dof);
        for (int i = 0; i < n_dof; ++i) {
            dt_[i] = s->type[i / 3];
            md[i] = dt_[i] == 0 ? s->ff.m_O : s->ff.m_H;
        }
        QHP_CUDA(cudaMemcpy(s->qtb_tw4, tw4.data(), sizeof(float2) * 2 * N, cudaMemcpyHostToDevice));
        QHP_CUDA(cudaMemcpy(s->qtb_tw2, tw2.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
        QHP_CUDA(cudaMemcpy(s->qtb_dof_type, dt_.data(), sizeof(int) * n_dof, cudaMemcpyHostToDevice));
        QHP_CUDA(cudaMemcpy(s->qtb_mdof, md.data(), sizeof(double) * n_dof, cudaMemcpyHostToDevice));
        QHP_CUDA(cudaFuncSetAttribute(k_qtb_generate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gen_smem(2048)));
        QHP_CUDA(cudaFuncSetAttribute(k_qtb_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem(2048)));
    }
    std::vector<double> g(2 * (size_t)(N + 1), s->th.gamma0);
    QHP_CUDA(cudaMemcpy(s->qtb_gamma, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemset(s->qtb_delta, 0, sizeof(double) * 2 * (N + 1)));
    QHP_CUDA(cudaMemset(s->qtb_v, 0, sizeof(float) * (size_t)N * n_dof));
    QHP_CUDA(cudaMemset(s->qtb_F, 0, sizeof(float) * (size_t)N * n_dof));
    s->qtb_ratio_first = 1;
    int rc = enqueue_filter(s);
    if (rc) return rc;
    rc = enqueue_generate(s, s->step / N);
    if (rc) return rc;
    QHP_CUDA(cudaStreamSynchronize(s->stream));
    return QHP_OK;
}

// Spectra of the finished segment, adaptation, filter and noise of the next segment.
cudaError_t launch_qtb_segment_end(qhp_system_s* s) {
    const int N = s->n_seg, n_dof = 3 * s->N;
    const int n_pairs = (n_dof + 1) / 2;
    const int blocks = std::min(SPEC_BLOCKS, n_pairs);
    k_qtb_spectra<<<blocks, 256, spec_smem(N), s->stream>>>(n_dof, N, ilog2(2 * N), s->th.dt_fs * 1e-3, s->qtb_dof_type,
                                                            s->qtb_mdof, s->qtb_gamma, s->qtb_v, s->qtb_F, s->qtb_tw2,
                                                            s->qtb_part);
    int nO = 0;
    for (int i = 0; i < s->N; ++i) nO += s->type[i] == 0;
    const double n_O = 3.0 * nO, n_H = 3.0 * (s->N - nO);
    const double wavg = exp(-N * s->th.dt_fs * 1e-3 / (s->th.tau_ratio_ps > 0 ? s->th.tau_ratio_ps : 1.0));
    k_qtb_adapt<<<(2 * (N + 1) + 127) / 128, 128, 0, s->stream>>>(
        blocks, N, s->qtb_part, n_O, n_H, s->ff.m_O, s->ff.m_H, s->th.adapt, s->th.a_gamma,
        s->th.gamma_min_frac * s->th.gamma0, wavg, s->qtb_ratio_first, s->qtb_gamma, s->qtb_avg, s->qtb_delta);
    s->launches += 2;
    if (s->th.adapt == QHP_ADAPT_RATIO) s->qtb_ratio_first = 0;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (enqueue_filter(s) != QHP_OK) return cudaErrorUnknown;
    // the step counter has already advanced past the segment: generate segment (step+1)/N
    return cudaSuccess;
}

int qtb_generate_segment(qhp_system_s* s, int64_t seg) { return enqueue_generate(s, seg); }

}  // namespace qhp
