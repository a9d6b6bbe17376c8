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
//
// FFTs are in place in shared memory, radix 2^2 (two radix-2 stages per pass, so half
// the passes and barriers of radix 2): the forward transform is decimation in frequency
// (natural order in, bit-reversed out) and the inverse decimation in time (bit-reversed
// in, natural out), so the pointwise product in between needs no permutation pass.
#include <math.h>

#include <algorithm>
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

// Shared-memory layout of the FFT buffers: element e lives at e + e/16 (one spare float2 per
// 16).  The strided passes touch elements 16a + b at once; the pad sends different a to
// different banks, which also holds for the four-consecutive-element butterflies of the
// shortest passes (threads 32 bytes apart), so no pass has bank conflicts.
__host__ __device__ __forceinline__ int fpad(int e) { return e + (e >> 4); }
__host__ __device__ __forceinline__ int fpad_len(int n) { return n + (n >> 4); }

// The spectrum of a real signal pairs bin k with bin -k.  In bit-reversed storage (the
// forward FFT's output) position p = brev(k) has its partner -k at the mirror of p
// within p's power-of-two block [b, 2b): pm = 3b - 1 - p.  Item q in [0, n/2] visits each
// pair once with p in the lower half of its block, so consecutive q read consecutive p
// and consecutive (descending) pm: no shared-memory bank conflicts.
__device__ __forceinline__ void pair_positions(int q, int& p, int& pm) {
    if (q < 2) {
        p = pm = q;   // k = 0 and k = n/2 are their own partners
        return;
    }
    const int qq = q - 1;
    const int b = 2 << (31 - __clz(qq));
    p = qq + (b >> 1);
    pm = 3 * b - 1 - p;
}

// Forward FFT in place, natural order in, bit-reversed order out (radix-2 decimation in
// frequency, stages fused in pairs).  tw[k] = exp(-2 pi i k / n), k < n/2.  NB buffers
// of n points are transformed together (more independent work per barrier).
template <int NB>
__device__ void fft_dif_fwd(float2* const (&x)[NB], int n, int logn, const float2* __restrict__ tw) {
    int h = n >> 1, lh = logn - 1, s = 1;   // stage half-size h = 2^lh, twiddle stride n/(2h)
    for (; h >= 2; h >>= 2, lh -= 2, s <<= 2) {
        __syncthreads();
        const int lq = lh - 1;              // q < h/2 = 2^lq
        for (int g = threadIdx.x; g < (n >> 2); g += blockDim.x) {
            const int q = g & ((1 << lq) - 1);
            const int i0 = ((g >> lq) << (lh + 1)) + q, i1 = i0 + (h >> 1), i2 = i0 + h, i3 = i2 + (h >> 1);
            const float2 wA = __ldg(&tw[q * s]), wB = __ldg(&tw[2 * q * s]);
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                float2* X = x[u];
                const float2 a0 = X[fpad(i0)], a1 = X[fpad(i1)], a2 = X[fpad(i2)], a3 = X[fpad(i3)];
                const float2 t0 = cadd(a0, a2), t2 = cmul(csub(a0, a2), wA);
                const float2 t1 = cadd(a1, a3);
                float2 t3 = cmul(csub(a1, a3), wA);
                t3 = make_float2(t3.y, -t3.x);   // times W^{n/4} = -i
                X[fpad(i0)] = cadd(t0, t1);
                X[fpad(i1)] = cmul(csub(t0, t1), wB);
                X[fpad(i2)] = cadd(t2, t3);
                X[fpad(i3)] = cmul(csub(t2, t3), wB);
            }
        }
    }
    if (h == 1) {   // odd number of stages: the last one alone (unit twiddles)
        __syncthreads();
        for (int g = threadIdx.x; g < (n >> 1); g += blockDim.x) {
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                float2* X = x[u];
                const float2 a = X[fpad(2 * g)], b = X[fpad(2 * g + 1)];
                X[fpad(2 * g)] = cadd(a, b);
                X[fpad(2 * g + 1)] = csub(a, b);
            }
        }
    }
    __syncthreads();
}

// Inverse FFT in place (unscaled), bit-reversed order in, natural order out (radix-2
// decimation in time with conjugate twiddles, stages fused in pairs).
__device__ void fft_dit_inv(float2* x, int n, int logn, const float2* __restrict__ tw) {
    int h = 1, lh = 0, s = n >> 1;          // stage half-size h = 2^lh, twiddle stride n/(2h)
    if (logn & 1) {                         // odd number of stages: the first one alone
        __syncthreads();
        for (int g = threadIdx.x; g < (n >> 1); g += blockDim.x) {
            const float2 a = x[fpad(2 * g)], b = x[fpad(2 * g + 1)];
            x[fpad(2 * g)] = cadd(a, b);
            x[fpad(2 * g + 1)] = csub(a, b);
        }
        h = 2;
        lh = 1;
        s = n >> 2;
    }
    for (; h < n; h <<= 2, lh += 2, s >>= 2) {   // stages h and 2h
        __syncthreads();
        for (int g = threadIdx.x; g < (n >> 2); g += blockDim.x) {
            const int q = g & (h - 1);
            const int i0 = ((g >> lh) << (lh + 2)) + q, i1 = i0 + h, i2 = i0 + 2 * h, i3 = i0 + 3 * h;
            const float2 w1 = cconj(__ldg(&tw[q * s])), w2 = cconj(__ldg(&tw[q * (s >> 1)]));
            const float2 a0 = x[fpad(i0)], a1 = x[fpad(i1)], a2 = x[fpad(i2)], a3 = x[fpad(i3)];
            const float2 b1 = cmul(a1, w1), b3 = cmul(a3, w1);
            const float2 u0 = cadd(a0, b1), u1 = csub(a0, b1), u2 = cadd(a2, b3), u3 = csub(a2, b3);
            const float2 c2 = cmul(u2, w2);
            float2 c3 = cmul(u3, w2);
            c3 = make_float2(-c3.y, c3.x);       // times W^{-n/4} = +i
            x[fpad(i0)] = cadd(u0, c2);
            x[fpad(i2)] = csub(u0, c2);
            x[fpad(i1)] = cadd(u1, c3);
            x[fpad(i3)] = csub(u1, c3);
        }
    }
    __syncthreads();
}

// White normal of dof at global noise index g (g >= -N): one Philox draw covers g pairs.
__device__ __forceinline__ float2 white_pair(uint64_t seed, uint32_t dof, uint64_t gs_even) {
    const uint4 x = philox_draw(seed, dof, gs_even >> 1, TAG_QTB_WHITE);
    return make_float2(normal_f32(x, 0), normal_f32(x, 1));
}

constexpr int GEN_PAIRS = 4;     // dof pairs per block -> 8 dofs = 32-byte output rows
constexpr int GEN_THREADS = 512;
constexpr int GEN_ROW = 9;       // floats per staged output row (8 dofs + 1 pad)

// One colored-noise segment k for all dofs.
__global__ void __launch_bounds__(GEN_THREADS) k_qtb_generate(int n_dof, int N, int log4n, int64_t seg,
                                                              uint64_t seed, const int* __restrict__ dof_type,
                                                              const float2* __restrict__ H /*[2][4N]*/,
                                                              const float2* __restrict__ tw4, float* __restrict__ u) {
    extern __shared__ float2 sm[];
    const int n = 4 * N;
    float2* buf = sm;                                  // [fpad_len(4N)]
    float* stage = reinterpret_cast<float*>(sm + fpad_len(n));   // [N][GEN_ROW]: 8 outputs, 1 pad
    float2* const bufs[1] = {buf};
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
            buf[fpad(t)] = make_float2(xa.x, xb.x);
            buf[fpad(t + 1)] = make_float2(xa.y, xb.y);
        }
        fft_dif_fwd<1>(bufs, n, log4n, tw4);   // bin k now sits at position brev(k)
        const int za = va ? dof_type[da] : 0, zb = vb ? dof_type[db] : 0;
        const float2* Ha = H + za * n;           // H is stored in the same bit-reversed order
        const float2* Hb = H + zb * n;
        for (int q = threadIdx.x; q <= n / 2; q += blockDim.x) {
            int pk, pm;
            pair_positions(q, pk, pm);
            const float2 Xk = buf[fpad(pk)], Xm = buf[fpad(pm)];
            const float2 Ak = make_float2(0.5f * (Xk.x + Xm.x), 0.5f * (Xk.y - Xm.y));   // (X_k + X*_-k)/2
            const float2 Bk = make_float2(0.5f * (Xk.y + Xm.y), -0.5f * (Xk.x - Xm.x));  // (X_k - X*_-k)/(2i)
            const float2 Yk = cadd(cmul(Ha[pk], Ak), cmul(make_float2(0.f, 1.f), cmul(Hb[pk], Bk)));
            if (pm != pk) {
                const float2 Am = cconj(Ak), Bm = cconj(Bk);                                 // spectra of real signals
                const float2 Ym = cadd(cmul(Ha[pm], Am), cmul(make_float2(0.f, 1.f), cmul(Hb[pm], Bm)));
                buf[fpad(pm)] = Ym;
            }
            buf[fpad(pk)] = Yk;
        }
        fft_dit_inv(buf, n, log4n, tw4);
        const float inv = 1.0f / (float)n;
        for (int m = threadIdx.x; m < N; m += blockDim.x) {
            const float2 y = buf[fpad(N + m)];
            stage[m * GEN_ROW + 2 * pp] = y.x * inv;   // rows of 9 floats: consecutive m in distinct banks
            stage[m * GEN_ROW + 2 * pp + 1] = y.y * inv;
        }
        __syncthreads();
    }
    // coalesced write of the staged block, 8 dofs per output row
    const int d0 = pair0 * 2;
    for (int e = threadIdx.x; e < N * 8; e += blockDim.x) {
        const int m = e >> 3, c = e & 7;
        if (d0 + c < n_dof) u[(size_t)m * n_dof + d0 + c] = stage[m * GEN_ROW + c];
    }
}

constexpr int SPEC_THREADS = 512;   // with 1,025 bins (n_seg 1024): three per thread, 32 warps per SM
constexpr int SPEC_DOFS = 4;   // dofs per tile: 16-byte row segments of v and F

// acc[z] += a, acc[2 + z] += b with constant indices (registers, not memory)
__device__ __forceinline__ void add_typed(float* acc, int z, float a, float b) {
    if (z == 0) {
        acc[0] += a;
        acc[2] += b;
    } else {
        acc[1] += a;
        acc[3] += b;
    }
}

// Per-block sums over dofs of |v~_k|^2 and Re(v~_k F~_k*) per type and bin (Eq. (22) without
// its dt/N factor; the per-type FDT deviation is linear in them and is formed from the
// sums in k_qtb_adapt).  Each thread owns the bins k = t, t + 512, ... (at most BPT): a
// tile of 4 dofs is summed in FP32, then added to FP64 running sums.  The block walks
// tiles of 4 dofs, read as [step][4] rows.
template <int BPT>
__global__ void __launch_bounds__(SPEC_THREADS) k_qtb_spectra(int n_dof, int N, int log2n,
                                                              const int* __restrict__ dof_type,
                                                              const float* __restrict__ v, const float* __restrict__ F,
                                                              const float2* __restrict__ tw2,
                                                              double* __restrict__ part) {
    extern __shared__ float2 sm[];
    const int n = 2 * N, nb = N + 1;
    float2* bv = sm;                                         // [fpad_len(2N)]
    float2* bf = sm + fpad_len(n);                           // [fpad_len(2N)]
    // tiles of SPEC_DOFS dofs, one row of N + 8 floats per dof (the pad puts the 4 rows of a
    // 32-element store in distinct banks; rows are read along the steps, contiguously)
    const int row = N + 8;
    float* tv = reinterpret_cast<float*>(sm + 2 * fpad_len(n));   // [SPEC_DOFS][N + 8]
    float* tf = tv + SPEC_DOFS * row;                            // [SPEC_DOFS][N + 8]
    float2* const bufs[2] = {bv, bf};
    double acc[BPT][4];
#pragma unroll
    for (int j = 0; j < BPT; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.0;
    const int n_tiles = (n_dof + SPEC_DOFS - 1) / SPEC_DOFS;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int d0 = tile * SPEC_DOFS;
        __syncthreads();
        for (int e = threadIdx.x; e < N * SPEC_DOFS; e += blockDim.x) {
            const int m = e / SPEC_DOFS, c = e % SPEC_DOFS;
            const bool ok = d0 + c < n_dof;
            tv[c * row + m] = ok ? v[(size_t)m * n_dof + d0 + c] : 0.0f;
            tf[c * row + m] = ok ? F[(size_t)m * n_dof + d0 + c] : 0.0f;
        }
        float ts[BPT][4];
#pragma unroll
        for (int j = 0; j < BPT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) ts[j][q] = 0.0f;
        for (int pp = 0; pp < SPEC_DOFS / 2; ++pp) {
            const int da = d0 + 2 * pp, db = da + 1;
            if (da >= n_dof) break;
            const bool vb = db < n_dof;
            __syncthreads();
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                float2 xv = make_float2(0.f, 0.f), xf = make_float2(0.f, 0.f);
                if (t < N) {
                    xv = make_float2(tv[(2 * pp) * row + t], tv[(2 * pp + 1) * row + t]);
                    xf = make_float2(tf[(2 * pp) * row + t], tf[(2 * pp + 1) * row + t]);
                }
                bv[fpad(t)] = xv;
                bf[fpad(t)] = xf;
            }
            fft_dif_fwd<2>(bufs, n, log2n, tw2);   // bin k at position brev(k)
            const int za = dof_type[da], zb = vb ? dof_type[db] : 0;
#pragma unroll
            for (int j = 0; j < BPT; ++j) {
                const int q = threadIdx.x + j * SPEC_THREADS;
                if (q >= nb) break;
                int pk, pm;
                pair_positions(q, pk, pm);
                const float2 Xk = bv[fpad(pk)], Xm = bv[fpad(pm)], Yk = bf[fpad(pk)], Ym = bf[fpad(pm)];
                // spectra of the a and b signals at bin k (twice their values: the 1/2 of
                // the real-pair split is applied squared, as 1/4, below)
                const float var = Xk.x + Xm.x, vai = Xk.y - Xm.y, vbr = Xk.y + Xm.y, vbi = Xm.x - Xk.x;
                const float far_ = Yk.x + Ym.x, fai = Yk.y - Ym.y, fbr = Yk.y + Ym.y, fbi = Ym.x - Yk.x;
                add_typed(ts[j], za, 0.25f * (var * var + vai * vai), 0.25f * (var * far_ + vai * fai));
                if (vb) add_typed(ts[j], zb, 0.25f * (vbr * vbr + vbi * vbi), 0.25f * (vbr * fbr + vbi * fbi));
            }
        }
#pragma unroll
        for (int j = 0; j < BPT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] += (double)ts[j][q];
    }
    // part[block][c][bin], c = (vv O, vv H, vF O, vF H); slot j holds bin min(k, n - k) of
    // the pair visited by item q
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
        const int q = threadIdx.x + j * SPEC_THREADS;
        if (q >= nb) break;
        int pk, pm;
        pair_positions(q, pk, pm);
        const int k = brev(pk, log2n), bin = min(k, n - k);
#pragma unroll
        for (int c = 0; c < 4; ++c) part[((size_t)blockIdx.x * 4 + c) * nb + bin] = acc[j][c];
    }
}

// Sum the block partials in fixed order, form the type means C_vv, C_vF (with the dt/N
// factor) and the FDT deviation Delta = (m gamma C_vv - Re C_vF) / 418.4 (Eq. (21); linear
// in the spectra, so the mean of the per-dof deviations), then adapt gamma.
__global__ void k_qtb_adapt(int nblocks, int N, double norm, const double* __restrict__ part, double n_O, double n_H,
                            double m_O, double m_H, int adapt, double a_gamma, double gmin, double wavg, int first,
                            double* gamma, double* avg, double* delta_out) {
    const int nb = N + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // (type, bin)
    if (e >= 2 * nb) return;
    const int z = e / nb, k = e % nb;
    double svv = 0.0, svf = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        svv += part[((size_t)b * 4 + z) * nb + k];
        svf += part[((size_t)b * 4 + 2 + z) * nb + k];
    }
    const double cnt = z == 0 ? n_O : n_H;
    if (cnt <= 0.0) return;
    const double cvv = norm * svv / cnt, cvf = norm * svf / cnt;
    double g = gamma[z * nb + k];
    const double dbar = ((z == 0 ? m_O : m_H) * g * cvv - cvf) / ACC;
    delta_out[z * nb + k] = dbar;
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

constexpr int TAP_THREADS = 128;

// Fixed-order block sum of one double per thread (TAP_THREADS threads).
__device__ __forceinline__ double block_sum(double x, double* sh) {
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = TAP_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    return sh[0];
}

// Filter taps of each type for the next segment: h_l, l in [-N, N); one block per tap.
__global__ void __launch_bounds__(TAP_THREADS) k_qtb_taps(int N, const double* __restrict__ sqrtS,
                                                          double* __restrict__ h /*[2][2N]*/) {
    __shared__ double sh[TAP_THREADS];
    const int nf = 2 * N, nb = N + 1;
    const int e = blockIdx.x;
    const int z = e / nf, li = e % nf;       // l = li - N
    const long long l = li - N;
    double acc = 0.0;
    for (int j = threadIdx.x; j < nf; j += TAP_THREADS) {
        const int bin = j < nf - j ? j : nf - j;
        long long jl = ((long long)j * l) % nf;
        if (jl < 0) jl += nf;
        acc += sqrtS[z * nb + bin] * cospi(2.0 * (double)jl / (double)nf);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) h[e] = acc / nf;
}

// Transfer function of the taps on the 4N-point grid (taps at circular index l mod 4N);
// one block per (type, bin).
__global__ void __launch_bounds__(TAP_THREADS) k_qtb_filter(int N, int log4n, const double* __restrict__ h,
                                                            float2* __restrict__ H /*[2][4N], bit-reversed bins*/) {
    __shared__ double sh[TAP_THREADS];
    const int n = 4 * N, nf = 2 * N;
    const int e = blockIdx.x;
    const int z = e / n, k = e % n;
    double re = 0.0, im = 0.0;
    for (int li = threadIdx.x; li < nf; li += TAP_THREADS) {
        const long long l = li - N;
        long long kl = ((long long)k * l) % n;
        if (kl < 0) kl += n;
        double sn, cs;
        sincospi(2.0 * (double)kl / (double)n, &sn, &cs);
        re += h[z * nf + li] * cs;
        im -= h[z * nf + li] * sn;
    }
    re = block_sum(re, sh);
    __syncthreads();
    im = block_sum(im, sh);
    if (threadIdx.x == 0) H[z * n + brev(k, log4n)] = make_float2((float)re, (float)im);
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

size_t gen_smem(int N) { return sizeof(float2) * fpad_len(4 * N) + sizeof(float) * GEN_ROW * N; }
size_t spec_smem(int N) { return sizeof(float2) * 2 * fpad_len(2 * N) + sizeof(float) * 2 * SPEC_DOFS * (N + 8); }
constexpr int SPEC_BLOCKS = 592;

// bins per thread of the spectra kernel for N (n_seg <= 2048): ceil((N + 1) / 512)
int spec_bpt(int N) {
    const int b = (N + 1 + SPEC_THREADS - 1) / SPEC_THREADS;
    return b <= 1 ? 1 : b <= 2 ? 2 : b <= 3 ? 3 : 5;
}

template <int B>
const void* spectra_kernel() { return (const void*)k_qtb_spectra<B>; }

const void* spectra_kernel_for(int N) {
    switch (spec_bpt(N)) {
        case 1: return spectra_kernel<1>();
        case 2: return spectra_kernel<2>();
        case 3: return spectra_kernel<3>();
        default: return spectra_kernel<5>();
    }
}

// Resident blocks of the spectra kernel (one wave; every block walks many tiles).
int spectra_blocks(qhp_system_s* s) {
    const int N = s->n_seg, n_dof = 3 * s->N;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spectra_kernel_for(N), SPEC_THREADS, spec_smem(N)) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int n_tiles = (n_dof + SPEC_DOFS - 1) / SPEC_DOFS;
    return std::max(1, std::min(std::min(SPEC_BLOCKS, n_tiles), per_sm * sm_count()));
}

cudaError_t launch_spectra(qhp_system_s* s, int blocks) {
    const int N = s->n_seg, n_dof = 3 * s->N;
    const size_t sm = spec_smem(N);
#define QHP_SPEC(B)                                                                                             \
    k_qtb_spectra<B><<<blocks, SPEC_THREADS, sm, s->stream>>>(n_dof, N, ilog2(2 * N), s->qtb_dof_type, s->qtb_v, \
                                                              s->qtb_F, s->qtb_tw2, s->qtb_part)
    switch (spec_bpt(N)) {
        case 1: QHP_SPEC(1); break;
        case 2: QHP_SPEC(2); break;
        case 3: QHP_SPEC(3); break;
        default: QHP_SPEC(5); break;
    }
#undef QHP_SPEC
    return cudaGetLastError();
}

int enqueue_filter(qhp_system_s* s) {
    const int N = s->n_seg;
    const double kT = KB * s->temperature;
    const double wcut = s->th.omega_cut_cm > 0.0 ? s->th.omega_cut_cm * CM1 : INFINITY;
    k_qtb_sqrtS<<<(2 * (N + 1) + 127) / 128, 128, 0, s->stream>>>(N, s->th.dt_fs * 1e-3, kT, HBAR, s->th.gamma0,
                                                                  wcut, s->qtb_gamma, s->qtb_sqrtS);
    k_qtb_taps<<<4 * N, TAP_THREADS, 0, s->stream>>>(N, s->qtb_sqrtS, s->qtb_h);
    k_qtb_filter<<<8 * N, TAP_THREADS, 0, s->stream>>>(N, ilog2(4 * N), s->qtb_h, s->qtb_H);
    s->launches += 3;
    QHP_CUDA(cudaGetLastError());
    return QHP_OK;
}

int enqueue_generate(qhp_system_s* s, int64_t seg) {
    const int N = s->n_seg, n_dof = 3 * s->N;
    const int n_pairs = (n_dof + 1) / 2;
    const int grid = (n_pairs + GEN_PAIRS - 1) / GEN_PAIRS;
    k_qtb_generate<<<grid, GEN_THREADS, gen_smem(N), s->stream>>>(n_dof, N, ilog2(4 * N), seg, s->seed, s->qtb_dof_type,
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
        QHP_CUDA(cudaFuncSetAttribute(k_qtb_spectra<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem(2048)));
        QHP_CUDA(cudaFuncSetAttribute(k_qtb_spectra<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem(2048)));
        QHP_CUDA(cudaFuncSetAttribute(k_qtb_spectra<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem(2048)));
        QHP_CUDA(cudaFuncSetAttribute(k_qtb_spectra<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem(2048)));
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
    const int blocks = spectra_blocks(s);
    {
        const cudaError_t e = launch_spectra(s, blocks);
        if (e != cudaSuccess) return e;
    }
    int nO = 0;
    for (int i = 0; i < s->N; ++i) nO += s->type[i] == 0;
    const double n_O = 3.0 * nO, n_H = 3.0 * (s->N - nO);
    const double wavg = exp(-N * s->th.dt_fs * 1e-3 / (s->th.tau_ratio_ps > 0 ? s->th.tau_ratio_ps : 1.0));
    k_qtb_adapt<<<(2 * (N + 1) + 127) / 128, 128, 0, s->stream>>>(
        blocks, N, s->th.dt_fs * 1e-3 / N, s->qtb_part, n_O, n_H, s->ff.m_O, s->ff.m_H, s->th.adapt, s->th.a_gamma,
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
