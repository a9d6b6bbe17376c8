// Device bodies of the per-atom-group stages of a time step, shared by the single-system
// kernels (modes.cu) and the batched one-launch step (forces.cu): the BAOAB integration with
// the bead positions (Eq. (17), Eq. (4)), the force projection (Eqs. (10)-(11)) and the
// batched list check.  A group is APB = 64/P whole atoms on BLOCK = 192 threads, one per
// (atom, dim, mode).  Bar is the group's barrier: the whole block (BlockBar) or, inside the
// one-launch step, the first 192 threads of a larger block (a named barrier).
#pragma once

#include "qhp_internal.cuh"

namespace qhp {
namespace {

struct BlockBar {
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};

constexpr int BLOCK = 192;
struct IntegrateArgs {
    int N, P, apb, n_seg;
    double half_dt_acc, inv_dt;
    uint64_t seed;
    const unsigned long long* step_ctr;
    double *Q, *Pm;
    const double* fmode;
    const int* type;
    const double* tab;     // per (atom type, mode): MT_* entries
    const double* anchor;
    const int* iperm;
    const double* Tm;      // sqrt(P) T[b][n]
    const float* Tmf;
    float4* pos_f4;
    double* pos_d;
    unsigned* dev_max;
    float* dev_atom;       // mixed: per sorted atom, max over beads of |x_ib - A_i|^2 (or null)
    const float* qtb_u;
    float *qtb_v, *qtb_F;
    const int* gate;       // if set, the kernel runs only when *gate != 0
    const double* fmode_s; // RESPA: slow mode forces kicked together with the fast ones
    double ws;             //        with weight ws (n_alt on the first inner step, else 0)
    const unsigned* status;
    long long* fzero;      // batched step: bead forces cleared here, before the forces add into them
};

template <class Bar = BlockBar>
__device__ __forceinline__ void block_max_atomic(float v, unsigned* out) {
    __shared__ float wmax[BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    Bar::sync();
    if (threadIdx.x == 0) {
        float m = wmax[0];
        for (int w = 1; w < BLOCK / 32; ++w) m = fmaxf(m, wmax[w]);
        atomicMax(out, __float_as_uint(m));   // m >= 0: float order == unsigned order
    }
}

// Dot products over the P modes / beads with four independent partial sums (the chains of
// dependent FMAs are what limits these short loops).
__device__ __forceinline__ float dot4(const float* __restrict__ a, int sa, const float* __restrict__ b, int k0,
                                      int k1) {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    int k = k0;
    for (; k + 3 < k1; k += 4) {
        s0 = fmaf(a[k * sa], b[k], s0);
        s1 = fmaf(a[(k + 1) * sa], b[k + 1], s1);
        s2 = fmaf(a[(k + 2) * sa], b[k + 2], s2);
        s3 = fmaf(a[(k + 3) * sa], b[k + 3], s3);
    }
    for (; k < k1; ++k) s0 = fmaf(a[k * sa], b[k], s0);
    return (s0 + s1) + (s2 + s3);
}
__device__ __forceinline__ double dot4(const double* __restrict__ a, int sa, const double* __restrict__ b, int k0,
                                       int k1) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = k0;
    for (; k + 3 < k1; k += 4) {
        s0 = fma(a[k * sa], b[k], s0);
        s1 = fma(a[(k + 1) * sa], b[k + 1], s1);
        s2 = fma(a[(k + 2) * sa], b[k + 2], s2);
        s3 = fma(a[(k + 3) * sa], b[k + 3], s3);
    }
    for (; k < k1; ++k) s0 = fma(a[k * sa], b[k], s0);
    return (s0 + s1) + (s2 + s3);
}

// FP32 <-> FP64 conversions from the bit patterns, on the integer pipes: the integrator's
// limit is its FP64 pipe (the B, A and O updates, 8 FP64 FMAs a mode), which these leave
// alone.  Values equal the hardware conversion's: IEEE round-to-nearest-even for
// double -> float, exact for float -> double.  Zeros, subnormal results, infinities and
// NaNs are left to the hardware conversion.
__device__ __forceinline__ float f64_to_f32(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;                  // biased float exponent
    if (e <= 0 || e >= 255) return (float)x;
    unsigned r = ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;                         // the 29 dropped bits
    r += (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ? 1u : 0u;   // a carry may reach the exponent
    return __uint_as_float((hi & 0x80000000u) | r);
}
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ bool finite_bits(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }

// Exact free flow over dt/2 (Eq. (9) without forces): drift for the centroid, the
// three-shear form of the rotation for n > 0 (determinant one whatever the rounding).
__device__ __forceinline__ void free_half(int n, const double* c, double& q, double& pm) {
    if (n == 0) {
        q += pm * c[MT_SA];
    } else {
        q += c[MT_SA] * pm;
        pm -= c[MT_SB] * q;
        q += c[MT_SA] * pm;
    }
}

// B(dt/2) A(dt/2) O(dt) A(dt/2) on each mode (Eq. (17)), then x = sqrt(P) T Q (Eq. (4)).
// INTEGRATE = false only recomputes bead positions (after a list rebuild or set_modes).
// One block of atoms (bx-th group of apb atoms); load_T = false keeps the transposed
// transform already staged in shared memory by the previous block of the same system.
template <bool MIXED, bool ADQTB, bool INTEGRATE, class Bar = BlockBar>
__device__ __forceinline__ void integrate_body(const IntegrateArgs& A, int bx, unsigned char* smem_raw,
                                               bool load_T) {
    const int P = A.P;
    double* qs = reinterpret_cast<double*>(smem_raw);                 // [BLOCK]
    float* qf = reinterpret_cast<float*>(qs + BLOCK);                 // [BLOCK]
    float* xr = qf + BLOCK;                                           // [BLOCK]
    float* Tsf = reinterpret_cast<float*>(smem_raw + BLOCK * 16);      // [P*P] (mixed), mode-major
    double* Tsd = reinterpret_cast<double*>(smem_raw + BLOCK * 16);    // [P*P] (fp64), mode-major

    const int t = threadIdx.x;
    const int la = t / (3 * P), d = (t / P) % 3, n = t % P;
    const int a = bx * A.apb + la;
    const bool valid = a < A.N;
    const int idx = (a * 3 + d) * P + n;

    __shared__ unsigned dev_s[BLOCK / 3];   // per atom of the group: max squared bead deviation
    if (t < A.apb) dev_s[t] = 0u;
    // transpose to [mode k][bead b] so that the lanes (beads) of a warp read consecutive words
    if (load_T)
        for (int e = t; e < P * P; e += BLOCK) {
            const int b = e / P, k = e % P;
            if (MIXED) Tsf[k * P + b] = A.Tmf[e];
            else Tsd[k * P + b] = A.Tm[e];
        }

    double q = 0.0, pm = 0.0;
    if (valid) {
        q = A.Q[idx];
        pm = A.Pm[idx];
        if (INTEGRATE) {
            const double* c = A.tab + ((size_t)A.type[a] * P + n) * MT_N;
            const unsigned long long step = *A.step_ctr;
            double f = A.fmode[idx];
            if (A.fmode_s) f += A.ws * A.fmode_s[idx];                // RESPA: B_s(n dt/2) B_f(dt/2)
            pm += A.half_dt_acc * f;                                  // B
            free_half(n, c, q, pm);                                   // A
            if (ADQTB) {                                              // O with colored noise
                const int dof = a * 3 + d;
                const int ms = (int)(step % (unsigned long long)A.n_seg);
                const size_t r = (size_t)ms * (size_t)(3 * A.N) + dof;
                const double kick = c[MT_AMP] * f32_to_f64(A.qtb_u[r]);
                const double pnew = c[MT_C1] * pm + kick;
                A.qtb_v[r] = f64_to_f32((pm + pnew) * c[MT_INV2M]);
                A.qtb_F[r] = f64_to_f32(kick * A.inv_dt);
                pm = pnew;
            } else {                                                  // O with white noise
                const uint4 x = philox_draw(A.seed, (uint32_t)idx, step, TAG_OSTEP);
                if (MIXED) {   // FP32 normal, widened once; the thermostat update itself is FP64
                    pm = fma(c[MT_AMP], f32_to_f64(normal_f32(x, 0)), c[MT_C1] * pm);
                } else {
                    pm = c[MT_C1] * pm + c[MT_AMP] * normal_f64(x, 0);
                }
            }
            free_half(n, c, q, pm);                                   // A
            A.Q[idx] = q;
            A.Pm[idx] = pm;
            if (A.fzero) A.fzero[idx] = 0;
        }
    }
    qs[t] = q;
    // mixed: the centroid slot carries the bead-independent FP64 centroid offset, rounded
    // once; the other slots the FP32 modes for the fluctuation sum
    if (MIXED) qf[t] = (n == 0) ? (valid ? f64_to_f32(q - A.anchor[a * 3 + d]) : 0.0f) : f64_to_f32(q);
    Bar::sync();

    float dv = 0.0f;
    if (valid) {
        const int base = la * 3 * P + d * P;
        if (MIXED) {
            // FP64 centroid offset + FP32 fluctuation sum: the bead position only feeds the
            // FP32 pair kernel, where 1e-7 relative on sub-Angstrom fluctuations is far
            // below the pair arithmetic's own rounding.
            float acc = 0.0f;
            acc = dot4(Tsf + n, P, qf + base, 1, P);
            xr[t] = qf[base] + acc;
        } else {
            double acc = 0.0;
            acc = dot4(Tsd + n, P, qs + base, 0, P);
            if (QHP_IN_BOUNDS(A.iperm[a], A.N, A.status)) A.pos_d[((size_t)d * A.N + A.iperm[a]) * P + n] = acc;
            xr[t] = f64_to_f32(acc - A.anchor[a * 3 + d]);
        }
    }
    Bar::sync();
    // mixed: the pair kernel's bead-pair records (bead_word layout), one component per thread
    if (MIXED && valid && QHP_IN_BOUNDS(A.iperm[a], A.N, A.status))
        reinterpret_cast<float*>(A.pos_f4)[bead_word(A.iperm[a], n, d, P)] = xr[t];
    if (valid && d == 0) {
        const int base = la * 3 * P;
        const float x0 = xr[base + n], x1 = xr[base + P + n], x2 = xr[base + 2 * P + n];
        dv = x0 * x0 + x1 * x1 + x2 * x2;
        if (A.dev_atom) atomicMax(&dev_s[la], __float_as_uint(dv));   // dv >= 0: float order == unsigned order
    }
    block_max_atomic<Bar>(dv, A.dev_max);   // ends with a barrier
    if (A.dev_atom && t < A.apb) {
        const int a2 = bx * A.apb + t;
        if (a2 < A.N && QHP_IN_BOUNDS(A.iperm[a2], A.N, A.status)) A.dev_atom[A.iperm[a2]] = __uint_as_float(dev_s[t]);
    }
}

__device__ __forceinline__ void batch_check(const CheckArgs& a) {
    const float dmax = __uint_as_float(atomicAdd(a.dev_max, 0u));   // coherent read of the blocks' maxima
    const int rebuild = !(dmax <= a.thr2);                          // NaN also triggers a rebuild
    *a.flag = rebuild;
    if (rebuild) {
        *a.dev_max = 0u;
        a.rebuild_count[0] += 1u;
        a.rebuild_count[1] += 1u;
    }
    cudaGraphSetConditional(a.cond, rebuild ? 1u : 0u);
}

struct ProjectArgs {
    int N, P, apb;
    double half_dt_acc;
    const double* Fd;
    const long long* Ffix;
    const double* Tp;      // T[b][n] / sqrt(P)
    const float* Tpf;
    double* fmode;
    double* Pm;
    unsigned* status;
    unsigned long long* step_ctr;
};

// f_n = (1/sqrt P) sum_b T_bn F_b (Eqs. (10)-(11)) and, with KICK, B(dt/2) P_n += dt/2 f_n.
template <bool MIXED, bool KICK, class Bar = BlockBar>
__device__ __forceinline__ void project_body(const ProjectArgs& A, int bx, unsigned char* smem_raw, bool load_T) {
    __shared__ double Fs[BLOCK];
    __shared__ long long Fi[BLOCK];
    __shared__ float Ff[BLOCK];
    const int P = A.P;
    float* Tsf = reinterpret_cast<float*>(smem_raw);
    double* Tsd = reinterpret_cast<double*>(smem_raw);
    const int t = threadIdx.x;
    const int la = t / (3 * P), d = (t / P) % 3, n = t % P;
    const int a = bx * A.apb + la;
    const bool valid = a < A.N;
    const int idx = (a * 3 + d) * P + n;
    if (load_T)
        for (int k = t; k < P * P; k += BLOCK) {
            if (MIXED) Tsf[k] = A.Tpf[k];
            else Tsd[k] = A.Tp[k];
        }
    long long v = 0;
    if (valid) {
        if (MIXED) {
            v = A.Ffix[idx];
            Fi[t] = v;
            Ff[t] = __ll2float_rn(v) * (1.0f / FIX_SCALE_F);   // one conversion per bead force
        } else {
            Fs[t] = A.Fd[idx];
        }
    }
    // f_0 = mean bead force: exact integer sum of the fixed-point forces; with P <= 32 the
    // P lanes of an (atom, dim) are an aligned group of one warp and add by shuffles
    if (MIXED && P <= 32)
        for (int off = 1; off < P; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    Bar::sync();
    if (valid) {
        const int base = la * 3 * P + d * P;
        double f;
        if (MIXED) {
            if (n == 0) {
                long long sum = v;
                if (P > 32) {
                    sum = 0;
                    for (int b = 0; b < P; ++b) sum += Fi[base + b];
                }
                f = (double)sum * (1.0 / (FIX_SCALE * (double)P));   // power of two: exact scaling
            } else {
                float acc = 0.0f;
                acc = dot4(Tsf + n, P, Ff + base, 0, P);
                f = f32_to_f64(acc);
            }
        } else {
            double acc = 0.0;
            acc = dot4(Tsd + n, P, Fs + base, 0, P);
            f = acc;
        }
        A.fmode[idx] = f;
        if (KICK) {
            const double p = A.Pm[idx] + A.half_dt_acc * f;
            A.Pm[idx] = p;
            if (!finite_bits(p)) atomicOr(A.status, ST_NONFINITE);
        }
    }
    if (KICK && bx == 0 && t == 0) *A.step_ctr += 1ull;
}

}  // namespace
}  // namespace qhp
