// Differentiation of the RPMD time step (FP64).
//
// * Gradients of U_P = (1/P) sum_b V(x_b) (Eq. (3)) with respect to the bead positions
//   and the force-field parameters theta = (eps, sigma, q_O, k_b, k_theta), q_H = -q_O/2.
// * The adjoint of a K-step BAOAB segment (Eq. (17)) with the thermostat noise held
//   fixed (same Philox counters), for the time average J = (1/K) sum_{k=1..K} a(Q_k) of
//   an observable: 0 = the potential energy at the centroid V(Q_0), 1 = the mean O-H
//   bond length over beads and bonds.  The forward trajectory is replayed from
//   checkpoints taken every `block` steps, so memory grows with block, not with K.
//
// One set of pair and bonded kernels serves everything: they are templates over the
// scalar type, instantiated with double (forces, energy and dU/dtheta) and with a dual
// number (value, derivative along a direction v), whose derivative part gives the
// Hessian-vector product -H v of the forces and d/dt dU/dtheta(x + t v) exactly, as
// the adjoint needs.
//
// Adjoint of one step (state (Q, P) after step k; h = dt/2 in force units; f = f(Q)
// the projected forces, symmetric Jacobian df/dQ = -d^2 U_P/dQ^2):
//     P' = P_{k-1} + h f(Q_{k-1});  (Q'', P'') = A(Q_{k-1}, P');  P''' = c1 P'' + noise;
//     (Q_k, P'''') = A(Q'', P''');  P_k = P'''' + h f(Q_k)
// backwards: lamQ_k += h (df/dQ)^T lamP_k (end of step k) and the same again from the
// start of step k + 1 (both use lamP_k), i.e. 2h for 0 < k < K; then A^T, c1, A^T.
// theta collects h (df/dtheta)^T lamP at the same points plus da/dtheta.
#include <math.h>

#include <vector>

#include "qhp_internal.cuh"

namespace qhp {

namespace {

// ------------------------------------------------------------------ dual numbers
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator/(double s, Dual b) {
    const double q = s / b.v;
    return {q, -q * b.d / b.v};
}
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(Dual x) { return x.v; }
__device__ __forceinline__ double der(double) { return 0.0; }
__device__ __forceinline__ double der(Dual x) { return x.d; }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ Dual sqrt_(Dual a) {
    const double r = sqrt(a.v);
    return {r, 0.5 * a.d / r};
}
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ Dual exp_(Dual a) {
    const double e = exp(a.v);
    return {e, e * a.d};
}
// d erfc(x)/dx = -(2/sqrt(pi)) exp(-x^2)
__device__ __forceinline__ double erfc_(double x) { return erfc(x); }
__device__ __forceinline__ Dual erfc_(Dual a) {
    return {erfc(a.v), -1.1283791670955126 * exp(-a.v * a.v) * a.d};
}
// d acos(x)/dx = -1/sqrt(1 - x^2)
__device__ __forceinline__ double acos_(double x) { return acos(fmin(1.0, fmax(-1.0, x))); }
__device__ __forceinline__ Dual acos_(Dual a) {
    return {acos(fmin(1.0, fmax(-1.0, a.v))), -a.d / sqrt(fmax(1e-300, 1.0 - a.v * a.v))};
}

template <class S>
__device__ __forceinline__ S load(const double* x, const double* v, size_t k);
template <>
__device__ __forceinline__ double load<double>(const double* x, const double*, size_t k) { return x[k]; }
template <>
__device__ __forceinline__ Dual load<Dual>(const double* x, const double* v, size_t k) { return {x[k], v[k]}; }
// shift a separation by whole boxes: the shift is a constant, the derivative is unchanged
__device__ __forceinline__ void shift(double& a, double s) { a -= s; }
__device__ __forceinline__ void shift(Dual& a, double s) { a.v -= s; }
__device__ __forceinline__ double reduce_warp(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

struct GradConsts {
    double L, invL, rc, rc2, alpha, c2a, sc, ecut, ke;
    double eps, sig, qO, lj12, lj6;   // lj12, lj6: (sigma/rc)^12, (sigma/rc)^6
    double kb, r0, kth, th0;
};

constexpr int NPART = 4;    // per (atom, bead): E, dE/deps, dE/dsigma, dE/dq_O
constexpr int NPARTB = 3;   // per (molecule, bead): E, dE/dk_b, dE/dk_theta

// Nonbonded terms, warp per (sorted atom i, bead b), lanes over i's list row.  F_i is
// written (value, and its derivative when S = Dual); partials hold half of every pair
// term (each pair is met from both ends): part[w][0..3] values, [4..7] derivatives.
template <class S>
__global__ void __launch_bounds__(128) k_grad_pairs(int N, int Pk, const double* __restrict__ x,
                                                    const double* __restrict__ v, const int* __restrict__ start,
                                                    const int* __restrict__ count, const int4* __restrict__ nbr,
                                                    const int* __restrict__ type_s, GradConsts c,
                                                    double* __restrict__ F, double* __restrict__ Ft,
                                                    double* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= N * Pk) return;
    const int i = w / Pk, b = w % Pk;
    S xi[3];
    for (int d = 0; d < 3; ++d) xi[d] = load<S>(x, v, ((size_t)d * N + i) * Pk + b);
    const bool Oi = type_s[i] == 0;
    const double ci = Oi ? 1.0 : -0.5;
    S f[3] = {S{}, S{}, S{}}, e{}, ge{}, gs{}, gq{};
    const int k0 = start[i], k1 = k0 + count[i];
    for (int k = k0 + lane; k < k1; k += 32) {
        const int ex = nbr[k].x;
        const int j = entry_partner(ex);
        const bool Oj = ex >= 0;   // bit 31 marks an H partner
        S dd[3];
        for (int d = 0; d < 3; ++d) {
            dd[d] = load<S>(x, v, ((size_t)d * N + j) * Pk + b) - xi[d];
            shift(dd[d], c.L * rint(val(dd[d]) * c.invL));
        }
        const S r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
        if (!(val(r2) < c.rc2)) continue;
        const S r = sqrt_(r2);
        const S rinv = 1.0 / r;
        const S ar = c.alpha * r;
        const S er = erfc_(ar);
        const S gauss = exp_(-(ar * ar));
        const double cc = ci * (Oj ? 1.0 : -0.5);
        const double qq = c.ke * c.qO * c.qO * cc;
        const S bracket = er * rinv - c.ecut + c.sc * (r - c.rc);   // DSF pair energy / qq
        S ep = qq * bracket;
        S g = qq * (er * rinv * rinv + c.c2a * gauss * rinv - c.sc) * rinv;   // -V'(r)/r
        gq = gq + (2.0 * c.ke * c.qO * cc) * bracket;
        if (Oi && Oj) {
            const S s2 = (c.sig * c.sig) * (rinv * rinv);
            const S s6 = s2 * s2 * s2;
            const S s12 = s6 * s6;
            ep = ep + 4.0 * c.eps * (s12 - s6) - 4.0 * c.eps * (c.lj12 - c.lj6);
            g = g + 24.0 * c.eps * (2.0 * s12 - s6) * (rinv * rinv);
            ge = ge + 4.0 * (s12 - s6) - 4.0 * (c.lj12 - c.lj6);
            gs = gs + (4.0 * c.eps / c.sig) * ((12.0 * s12 - 6.0 * s6) - (12.0 * c.lj12 - 6.0 * c.lj6));
        }
        for (int d = 0; d < 3; ++d) f[d] = f[d] - g * dd[d];
        e = e + ep;
    }
    double out[2 * (3 + NPART)];
    const S acc[3 + NPART] = {f[0], f[1], f[2], e, ge, gs, gq};
    for (int q = 0; q < 3 + NPART; ++q) {
        out[q] = reduce_warp(val(acc[q]));
        out[3 + NPART + q] = reduce_warp(der(acc[q]));
    }
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) {
            F[((size_t)d * N + i) * Pk + b] = out[d];
            if (Ft) Ft[((size_t)d * N + i) * Pk + b] = out[3 + NPART + d];
        }
        for (int q = 0; q < NPART; ++q) {
            part[(size_t)w * 2 * NPART + q] = 0.5 * out[3 + q];
            part[(size_t)w * 2 * NPART + NPART + q] = 0.5 * out[3 + NPART + 3 + q];
        }
    }
}

// Bonds and angle per (molecule, bead): forces added to F (and Ft), partials per thread.
template <class S>
__global__ void k_grad_bonded(int n_mol, int N, int Pk, const double* __restrict__ x, const double* __restrict__ v,
                              const int* __restrict__ iperm, GradConsts c, double* __restrict__ F,
                              double* __restrict__ Ft, double* __restrict__ partb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_mol * Pk) return;
    const int m = t / Pk, b = t % Pk;
    const int sO = iperm[3 * m], s1 = iperm[3 * m + 1], s2 = iperm[3 * m + 2];
    S d1[3], d2[3];
    for (int d = 0; d < 3; ++d) {
        const S xo = load<S>(x, v, ((size_t)d * N + sO) * Pk + b);
        d1[d] = load<S>(x, v, ((size_t)d * N + s1) * Pk + b) - xo;
        d2[d] = load<S>(x, v, ((size_t)d * N + s2) * Pk + b) - xo;
        shift(d1[d], c.L * rint(val(d1[d]) * c.invL));
        shift(d2[d], c.L * rint(val(d2[d]) * c.invL));
    }
    const S r1 = sqrt_(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
    const S r2 = sqrt_(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
    const S ir12 = 1.0 / (r1 * r2);
    S cs = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) * ir12;
    const S th = acos_(cs);
    const S sn = sqrt_(1.0 - cs * cs);
    const S u1 = r1 - c.r0, u2 = r2 - c.r0, uth = th - c.th0;
    const S pb1 = -c.kb * u1 / r1, pb2 = -c.kb * u2 / r2;   // bond force / r along d
    const S pa = c.kth * uth / sn;                           // angle: k (th - th0) / sin(th)
    const S ir1s = 1.0 / (r1 * r1), ir2s = 1.0 / (r2 * r2);
    for (int d = 0; d < 3; ++d) {
        const S f1 = pb1 * d1[d] + pa * (d2[d] * ir12 - cs * d1[d] * ir1s);
        const S f2 = pb2 * d2[d] + pa * (d1[d] * ir12 - cs * d2[d] * ir2s);
        const S fo = -(f1 + f2);
        const size_t k1 = ((size_t)d * N + s1) * Pk + b, k2 = ((size_t)d * N + s2) * Pk + b,
                     ko = ((size_t)d * N + sO) * Pk + b;
        F[k1] += val(f1);
        F[k2] += val(f2);
        F[ko] += val(fo);
        if (Ft) {
            Ft[k1] += der(f1);
            Ft[k2] += der(f2);
            Ft[ko] += der(fo);
        }
    }
    const S sb = 0.5 * (u1 * u1 + u2 * u2);
    const S sa = 0.5 * (uth * uth);
    const S en = c.kb * sb + c.kth * sa;
    const S acc[NPARTB] = {en, sb, sa};
    for (int q = 0; q < NPARTB; ++q) {
        partb[(size_t)t * 2 * NPARTB + q] = val(acc[q]);
        partb[(size_t)t * 2 * NPARTB + NPARTB + q] = der(acc[q]);
    }
}

// out[c] = sum over rows of in[r * cols + c], one block per column, fixed order.
__global__ void k_colsum(const double* __restrict__ in, int rows, int cols, double* __restrict__ out) {
    __shared__ double sh[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < rows; r += 256) s += in[(size_t)r * cols + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

// x_b = sum_n Tm[b][n] Q_n (Eq. (4)); out [3][N][P] in sorted atom order.
__global__ void k_modes_to_x(int N, int P, const double* __restrict__ Q, const double* __restrict__ Tm,
                             const int* __restrict__ iperm, double* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3 * P) return;
    const int b = idx % P, dof = idx / P, a = dof / 3, d = dof % 3;
    double acc = 0.0;
    for (int n = 0; n < P; ++n) acc = fma(Tm[b * P + n], Q[(size_t)dof * P + n], acc);
    out[((size_t)d * N + iperm[a]) * P + b] = acc;
}

// Q_n = (1/P) sum_b Tm[b][n] x_b (inverse of Eq. (4)); x [P][N][3] in atom order.
__global__ void k_beads_to_modes(int N, int P, const double* __restrict__ x, const double* __restrict__ Tm,
                                 double* __restrict__ Q) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3 * P) return;
    const int n = idx % P, dof = idx / P, a = dof / 3, d = dof % 3;
    double acc = 0.0;
    for (int b = 0; b < P; ++b) acc = fma(Tm[b * P + n], x[((size_t)b * N + a) * 3 + d], acc);
    Q[idx] = acc / P;
}

// out[(a*3+d)*P + n] (+)= scale * sum_b Tm[b][n] G[d][iperm[a]][b]
__global__ void k_project_g(int N, int P, const double* __restrict__ G, const double* __restrict__ Tm,
                            const int* __restrict__ iperm, double scale, int accumulate, double* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3 * P) return;
    const int n = idx % P, dof = idx / P, a = dof / 3, d = dof % 3;
    const double* g = G + ((size_t)d * N + iperm[a]) * P;
    double acc = 0.0;
    for (int b = 0; b < P; ++b) acc = fma(Tm[b * P + n], g[b], acc);
    out[idx] = accumulate ? out[idx] + scale * acc : scale * acc;
}

// out[(b*N + a)*3 + d] = scale * G[d][iperm[a]][b]
__global__ void k_sorted_to_beads(int N, int P, const double* __restrict__ G, const int* __restrict__ iperm,
                                  double scale, double* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3 * P) return;
    const int d = idx % 3, a = (idx / 3) % N, b = idx / (3 * N);
    out[idx] = scale * G[((size_t)d * N + iperm[a]) * P + b];
}

// centroid configuration x1 [3][N] (sorted) = Q_0
__global__ void k_centroid_x(int N, int P, const double* __restrict__ Q, const int* __restrict__ iperm,
                             double* __restrict__ x1) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3) return;
    const int a = idx / 3, d = idx % 3;
    x1[(size_t)d * N + iperm[a]] = Q[(size_t)idx * P];
}

// lamQ[a][d][0] += w * (-F1): the gradient of V(Q_0) with respect to the centroid mode
__global__ void k_add_centroid_grad(int N, int P, const double* __restrict__ F1, const int* __restrict__ iperm,
                                    double w, double* __restrict__ lamQ) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3) return;
    const int a = idx / 3, d = idx % 3;
    lamQ[(size_t)idx * P] -= w * F1[(size_t)d * N + iperm[a]];
}

// O-H lengths per (molecule, bead) and w * their gradient in G [3][N][P] (sorted; zeroed before)
__global__ void k_oh_grad(int n_mol, int N, int P, const double* __restrict__ x, const int* __restrict__ iperm,
                          double L, double w, double* __restrict__ G, double* __restrict__ parto) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_mol * P) return;
    const int m = t / P, b = t % P;
    const int sO = iperm[3 * m];
    double sum = 0.0;
    for (int h = 1; h <= 2; ++h) {
        const int sh = iperm[3 * m + h];
        double dd[3];
        for (int d = 0; d < 3; ++d) {
            dd[d] = x[((size_t)d * N + sh) * P + b] - x[((size_t)d * N + sO) * P + b];
            dd[d] -= L * rint(dd[d] / L);
        }
        const double r = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        sum += r;
        for (int d = 0; d < 3; ++d) {
            G[((size_t)d * N + sh) * P + b] += w * dd[d] / r;
            G[((size_t)d * N + sO) * P + b] -= w * dd[d] / r;
        }
    }
    parto[t] = sum;
}

// Transpose of the exact free flow A(dt/2) of one mode (the three shears in reverse order).
__device__ __forceinline__ void free_half_adjoint(int n, const double* c, double& lq, double& lp) {
    if (n == 0) {
        lp += c[MT_SA] * lq;
    } else {
        lp += c[MT_SA] * lq;
        lq -= c[MT_SB] * lp;
        lp += c[MT_SA] * lq;
    }
}

// Backward through A, O, A of one step: (lamQ, lamP) <- A^T c1 A^T (lamQ, lamP).
__global__ void k_adj_linear(int N, int P, const int* __restrict__ type, const double* __restrict__ tab,
                             double* __restrict__ lamQ, double* __restrict__ lamP) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3 * P) return;
    const int n = idx % P, a = idx / (3 * P);
    const double* c = tab + ((size_t)type[a] * P + n) * MT_N;
    double lq = lamQ[idx], lp = lamP[idx];
    free_half_adjoint(n, c, lq, lp);
    lp *= c[MT_C1];
    free_half_adjoint(n, c, lq, lp);
    lamQ[idx] = lq;
    lamP[idx] = lp;
}

// acc[1 + k] += scale * s[k] for the five parameter slots taken from the column sums.
//   sums[0..7]: pair partials (E, eps, sigma, q) values then derivatives;
//   sums[8..13]: bonded partials (E, k_b, k_theta) values then derivatives.
// which = 0 takes values, 1 derivatives; e_scale adds scale_e * (E_pair + E_bond + e_add) to
// acc[0]; dq_add is added to the q_O slot (self term).
__global__ void k_accumulate(const double* __restrict__ sums, int which, double scale, double scale_e, double e_add,
                             double dq_add, double* __restrict__ acc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int o = which ? NPART : 0, ob = which ? NPARTB : 0;
    const double* sp = sums;
    const double* sb = sums + 2 * NPART;
    acc[0] += scale_e * (sp[o + 0] + sb[ob + 0] + e_add);
    acc[1] += scale * sp[o + 1];
    acc[2] += scale * sp[o + 2];
    acc[3] += scale * (sp[o + 3] + dq_add);
    acc[4] += scale * sb[ob + 1];
    acc[5] += scale * sb[ob + 2];
}

__global__ void k_accumulate_value(const double* __restrict__ sums, double scale, double* __restrict__ acc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) acc[0] += scale * sums[0];
}

// ------------------------------------------------------------------ host side

int grad_prepare(qhp_system_s* s, int qbuf_steps) {
    GradBuffers& g = s->grad;
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    if (!g.ready) {
        TRY(dalloc(s, &g.x, NP3));
        TRY(dalloc(s, &g.v, NP3));
        TRY(dalloc(s, &g.F, NP3));
        TRY(dalloc(s, &g.Ft, NP3));
        TRY(dalloc(s, &g.part, (size_t)s->N * s->P * 2 * NPART));
        TRY(dalloc(s, &g.partb, (size_t)s->n_mol * s->P * 2 * NPARTB));
        TRY(dalloc(s, &g.x1, (size_t)s->N * 3));
        TRY(dalloc(s, &g.F1, (size_t)s->N * 3));
        TRY(dalloc(s, &g.part1, (size_t)s->N * 2 * NPART));
        TRY(dalloc(s, &g.partb1, (size_t)s->n_mol * 2 * NPARTB));
        TRY(dalloc(s, &g.G, NP3));
        TRY(dalloc(s, &g.parto, (size_t)s->n_mol * s->P));
        TRY(dalloc(s, &g.lamQ, NP3));
        TRY(dalloc(s, &g.lamP, NP3));
        TRY(dalloc(s, &g.sums, 32));
        TRY(dalloc(s, &g.acc, 8));
        g.ready = true;
    }
    if (qbuf_steps > g.qbuf_steps) {
        TRY(dalloc(s, &g.Qbuf, NP3 * (size_t)(qbuf_steps + 1)));
        g.qbuf_steps = qbuf_steps;
    }
    return QHP_OK;
}

GradConsts grad_consts(const qhp_system_s* s, const double* theta = nullptr) {
    qhp_ff f = s->ff;
    if (theta) {   // another parameter set (eps, sigma, q_O, k_b, k_theta) on the same system
        f.eps = theta[0];
        f.sigma = theta[1];
        f.q_O = theta[2];
        f.k_b = theta[3];
        f.k_theta = theta[4];
    }
    GradConsts c;
    const double rc = f.rc, a = f.alpha;
    c.L = s->L;
    c.invL = 1.0 / s->L;
    c.rc = rc;
    c.rc2 = rc * rc;
    c.alpha = a;
    c.c2a = 2.0 * a / sqrt(M_PI);
    c.sc = erfc(a * rc) / (rc * rc) + c.c2a * exp(-(a * rc) * (a * rc)) / rc;
    c.ecut = erfc(a * rc) / rc;
    c.ke = COULOMB;
    c.eps = f.eps;
    c.sig = f.sigma;
    c.qO = f.q_O;
    const double s6 = pow(f.sigma / rc, 6.0);
    c.lj6 = s6;
    c.lj12 = s6 * s6;
    c.kb = f.k_b;
    c.r0 = f.r0;
    c.kth = f.k_theta;
    c.th0 = f.theta0;
    return c;
}

// DSF self energy -(erfc(a rc)/(2 rc) + a/sqrt(pi)) k_e q_O^2 sum_i c_i^2 = coef * q_O^2.
double self_coef(const qhp_system_s* s) {
    const double a = s->ff.alpha, rc = s->ff.rc;
    double c2 = 0.0;
    for (int i = 0; i < s->N; ++i) c2 += s->type[i] == 0 ? 1.0 : 0.25;
    return -(erfc(a * rc) / (2.0 * rc) + a / sqrt(M_PI)) * COULOMB * c2;
}

inline int blocks(int64_t n, int tb) { return (int)((n + tb - 1) / tb); }

// out[0] = sum over rows b, b + stride, ... of column col (one bead's rows of a partial array)
__global__ void k_colsum_stride(const double* __restrict__ in, int rows, int stride, int cols, int col,
                                double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int r = threadIdx.x * stride; r < rows; r += 256 * stride) s += in[(size_t)r * cols + col];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// Pair + bonded terms at the configuration in g.x (Pk beads; with tangent g.v when dual),
// then the column sums of both partial arrays into g.sums[0..13].
cudaError_t eval_terms(qhp_system_s* s, int Pk, bool dual, const double* x, const double* v, double* F, double* Ft,
                       double* part, double* partb, const double* theta = nullptr) {
    GradBuffers& g = s->grad;
    const GradConsts c = grad_consts(s, theta);
    const int N = s->N;
    const int warps = N * Pk;
    if (dual)
        k_grad_pairs<Dual><<<blocks((int64_t)warps * 32, 128), 128, 0, s->stream>>>(
            N, Pk, x, v, s->nbr_start, s->nbr_count, s->nbr, s->type_s, c, F, Ft, part);
    else
        k_grad_pairs<double><<<blocks((int64_t)warps * 32, 128), 128, 0, s->stream>>>(
            N, Pk, x, nullptr, s->nbr_start, s->nbr_count, s->nbr, s->type_s, c, F, nullptr, part);
    const int nt = s->n_mol * Pk;
    if (dual)
        k_grad_bonded<Dual><<<blocks(nt, 128), 128, 0, s->stream>>>(s->n_mol, N, Pk, x, v, s->iperm, c, F, Ft, partb);
    else
        k_grad_bonded<double><<<blocks(nt, 128), 128, 0, s->stream>>>(s->n_mol, N, Pk, x, nullptr, s->iperm, c, F,
                                                                      nullptr, partb);
    k_colsum<<<2 * NPART, 256, 0, s->stream>>>(part, N * Pk, 2 * NPART, g.sums);
    k_colsum<<<2 * NPARTB, 256, 0, s->stream>>>(partb, nt, 2 * NPARTB, g.sums + 2 * NPART);
    s->launches += 4;
    return cudaGetLastError();
}

// The list must cover the configuration about to be evaluated: it is rebuilt around the
// current modes (the rows depend on the centroids in both list modes).
int ensure_list_for_current_modes(qhp_system_s* s) { return rebuild_list_now(s); }

// Hessian-vector product at the modes Qk along lamP with weight w:
//   lamQ += w (df/dQ)^T lamP,  acc[1..5] += w (df/dtheta)^T lamP.
int hvp(qhp_system_s* s, const double* Qk, double w) {
    GradBuffers& g = s->grad;
    const int N = s->N, P = s->P;
    const int64_t n = (int64_t)N * 3 * P;
    k_modes_to_x<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, Qk, s->Tmat, s->iperm, g.x);
    k_modes_to_x<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, g.lamP, s->Tmat, s->iperm, g.v);
    s->launches += 2;
    QHP_CUDA(eval_terms(s, P, true, g.x, g.v, g.F, g.Ft, g.part, g.partb));
    // f_n = (1/P) sum_b Tm[b][n] F_b, so (df/dQ) lamP = (1/P) sum_b Tm[b][n] dF_b
    k_project_g<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, g.Ft, s->Tmat, s->iperm, w / P, 1, g.lamQ);
    // (df/dtheta)^T lamP = -d/dt dU_P/dtheta (x + t v)
    k_accumulate<<<1, 32, 0, s->stream>>>(g.sums, 1, -w / P, 0.0, 0.0, 0.0, g.acc);
    s->launches += 2;
    QHP_CUDA(cudaGetLastError());
    return QHP_OK;
}

// Observable a at the modes Qk with weight wK (= 1/K): acc[0] += wK a, lamQ += wK da/dQ,
// acc[1..5] += wK da/dtheta.
int observe(qhp_system_s* s, const double* Qk, int which, double wK, double scoef) {
    GradBuffers& g = s->grad;
    const int N = s->N, P = s->P;
    const int64_t n = (int64_t)N * 3 * P;
    if (which == 0) {
        k_centroid_x<<<blocks((int64_t)N * 3, 256), 256, 0, s->stream>>>(N, P, Qk, s->iperm, g.x1);
        s->launches++;
        QHP_CUDA(eval_terms(s, 1, false, g.x1, nullptr, g.F1, nullptr, g.part1, g.partb1));
        const double qO = s->ff.q_O;
        k_accumulate<<<1, 32, 0, s->stream>>>(g.sums, 0, wK, wK, scoef * qO * qO, 2.0 * scoef * qO, g.acc);
        k_add_centroid_grad<<<blocks((int64_t)N * 3, 256), 256, 0, s->stream>>>(N, P, g.F1, s->iperm, wK, g.lamQ);
        s->launches += 2;
    } else {
        const double wa = 1.0 / (2.0 * s->n_mol * P);   // mean over beads and bonds
        k_modes_to_x<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, Qk, s->Tmat, s->iperm, g.x);
        QHP_CUDA(cudaMemsetAsync(g.G, 0, sizeof(double) * n, s->stream));
        k_oh_grad<<<blocks((int64_t)s->n_mol * P, 128), 128, 0, s->stream>>>(s->n_mol, N, P, g.x, s->iperm, s->L,
                                                                             wK * wa, g.G, g.parto);
        k_colsum<<<1, 256, 0, s->stream>>>(g.parto, s->n_mol * P, 1, g.sums + 16);
        k_accumulate_value<<<1, 32, 0, s->stream>>>(g.sums + 16, wK * wa, g.acc);
        // da/dQ_n = sum_b Tm[b][n] da/dx_b
        k_project_g<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, g.G, s->Tmat, s->iperm, 1.0, 1, g.lamQ);
        s->launches += 5;
    }
    QHP_CUDA(cudaGetLastError());
    return QHP_OK;
}

int load_modes(qhp_system_s* s, const double* Qk) {
    QHP_CUDA(cudaMemcpyAsync(s->Q, Qk, sizeof(double) * (size_t)s->N * 3 * s->P, cudaMemcpyDeviceToDevice,
                             s->stream));
    s->forces_valid = false;
    s->list_valid = false;
    return ensure_list_for_current_modes(s);
}

}  // namespace

}  // namespace qhp

using namespace qhp;

extern "C" {

int qhp_energy_grad_device(qhp_sys s, const double* x, double* energy, double* dE_dx, double* dE_dtheta) {
    TraceRange tr("qhp_energy_grad_device");
    if (!s || !s->beads_set) {
        set_error("qhp_energy_grad: system not initialised");
        return QHP_ERR_STATE;
    }
    TRY(grad_prepare(s, 0));
    GradBuffers& g = s->grad;
    const int N = s->N, P = s->P;
    const int64_t n = (int64_t)N * 3 * P;
    if (x) {
        // the bead positions become the system's state (momenta kept)
        k_beads_to_modes<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, x, s->Tmat, s->Q);
        s->launches++;
        QHP_CUDA(cudaGetLastError());
        s->forces_valid = false;
        s->list_valid = false;
    }
    TRY(ensure_list_for_current_modes(s));
    k_modes_to_x<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, s->Q, s->Tmat, s->iperm, g.x);
    s->launches++;
    QHP_CUDA(eval_terms(s, P, false, g.x, nullptr, g.F, nullptr, g.part, g.partb));
    QHP_CUDA(cudaMemsetAsync(g.acc, 0, sizeof(double) * 8, s->stream));
    const double sc = self_coef(s), qO = s->ff.q_O;
    // U_P = (1/P) sum_b V(x_b); the self term is the same for every bead
    k_accumulate<<<1, 32, 0, s->stream>>>(g.sums, 0, 1.0 / P, 1.0 / P, P * sc * qO * qO, P * 2.0 * sc * qO, g.acc);
    s->launches++;
    if (dE_dx) {
        k_sorted_to_beads<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, g.F, s->iperm, -1.0 / P, dE_dx);
        s->launches++;
    }
    QHP_CUDA(cudaGetLastError());
    double acc[6];
    QHP_CUDA(cudaMemcpyAsync(acc, g.acc, sizeof acc, cudaMemcpyDeviceToHost, s->stream));
    QHP_CUDA(cudaStreamSynchronize(s->stream));
    if (energy) *energy = acc[0];
    if (dE_dtheta)
        for (int k = 0; k < 5; ++k) dE_dtheta[k] = acc[1 + k];
    return QHP_OK;
}

int qhp_energy_grad(qhp_sys s, double* energy, double* dE_dx, double* dE_dtheta) {
    if (!s || !s->beads_set) {
        set_error("qhp_energy_grad: system not initialised");
        return QHP_ERR_STATE;
    }
    double* dev = nullptr;
    const size_t n = (size_t)s->N * 3 * s->P;
    if (dE_dx) {
        TRY(grad_prepare(s, 0));
        dev = s->grad.G;
    }
    TRY(qhp_energy_grad_device(s, nullptr, energy, dev, dE_dtheta));
    if (dE_dx) QHP_CUDA(cudaMemcpy(dE_dx, dev, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return QHP_OK;
}

int qhp_state_energies(qhp_sys s, const double* theta_A, const double* theta_B, double* out) {
    if (!s || !s->beads_set || !theta_A || !theta_B || !out) {
        set_error("qhp_state_energies: need an initialised system and two parameter sets");
        return QHP_ERR_ARG;
    }
    TRY(grad_prepare(s, 0));
    GradBuffers& g = s->grad;
    const int N = s->N, P = s->P;
    const int64_t n = (int64_t)N * 3 * P;
    if (!s->list_valid) TRY(rebuild_list_now(s));   // after a step the list covers the beads
    k_modes_to_x<<<blocks(n, 256), 256, 0, s->stream>>>(N, P, s->Q, s->Tmat, s->iperm, g.x);
    s->launches++;
    const double sc = self_coef(s);
    const double* th[2] = {theta_A, theta_B};
    double h[2][4];
    for (int k = 0; k < 2; ++k) {
        QHP_CUDA(eval_terms(s, P, false, g.x, nullptr, g.F, nullptr, g.part, g.partb, th[k]));
        // bead 0 alone: rows w = i P + 0 of the pair partials, t = m P + 0 of the bonded ones
        k_colsum_stride<<<1, 256, 0, s->stream>>>(g.part, N * P, P, 2 * NPART, 0, g.sums + 16);
        k_colsum_stride<<<1, 256, 0, s->stream>>>(g.partb, s->n_mol * P, P, 2 * NPARTB, 0, g.sums + 17);
        s->launches += 2;
        QHP_CUDA(cudaGetLastError());
        double r[18];
        QHP_CUDA(cudaMemcpyAsync(r, g.sums, sizeof r, cudaMemcpyDeviceToHost, s->stream));
        QHP_CUDA(cudaStreamSynchronize(s->stream));
        const double qO = th[k][2];
        h[k][0] = (r[0] + r[2 * NPART]) / P + sc * qO * qO;   // U_P (Eq. (3))
        h[k][1] = r[16] + r[17] + sc * qO * qO;               // V(x_0)
    }
    out[0] = h[0][0];
    out[1] = h[1][0];
    out[2] = h[0][1];
    out[3] = h[1][1];
    return QHP_OK;
}

int qhp_segment_grad(qhp_sys s, int K, int block, int observable, double* J, double* dJ_dtheta) {
    TraceRange tr("qhp_segment_grad");
    if (!s || !s->beads_set) {
        set_error("qhp_segment_grad: system not initialised");
        return QHP_ERR_STATE;
    }
    if (K < 1 || block < 1 || (observable != 0 && observable != 1)) {
        set_error("qhp_segment_grad: need K >= 1, block >= 1 and observable 0 or 1");
        return QHP_ERR_ARG;
    }
    if (s->precision != QHP_FP64 || s->th.kind == QHP_THERMO_ADQTB) {
        set_error("qhp_segment_grad: needs an FP64 system with the PILE or NVE thermostat");
        return QHP_ERR_STATE;
    }
    if (block > K) block = K;
    TRY(grad_prepare(s, block));
    GradBuffers& g = s->grad;
    const int N = s->N, P = s->P;
    const size_t NP3 = (size_t)N * 3 * P;
    const double h = 0.5 * s->th.dt_fs * 1e-3 * ACC;   // B kick: P += h f
    const double wK = 1.0 / K, scoef = self_coef(s);

    // checkpoints every `block` steps (host blobs of the whole dynamical state)
    size_t bytes = 0;
    TRY(qhp_get_state(s, nullptr, &bytes));
    const int nb = (K + block - 1) / block;
    std::vector<std::vector<unsigned char>> ck(nb, std::vector<unsigned char>(bytes));
    TRY(qhp_get_state(s, ck[0].data(), &bytes));
    for (int c = 1; c < nb; ++c) {
        TRY(qhp_step_rpmd(s, block));
        TRY(qhp_get_state(s, ck[c].data(), &bytes));
    }

    QHP_CUDA(cudaMemsetAsync(g.lamQ, 0, sizeof(double) * NP3, s->stream));
    QHP_CUDA(cudaMemsetAsync(g.lamP, 0, sizeof(double) * NP3, s->stream));
    QHP_CUDA(cudaMemsetAsync(g.acc, 0, sizeof(double) * 8, s->stream));
    int rc = QHP_OK;
    for (int c = nb - 1; c >= 0 && rc == QHP_OK; --c) {
        const int k0 = c * block, k1 = std::min(K, k0 + block);
        // replay the block forward, keeping the modes after every step
        rc = qhp_set_state(s, ck[c].data(), bytes);
        if (rc != QHP_OK) break;
        QHP_CUDA(cudaMemcpyAsync(g.Qbuf, s->Q, sizeof(double) * NP3, cudaMemcpyDeviceToDevice, s->stream));
        for (int k = k0 + 1; k <= k1 && rc == QHP_OK; ++k) {
            rc = qhp_step_rpmd(s, 1);
            if (rc == QHP_OK)
                QHP_CUDA(cudaMemcpyAsync(g.Qbuf + (size_t)(k - k0) * NP3, s->Q, sizeof(double) * NP3,
                                         cudaMemcpyDeviceToDevice, s->stream));
        }
        if (rc == QHP_OK) rc = qhp_sync(s);
        // backwards through the block
        for (int k = k1; k > k0 && rc == QHP_OK; --k) {
            const double* Qk = g.Qbuf + (size_t)(k - k0) * NP3;
            rc = load_modes(s, Qk);
            if (rc == QHP_OK) rc = observe(s, Qk, observable, wK, scoef);
            if (rc == QHP_OK && k < K) rc = hvp(s, Qk, 2.0 * h);
            if (rc == QHP_OK) {
                k_adj_linear<<<blocks((int64_t)NP3, 256), 256, 0, s->stream>>>(N, P, s->type_d, s->mode_tab, g.lamQ,
                                                                               g.lamP);
                s->launches++;
                const cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) rc = cuda_fail(e, "k_adj_linear");
            }
        }
        // start of the segment: only the theta part of the first kick matters
        if (c == 0 && rc == QHP_OK) {
            rc = load_modes(s, g.Qbuf);
            if (rc == QHP_OK) rc = hvp(s, g.Qbuf, h);
        }
    }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (rc == QHP_OK) {
        QHP_CUDA(cudaMemcpyAsync(acc, g.acc, sizeof acc, cudaMemcpyDeviceToHost, s->stream));
        QHP_CUDA(cudaStreamSynchronize(s->stream));
    }
    // leave the system exactly as it was
    const int rc2 = qhp_set_state(s, ck[0].data(), bytes);
    if (rc != QHP_OK) return rc;
    if (rc2 != QHP_OK) return rc2;
    if (J) *J = acc[0];
    if (dJ_dtheta)
        for (int k = 0; k < 5; ++k) dJ_dtheta[k] = acc[1 + k];
    return QHP_OK;
}

}  // extern "C"
