// Bead-batched forces: nonbonded pairs from the centroid list and bonded terms.
//
// Pair kernel mapping: one warp per sorted atom i.  The centroid list is shared
// by all beads (Sec. III.A.3), so the lanes of a warp take the *beads* of i:
// for P >= 32 every lane owns P/32 beads and all lanes walk the same list entry
// (no divergence, one coalesced 128-byte load per coordinate plane); for P < 32
// the warp takes 32/P list entries at a time, lane = (entry slot, bead).  The
// full list is walked (each pair twice), so forces on i accumulate in registers
// and are written once: no atomics, and the result does not depend on timing.
//
// Mixed precision: positions are FP32 offsets from the atom's anchor (its
// centroid at the last list build), each list entry carries the FP32 anchor
// separation D_ij (rounded once from FP64), so d = D_ij + (x_j - x_i) stays
// accurate to ~5e-7 A in boxes of any size.  Pair math is FP32; the per-lane
// sum is converted once to int64 fixed point (2^-34 kcal/mol/A), to which the
// bonded kernel adds its own integer contribution, so bead sums are exact.
//
// FP64 path: absolute FP64 positions, minimum image per pair, FP64 math and
// FP64 forces.
#include <math.h>

#include <algorithm>
#include <vector>

#include "qhp_internal.cuh"

namespace qhp {

namespace {

struct PairConsts {
    float rc2, rc, alpha, c2a, sc, ecut, sig2, eps4, eps24, ljshift, L, invL;
    double rc2_d, rc_d, alpha_d, c2a_d, sc_d, ecut_d, sig2_d, eps4_d, eps24_d, ljshift_d, L_d, invL_d, ke_d;
    float ke, qO_ke, qH_ke;
    float p_alpha;        // A&S 7.1.26 p times alpha
    float neg_a2_log2e;   // -alpha^2 log2(e)
};

// List entries carry the partner's sorted index in the low 31 bits and "partner is H"
// in bit 31, so the partner's charge and LJ flag need no extra load.
__device__ __forceinline__ int entry_j(int x) { return x & 0x7fffffff; }
__device__ __forceinline__ bool entry_is_h(int x) { return x < 0; }

// Hardware approximations of the special-function unit, flush-to-zero (pair distances
// are never denormal): reciprocal square root (rel. error < 2^-22.9), reciprocal and
// base-2 exponential (a few ulp), written as PTX so that no range fix-up code surrounds them.
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// erfc(a r) for a r >= 0 with absolute error below 1.5e-7: the rational approximation
// 7.1.26 of Abramowitz & Stegun (Handbook of Mathematical Functions, 1964; from Hastings),
// erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2), t = 1/(1 + p x).
// The factor exp(-a^2 r^2) is the Gaussian the DSF force needs anyway: it is formed from
// r^2 directly (exponent -a^2 log2(e) r^2 for the base-2 exponential); gauss receives it.
__device__ __forceinline__ float erfc_as(float r, float r2, const PairConsts& c, float& gauss) {
    const float t = rcp_fast(fmaf(c.p_alpha, r, 1.0f));
    float p = 1.061405429f;
    p = fmaf(p, t, -1.453152027f);
    p = fmaf(p, t, 1.421413741f);
    p = fmaf(p, t, -0.284496736f);
    p = fmaf(p, t, 0.254829592f);
    gauss = ex2_fast(c.neg_a2_log2e * r2);
    return t * p * gauss;
}

// One bead pair: DSF Coulomb (+ shifted LJ on O-O), force on i accumulated as -g d.
template <bool ALL, bool ENERGY>
__device__ __forceinline__ void pair_term(float dx, float dy, float dz, float qq, bool lj, const PairConsts& c,
                                          float& fx, float& fy, float& fz, float& en) {
    if (ALL) {
        dx -= c.L * rintf(dx * c.invL);
        dy -= c.L * rintf(dy * c.invL);
        dz -= c.L * rintf(dz * c.invL);
    }
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < c.rc2) {
        const float rinv = rsqrt_fast(r2);
        const float r = r2 * rinv;
        float gauss;
        const float erfc_ar = erfc_as(r, r2, c, gauss);
        const float rinv2 = rinv * rinv;
        // -V'(r)/r = qq (erfc(a r)/r^2 + (2a/sqrt(pi)) e^{-a^2 r^2}/r - S_c) / r
        float g = qq * fmaf(erfc_ar, rinv2, fmaf(c.c2a * gauss, rinv, -c.sc)) * rinv;
        float ep = 0.0f;
        if (ENERGY) ep = qq * (erfc_ar * rinv - c.ecut + c.sc * (r - c.rc));
        if (lj) {
            const float s2 = c.sig2 * rinv2;
            const float s6 = s2 * s2 * s2;
            g = fmaf(c.eps24 * fmaf(2.0f * s6, s6, -s6), rinv2, g);
            if (ENERGY) ep += c.eps4 * (s6 * s6 - s6) - c.ljshift;
        }
        fx = fmaf(-g, dx, fx);
        fy = fmaf(-g, dy, fy);
        fz = fmaf(-g, dz, fz);
        if (ENERGY) en = fmaf(0.5f, ep, en);
    }
}

constexpr int PAIR_WARPS = 4;   // warps per block
constexpr int PAIR_RED = PAIR_WARPS * 4 * 64;   // floats of the cross-warp reduction buffer

// Warps that share one atom's list (W): with many beads (P >= 16) four warps split the
// list; with few beads one warp takes a whole list (32/P entries per iteration) and a
// block holds four atoms.  This is the default; the autotuner may pick another W.
__host__ __device__ constexpr int pair_warps_default(int P) { return P >= 16 ? 4 : 1; }

struct PairArgs {
    int N, P, W, all;
    const float4* pos;
    const int *start, *count;
    const int4* nbr;
    const float* charge_s;
    const int *type_s, *perm;
    long long* F;
    float* epair;
    const unsigned* status;
    PairConsts c;
};

// One block (bx) of the pair kernel: APB = PAIR_WARPS / W atoms.  red: PAIR_RED floats.
template <int P, int W, bool ALL, bool ENERGY>
__device__ __forceinline__ void pair_body(const PairArgs& A, int bx, float* red_raw) {
    constexpr int JPW = P >= 32 ? 1 : 32 / P;
    constexpr int BPL = P > 32 ? P / 32 : 1;
    constexpr int NB = P > 32 ? P : 32;                   // bead slots reduced across warps
    constexpr int APB = PAIR_WARPS / W;                   // atoms per block
    float(*red)[4][NB] = reinterpret_cast<float(*)[4][NB]>(red_raw);
    const int N = A.N;
    const float4* __restrict__ pos = A.pos;
    const int* __restrict__ start = A.start;
    const int* __restrict__ count = A.count;
    const int4* __restrict__ nbr = A.nbr;
    const float* __restrict__ charge_s = A.charge_s;
    const int* __restrict__ type_s = A.type_s;
    const int* __restrict__ perm = A.perm;
    long long* __restrict__ F = A.F;
    float* __restrict__ epair = A.epair;
    const PairConsts& c = A.c;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int wa = w % W;                                 // this warp's chunk of the atom's list
    const int i_raw = bx * APB + w / W;
    const bool live = i_raw < N;
    const int i = live ? i_raw : N - 1;                   // idle warps still reach the barrier
    const int b0 = P >= 32 ? lane : (lane % P);
    const int jsub = P >= 32 ? 0 : lane / P;
    const bool ok = live && (*A.status & ST_LIST_OVERFLOW) == 0u;
    // N * P < 2^30 is checked at set-up, so 32-bit element offsets suffice
    const float4* __restrict__ pl = pos + b0;

    float xi[BPL], yi[BPL], zi[BPL], fx[BPL], fy[BPL], fz[BPL], en[BPL];
#pragma unroll
    for (int u = 0; u < BPL; ++u) {
        const float4 p = pl[i * P + 32 * u];
        xi[u] = p.x;
        yi[u] = p.y;
        zi[u] = p.z;
        fx[u] = fy[u] = fz[u] = en[u] = 0.0f;
    }
    const float qi = charge_s[i];
    const bool Oi = type_s[i] == 0;
    const float qO = qi * c.qO_ke, qH = qi * c.qH_ke;
    // the list of i is cut into W contiguous chunks, one per warp
    const int ka = start[i], kb = ok ? ka + count[i] : ka;
    const int chunk = ((kb - ka + W - 1) / W + JPW - 1) / JPW * JPW;
    const int kw0 = min(kb, ka + wa * chunk), k1 = min(kb, kw0 + chunk);
    int k = kw0 + jsub;
    if (P == 2 || P == 4) {
        // few beads: little arithmetic per entry, so the loop waits on the list stream and the
        // dependent position gathers; four entries per lane in flight.  (With P = 1 the extra
        // registers cost more occupancy than the deeper pipeline gains: measured slower.)
        for (; k + 3 * JPW < k1; k += 4 * JPW) {
            int4 e[4];
            float4 q[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) e[v] = __ldg(&nbr[k + v * JPW]);
#pragma unroll
            for (int v = 0; v < 4; ++v) q[v] = __ldg(&pl[entry_j(e[v].x) * P]);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const bool h = entry_is_h(e[v].x);
                pair_term<ALL, ENERGY>(__int_as_float(e[v].y) + (q[v].x - xi[0]), __int_as_float(e[v].z) + (q[v].y - yi[0]),
                                       __int_as_float(e[v].w) + (q[v].z - zi[0]), h ? qH : qO, Oi && !h, c, fx[0], fy[0],
                                       fz[0], en[0]);
            }
        }
    }
    if (P >= 32) {
        // all lanes walk the same entry: the warp's entries are staged in shared memory 32 at
        // a time by asynchronous copies issued one block ahead, so that only the dependent
        // position gather is left on the loop's critical path.  Same entry order and pairing
        // as the loop below, hence the same sums.
        __shared__ int4 s_e[PAIR_WARPS][2][32];
        int4(*ring)[32] = s_e[w];
        const auto stage = [&](int kb0, int slot) {
            const int kk = kb0 + lane;
            const bool in = kk < k1;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&ring[slot][lane]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(nbr + (in ? kk : kb0)),
                         "r"(in ? 16 : 0)
                         : "memory");
        };
        int slot = 0;
        if (k < k1) stage(k, 0);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        for (int kb0 = k; kb0 < k1; kb0 += 32, slot ^= 1) {
            if (kb0 + 32 < k1) stage(kb0 + 32, slot ^ 1);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this block's copies are done
            __syncwarp();
            const int n = min(32, k1 - kb0);
            int q = 0;
            for (; q + 1 < n; q += 2) {
                const int4 e0 = ring[slot][q];
                const int4 e1 = ring[slot][q + 1];
                const int j0 = entry_j(e0.x) * P, j1 = entry_j(e1.x) * P;
                const bool h0 = entry_is_h(e0.x), h1 = entry_is_h(e1.x);
#pragma unroll
                for (int u = 0; u < BPL; ++u) {
                    const float4 a = __ldg(&pl[j0 + 32 * u]);
                    const float4 b = __ldg(&pl[j1 + 32 * u]);
                    pair_term<ALL, ENERGY>(__int_as_float(e0.y) + (a.x - xi[u]), __int_as_float(e0.z) + (a.y - yi[u]),
                                           __int_as_float(e0.w) + (a.z - zi[u]), h0 ? qH : qO, Oi && !h0, c, fx[u],
                                           fy[u], fz[u], en[u]);
                    pair_term<ALL, ENERGY>(__int_as_float(e1.y) + (b.x - xi[u]), __int_as_float(e1.z) + (b.y - yi[u]),
                                           __int_as_float(e1.w) + (b.z - zi[u]), h1 ? qH : qO, Oi && !h1, c, fx[u],
                                           fy[u], fz[u], en[u]);
                }
            }
            if (q < n) {
                const int4 e0 = ring[slot][q];
                const int j0 = entry_j(e0.x) * P;
                const bool h0 = entry_is_h(e0.x);
#pragma unroll
                for (int u = 0; u < BPL; ++u) {
                    const float4 a = __ldg(&pl[j0 + 32 * u]);
                    pair_term<ALL, ENERGY>(__int_as_float(e0.y) + (a.x - xi[u]), __int_as_float(e0.z) + (a.y - yi[u]),
                                           __int_as_float(e0.w) + (a.z - zi[u]), h0 ? qH : qO, Oi && !h0, c, fx[u],
                                           fy[u], fz[u], en[u]);
                }
            }
            __syncwarp();   // every lane is done with this slot before it is refilled
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        k = k1;
    }
    // two list entries per iteration: both entries and all their loads are in flight together
    for (; k + JPW < k1; k += 2 * JPW) {
        const int4 e0 = __ldg(&nbr[k]);
        const int4 e1 = __ldg(&nbr[k + JPW]);
        const int j0 = entry_j(e0.x) * P, j1 = entry_j(e1.x) * P;
        const bool h0 = entry_is_h(e0.x), h1 = entry_is_h(e1.x);
#pragma unroll
        for (int u = 0; u < BPL; ++u) {
            const float4 a = __ldg(&pl[j0 + 32 * u]);
            const float4 b = __ldg(&pl[j1 + 32 * u]);
            pair_term<ALL, ENERGY>(__int_as_float(e0.y) + (a.x - xi[u]), __int_as_float(e0.z) + (a.y - yi[u]),
                                   __int_as_float(e0.w) + (a.z - zi[u]), h0 ? qH : qO, Oi && !h0, c, fx[u], fy[u],
                                   fz[u], en[u]);
            pair_term<ALL, ENERGY>(__int_as_float(e1.y) + (b.x - xi[u]), __int_as_float(e1.z) + (b.y - yi[u]),
                                   __int_as_float(e1.w) + (b.z - zi[u]), h1 ? qH : qO, Oi && !h1, c, fx[u], fy[u],
                                   fz[u], en[u]);
        }
    }
    if (k < k1) {
        const int4 e0 = __ldg(&nbr[k]);
        const int j0 = entry_j(e0.x) * P;
        const bool h0 = entry_is_h(e0.x);
#pragma unroll
        for (int u = 0; u < BPL; ++u) {
            const float4 a = __ldg(&pl[j0 + 32 * u]);
            pair_term<ALL, ENERGY>(__int_as_float(e0.y) + (a.x - xi[u]), __int_as_float(e0.z) + (a.y - yi[u]),
                                   __int_as_float(e0.w) + (a.z - zi[u]), h0 ? qH : qO, Oi && !h0, c, fx[u], fy[u],
                                   fz[u], en[u]);
        }
    }
    if (P < 32) {
#pragma unroll
        for (int off = (P < 32 ? P : 16); off < 32; off <<= 1) {
            fx[0] += __shfl_xor_sync(0xffffffffu, fx[0], off);
            fy[0] += __shfl_xor_sync(0xffffffffu, fy[0], off);
            fz[0] += __shfl_xor_sync(0xffffffffu, fz[0], off);
            if (ENERGY) en[0] += __shfl_xor_sync(0xffffffffu, en[0], off);
        }
    }
    if (jsub == 0) {
#pragma unroll
        for (int u = 0; u < BPL; ++u) {
            const int b = b0 + 32 * u;
            red[w][0][b] = fx[u];
            red[w][1][b] = fy[u];
            red[w][2][b] = fz[u];
            red[w][3][b] = en[u];
        }
    }
    __syncthreads();
    // the first warp of each atom adds the chunks in a fixed order and writes each bead force once
    if (live && wa == 0 && jsub == 0) {
        const int a = perm[i];
#pragma unroll
        for (int u = 0; u < BPL; ++u) {
            const int b = b0 + 32 * u;
            float sx = red[w][0][b], sy = red[w][1][b], sz = red[w][2][b], se = red[w][3][b];
#pragma unroll
            for (int v = 1; v < W; ++v) {
                sx += red[w + v][0][b];
                sy += red[w + v][1][b];
                sz += red[w + v][2][b];
                se += red[w + v][3][b];
            }
            F[((size_t)a * 3 + 0) * P + b] = __float2ll_rn(sx * FIX_SCALE_F);
            F[((size_t)a * 3 + 1) * P + b] = __float2ll_rn(sy * FIX_SCALE_F);
            F[((size_t)a * 3 + 2) * P + b] = __float2ll_rn(sz * FIX_SCALE_F);
            if (ENERGY) epair[(size_t)i * P + b] = se;
        }
    }
}

// Residency: with P = 16 or 32 (one atom per block, lanes = beads) the loop is latency bound
// and 16 resident blocks (64 warps, 32 registers a thread) measured 12% faster than 10-12
// (with the staged entries of P = 32: 0.300 ms at 16 blocks, 0.318 ms at 12); with few
// beads the compiler's default allocation (minimum 0) is faster, and P = 64 (two beads a
// lane) would spill.
template <int P>
__host__ __device__ constexpr int pair_min_blocks() { return (P == 16 || P == 32) ? 16 : 0; }

template <int P, int W, bool ALL, bool ENERGY>
__global__ void __launch_bounds__(32 * PAIR_WARPS, pair_min_blocks<P>()) k_pair_mixed(const __grid_constant__ PairArgs A) {
    __shared__ float red[PAIR_RED];
    pair_body<P, W, ALL, ENERGY>(A, blockIdx.x, red);
}

// Batched systems: one persistent launch per (bead count, small-box path, warps per atom)
// present, over the (system, block) items of the systems of that kind.  Each launch carries
// one specialisation, so it runs at that specialisation's registers and residency (the same
// as the single-system kernel).
// The persistent item loop keeps a few more values live than the single-system kernel:
// 12 resident blocks (40 registers) for P = 16 and 32 instead of 16.
template <int P>
__host__ __device__ constexpr int pair_batch_min_blocks() { return (P == 16 || P == 32) ? 12 : 0; }

template <int P, int W, bool ALL>
__global__ void __launch_bounds__(32 * PAIR_WARPS, pair_batch_min_blocks<P>()) k_pair_batch(const PairArgs* __restrict__ args,
                                                                                      const int2* __restrict__ items,
                                                                                      const int* __restrict__ ranges) {
    __shared__ float red[PAIR_RED];
    for (int it = ranges[blockIdx.x]; it < ranges[blockIdx.x + 1]; ++it) {
        const int2 w = items[it];
        __syncthreads();   // the previous item's reduction has been read
        pair_body<P, W, ALL, false>(args[w.x], w.y, red);
    }
}

// FP64 path, small boxes: one warp per (sorted atom i, bead b), its lanes over i's list row,
// then a fixed shuffle tree.  Every bead is its own warp, so a few hundred atoms still fill the
// GPU (at 4,096 waters the gathers of single words measured 1.6x slower than the bead lanes).
template <bool ENERGY>
__global__ void __launch_bounds__(128) k_pair_fp64_rows(int N, int P, const double* __restrict__ pos,
                                                   const int* __restrict__ start, const int* __restrict__ count,
                                                   const int4* __restrict__ nbr,
                                                   const float* __restrict__ charge_s, const int* __restrict__ type_s,
                                                   const int* __restrict__ perm, const double q_O, const double q_H,
                                                   double* __restrict__ F, double* __restrict__ epair, PairConsts c,
                                                   const unsigned* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int w = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= N * P) return;   // whole warps
    const int i = w / P, b = w % P;
    const bool ok = (*status & ST_LIST_OVERFLOW) == 0u;
    const double qi = (type_s[i] == 0 ? q_O : q_H) * c.ke_d;
    const bool Oi = type_s[i] == 0;
    const int k0 = start[i], k1 = ok ? k0 + count[i] : k0;
    const double xi = pos[((size_t)0 * N + i) * P + b];
    const double yi = pos[((size_t)1 * N + i) * P + b];
    const double zi = pos[((size_t)2 * N + i) * P + b];
    double fx = 0.0, fy = 0.0, fz = 0.0, en = 0.0;
    for (int k = k0 + lane; k < k1; k += 32) {
        const int ex = __ldg(&nbr[k].x);
        const int j = entry_j(ex);
        const bool Oj = !entry_is_h(ex);
        const double qq = qi * (Oj ? q_O : q_H);
        double dx = pos[((size_t)0 * N + j) * P + b] - xi;
        double dy = pos[((size_t)1 * N + j) * P + b] - yi;
        double dz = pos[((size_t)2 * N + j) * P + b] - zi;
        dx -= c.L_d * rint(dx * c.invL_d);
        dy -= c.L_d * rint(dy * c.invL_d);
        dz -= c.L_d * rint(dz * c.invL_d);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < c.rc2_d) {
            const double r = sqrt(r2);
            const double rinv = 1.0 / r;
            const double ar = c.alpha_d * r;
            const double erfc_ar = erfc(ar);
            const double ex2 = exp(-ar * ar);
            const double rinv2 = rinv * rinv;
            double g = qq * (erfc_ar * rinv2 + c.c2a_d * ex2 * rinv - c.sc_d) * rinv;
            double ep = 0.0;
            if (ENERGY) ep = qq * (erfc_ar * rinv - c.ecut_d + c.sc_d * (r - c.rc_d));
            if (Oi && Oj) {
                const double s2 = c.sig2_d * rinv2;
                const double s6 = s2 * s2 * s2;
                g += c.eps24_d * (2.0 * s6 * s6 - s6) * rinv2;
                if (ENERGY) ep += c.eps4_d * (s6 * s6 - s6) - c.ljshift_d;
            }
            fx -= g * dx;
            fy -= g * dy;
            fz -= g * dz;
            if (ENERGY) en += 0.5 * ep;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, off);
        fy += __shfl_xor_sync(0xffffffffu, fy, off);
        fz += __shfl_xor_sync(0xffffffffu, fz, off);
        if (ENERGY) en += __shfl_xor_sync(0xffffffffu, en, off);
    }
    if (lane == 0) {
        const int a = perm[i];
        F[((size_t)a * 3 + 0) * P + b] = fx;
        F[((size_t)a * 3 + 1) * P + b] = fy;
        F[((size_t)a * 3 + 2) * P + b] = fz;
        if (ENERGY) epair[(size_t)i * P + b] = en;
    }
}

// FP64 path, large boxes: one warp per sorted atom, lanes = (entry slot, bead) as in the
// mixed kernel (P <= 32 by slots, P = 64 two beads a lane), so a partner's beads load as
// consecutive words.
template <bool ENERGY>
__global__ void __launch_bounds__(128) k_pair_fp64_beads(int N, int P, const double* __restrict__ pos,
                                                   const int* __restrict__ start, const int* __restrict__ count,
                                                   const int4* __restrict__ nbr,
                                                   const float* __restrict__ charge_s, const int* __restrict__ type_s,
                                                   const int* __restrict__ perm, const double q_O, const double q_H,
                                                   double* __restrict__ F, double* __restrict__ epair, PairConsts c,
                                                   const unsigned* __restrict__ status) {
    // lane = (entry slot, bead) as in the mixed kernel, with P <= 32 handled by slots and
    // P = 64 by two beads per lane.
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const int JPW = P >= 32 ? 1 : 32 / P;
    const int BPL = P > 32 ? P / 32 : 1;
    const int b0 = P >= 32 ? lane : (lane % P);
    const int jsub = P >= 32 ? 0 : lane / P;
    const bool ok = (*status & ST_LIST_OVERFLOW) == 0u;
    const double qi = (type_s[i] == 0 ? q_O : q_H) * c.ke_d;
    const bool Oi = type_s[i] == 0;
    const int k0 = start[i], k1 = ok ? k0 + count[i] : k0;
    for (int u = 0; u < BPL; ++u) {
        const int b = b0 + 32 * u;
        const double xi = pos[((size_t)0 * N + i) * P + b];
        const double yi = pos[((size_t)1 * N + i) * P + b];
        const double zi = pos[((size_t)2 * N + i) * P + b];
        double fx = 0.0, fy = 0.0, fz = 0.0, en = 0.0;
        for (int k = k0 + jsub; k < k1; k += JPW) {
            const int ex = __ldg(&nbr[k].x);
            const int j = entry_j(ex);
            const bool Oj = !entry_is_h(ex);
            const double qq = qi * (Oj ? q_O : q_H);
            double dx = pos[((size_t)0 * N + j) * P + b] - xi;
            double dy = pos[((size_t)1 * N + j) * P + b] - yi;
            double dz = pos[((size_t)2 * N + j) * P + b] - zi;
            dx -= c.L_d * rint(dx * c.invL_d);
            dy -= c.L_d * rint(dy * c.invL_d);
            dz -= c.L_d * rint(dz * c.invL_d);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < c.rc2_d) {
                const double r = sqrt(r2);
                const double rinv = 1.0 / r;
                const double ar = c.alpha_d * r;
                const double erfc_ar = erfc(ar);
                const double ex = exp(-ar * ar);
                const double rinv2 = rinv * rinv;
                double g = qq * (erfc_ar * rinv2 + c.c2a_d * ex * rinv - c.sc_d) * rinv;
                double ep = 0.0;
                if (ENERGY) ep = qq * (erfc_ar * rinv - c.ecut_d + c.sc_d * (r - c.rc_d));
                if (Oi && Oj) {
                    const double s2 = c.sig2_d * rinv2;
                    const double s6 = s2 * s2 * s2;
                    g += c.eps24_d * (2.0 * s6 * s6 - s6) * rinv2;
                    if (ENERGY) ep += c.eps4_d * (s6 * s6 - s6) - c.ljshift_d;
                }
                fx -= g * dx;
                fy -= g * dy;
                fz -= g * dz;
                if (ENERGY) en += 0.5 * ep;
            }
        }
        for (int off = (P < 32 ? P : 32); off < 32; off <<= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, off);
            fy += __shfl_xor_sync(0xffffffffu, fy, off);
            fz += __shfl_xor_sync(0xffffffffu, fz, off);
            if (ENERGY) en += __shfl_xor_sync(0xffffffffu, en, off);
        }
        if (jsub == 0) {
            const int a = perm[i];
            F[((size_t)a * 3 + 0) * P + b] = fx;
            F[((size_t)a * 3 + 1) * P + b] = fy;
            F[((size_t)a * 3 + 2) * P + b] = fz;
            if (ENERGY) epair[(size_t)i * P + b] = en;
        }
    }
}

struct BondConsts {
    double kb, r0, kth, th0, L;
};

// Bonded terms per (molecule, bead); each thread owns the forces of its three atoms at its bead.
struct BondArgs {
    int n_mol, N, P;
    const float4* pos_f;
    const double* pos_d;
    const float* dA;
    const int* iperm;
    long long* Ffix;
    double* Fd;
    double* ebond;
    BondConsts c;
    int overwrite;   // mixed: store the bonded forces instead of adding them to the pair forces
};

template <bool MIXED, bool ENERGY>
__device__ __forceinline__ void bonded_body(const BondArgs& A, int t) {
    const int n_mol = A.n_mol, N = A.N, P = A.P;
    const float4* __restrict__ pos_f = A.pos_f;
    const double* __restrict__ pos_d = A.pos_d;
    const float* __restrict__ dA = A.dA;
    const int* __restrict__ iperm = A.iperm;
    long long* Ffix = A.Ffix;
    double* Fd = A.Fd;
    double* ebond = A.ebond;
    const BondConsts& c = A.c;
    if (t >= n_mol * P) return;
    const int m = t / P, b = t % P;
    const int aO = 3 * m, aH1 = aO + 1, aH2 = aO + 2;
    const int sO = iperm[aO], s1 = iperm[aH1], s2 = iperm[aH2];
    if (MIXED) {
        float d1[3], d2[3];
        const float4 xo = pos_f[(size_t)sO * P + b], x1 = pos_f[(size_t)s1 * P + b], x2 = pos_f[(size_t)s2 * P + b];
        const float4 a1 = reinterpret_cast<const float4*>(dA)[(size_t)m * 2 + 0];
        const float4 a2 = reinterpret_cast<const float4*>(dA)[(size_t)m * 2 + 1];
        d1[0] = (x1.x - xo.x) + a1.x;
        d1[1] = (x1.y - xo.y) + a1.y;
        d1[2] = (x1.z - xo.z) + a1.z;
        d2[0] = (x2.x - xo.x) + a2.x;
        d2[1] = (x2.y - xo.y) + a2.y;
        d2[2] = (x2.z - xo.z) + a2.z;
        const float r1 = sqrtf(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        const float r2 = sqrtf(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
        float cs = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (r1 * r2);
        cs = fminf(1.0f, fmaxf(-1.0f, cs));
        const float th = acosf(cs);
        const float sn = sqrtf(fmaxf(1e-30f, 1.0f - cs * cs));
        const float kb = (float)c.kb, r0 = (float)c.r0, kth = (float)c.kth, th0 = (float)c.th0;
        const float pb1 = -kb * (r1 - r0) / r1, pb2 = -kb * (r2 - r0) / r2;
        const float pa = kth * (th - th0) / sn;
        const float ir12 = 1.0f / (r1 * r2);
        for (int d = 0; d < 3; ++d) {
            const float f1 = pb1 * d1[d] + pa * (d2[d] * ir12 - cs * d1[d] / (r1 * r1));
            const float f2 = pb2 * d2[d] + pa * (d1[d] * ir12 - cs * d2[d] / (r2 * r2));
            const long long i1 = __float2ll_rn(f1 * FIX_SCALE_F), i2 = __float2ll_rn(f2 * FIX_SCALE_F);
            if (A.overwrite) {
                Ffix[((size_t)aH1 * 3 + d) * P + b] = i1;
                Ffix[((size_t)aH2 * 3 + d) * P + b] = i2;
                Ffix[((size_t)aO * 3 + d) * P + b] = -(i1 + i2);
            } else {
                Ffix[((size_t)aH1 * 3 + d) * P + b] += i1;
                Ffix[((size_t)aH2 * 3 + d) * P + b] += i2;
                Ffix[((size_t)aO * 3 + d) * P + b] -= i1 + i2;
            }
        }
        if (ENERGY)
            ebond[t] = 0.5 * c.kb * ((double)(r1 - r0) * (r1 - r0) + (double)(r2 - r0) * (r2 - r0)) +
                       0.5 * c.kth * (double)(th - th0) * (th - th0);
    } else {
        double d1[3], d2[3];
        for (int d = 0; d < 3; ++d) {
            const double xo = pos_d[((size_t)d * N + sO) * P + b];
            double a1 = pos_d[((size_t)d * N + s1) * P + b] - xo;
            double a2 = pos_d[((size_t)d * N + s2) * P + b] - xo;
            d1[d] = a1 - c.L * rint(a1 / c.L);
            d2[d] = a2 - c.L * rint(a2 / c.L);
        }
        const double r1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        const double r2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
        double cs = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (r1 * r2);
        cs = fmin(1.0, fmax(-1.0, cs));
        const double th = acos(cs);
        const double sn = sqrt(fmax(1e-300, 1.0 - cs * cs));
        const double pb1 = -c.kb * (r1 - c.r0) / r1, pb2 = -c.kb * (r2 - c.r0) / r2;
        const double pa = c.kth * (th - c.th0) / sn;
        const double ir12 = 1.0 / (r1 * r2);
        for (int d = 0; d < 3; ++d) {
            const double f1 = pb1 * d1[d] + pa * (d2[d] * ir12 - cs * d1[d] / (r1 * r1));
            const double f2 = pb2 * d2[d] + pa * (d1[d] * ir12 - cs * d2[d] / (r2 * r2));
            Fd[((size_t)aH1 * 3 + d) * P + b] += f1;
            Fd[((size_t)aH2 * 3 + d) * P + b] += f2;
            Fd[((size_t)aO * 3 + d) * P + b] -= f1 + f2;
        }
        if (ENERGY)
            ebond[t] = 0.5 * c.kb * ((r1 - c.r0) * (r1 - c.r0) + (r2 - c.r0) * (r2 - c.r0)) +
                       0.5 * c.kth * (th - c.th0) * (th - c.th0);
    }
}

template <bool MIXED, bool ENERGY>
__global__ void k_bonded(const __grid_constant__ BondArgs A) {
    bonded_body<MIXED, ENERGY>(A, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_bonded_batch(const BondArgs* __restrict__ args, const int2* __restrict__ items,
                               const int* __restrict__ ranges) {
    for (int it = ranges[blockIdx.x]; it < ranges[blockIdx.x + 1]; ++it) {
        const int2 w = items[it];
        bonded_body<true, false>(args[w.x], w.y * (int)blockDim.x + threadIdx.x);
    }
}

// Count in-cutoff bead pairs j > i (lane = bead, one list entry at a time); not on the step path.
__global__ void k_count_pairs(int N, int P, int mixed, int all, const float4* __restrict__ pos_f,
                              const double* __restrict__ pos_d, const int* __restrict__ start,
                              const int* __restrict__ count,
                              const int4* __restrict__ nbr, const int* __restrict__ type_s, PairConsts c,
                              unsigned long long* out2) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    unsigned long long n = 0, noo = 0;
    for (int b = lane; b < P; b += 32) {
        for (int k = start[i]; k < start[i] + count[i]; ++k) {
            const int4 e = nbr[k];
            const int j = entry_j(e.x);
            if (j <= i) continue;
            double r2;
            if (mixed) {
                const float4 pj = pos_f[(size_t)j * P + b], pi = pos_f[(size_t)i * P + b];
                float dx = __int_as_float(e.y) + (pj.x - pi.x);
                float dy = __int_as_float(e.z) + (pj.y - pi.y);
                float dz = __int_as_float(e.w) + (pj.z - pi.z);
                if (all) {
                    dx -= c.L * rintf(dx * c.invL);
                    dy -= c.L * rintf(dy * c.invL);
                    dz -= c.L * rintf(dz * c.invL);
                }
                r2 = (double)(dx * dx + dy * dy + dz * dz);
                if (!((float)r2 < c.rc2)) continue;
            } else {
                double d[3];
                for (int q = 0; q < 3; ++q) {
                    d[q] = pos_d[((size_t)q * N + j) * P + b] - pos_d[((size_t)q * N + i) * P + b];
                    d[q] -= c.L_d * rint(d[q] * c.invL_d);
                }
                r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < c.rc2_d)) continue;
            }
            ++n;
            noo += (type_s[i] == 0 && type_s[j] == 0);
        }
    }
    atomicAdd(&out2[0], n);
    atomicAdd(&out2[1], noo);
}

PairConsts make_pair_consts(const qhp_system_s* s) {
    const qhp_ff& f = s->ff;
    PairConsts c;
    const double rc = f.rc, a = f.alpha;
    const double sc = erfc(a * rc) / (rc * rc) + 2.0 * a / sqrt(M_PI) * exp(-(a * rc) * (a * rc)) / rc;
    const double ecut = erfc(a * rc) / rc;
    const double sr6 = pow(f.sigma / rc, 6.0);
    const double ljs = 4.0 * f.eps * (sr6 * sr6 - sr6);
    c.rc2_d = rc * rc;
    c.rc_d = rc;
    c.alpha_d = a;
    c.c2a_d = 2.0 * a / sqrt(M_PI);
    c.sc_d = sc;
    c.ecut_d = ecut;
    c.sig2_d = f.sigma * f.sigma;
    c.eps4_d = 4.0 * f.eps;
    c.eps24_d = 24.0 * f.eps;
    c.ljshift_d = ljs;
    c.L_d = s->L;
    c.invL_d = 1.0 / s->L;
    c.ke_d = COULOMB;
    c.rc2 = (float)c.rc2_d;
    c.rc = (float)rc;
    c.alpha = (float)a;
    c.c2a = (float)c.c2a_d;
    c.sc = (float)sc;
    c.ecut = (float)ecut;
    c.sig2 = (float)c.sig2_d;
    c.eps4 = (float)c.eps4_d;
    c.eps24 = (float)c.eps24_d;
    c.ljshift = (float)ljs;
    c.L = (float)s->L;
    c.invL = (float)(1.0 / s->L);
    c.ke = (float)COULOMB;
    c.qO_ke = (float)(COULOMB * f.q_O);
    c.qH_ke = (float)(COULOMB * (-0.5 * f.q_O));
    c.p_alpha = (float)(0.3275911 * a);
    c.neg_a2_log2e = (float)(-a * a * 1.4426950408889634);
    return c;
}

PairArgs make_pair_args(const qhp_system_s* s) {
    PairArgs A;
    A.N = s->N;
    A.P = s->P;
    A.W = s->pair_w > 0 ? s->pair_w : pair_warps_default(s->P);
    A.all = s->list_mode ? 0 : 1;
    A.pos = s->pos_f4;
    A.start = s->nbr_start;
    A.count = s->nbr_count;
    A.nbr = s->nbr;
    A.charge_s = s->charge_s;
    A.type_s = s->type_s;
    A.perm = s->perm;
    A.F = s->Ffix;
    A.epair = s->e_pair;
    A.status = s->status;
    A.c = make_pair_consts(s);
    return A;
}

template <int P, int W>
void pair_mixed_launch(const PairArgs& A, bool energy, cudaStream_t st) {
    const int grid = (A.N + PAIR_WARPS / W - 1) / (PAIR_WARPS / W);
    if (A.all) {
        if (energy) k_pair_mixed<P, W, true, true><<<grid, 32 * PAIR_WARPS, 0, st>>>(A);
        else k_pair_mixed<P, W, true, false><<<grid, 32 * PAIR_WARPS, 0, st>>>(A);
    } else {
        if (energy) k_pair_mixed<P, W, false, true><<<grid, 32 * PAIR_WARPS, 0, st>>>(A);
        else k_pair_mixed<P, W, false, false><<<grid, 32 * PAIR_WARPS, 0, st>>>(A);
    }
}

template <int P>
void pair_mixed_dispatch(const PairArgs& A, bool energy, cudaStream_t st) {
    if (A.W == 4) pair_mixed_launch<P, 4>(A, energy, st);
    else if (A.W == 2) pair_mixed_launch<P, 2>(A, energy, st);
    else pair_mixed_launch<P, 1>(A, energy, st);
}

BondArgs make_bond_args(const qhp_system_s* s) {
    BondArgs B;
    B.n_mol = s->n_mol;
    B.N = s->N;
    B.P = s->P;
    B.pos_f = s->pos_f4;
    B.pos_d = s->pos_d;
    B.dA = s->dA;
    B.iperm = s->iperm;
    B.Ffix = s->Ffix;
    B.Fd = s->Fd;
    B.ebond = s->e_bond;
    B.c = BondConsts{s->ff.k_b, s->ff.r0, s->ff.k_theta, s->ff.theta0, s->L};
    B.overwrite = 0;
    return B;
}

}  // namespace

// FP64 pair mapping: bead lanes from this many atoms up (16 warps per SM of 148), row lanes
// below.  Measured: 64 waters 0.186 -> 0.088 ms and 216 waters 1.72 -> 1.29 ms with row lanes;
// 4,096 waters 32.8 ms with bead lanes against 52.6 ms with row lanes.
constexpr int FP64_BEAD_LANES_MIN_ATOMS = 148 * 16;

cudaError_t launch_pair(qhp_system_s* s, bool energy) {
    const PairConsts c = make_pair_consts(s);
    const int grid = (s->N * 32 + 127) / 128;
    if (s->precision == QHP_MIXED) {
        const PairArgs A = make_pair_args(s);
        switch (s->P) {
            case 1: pair_mixed_dispatch<1>(A, energy, s->stream); break;
            case 2: pair_mixed_dispatch<2>(A, energy, s->stream); break;
            case 4: pair_mixed_dispatch<4>(A, energy, s->stream); break;
            case 8: pair_mixed_dispatch<8>(A, energy, s->stream); break;
            case 16: pair_mixed_dispatch<16>(A, energy, s->stream); break;
            case 32: pair_mixed_dispatch<32>(A, energy, s->stream); break;
            case 64: pair_mixed_dispatch<64>(A, energy, s->stream); break;
            default: return cudaErrorInvalidValue;
        }
    } else if (s->N >= FP64_BEAD_LANES_MIN_ATOMS) {   // a warp per atom fills the GPU
        if (energy)
            k_pair_fp64_beads<true><<<grid, 128, 0, s->stream>>>(s->N, s->P, s->pos_d, s->nbr_start, s->nbr_count, s->nbr,
                                                                 s->charge_s, s->type_s, s->perm, s->ff.q_O, -0.5 * s->ff.q_O,
                                                                 s->Fd, s->e_pair_d, c, s->status);
        else
            k_pair_fp64_beads<false><<<grid, 128, 0, s->stream>>>(s->N, s->P, s->pos_d, s->nbr_start, s->nbr_count, s->nbr,
                                                                  s->charge_s, s->type_s, s->perm, s->ff.q_O, -0.5 * s->ff.q_O,
                                                                  s->Fd, s->e_pair_d, c, s->status);
    } else {   // a warp per (atom, bead)
        const int grid_rows = (int)(((int64_t)s->N * s->P * 32 + 127) / 128);
        if (energy)
            k_pair_fp64_rows<true><<<grid_rows, 128, 0, s->stream>>>(s->N, s->P, s->pos_d, s->nbr_start, s->nbr_count, s->nbr,
                                                                     s->charge_s, s->type_s, s->perm, s->ff.q_O,
                                                                     -0.5 * s->ff.q_O, s->Fd, s->e_pair_d, c, s->status);
        else
            k_pair_fp64_rows<false><<<grid_rows, 128, 0, s->stream>>>(s->N, s->P, s->pos_d, s->nbr_start, s->nbr_count, s->nbr,
                                                                      s->charge_s, s->type_s, s->perm, s->ff.q_O,
                                                                      -0.5 * s->ff.q_O, s->Fd, s->e_pair_d, c, s->status);
    }
    s->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_bonded(qhp_system_s* s, bool energy) {
    const BondArgs B = make_bond_args(s);
    const int g2 = (s->n_mol * s->P + 127) / 128;
    if (s->precision == QHP_MIXED) {
        if (energy) k_bonded<true, true><<<g2, 128, 0, s->stream>>>(B);
        else k_bonded<true, false><<<g2, 128, 0, s->stream>>>(B);
    } else {
        if (energy) k_bonded<false, true><<<g2, 128, 0, s->stream>>>(B);
        else k_bonded<false, false><<<g2, 128, 0, s->stream>>>(B);
    }
    s->launches += 1;
    return cudaGetLastError();
}

// Batched stages (mixed precision).  Pair items are blocks of PAIR_WARPS / W atoms, costed
// by the bead-pair work of their list rows (row length x max(P, 32) lanes); one stage per
// (log2 P, small-box path, W), index batch_pair_stage(lp, all, W).
int batch_pair_stage(int lp, int all, int W) { return (lp * 2 + all) * 3 + (W == 4 ? 2 : W == 2 ? 1 : 0); }

template <int P>
struct PairBatchVariants {
    template <int W, bool ALL>
    static void go(const BatchStage* s, cudaStream_t st, const void** ptr) {
        if (ptr) *ptr = (const void*)k_pair_batch<P, W, ALL>;
        else k_pair_batch<P, W, ALL><<<s->grid, 32 * PAIR_WARPS, 0, st>>>((const PairArgs*)s->args, s->items, s->ranges);
    }
    // launch stage s (ptr == nullptr) or return its kernel (ptr != nullptr)
    static void dispatch(int all, int W, const BatchStage* s, cudaStream_t st, const void** ptr) {
        if (all) {
            if (W == 4) go<4, true>(s, st, ptr);
            else if (W == 2) go<2, true>(s, st, ptr);
            else go<1, true>(s, st, ptr);
        } else {
            if (W == 4) go<4, false>(s, st, ptr);
            else if (W == 2) go<2, false>(s, st, ptr);
            else go<1, false>(s, st, ptr);
        }
    }
};

void pair_batch_dispatch(int lp, int all, int W, const BatchStage* s, cudaStream_t st, const void** ptr) {
    switch (lp) {
        case 0: PairBatchVariants<1>::dispatch(all, W, s, st, ptr); break;
        case 1: PairBatchVariants<2>::dispatch(all, W, s, st, ptr); break;
        case 2: PairBatchVariants<4>::dispatch(all, W, s, st, ptr); break;
        case 3: PairBatchVariants<8>::dispatch(all, W, s, st, ptr); break;
        case 4: PairBatchVariants<16>::dispatch(all, W, s, st, ptr); break;
        case 5: PairBatchVariants<32>::dispatch(all, W, s, st, ptr); break;
        default: PairBatchVariants<64>::dispatch(all, W, s, st, ptr); break;
    }
}

int batch_stage_pair(const std::vector<qhp_system_s*>& v, BatchStage* st /*[BATCH_PAIR_STAGES]*/) {
    const int Ws[3] = {1, 2, 4};
    for (int lp = 0; lp < 7; ++lp)
        for (int all = 0; all < 2; ++all)
            for (int W : Ws) {
                const int P = 1 << lp;
                BatchStage& S = st[batch_pair_stage(lp, all, W)];
                std::vector<PairArgs> a;
                std::vector<int2> items;
                std::vector<double> cost;
                for (size_t k = 0; k < v.size(); ++k) {
                    const qhp_system_s* s = v[k];
                    if (s->P != P) continue;
                    const PairArgs A = make_pair_args(s);
                    if (A.all != all || A.W != W) continue;
                    const int idx = (int)a.size();
                    a.push_back(A);
                    const int apb = PAIR_WARPS / W;
                    const int nb = (s->N + apb - 1) / apb;
                    std::vector<int> cnt(s->N);
                    QHP_CUDA(cudaMemcpy(cnt.data(), s->nbr_count, sizeof(int) * s->N, cudaMemcpyDeviceToHost));
                    const double lanes = (double)std::max(P, 32) / 32.0;
                    for (int b = 0; b < nb; ++b) {
                        double c = 0.0;
                        for (int i = b * apb; i < std::min(s->N, (b + 1) * apb); ++i) c += (double)cnt[i] * lanes;
                        items.push_back(make_int2(idx, b));
                        cost.push_back(c + 8.0);
                    }
                }
                if (a.empty()) {
                    stage_free(S);
                    continue;
                }
                const void* fn = nullptr;
                pair_batch_dispatch(lp, all, W, nullptr, nullptr, &fn);
                int per_sm = 0;
                QHP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * PAIR_WARPS, 0));
                S.smem = 0;
                TRY(stage_upload(S, a.data(), sizeof(PairArgs) * a.size(), items, cost, std::max(1, per_sm) * sm_count()));
            }
    return QHP_OK;
}

int batch_stage_bonded(const std::vector<qhp_system_s*>& v, BatchStage& st) {
    std::vector<BondArgs> a;
    std::vector<int2> items;
    std::vector<double> cost;
    for (size_t k = 0; k < v.size(); ++k) {
        a.push_back(make_bond_args(v[k]));
        const int nb = (v[k]->n_mol * v[k]->P + 127) / 128;
        for (int b = 0; b < nb; ++b) {
            items.push_back(make_int2((int)k, b));
            cost.push_back(1.0);
        }
    }
    int per_sm = 0;
    QHP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bonded_batch, 128, 0));
    st.smem = 0;
    return stage_upload(st, a.data(), sizeof(BondArgs) * a.size(), items, cost, std::max(1, per_sm) * sm_count());
}

cudaError_t launch_batch_pair(const BatchStage* st, cudaStream_t stream) {
    const int Ws[3] = {1, 2, 4};
    for (int lp = 0; lp < 7; ++lp)
        for (int all = 0; all < 2; ++all)
            for (int W : Ws) {
                const BatchStage& S = st[batch_pair_stage(lp, all, W)];
                if (S.n_items == 0) continue;
                pair_batch_dispatch(lp, all, W, &S, stream, nullptr);
                const cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

cudaError_t launch_batch_bonded(const BatchStage& st, cudaStream_t stream) {
    k_bonded_batch<<<st.grid, 128, 0, stream>>>((const BondArgs*)st.args, st.items, st.ranges);
    return cudaGetLastError();
}

cudaError_t launch_forces(qhp_system_s* s, bool energy) {
    cudaError_t e = launch_pair(s, energy);
    if (e != cudaSuccess) return e;
    if (s->prof_on) {
        e = record_stage(s, 3);
        if (e != cudaSuccess) return e;
    }
    return launch_bonded(s, energy);
}

// RESPA: the bonded (fast) forces alone into the fixed-point bead forces.
cudaError_t launch_bonded_fast(qhp_system_s* s) {
    BondArgs B = make_bond_args(s);
    B.overwrite = 1;
    const int g2 = (s->n_mol * s->P + 127) / 128;
    k_bonded<true, false><<<g2, 128, 0, s->stream>>>(B);
    s->launches += 1;
    return cudaGetLastError();
}

// RESPA with contraction: the nonbonded (slow) forces on the Pc contracted beads.
cudaError_t launch_pair_contracted(qhp_system_s* s) {
    PairArgs A = make_pair_args(s);
    A.P = s->pc;
    A.W = s->pair_w > 0 ? s->pair_w : pair_warps_default(s->pc);
    A.pos = s->pos_c;
    A.F = s->Ffix_s;
    switch (s->pc) {
        case 1: pair_mixed_dispatch<1>(A, false, s->stream); break;
        case 2: pair_mixed_dispatch<2>(A, false, s->stream); break;
        case 4: pair_mixed_dispatch<4>(A, false, s->stream); break;
        case 8: pair_mixed_dispatch<8>(A, false, s->stream); break;
        case 16: pair_mixed_dispatch<16>(A, false, s->stream); break;
        case 32: pair_mixed_dispatch<32>(A, false, s->stream); break;
        case 64: pair_mixed_dispatch<64>(A, false, s->stream); break;
        default: return cudaErrorInvalidValue;
    }
    s->launches += 1;
    return cudaGetLastError();
}

// In-cutoff bead pairs (each unordered pair once) and how many of them are O-O.
cudaError_t launch_count_pairs(qhp_system_s* s, unsigned long long* out2) {
    const PairConsts c = make_pair_consts(s);
    const int grid = (s->N * 32 + 127) / 128;
    k_count_pairs<<<grid, 128, 0, s->stream>>>(s->N, s->P, s->precision == QHP_MIXED, s->list_mode, s->pos_f4, s->pos_d,
                                               s->nbr_start, s->nbr_count, s->nbr, s->type_s, c, out2);
    s->launches += 1;
    return cudaGetLastError();
}

}  // namespace qhp
