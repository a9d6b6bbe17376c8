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
#include "step_bodies.cuh"

namespace qhp {

namespace {

// Coefficients of the two even functions of the DSF Coulomb pair, fitted on [0, rc^2] in
// t = r^2 (2/rc^2) - 1 (see make_pair_consts): with erfc = 1 - erf,
//   -V'(r)/r / (q_i q_j k_e) = 1/r^3 - S_c/r - G(r^2),  G(s) = erf(a sqrt s)/s^(3/2) - (2a/sqrt(pi)) e^(-a^2 s)/s,
//   V(r) / (q_i q_j k_e)     = 1/r - E(r^2) - erfc(a rc)/rc + S_c (r - rc),  E(s) = erf(a sqrt s)/sqrt s.
// G and E are entire functions of s (their series in a^2 s have no odd powers of r), so a
// degree-8 polynomial reaches 2.5e-8 of G(0) on the cutoff sphere, below the FP32 rounding of
// its own evaluation; the pair then needs one special-function operation, the 1/sqrt(r^2).
constexpr int NPOLY = 9;

struct PairConsts {
    float rc2, rc, sc, ecut, sig2, eps4, neps24, ljshift, L, invL;
    double rc2_d, rc_d, alpha_d, c2a_d, sc_d, ecut_d, sig2_d, eps4_d, eps24_d, ljshift_d, L_d, invL_d, ke_d;
    float qO_ke, qH_ke;
    float tscale;           // 2 / rc^2
    float bucket_lo, bucket_inv;   // the row order's distance buckets (list_bucket)
    float gpoly[NPOLY];     // G in powers of t
    float epoly[NPOLY];     // E in powers of t
};

// The partner's sorted index of a list entry (entry_partner); its type rides in bit 31 and
// its distance bucket in bits 26-30, so neither needs an extra load.
__device__ __forceinline__ int entry_j(int x) { return entry_partner(x); }

// Reciprocal square root of the special-function unit, flush-to-zero (pair distances are
// never denormal), relative error below 2^-22.9, written as PTX so that no range fix-up
// code surrounds it.
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32x2 arithmetic (one instruction for the two beads a lane carries).
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// round(x 2^34) as int64, the same value as __float2ll_rn(x * FIX_SCALE_F), for |x| < 2^29,
// from two 32-bit conversions (64-bit conversions run on the FP64 pipe, which this part has
// little of).  v = x 2^34 is split exactly into h 2^32 + l with h = floor(v 2^-32) and
// 0 <= l < 2^32: l is made of v's own mantissa bits, so the FMA forming it is exact, and only
// l's fraction (below 2^-1 only when |v| < 2^24) is rounded, half to even as for v itself.
__device__ __forceinline__ long long fix64(float x) {
    const float v = x * FIX_SCALE_F;
    const float h = floorf(v * 0x1p-32f);
    const float l = fmaf(h, -0x1p32f, v);
    return (long long)((unsigned long long)(unsigned)__float2int_rz(h) << 32) + (long long)__float2uint_rn(l);
}

constexpr int PAIR_WARPS = 4;   // warps per block
constexpr int PAIR_SUB = 32;    // list entries read (and staged) at a time

// Warps that share one atom's list (W): with many beads (P >= 16) four warps split the
// list; with few beads one warp takes a whole list and a block holds four atoms.  This is
// the default; the autotuner may pick another W.  Forces do not depend on W.
__host__ __device__ constexpr int pair_warps_default(int P) { return P >= 16 ? 4 : 1; }

struct PairArgs {
    int N, P, W, all;
    const float4* pos;
    const int *start, *count, *nO;
    const int4* nbr;
    const float* charge_s;
    const int *type_s, *perm;
    long long* F;
    float* epair;
    const unsigned* status;
    const unsigned* dev_max;   // running max |x_ib - A_i|^2 since the list build, or null
    const float* dev_atom;     // per sorted atom, max over its beads of |x_ib - A_i|^2 this step, or null
    int skip;                  // 1: entries beyond every bead pair's reach are dropped, 0: evaluated
    PairConsts c;
};

struct PairSmem {
    float4 ent[PAIR_WARPS][PAIR_SUB][2];   // staged entries {Dx, Dx, Dy, Dy}, {Dz, Dz, j, -}
    long long acc[PAIR_WARPS][3][64];      // per warp and bead: int64 sum of the block sums
    float esum[PAIR_WARPS][64];            // per warp and bead: pair energy (ENERGY)
};

// The pair terms of one list entry for the two beads of a lane (Eq. (3)'s V on every bead):
// DSF Coulomb, plus the shifted LJ when LJ; the force on i, -g d, accumulates in f.  A bead
// beyond rc adds nothing.  ONE: a single bead (P = 1), carried in .x.
template <bool LJ, bool ENERGY, bool ONE>
__device__ __forceinline__ void pair2(float2 dx, float2 dy, float2 dz, float2 qq, const PairConsts& c,
                                      float2& fx, float2& fy, float2& fz, float2& en) {
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    const bool in0 = r2.x < c.rc2, in1 = !ONE && r2.y < c.rc2;
    if (in0 || in1) {
        const float2 rinv = make_float2(rsqrt_fast(r2.x), ONE ? 1.0f : rsqrt_fast(r2.y));
        const float2 rinv2 = mul2(rinv, rinv);
        const float2 t = fma2(r2, f2(c.tscale), f2(-1.0f));
        float2 p = f2(c.gpoly[NPOLY - 1]);
#pragma unroll
        for (int k = NPOLY - 2; k >= 0; --k) p = fma2(p, t, f2(c.gpoly[k]));
        // -g = qq (G - 1/r^3 + S_c/r)
        const float2 u = mul2(rinv, add2(rinv2, f2(-c.sc)));
        float2 ng = mul2(qq, fma2(u, f2(-1.0f), p));
        float2 ep = f2(0.0f);
        if (ENERGY) {
            float2 pe = f2(c.epoly[NPOLY - 1]);
#pragma unroll
            for (int k = NPOLY - 2; k >= 0; --k) pe = fma2(pe, t, f2(c.epoly[k]));
            const float2 r = mul2(r2, rinv);
            ep = mul2(qq, add2(add2(rinv, fma2(pe, f2(-1.0f), f2(-c.ecut))), mul2(f2(c.sc), add2(r, f2(-c.rc)))));
        }
        if (LJ) {
            const float2 s2 = mul2(f2(c.sig2), rinv2);
            const float2 s6 = mul2(mul2(s2, s2), s2);
            // -24 eps (2 s^12 - s^6) / r^2
            ng = fma2(mul2(f2(c.neps24), rinv2), mul2(s6, fma2(s6, f2(2.0f), f2(-1.0f))), ng);
            if (ENERGY) ep = add2(ep, fma2(f2(c.eps4), mul2(s6, add2(s6, f2(-1.0f))), f2(-c.ljshift)));
        }
        if (!in0) ng.x = 0.0f, ep.x = 0.0f;
        if (!in1) ng.y = 0.0f, ep.y = 0.0f;
        fx = fma2(ng, dx, fx);
        fy = fma2(ng, dy, fy);
        fz = fma2(ng, dz, fz);
        if (ENERGY) en = fma2(f2(0.5f), ep, en);
    }
}

// The partner's two beads of lane bp: the xy plane's float4 and the z plane's float2
// (bead_word layout); one bead (P = 1) is carried in .x and .y alike.
template <int P>
__device__ __forceinline__ void load_pair_beads(const float* __restrict__ pw, int j, int bp, float2& x, float2& y,
                                                float2& z) {
    if (P == 1) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(pw) + j);
        x = f2(q.x), y = f2(q.y), z = f2(q.z);
    } else {
        const float* rec = pw + (size_t)j * bead_stride(P);
        const float4 q = __ldg(reinterpret_cast<const float4*>(rec) + bp);
        x = make_float2(q.x, q.y), y = make_float2(q.z, q.w);
        z = __ldg(reinterpret_cast<const float2*>(rec + 2 * P) + bp);
    }
}

// The same terms for a single bead (P = 1) in scalar FP32.
template <bool LJ, bool ENERGY>
__device__ __forceinline__ void pair1(float dx, float dy, float dz, float qq, const PairConsts& c, float& fx, float& fy,
                                      float& fz, float& en) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < c.rc2) {
        const float rinv = rsqrt_fast(r2);
        const float rinv2 = rinv * rinv;
        const float t = fmaf(r2, c.tscale, -1.0f);
        float p = c.gpoly[NPOLY - 1];
#pragma unroll
        for (int k = NPOLY - 2; k >= 0; --k) p = fmaf(p, t, c.gpoly[k]);
        float ng = qq * fmaf(rinv, c.sc - rinv2, p);   // qq (G - 1/r^3 + S_c/r)
        float ep = 0.0f;
        if (ENERGY) {
            float pe = c.epoly[NPOLY - 1];
#pragma unroll
            for (int k = NPOLY - 2; k >= 0; --k) pe = fmaf(pe, t, c.epoly[k]);
            ep = qq * (rinv - pe - c.ecut + c.sc * (r2 * rinv - c.rc));
        }
        if (LJ) {
            const float s2 = c.sig2 * rinv2;
            const float s6 = s2 * s2 * s2;
            ng = fmaf(c.neps24 * rinv2, s6 * fmaf(s6, 2.0f, -1.0f), ng);
            if (ENERGY) ep += fmaf(c.eps4, s6 * (s6 - 1.0f), -c.ljshift);
        }
        fx = fmaf(ng, dx, fx);
        fy = fmaf(ng, dy, fy);
        fz = fmaf(ng, dz, fz);
        if (ENERGY) en = fmaf(0.5f, ep, en);
    }
}

// One list entry for a single bead: partner position p, anchor separation D.
template <bool ALL, bool LJ, bool ENERGY>
__device__ __forceinline__ void pair_entry1(float Dx, float Dy, float Dz, float4 p, float2 nxi, float2 nyi, float2 nzi,
                                            float qq, const PairConsts& c, float2& fx, float2& fy, float2& fz, float2& en) {
    float dx = Dx + (p.x + nxi.x), dy = Dy + (p.y + nyi.x), dz = Dz + (p.z + nzi.x);
    if (ALL) {
        dx = fmaf(-c.L, rintf(dx * c.invL), dx);
        dy = fmaf(-c.L, rintf(dy * c.invL), dy);
        dz = fmaf(-c.L, rintf(dz * c.invL), dz);
    }
    pair1<LJ, ENERGY>(dx, dy, dz, qq, c, fx.x, fy.x, fz.x, en.x);
}

// One list entry (anchor separation D) for the lane's two beads, the partner's beads given.
// wrap: a bead pair may need another image than D's (small boxes; otherwise every |d_c| < L/2
// and the minimum image changes nothing, so skipping it changes no bit).
template <int P, bool ALL, bool LJ, bool ENERGY>
__device__ __forceinline__ void pair_entry_at(float2 Dx, float2 Dy, float2 Dz, float2 px, float2 py, float2 pz,
                                              float2 nxi, float2 nyi, float2 nzi, float2 qq, const PairConsts& c,
                                              float2& fx, float2& fy, float2& fz, float2& en, bool wrap = true) {
    // d = D_ij + (x_jb - x_ib): anchor separation plus the two bead offsets
    float2 dx = add2(add2(px, nxi), Dx);
    float2 dy = add2(add2(py, nyi), Dy);
    float2 dz = add2(add2(pz, nzi), Dz);
    if (ALL && wrap) {   // small boxes: minimum image per bead pair
        dx = fma2(f2(-c.L), make_float2(rintf(dx.x * c.invL), rintf(dx.y * c.invL)), dx);
        dy = fma2(f2(-c.L), make_float2(rintf(dy.x * c.invL), rintf(dy.y * c.invL)), dy);
        dz = fma2(f2(-c.L), make_float2(rintf(dz.x * c.invL), rintf(dz.y * c.invL)), dz);
    }
    pair2<LJ, ENERGY, P == 1>(dx, dy, dz, qq, c, fx, fy, fz, en);
}

// One list entry (anchor separation D, partner j) for the lane's two beads.
template <int P, bool ALL, bool LJ, bool ENERGY>
__device__ __forceinline__ void pair_entry(float2 Dx, float2 Dy, float2 Dz, int j, const float* __restrict__ pw,
                                           int bp, float2 nxi, float2 nyi, float2 nzi, float2 qq, const PairConsts& c,
                                           float2& fx, float2& fy, float2& fz, float2& en, bool wrap) {
    float2 px, py, pz;
    load_pair_beads<P>(pw, j, bp, px, py, pz);
    pair_entry_at<P, ALL, LJ, ENERGY>(Dx, Dy, Dz, px, py, pz, nxi, nyi, nzi, qq, c, fx, fy, fz, en, wrap);
}

// Entries per deterministic partial sum: 32, or for few beads as many as make eight entries
// per lane (32 with one lane per entry, P <= 2), so that the per-block reduction stays a small
// share of the work.
__host__ __device__ constexpr int pair_block(int P) { return P >= 16 ? 32 : (P <= 2 ? 1024 : 512 / P); }

// Per-warp state of one atom's row walk.
struct PairLane {
    float2 nxi, nyi, nzi;   // minus the lane's own two bead offsets
    int i, slot, bp;
    int b_stop;             // the row walk ends at the first 32 entries from this bucket on
    int b_act;              // entries from this bucket on lie beyond reach of every bead pair
    float reach_i;          // rc + max_b |x_ib - A_i| (+ margin), or 0: no per-entry test
};

// Adds the FP32 sums (fx, fy, fz) of one block to the warp's int64 accumulators: the slots
// first in a fixed tree, then one int64 conversion per value; value v = (dim v % 3, bead
// 2 bp + v / 3), slot s < S takes values s R .. s R + R - 1, chosen by a select so that every
// lane runs the same R conversions.
template <int P>
__device__ __forceinline__ void pair_block_sum(float2 fx, float2 fy, float2 fz, int slot, int bp, long long (*acc)[64]) {
    constexpr int LPE = P == 1 ? 1 : P / 2;
    constexpr int EPI = 32 / LPE;
#pragma unroll
    for (int off = LPE; off < 32; off <<= 1) {
        fx.x += __shfl_xor_sync(0xffffffffu, fx.x, off);
        fx.y += __shfl_xor_sync(0xffffffffu, fx.y, off);
        fy.x += __shfl_xor_sync(0xffffffffu, fy.x, off);
        fy.y += __shfl_xor_sync(0xffffffffu, fy.y, off);
        fz.x += __shfl_xor_sync(0xffffffffu, fz.x, off);
        fz.y += __shfl_xor_sync(0xffffffffu, fz.y, off);
    }
    const float vals[6] = {fx.x, fy.x, fz.x, fx.y, fy.y, fz.y};
    constexpr int NV = P == 1 ? 3 : 6;
    constexpr int S = EPI < NV ? EPI : NV;
    constexpr int R = (NV + S - 1) / S;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = slot * R + r;
        float x = vals[r];
#pragma unroll
        for (int s2 = 1; s2 < S; ++s2)
            if (s2 * R + r < NV) x = (slot == s2) ? vals[s2 * R + r] : x;
        if (slot < S && v < NV) acc[v % 3][2 * bp + v / 3] += fix64(x);
    }
}

// The blocks of one group of atom i's row, [k_begin, k_end), that belong to this warp: the
// first is block `first` of the group, then every W-th.  Entries are read 32 at a time (lane
// k: entry k); when several lanes share an entry it is staged in shared memory, and slots past
// the group's end hold a dummy partner (atom i itself, L/2 away in each dimension: beyond rc
// in every image), so every iteration runs unchecked.  Within the group entries come by |D|^2
// bucket: at the first 32 entries that all lie beyond reach the group ends for this warp.
template <int P, int W, bool ALL, bool LJ, bool ENERGY>
__device__ __forceinline__ void pair_group(const PairArgs& A, const PairLane& L, int k_begin, int k_end, int first,
                                           float qqs, float4 (*ent)[2], long long (*acc)[64], float2& en) {
    constexpr int LPE = P == 1 ? 1 : P / 2;
    constexpr int EPI = 32 / LPE;
    constexpr int BLK = pair_block(P);
    const PairConsts& c = A.c;
    const float* __restrict__ pw = reinterpret_cast<const float*>(A.pos);
    const int lane = threadIdx.x & 31;
    const float2 qq = f2(qqs);
    for (int kb = k_begin + first * BLK; kb < k_end; kb += W * BLK) {
        const int bend = min(k_end, kb + BLK);
        float2 fx = f2(0.0f), fy = f2(0.0f), fz = f2(0.0f);
        bool beyond = false;
        if (LPE == 1) {
            // one lane per entry, two entries per lane in flight: 64 entries at a time (a lane
            // still adds its entries in index order), both partners gathered before either is used
            for (int sb = kb; sb < bend; sb += 64) {
                const int n0 = min(32, bend - sb), n1 = min(32, bend - sb - 32);
                int4 e0 = make_int4(0, 0, 0, 0), e1 = make_int4(0, 0, 0, 0);
                bool a0 = false, a1 = false;
                if (lane < n0) {
                    e0 = __ldg(&A.nbr[sb + lane]);
                    a0 = entry_bucket(e0.x) < L.b_stop;
                }
                if (lane < n1) {
                    e1 = __ldg(&A.nbr[sb + 32 + lane]);
                    a1 = entry_bucket(e1.x) < L.b_stop;
                }
                const unsigned am0 = __ballot_sync(0xffffffffu, a0);
                const unsigned am1 = __ballot_sync(0xffffffffu, a1);
                if (a0) a0 = QHP_IN_BOUNDS(entry_j(e0.x), A.N, A.status);
                if (a1) a1 = QHP_IN_BOUNDS(entry_j(e1.x), A.N, A.status);
                if (am0 == 0u) {
                    beyond = true;
                    break;
                }
                if (P == 1) {
                    const float4 p0 = __ldg(reinterpret_cast<const float4*>(pw) + (a0 ? entry_j(e0.x) : L.i));
                    const float4 p1 = __ldg(reinterpret_cast<const float4*>(pw) + (a1 ? entry_j(e1.x) : L.i));
                    if (a0)
                        pair_entry1<ALL, LJ, ENERGY>(__int_as_float(e0.y), __int_as_float(e0.z), __int_as_float(e0.w), p0, L.nxi,
                                                     L.nyi, L.nzi, qqs, c, fx, fy, fz, en);
                    if (a1)
                        pair_entry1<ALL, LJ, ENERGY>(__int_as_float(e1.y), __int_as_float(e1.z), __int_as_float(e1.w), p1, L.nxi,
                                                     L.nyi, L.nzi, qqs, c, fx, fy, fz, en);
                } else {
                    float2 px0, py0, pz0, px1, py1, pz1;
                    load_pair_beads<P>(pw, a0 ? entry_j(e0.x) : L.i, L.bp, px0, py0, pz0);
                    load_pair_beads<P>(pw, a1 ? entry_j(e1.x) : L.i, L.bp, px1, py1, pz1);
                    if (a0)
                        pair_entry_at<P, ALL, LJ, ENERGY>(f2(__int_as_float(e0.y)), f2(__int_as_float(e0.z)), f2(__int_as_float(e0.w)),
                                                          px0, py0, pz0, L.nxi, L.nyi, L.nzi, qq, c, fx, fy, fz, en);
                    if (a1)
                        pair_entry_at<P, ALL, LJ, ENERGY>(f2(__int_as_float(e1.y)), f2(__int_as_float(e1.z)), f2(__int_as_float(e1.w)),
                                                          px1, py1, pz1, L.nxi, L.nyi, L.nzi, qq, c, fx, fy, fz, en);
                }
                if (am1 == 0u && n1 > 0) {   // the second 32 and all after them lie beyond reach
                    beyond = true;
                    break;
                }
            }
        } else {
            for (int sb = kb; sb < bend; sb += 32) {
                const int n = min(32, bend - sb);
                int4 e = make_int4(0, 0, 0, 0);
                bool valid = false, near = false, act = false, wrap = true;
                if (lane < n) {
                    e = __ldg(&A.nbr[sb + lane]);
                    valid = QHP_IN_BOUNDS(entry_j(e.x), A.N, A.status);
                    near = entry_bucket(e.x) < L.b_stop;
                    act = valid && entry_bucket(e.x) < L.b_act;
                    if (act && L.reach_i > 0.0f) {
                        // e_ij = dev_i + dev_j (+ margin) bounds |(x_jb - A_j) - (x_ib - A_i)|
                        const float dx = __int_as_float(e.y), dy = __int_as_float(e.z), dz = __int_as_float(e.w);
                        const float r = L.reach_i + sqrtf(__ldg(&A.dev_atom[entry_j(e.x)])) * 1.000001f;
                        act = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < r * r;
                        if (ALL) wrap = fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))) + (r - c.rc) >= 0.499f * c.L;
                    }
                }
                if (__ballot_sync(0xffffffffu, near) == 0u) {   // rows come in bucket order
                    beyond = true;
                    break;
                }
                // Entries within reach first, in row order, then (skipping off) the others, which
                // add exactly zero: the slots' summation order is the same either way.
                const unsigned am = __ballot_sync(0xffffffffu, act);
                const unsigned vm = __ballot_sync(0xffffffffu, valid);
                const unsigned lt = (1u << lane) - 1u;
                const int na = __popc(am);
                const int cnt = A.skip ? na : __popc(vm);
                int rank = -1;
                if (act) rank = __popc(am & lt);
                else if (!A.skip && valid) rank = na + __popc(vm & ~am & lt);
                const int nit = (cnt + EPI - 1) / EPI;
                __syncwarp();
                if (rank >= 0) {
                    const float dx = __int_as_float(e.y), dy = __int_as_float(e.z), dz = __int_as_float(e.w);
                    ent[rank][0] = make_float4(dx, dx, dy, dy);
                    ent[rank][1] = make_float4(dz, dz, __int_as_float(entry_j(e.x)), wrap ? 1.0f : 0.0f);
                }
                if (lane >= cnt) {   // the last pass's spare slots: atom i itself, L/2 away
                    const float h = 0.5f * c.L;
                    ent[lane][0] = make_float4(h, h, h, h);
                    ent[lane][1] = make_float4(h, h, __int_as_float(L.i), 0.0f);
                }
                __syncwarp();
                for (int it = 0; it < nit; ++it) {
                    const float4 a = ent[it * EPI + L.slot][0], b = ent[it * EPI + L.slot][1];
                    pair_entry<P, ALL, LJ, ENERGY>(make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                                                   __float_as_int(b.z), pw, L.bp, L.nxi, L.nyi, L.nzi, qq, c, fx, fy, fz, en,
                                                   b.w != 0.0f);
                }
            }
        }
        pair_block_sum<P>(fx, fy, fz, L.slot, L.bp, acc);
        if (beyond) break;
    }
}

// One block (bx) of the pair kernel: APB = PAIR_WARPS / W atoms, W warps per atom.
//
// Lanes: with P >= 2 a lane carries beads 2bp and 2bp + 1 of one list entry (LPE = P/2 lanes
// per entry) and a warp takes EPI = 64/P entries at a time; with P = 1 a lane takes one entry.
// The row of atom i holds its O partners first, then its H partners (k_list_sort), so the
// charge product and the LJ switch are fixed within each group.  Each group is cut into
// blocks of pair_block(P) entries; block q of the row (O blocks first) belongs to warp q mod W.
// A block's FP32 sum is converted to int64 once and the integers are added, so the forces do
// not depend on W.  Entries beyond rc + 2 max|x_ib - A_i| (+ margin) of every bead pair are
// skipped (pair_group): they would add exactly zero.
template <int P, int W, bool ALL, bool ENERGY, bool ACC = false, class Bar = BlockBar>
__device__ __forceinline__ void pair_body(const PairArgs& A, int bx, PairSmem& sm, int tid) {
    constexpr bool ONE = P == 1;
    constexpr int LPE = ONE ? 1 : P / 2;
    constexpr int APB = PAIR_WARPS / W;
    constexpr int BLK = pair_block(P);
    const PairConsts& c = A.c;
    const float* __restrict__ pw = reinterpret_cast<const float*>(A.pos);
    const int lane = tid & 31, w = tid >> 5;
    const int wa = w % W;
    const int i_raw = bx * APB + w / W;
    const bool live = i_raw < A.N;
    PairLane L;
    L.i = live ? i_raw : A.N - 1;      // idle warps still reach the barrier
    L.slot = lane / LPE;
    L.bp = lane % LPE;
    const int i = L.i, slot = L.slot, bp = L.bp;
    const bool ok = live && (*A.status & ST_LIST_OVERFLOW) == 0u;
    load_pair_beads<P>(pw, i, bp, L.nxi, L.nyi, L.nzi);
    L.nxi = make_float2(-L.nxi.x, -L.nxi.y), L.nyi = make_float2(-L.nyi.x, -L.nyi.y);
    L.nzi = make_float2(-L.nzi.x, -L.nzi.y);
    const float qi = A.charge_s[i];
    const bool Oi = A.type_s[i] == 0;
    if (slot == 0) {
        sm.acc[w][0][2 * bp] = sm.acc[w][1][2 * bp] = sm.acc[w][2][2 * bp] = 0;
        sm.acc[w][0][2 * bp + 1] = sm.acc[w][1][2 * bp + 1] = sm.acc[w][2][2 * bp + 1] = 0;
    }
    // Reach: a bead pair of entry (i, j) lies at |D_ij + (x_jb - A_j) - (x_ib - A_i)| >=
    // |D_ij| - dev_j - dev_i, so beyond rc + dev_i + dev_j no bead pair comes within rc and
    // the entry adds exactly zero.  The row's bucket bound uses dev_i and the global maximum
    // for dev_j (LIST_BUCKETS + 2: no bound); the per-entry test each partner's own dev_j.
    L.b_stop = L.b_act = LIST_BUCKETS + 2;
    L.reach_i = 0.0f;
    if (A.dev_max) {   // |D| is the anchors' minimum image: the bound holds for every image
        const float m2 = __uint_as_float(*A.dev_max);
        const float di2 = A.dev_atom ? A.dev_atom[i] : m2;
        if (m2 >= 0.0f && m2 <= 1.0e4f && di2 >= 0.0f && di2 <= m2) {
            const float ri = c.rc + sqrtf(di2) * 1.000001f + 1.0e-3f;
            const float reach = ri + sqrtf(m2) * 1.000001f;
            L.b_act = list_bucket_d2(reach * reach, c.bucket_lo, c.bucket_inv) + 1;   // above reach's own bucket
            if (A.dev_atom) L.reach_i = ri;
            if (A.skip) L.b_stop = L.b_act;
        }
    }
    const int ka = A.start[i];
    int cnt = ok ? A.count[i] : 0;
    if (!QHP_IN_BOUNDS(cnt, A.start[i + 1] - ka + 1, A.status)) cnt = 0;   // a row never passes its slot
    const int nO = ok ? min(A.nO[i], cnt) : 0;
    float2 en = f2(0.0f);
    // O partners: blocks wa, wa + W, ... of the group; H partners: numbered after the O blocks
    if (Oi) pair_group<P, W, ALL, true, ENERGY>(A, L, ka, ka + nO, wa, qi * c.qO_ke, sm.ent[w], sm.acc[w], en);
    else pair_group<P, W, ALL, false, ENERGY>(A, L, ka, ka + nO, wa, qi * c.qO_ke, sm.ent[w], sm.acc[w], en);
    const int nb0 = (nO + BLK - 1) / BLK;
    pair_group<P, W, ALL, false, ENERGY>(A, L, ka + nO, ka + cnt, ((wa - nb0 % W) + W) % W, qi * c.qH_ke, sm.ent[w],
                                         sm.acc[w], en);
    if (ENERGY) {
#pragma unroll
        for (int off = LPE; off < 32; off <<= 1) {
            en.x += __shfl_xor_sync(0xffffffffu, en.x, off);
            en.y += __shfl_xor_sync(0xffffffffu, en.y, off);
        }
        if (slot == 0) {
            sm.esum[w][2 * bp] = en.x;
            if (!ONE) sm.esum[w][2 * bp + 1] = en.y;
        }
    }
    if (W > 1) Bar::sync();
    else __syncwarp();
    // the first warp of each atom adds the W integer sums and writes each bead force once
    if (live && wa == 0 && slot == 0) {
        const int a = A.perm[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            long long s0 = sm.acc[w][d][2 * bp], s1 = ONE ? 0 : sm.acc[w][d][2 * bp + 1];
#pragma unroll
            for (int v = 1; v < W; ++v) {
                s0 += sm.acc[w + v][d][2 * bp];
                if (!ONE) s1 += sm.acc[w + v][d][2 * bp + 1];
            }
            long long* out = A.F + ((size_t)a * 3 + d) * P + 2 * bp;
            if (ACC) {   // batched step: integer adds into forces cleared by the integrate stage
                atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)s0);
                if (!ONE) atomicAdd(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)s1);
            } else if (ONE) {
                out[0] = s0;
            } else {
                *reinterpret_cast<longlong2*>(out) = make_longlong2(s0, s1);
            }
        }
        if (ENERGY) {
            float e0 = sm.esum[w][2 * bp], e1 = ONE ? 0.0f : sm.esum[w][2 * bp + 1];
#pragma unroll
            for (int v = 1; v < W; ++v) {
                e0 += sm.esum[w + v][2 * bp];
                if (!ONE) e1 += sm.esum[w + v][2 * bp + 1];
            }
            A.epair[(size_t)i * P + 2 * bp] = e0;
            if (!ONE) A.epair[(size_t)i * P + 2 * bp + 1] = e1;
        }
    }
}

// Residency: with two beads per lane the loop holds twice the scalar state, and the compiler's
// choice (48-62 registers, 8-10 blocks per SM) left the gathers' latency exposed; 12 blocks
// (40 registers, a few spilled words) measured 5-10% faster at P = 32.  P <= 2 keep the
// compiler's allocation.
#ifndef QHP_PAIR_MIN_BLOCKS
#define QHP_PAIR_MIN_BLOCKS 12
#endif
template <int P>
__host__ __device__ constexpr int pair_min_blocks() { return P >= 4 ? QHP_PAIR_MIN_BLOCKS : 0; }

template <int P, int W, bool ALL, bool ENERGY>
__global__ void __launch_bounds__(32 * PAIR_WARPS, pair_min_blocks<P>()) k_pair_mixed(const __grid_constant__ PairArgs A) {
    __shared__ PairSmem sm;
    pair_body<P, W, ALL, ENERGY>(A, blockIdx.x, sm, threadIdx.x);
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
        if (!QHP_IN_BOUNDS(j, N, status)) continue;
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
            if (!QHP_IN_BOUNDS(j, N, status)) continue;
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
    const unsigned* status;
};

template <bool MIXED, bool ENERGY, bool ACC = false>
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
    if (!(QHP_IN_BOUNDS(sO, N, A.status) && QHP_IN_BOUNDS(s1, N, A.status) && QHP_IN_BOUNDS(s2, N, A.status))) return;
    if (MIXED) {
        float d1[3], d2[3];
        const float* pw = reinterpret_cast<const float*>(pos_f);
        const float3 xo = make_float3(pw[bead_word(sO, b, 0, P)], pw[bead_word(sO, b, 1, P)], pw[bead_word(sO, b, 2, P)]);
        const float3 x1 = make_float3(pw[bead_word(s1, b, 0, P)], pw[bead_word(s1, b, 1, P)], pw[bead_word(s1, b, 2, P)]);
        const float3 x2 = make_float3(pw[bead_word(s2, b, 0, P)], pw[bead_word(s2, b, 1, P)], pw[bead_word(s2, b, 2, P)]);
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
            } else if (ACC) {   // batched step: the pair terms of the same atoms add concurrently
                atomicAdd(reinterpret_cast<unsigned long long*>(&Ffix[((size_t)aH1 * 3 + d) * P + b]), (unsigned long long)i1);
                atomicAdd(reinterpret_cast<unsigned long long*>(&Ffix[((size_t)aH2 * 3 + d) * P + b]), (unsigned long long)i2);
                atomicAdd(reinterpret_cast<unsigned long long*>(&Ffix[((size_t)aO * 3 + d) * P + b]),
                          (unsigned long long)(-(i1 + i2)));
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

// ------------------------------------------------------------------ one-launch batched step
// A batched step over many systems in one cooperative launch of STEP_THREADS threads per block,
// three phases separated by grid barriers:
//   1. integrate: B-A-O-A and bead positions of every system's atom groups (threads 0..191);
//      the block that finishes a system's last group runs its list check (batch_check);
//   2. forces: the two 128-thread halves of each block walk their own ranges of pair items
//      (every bead count, small-box path and warps-per-atom setting) and bonded items, adding
//      int64 fixed-point forces atomically into the forces phase 1 cleared;
//   3. projection and the closing B of every system (threads 0..191).
// A system whose check fired skips phases 2 and 3 here: its conditional graph node rebuilds the
// list and computes its forces and projection with the single-system kernels after the launch.
// Integer addition is exact, so the order of the items (and which block runs which) cannot
// change a bit: every member ends the step bit-identical to stepping it alone.
constexpr int STEP_THREADS = 256;

struct ForceArgs {
    PairArgs p;
    BondArgs b;
};

// Item kind: batch_pair_stage(log2 P, small-box path, W) for pair items, FORCE_BONDED_VARIANT
// for bonded ones.
__host__ __device__ constexpr int batch_pair_stage(int lp, int all, int W) {
    return (lp * 2 + all) * 3 + (W == 4 ? 2 : W == 2 ? 1 : 0);
}

// Barriers of the step's sub-blocks: the 192 threads of the integrate / project groups, and
// the two 128-thread halves of the force phase (named barriers 1, 2 and 3; 0 is the block's).
struct GroupBar {
    __device__ __forceinline__ static void sync() { asm volatile("bar.sync 1, 192;" ::: "memory"); }
};
struct HalfBar {
    __device__ __forceinline__ static void sync() {
        asm volatile("bar.sync %0, 128;" ::"r"(2 + (int)(threadIdx.x >> 7)) : "memory");
    }
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier for a co-resident grid: every block's thread 0 reads the generation, counts
// itself in and waits for the generation to move; the expected-th arrival resets the count,
// stamps the phase and moves the generation.  A wait longer than wait_ns gives up: it sets
// ST_TIMEOUT and the block leaves the step (so do the others when they see the bit), so a lost
// block ends the launch with an error instead of a hang.  Returns false when the step ends.
__device__ bool grid_sync(StepBatchState* st, unsigned expected, long long wait_ns, int stamp) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = &st->bar[1];
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&st->bar[0], 1u) == expected - 1u) {
            atomicExch(&st->bar[0], 0u);
            if (stamp >= 0) st->ts[stamp] = global_ns();
            __threadfence();
            atomicAdd(&st->bar[1], 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if ((long long)(global_ns() - t0) > wait_ns) {
                    atomicOr(&st->status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile unsigned*)&st->status & ST_TIMEOUT) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

struct StepBatchArgs {
    const IntegrateArgs* iargs;
    const int2* iitems;
    const int* iranges;   // per block
    const ForceArgs* fargs;
    const int2* fitems;
    const int* franges;   // per half block
    const ProjectArgs* pargs;
    const int2* pitems;
    const int* pranges;   // per block
    const CheckArgs* checks;
    int* done;            // integrate items finished per system (reset by the last one)
    const int* nitems;    // integrate items per system
    StepBatchState* st;
    long long wait_ns;
};

#define QHP_FORCE_CASE(LP, AL, WS)                                                                          \
    case ((LP) * 2 + (AL)) * 3 + (WS):                                                                     \
        pair_body<(1 << (LP)), ((WS) == 2 ? 4 : (WS) == 1 ? 2 : 1), ((AL) != 0), false, true, HalfBar>(A.p, bx, \
                                                                                                      sm, lt); \
        break;
#define QHP_FORCE_CASES_W(LP, AL) QHP_FORCE_CASE(LP, AL, 0) QHP_FORCE_CASE(LP, AL, 1) QHP_FORCE_CASE(LP, AL, 2)
#define QHP_FORCE_CASES_P(LP) QHP_FORCE_CASES_W(LP, 0) QHP_FORCE_CASES_W(LP, 1)
// 4 resident blocks of 256 threads (64 registers): the 42 inlined pair specialisations and the
// per-item arguments, read from global memory rather than the parameter bank, spill heavily at
// 40 registers.
#ifndef QHP_STEP_MIN_BLOCKS
#define QHP_STEP_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(STEP_THREADS, QHP_STEP_MIN_BLOCKS) k_step_batch(const __grid_constant__ StepBatchArgs S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const unsigned nblk = gridDim.x;
    if (blockIdx.x == 0 && tid == 0) S.st->ts[0] = global_ns();
    // phase 1: integrate, and each system's list check by the block finishing its last group
    if (tid < BLOCK) {
        int prev = -1;
        for (int it = S.iranges[blockIdx.x]; it < S.iranges[blockIdx.x + 1]; ++it) {
            const int2 w = S.iitems[it];
            GroupBar::sync();   // the previous group is done with shared memory
            integrate_body<true, false, true, GroupBar>(S.iargs[w.x], w.y, smem_raw, w.x != prev);
            prev = w.x;
            GroupBar::sync();   // every thread of the group has written its modes, positions and forces
            if (tid == 0) {
                __threadfence();
                if (atomicAdd(&S.done[w.x], 1) == S.nitems[w.x] - 1) {
                    __threadfence();
                    batch_check(S.checks[w.x]);
                    S.done[w.x] = 0;   // for the next step
                }
            }
        }
    }
    if (!grid_sync(S.st, nblk, S.wait_ns, 1)) return;
    // phase 2: forces, one item at a time per 128-thread half
    {
        const int h = tid >> 7, lt = tid & 127;
        PairSmem& sm = reinterpret_cast<PairSmem*>(smem_raw)[h];
        const int v = (int)blockIdx.x * 2 + h;
        for (int it = S.franges[v]; it < S.franges[v + 1]; ++it) {
            const int2 w = S.fitems[it];
            const int sys = w.x & 0xffff, kind = w.x >> 16, bx = w.y;
            HalfBar::sync();   // the previous item's sums have been read
            if (*S.checks[sys].flag) continue;   // rebuilt this step: computed after the launch
            const ForceArgs& A = S.fargs[sys];
            if (kind == FORCE_BONDED_VARIANT) {
                bonded_body<true, false, true>(A.b, bx * 128 + lt);
                continue;
            }
            switch (kind) {
                QHP_FORCE_CASES_P(0) QHP_FORCE_CASES_P(1) QHP_FORCE_CASES_P(2) QHP_FORCE_CASES_P(3)
                QHP_FORCE_CASES_P(4) QHP_FORCE_CASES_P(5) QHP_FORCE_CASES_P(6)
                default: break;
            }
        }
    }
    if (!grid_sync(S.st, nblk, S.wait_ns, 2)) return;
    // phase 3: projection and the closing B
    if (tid < BLOCK) {
        int prev = -1;
        for (int it = S.pranges[blockIdx.x]; it < S.pranges[blockIdx.x + 1]; ++it) {
            const int2 w = S.pitems[it];
            if (*S.checks[w.x].flag) continue;
            GroupBar::sync();
            project_body<true, true, GroupBar>(S.pargs[w.x], w.y, smem_raw, w.x != prev);
            prev = w.x;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&S.st->bar[2], 1u) == nblk - 1u) {
            S.st->ts[3] = global_ns();
            S.st->bar[2] = 0u;
        }
    }
}
#undef QHP_FORCE_CASE
#undef QHP_FORCE_CASES_W
#undef QHP_FORCE_CASES_P

// Self-test of the barrier's time limit: the blocks wait for one arrival more than the grid
// has, so every wait runs out after wait_ns and sets ST_TIMEOUT.
__global__ void k_grid_sync_selftest(StepBatchState* st, long long wait_ns) {
    grid_sync(st, gridDim.x + 1u, wait_ns, -1);
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
                const float* pw = reinterpret_cast<const float*>(pos_f);
                float dx = __int_as_float(e.y) + (pw[bead_word(j, b, 0, P)] - pw[bead_word(i, b, 0, P)]);
                float dy = __int_as_float(e.z) + (pw[bead_word(j, b, 1, P)] - pw[bead_word(i, b, 1, P)]);
                float dz = __int_as_float(e.w) + (pw[bead_word(j, b, 2, P)] - pw[bead_word(i, b, 2, P)]);
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

// Degree NPOLY - 1 interpolant of f(t) on [-1, 1] at the NPOLY Chebyshev nodes, in powers of t.
template <class Fn>
void chebyshev_fit(Fn f, float* out) {
    constexpr int n = NPOLY;
    double cc[n];
    for (int k = 0; k < n; ++k) {
        double sum = 0.0;
        for (int m = 0; m < n; ++m) {
            const double th = M_PI * (m + 0.5) / n;
            sum += f(cos(th)) * cos(k * th);
        }
        cc[k] = (k == 0 ? 1.0 : 2.0) * sum / n;
    }
    double T[n][n] = {};   // T[k][p]: coefficient of t^p in the Chebyshev polynomial T_k
    T[0][0] = 1.0;
    T[1][1] = 1.0;
    for (int k = 2; k < n; ++k)
        for (int p = 0; p < n; ++p) T[k][p] = (p > 0 ? 2.0 * T[k - 1][p - 1] : 0.0) - T[k - 2][p];
    for (int p = 0; p < n; ++p) {
        double sum = 0.0;
        for (int k = 0; k < n; ++k) sum += cc[k] * T[k][p];
        out[p] = (float)sum;
    }
}

// G(s) = erf(a sqrt s)/s^(3/2) - (2a/sqrt(pi)) e^(-a^2 s)/s and E(s) = erf(a sqrt s)/sqrt s, with
// their power series in x = a^2 s (G = a^3 (4/sqrt(pi)) sum (-x)^m/(m!(2m+3)),
// E = a (2/sqrt(pi)) sum (-x)^m/(m!(2m+1))) where the closed forms cancel.
double dsf_G(double a, double s) {
    const double x = a * a * s;
    if (x < 0.5) {
        double sum = 0.0, term = 1.0;
        for (int m = 0; m < 20; ++m) {
            sum += term / (2 * m + 3);
            term *= -x / (m + 1);
        }
        return a * a * a * 4.0 / sqrt(M_PI) * sum;
    }
    const double r = sqrt(s);
    return erf(a * r) / (s * r) - 2.0 * a / sqrt(M_PI) * exp(-x) / s;
}
double dsf_E(double a, double s) {
    const double x = a * a * s;
    if (x < 0.5) {
        double sum = 0.0, term = 1.0;
        for (int m = 0; m < 20; ++m) {
            sum += term / (2 * m + 1);
            term *= -x / (m + 1);
        }
        return a * 2.0 / sqrt(M_PI) * sum;
    }
    return erf(a * sqrt(s)) / sqrt(s);
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
    c.sc = (float)sc;
    c.ecut = (float)ecut;
    c.sig2 = (float)c.sig2_d;
    c.eps4 = (float)c.eps4_d;
    c.neps24 = (float)(-c.eps24_d);
    c.ljshift = (float)ljs;
    c.L = (float)s->L;
    c.invL = (float)(1.0 / s->L);
    c.qO_ke = (float)(COULOMB * f.q_O);
    c.qH_ke = (float)(COULOMB * (-0.5 * f.q_O));
    c.tscale = (float)(2.0 / (rc * rc));
    list_bucket_params(s, &c.bucket_lo, &c.bucket_inv);
    const double half = 0.5 * rc * rc;   // s = (t + 1) rc^2 / 2
    chebyshev_fit([&](double t) { return dsf_G(a, (t + 1.0) * half); }, c.gpoly);
    chebyshev_fit([&](double t) { return dsf_E(a, (t + 1.0) * half); }, c.epoly);
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
    A.nO = s->nbr_nO;
    A.nbr = s->nbr;
    A.charge_s = s->charge_s;
    A.type_s = s->type_s;
    A.perm = s->perm;
    A.F = s->Ffix;
    A.epair = s->e_pair;
    A.status = s->status;
    A.dev_max = s->dev_max;
    A.dev_atom = s->dev_atom;
    A.skip = s->pair_skip;
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
    B.status = s->status;
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

// The batched force stage (mixed precision): pair items are blocks of PAIR_WARPS / W atoms,
// costed by the warp passes of their list rows (a pass evaluates 32 / max(1, P/2) entries);
// bonded items are blocks of 128 (molecule, bead) pairs.  Every resident block gets an equal
// share of every specialisation's items, specialisation by specialisation.
int batch_stage_force(const std::vector<qhp_system_s*>& v, BatchStage& st, int* n_pair_items, int halves) {
    if (v.size() > 0xffff) {
        set_error("a batch holds at most 65535 systems");
        return QHP_ERR_ARG;
    }
    std::vector<ForceArgs> a;
    std::vector<int2> items;
    std::vector<double> cost;
    for (size_t k = 0; k < v.size(); ++k) {
        const qhp_system_s* s = v[k];
        ForceArgs fa;
        fa.p = make_pair_args(s);
        fa.b = make_bond_args(s);
        a.push_back(fa);
        const int P = s->P, W = fa.p.W, lp = __builtin_ctz((unsigned)P);
        const int kind = batch_pair_stage(lp, fa.p.all, W);
        const int apb = PAIR_WARPS / W;
        const int nb = (s->N + apb - 1) / apb;
        std::vector<int> cnt(s->N);
        QHP_CUDA(cudaMemcpy(cnt.data(), s->nbr_count, sizeof(int) * s->N, cudaMemcpyDeviceToHost));
        // warp passes per entry: a pass evaluates 32 / LPE entries, LPE = max(1, P / 2) lanes each
        const double passes = (double)std::max(1, P / 2) / 32.0;
        for (int b = 0; b < nb; ++b) {
            double c = 0.0;
            for (int i = b * apb; i < std::min(s->N, (b + 1) * apb); ++i) c += (double)cnt[i] * passes;
            items.push_back(make_int2((kind << 16) | (int)k, b));
            cost.push_back(c / PAIR_WARPS + 2.0);   // per warp of the block, plus the row set-up and sums
        }
        const int nbb = (s->n_mol * P + 127) / 128;
        for (int b = 0; b < nbb; ++b) {
            items.push_back(make_int2((FORCE_BONDED_VARIANT << 16) | (int)k, b));
            cost.push_back(1.0);
        }
    }
    if (n_pair_items) {
        *n_pair_items = 0;
        for (const int2& w : items) *n_pair_items += (w.x >> 16) != FORCE_BONDED_VARIANT;
    }
    st.smem = 0;
    const int grid = halves;
    // one phase per specialisation present (in kind order, bonded last): the blocks of an SM run
    // the same code at about the same time instead of a mix of the 43 bodies
    std::vector<int> kinds;
    for (const int2& w : items) kinds.push_back(w.x >> 16);
    std::vector<int> uniq(kinds);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    std::vector<int> phase(items.size());
    for (size_t i = 0; i < items.size(); ++i)
        phase[i] = (int)(std::lower_bound(uniq.begin(), uniq.end(), kinds[i]) - uniq.begin());
    return stage_upload_phased(st, a.data(), sizeof(ForceArgs) * a.size(), items, cost, phase, grid);
}

// Shared memory of the step kernel (the larger of the integrate / project group's and the two
// halves' pair sums) and its co-resident grid: every block must be resident at once for the
// grid barriers, which a cooperative launch of at most this many blocks guarantees.
int step_batch_config(int maxP, int* grid, size_t* smem) {
    const size_t sm = std::max(batch_group_smem(maxP), 2 * sizeof(PairSmem));
    if (sm > 48 * 1024) QHP_CUDA(cudaFuncSetAttribute(k_step_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    QHP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batch, STEP_THREADS, sm));
    if (per_sm < 1) {
        set_error("the batched step kernel does not fit on an SM");
        return QHP_ERR_STATE;
    }
    *grid = per_sm * sm_count();
    *smem = sm;
    return QHP_OK;
}

cudaError_t launch_step_batch(const BatchStage& integ, const BatchStage& force, const BatchStage& proj,
                              const CheckArgs* checks, int* done, const int* nitems, StepBatchState* state,
                              long long wait_ns, int grid, size_t smem, cudaStream_t stream) {
    StepBatchArgs S;
    S.iargs = (const IntegrateArgs*)integ.args;
    S.iitems = integ.items;
    S.iranges = integ.ranges;
    S.fargs = (const ForceArgs*)force.args;
    S.fitems = force.items;
    S.franges = force.ranges;
    S.pargs = (const ProjectArgs*)proj.args;
    S.pitems = proj.items;
    S.pranges = proj.ranges;
    S.checks = checks;
    S.done = done;
    S.nitems = nitems;
    S.st = state;
    S.wait_ns = wait_ns;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(STEP_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_batch, S);
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
    A.dev_atom = s->dev_atom_c;
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

using namespace qhp;

extern "C" int qhp_selftest_grid_barrier(long long wait_ns, unsigned* status_out) {
    if (wait_ns < 1000 || wait_ns > 10000000000LL) {
        set_error("qhp_selftest_grid_barrier: wait_ns must lie in [1e3, 1e10]");
        return QHP_ERR_ARG;
    }
    StepBatchState* st = nullptr;
    QHP_CUDA(cudaMalloc(&st, sizeof(StepBatchState)));
    cudaError_t e = cudaMemset(st, 0, sizeof(StepBatchState));
    if (e == cudaSuccess) {
        void* args[] = {&st, &wait_ns};
        e = cudaLaunchCooperativeKernel((const void*)k_grid_sync_selftest, dim3(2), dim3(32), args, 0, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    StepBatchState h = {};
    if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(st);
    if (e != cudaSuccess) return cuda_fail(e, "grid barrier self-test");
    if (status_out) *status_out = h.status;
    if (h.status & ST_TIMEOUT) {
        set_error("grid barrier wait ran out after %lld ns (self-test: one arrival never comes)", wait_ns);
        return QHP_ERR_TIMEOUT;
    }
    return QHP_OK;
}
