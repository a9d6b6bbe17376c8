// Centroid cell grid, counting sort and Verlet list (Sec. III.A.3: one list on
// ring-polymer centroids serves every bead).
//
// Every kernel of the rebuild chain reads the device rebuild flag first and
// returns at once when it is clear, so the chain can sit inside a captured
// CUDA graph that replays every step.
//
// Bit-exactness with the definition: the cell of a centroid C is
//   t = C/L, frac = t - floor(t) (0 if it rounds to 1), c = min(floor(frac n_c), n_c - 1),
// and (i, j) is listed iff molecules differ and
//   d = C_j - C_i - L rint((C_j - C_i)/L), (dx*dx + dy*dy) + dz*dz < r_list^2,
// with each operation rounded on its own (explicit _rn intrinsics, no FMA).  An
// FP32 prefilter on wrapped centroids decides the candidates that are more than
// 1e-3 A away from r_list; the rest get the exact FP64 test above.
#include <algorithm>
#include <vector>

#include "qhp_internal.cuh"

namespace qhp {

namespace {

__device__ __forceinline__ double min_image_rn(double d, double L) {
    return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// Error-free transformation a + b = s + e (Knuth's TwoSum; additions only, so no FMA
// contraction can alter it).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hj + lj) + (sh + sl) - (hi + li), the result small while the terms are up to a box
// length: the large parts are combined exactly, so the FP32 result is essentially the
// correctly rounded separation.
__device__ __forceinline__ float sep_df(float hj, float lj, float hi, float li, float sh, float sl) {
    float s1, e1, s2, e2;
    two_sum(hj, sh, s1, e1);
    two_sum(s1, -hi, s2, e2);
    return s2 + ((e1 + e2) + ((lj - li) + sl));
}

// Same image for |d| < L/2 - tiny, by a multiply instead of a correctly rounded divide;
// used for the anchor separations stored in list entries, which need accuracy, not bit
// equality with the list definition (FP64 division is expensive on this part).
__device__ __forceinline__ double min_image_fast(double d, double L, double invL) {
    return fma(-L, rint(d * invL), d);
}

__device__ __forceinline__ int cell_coord(double C, double L, int n_c, double* frac_out) {
    const double t = __ddiv_rn(C, L);
    double frac = __dsub_rn(t, floor(t));
    // 1.0 can come from rounding; a NaN or infinite coordinate (a blown-up state, which the
    // status word reports) goes to cell 0, so that no index is ever formed from it
    if (!(frac >= 0.0 && frac < 1.0)) frac = 0.0;
    *frac_out = frac;
    int c = (int)floor(__dmul_rn(frac, (double)n_c));
    return c < n_c - 1 ? c : n_c - 1;
}

// Decide whether the list must be rebuilt; clear the deviation maximum if so.  Inside a
// step graph the decision also drives the conditional node that holds the rebuild chain.
__global__ void k_check(unsigned* dev_max, float thr2, int* flag, int force, unsigned* rebuild_count,
                        cudaGraphConditionalHandle cond, int use_cond) {
    const float dmax = __uint_as_float(*dev_max);
    const int rebuild = force || !(dmax <= thr2);   // NaN also triggers a rebuild
    *flag = rebuild;
    if (rebuild) {
        *dev_max = 0u;
        *rebuild_count += 1u;
    }
    if (use_cond) {
        cudaGraphSetConditional(cond, rebuild ? 1u : 0u);
        if (rebuild) rebuild_count[1] += 1u;   // rebuild chains run inside the step graph
    }
}

// Right after a rebuild the deviation maximum is measured from the new anchors; the list
// covers every bead pair within rc only if no bead lies farther than skin/2 from its anchor.
__global__ void k_check_cover(const int* flag, const unsigned* dev_max, float thr2, unsigned* status) {
    if (!*flag) return;
    if (!(__uint_as_float(*dev_max) <= thr2)) atomicOr(status, ST_SPREAD);
}

__global__ void k_zero_ints(const int* flag, int* a, int n) {
    if (!*flag) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0;
}

// New anchors = current centroids Q_0 (or, with keep, the stored anchors of a
// checkpoint); cell of every atom (list mode).
__global__ void k_cells(const int* flag, int N, int P, const double* Q, double L, int n_c, int list_mode,
                        double* anchor, int* cell, int* cell_count, int keep) {
    if (!*flag) return;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    int c3[3];
    for (int d = 0; d < 3; ++d) {
        const double C = keep ? anchor[a * 3 + d] : Q[((size_t)a * 3 + d) * P];
        if (!keep) anchor[a * 3 + d] = C;
        double fr;
        c3[d] = cell_coord(C, L, n_c, &fr);
    }
    if (list_mode) {
        const int c = (c3[2] * n_c + c3[1]) * n_c + c3[0];
        cell[a] = c;
        atomicAdd(&cell_count[c], 1);
    }
}

// Exclusive scan of n values (single block of 1024 threads).
__global__ void k_scan(const int* flag, const int* in, int* out, int n, int64_t cap, int* total, unsigned* status) {
    if (!*flag) return;
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int v = i < n ? in[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int excl = carry + x - v + (w > 0 ? warp_sums[w - 1] : 0);
        if (i < n) out[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[n] = carry;
        if (total) *total = carry;
        if (cap >= 0 && (int64_t)carry > cap) atomicOr(status, ST_LIST_OVERFLOW);
    }
}

__global__ void k_cell_scatter(const int* flag, int N, const int* cell, const int* cell_start, int* cell_fill,
                               int* tmp, const unsigned* status) {
    if (!*flag) return;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    const int c = cell[a];
    const int slot = atomicAdd(&cell_fill[c], 1);
    if (QHP_IN_BOUNDS(cell_start[c] + slot, N, status)) tmp[cell_start[c] + slot] = a;
}

// Order each cell's atoms by index: rank = number of smaller indices in the cell.
__global__ void k_cell_sort(const int* flag, const int* cell_start, const int* tmp, int* perm, int* iperm) {
    if (!*flag) return;
    const int c = blockIdx.x;
    const int s0 = cell_start[c], s1 = cell_start[c + 1];
    for (int e = s0 + threadIdx.x; e < s1; e += blockDim.x) {
        const int a = tmp[e];
        int rank = 0;
        for (int k = s0; k < s1; ++k) rank += tmp[k] < a;
        perm[s0 + rank] = a;
        iperm[a] = s0 + rank;
    }
}

__global__ void k_identity_order(const int* flag, int N, int* perm, int* iperm) {
    if (!*flag) return;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    perm[a] = a;
    iperm[a] = a;
}

// Sorted per-atom attributes, FP32 wrapped centroids and (mixed) intramolecular anchor offsets.
__global__ void k_sorted_attrs(const int* flag, int N, double L, const int* perm, const int* type, const int* mol,
                               const double* anchor, float q_O, float q_H, float* charge_s, int* type_s, int* mol_s,
                               float4* cw, float4* cwl, float* dA) {
    if (!*flag) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int a = perm[s];
    const int ty = type[a];
    charge_s[s] = ty == 0 ? q_O : q_H;
    type_s[s] = ty;
    mol_s[s] = mol[a];
    double w[3];
    for (int d = 0; d < 3; ++d) {   // wrapped coordinate frac * L, consistent with the cell index
        double fr;
        (void)cell_coord(anchor[a * 3 + d], L, 1, &fr);
        w[d] = fr * L;
    }
    const float h0 = (float)w[0], h1 = (float)w[1], h2 = (float)w[2];
    cw[s] = make_float4(h0, h1, h2, 0.0f);
    cwl[s] = make_float4((float)(w[0] - (double)h0), (float)(w[1] - (double)h1), (float)(w[2] - (double)h2), 0.0f);
    if (dA && (a % 3) != 0) {     // H atom: min-image A_H - A_O of its molecule
        const int o = a - (a % 3);
        float* out = dA + ((size_t)(a / 3) * 2 + (a % 3) - 1) * 4;
        for (int d = 0; d < 3; ++d) out[d] = (float)min_image_rn(anchor[a * 3 + d] - anchor[o * 3 + d], L);
        out[3] = 0.0f;
    }
}

// Centroid Verlet list, one block per cell: the 125 stencil cells' candidates are staged
// in shared memory (in stencil order, ascending index within a cell, i.e. the same order as
// the oracle's per-atom scan) and every atom of the cell tests them from there.  FILL = false
// counts (set-up), true writes the rows.  A warp tests 32 candidates at a time; the accepted
// ones go to a per-warp queue and entries are written 32 at a time from the queue, so the
// separation arithmetic runs on full warps (a quarter of the candidates are accepted).
constexpr int LC_THREADS = 256;
constexpr int LC_WARPS = LC_THREADS / 32;
constexpr int LC_MAXA = 8;     // atoms per warp in one pass over the staged candidates
constexpr int LC_CHUNK = 768;   // 3 x 768 x 16 B of staged candidates: within the 48 KB static limit

template <bool FILL>
__global__ void __launch_bounds__(LC_THREADS, 4) k_list_cells(
    const int* flag, int N, double L, int n_c, double r2max, float lo2, float hi2, const int* perm,
    const int* cell_start, const float4* cw, const float4* cwl, const int* mol_s, const int* type_s,
    const double* anchor, int* count, const int* start, int4* nbr, int row_cap, unsigned* status) {
    if (!*flag) return;
    __shared__ int c_beg[125], c_cnt[125], c_off[126];
    __shared__ float4 c_sh[125], c_lo[125];   // periodic shift of each stencil cell (hi, lo parts)
    __shared__ float4 s_w[LC_CHUNK];     // shifted wrapped centroid (prefilter), .w = mol as int bits
    __shared__ float4 s_l[LC_CHUNK];     // low parts, .w = j | H bit as int bits
    __shared__ float4 s_s[LC_CHUNK];     // unshifted wrapped centroid (hi), .w = stencil cell as int bits
    __shared__ int s_q[LC_WARPS][32];    // per-warp queue of accepted candidates
    __shared__ int s_cnt[LC_WARPS][LC_MAXA];   // row lengths so far of the warp's atoms
    const int c = blockIdx.x;
    const int i0 = cell_start[c], i1 = cell_start[c + 1];
    if (i0 == i1) return;
    const int cx = c % n_c, cy = (c / n_c) % n_c, cz = c / (n_c * n_c);
    const float Lf = (float)L;
    const float Llo = (float)(L - (double)Lf);
    const int t = threadIdx.x;
    if (t < 125) {
        const int dx = t % 5 - 2, dy = (t / 5) % 5 - 2, dz = t / 25 - 2;   // stencil order dz, dy, dx
        int x = cx + dx, y = cy + dy, z = cz + dz;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        if (x < 0) { x += n_c; sx = -Lf; } else if (x >= n_c) { x -= n_c; sx = Lf; }
        if (y < 0) { y += n_c; sy = -Lf; } else if (y >= n_c) { y -= n_c; sy = Lf; }
        if (z < 0) { z += n_c; sz = -Lf; } else if (z >= n_c) { z -= n_c; sz = Lf; }
        const int cj = (z * n_c + y) * n_c + x;
        c_beg[t] = cell_start[cj];
        c_cnt[t] = cell_start[cj + 1] - c_beg[t];
        c_sh[t] = make_float4(sx, sy, sz, 0.f);
        c_lo[t] = make_float4(sx > 0.f ? Llo : (sx < 0.f ? -Llo : 0.f), sy > 0.f ? Llo : (sy < 0.f ? -Llo : 0.f),
                              sz > 0.f ? Llo : (sz < 0.f ? -Llo : 0.f), 0.f);
    }
    __syncthreads();
    if (t == 0) {
        int o = 0;
        for (int k = 0; k < 125; ++k) {
            c_off[k] = o;
            o += c_cnt[k];
        }
        c_off[125] = o;
    }
    __syncthreads();
    const int M = c_off[125];
    const int lane = t & 31, w = t >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int ib = i0; ib < i1; ib += LC_WARPS * LC_MAXA) {
        if (lane < LC_MAXA) s_cnt[w][lane] = 0;
        for (int m0 = 0; m0 < M; m0 += LC_CHUNK) {
            const int mc = min(LC_CHUNK, M - m0);
            const int mpad = (mc + 31) & ~31;   // slots mc .. mpad-1 hold candidates that never pass
            __syncthreads();
            for (int e = t; e < mpad; e += LC_THREADS) {
                if (e >= mc) {
                    s_w[e] = make_float4(INFINITY, 0.f, 0.f, __int_as_float(-1));
                    continue;
                }
                const int m = m0 + e;
                int lo = 0, hi = 124;   // stencil cell of candidate m (binary search over 125 offsets)
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (c_off[mid] <= m) lo = mid;
                    else hi = mid - 1;
                }
                const int k = lo;
                const int j = c_beg[k] + (m - c_off[k]);
                const float4 wj = cw[j];
                const float4 lj = cwl[j];
                const float4 sh = c_sh[k];
                s_w[e] = make_float4(wj.x + sh.x, wj.y + sh.y, wj.z + sh.z, __int_as_float(mol_s[j]));
                s_l[e] = make_float4(lj.x, lj.y, lj.z, __int_as_float(j | (type_s[j] ? (int)0x80000000u : 0)));
                s_s[e] = make_float4(wj.x, wj.y, wj.z, __int_as_float(k));
            }
            __syncthreads();
            for (int a = 0; a < LC_MAXA; ++a) {
                const int i = ib + w + LC_WARPS * a;
                if (i >= i1) break;
                const float4 wi = cw[i];
                const int mi = mol_s[i];
                const int ai = perm[i];
                __syncwarp();
                int cnt = s_cnt[w][a];
                int base = 0, lim = 0, qn = 0;
                float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
                if (FILL) {
                    base = start[i] + cnt;
                    lim = start[i] + row_cap;
                    li = cwl[i];
                }
                // write the first n queued candidates as entries base .. base + n - 1
                auto flush = [&](int n) {
                    __syncwarp();
                    if (lane < n) {
                        const int e = s_q[w][lane];
                        const int pos = base + lane;
                        if (pos < lim) {
                            const float4 sl = s_l[e];
                            const float4 wj = s_s[e];
                            const int k = __float_as_int(wj.w);
                            const float4 sh = c_sh[k], lo = c_lo[k];
                            const float Dx = sep_df(wj.x, sl.x, wi.x, li.x, sh.x, lo.x);
                            const float Dy = sep_df(wj.y, sl.y, wi.y, li.y, sh.y, lo.y);
                            const float Dz = sep_df(wj.z, sl.z, wi.z, li.z, sh.z, lo.z);
                            nbr[pos] = make_int4(__float_as_int(sl.w), __float_as_int(Dx), __float_as_int(Dy),
                                                 __float_as_int(Dz));
                        }
                    }
                    base += n;
                    __syncwarp();
                };
                for (int eb = 0; eb < mpad; eb += 32) {
                    const int e = eb + lane;
                    const float4 sw = s_w[e];
                    const float ddx = sw.x - wi.x, ddy = sw.y - wi.y, ddz = sw.z - wi.z;
                    const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    const bool other = __float_as_int(sw.w) != mi;
                    bool acc = other && r2 < lo2;
                    const bool band = other && r2 >= lo2 && r2 <= hi2;
                    if (__any_sync(0xffffffffu, band) && band) {   // borderline: the exact FP64 definition decides
                        const int j = __float_as_int(s_l[e].w) & 0x7fffffff;
                        const int aj = perm[j];
                        const double ex = min_image_rn(__dsub_rn(anchor[aj * 3], anchor[ai * 3]), L);
                        const double ey = min_image_rn(__dsub_rn(anchor[aj * 3 + 1], anchor[ai * 3 + 1]), L);
                        const double ez = min_image_rn(__dsub_rn(anchor[aj * 3 + 2], anchor[ai * 3 + 2]), L);
                        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                        acc = d2 < r2max;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, acc);
                    const int nacc = __popc(bal);
                    if (FILL) {
                        // queue slots qn, qn+1, ... in candidate order; a full queue is written at once
                        const int slot = qn + __popc(bal & lt_mask);
                        if (acc && slot < 32) s_q[w][slot] = e;
                        if (qn + nacc >= 32) {
                            flush(32);
                            if (acc && slot >= 32) s_q[w][slot - 32] = e;
                            qn += nacc - 32;
                        } else {
                            qn += nacc;
                        }
                    }
                    cnt += nacc;
                }
                if (FILL && qn > 0) flush(qn);   // the staged candidates are replaced by the next chunk
                __syncwarp();
                if (lane == 0) s_cnt[w][a] = cnt;
            }
        }
        __syncwarp();
        if (lane < LC_MAXA) {
            const int i = ib + w + LC_WARPS * lane;
            if (i < i1) {
                const int cnt = s_cnt[w][lane];
                // a row is never longer than its slot: an overrun is reported, not read
                if (FILL && cnt > row_cap) atomicOr(status, ST_LIST_OVERFLOW);
                count[i] = FILL ? min(cnt, row_cap) : cnt;
            }
        }
    }
}

// Small boxes (no cell grid), warp per atom, identity order: every atom of another
// molecule whose minimum-image anchor distance is below r_list, by brute force with the
// same FP64 operation order as the cell path.  The pair kernel then applies a per-bead
// minimum image, which r_list >= L/2 makes necessary.
template <bool FILL>
__global__ void k_list_all(const int* flag, int N, double L, double r2max, const int* mol_s, const int* type_s,
                           const double* anchor, int* count, const int* start, int4* nbr, int row_cap,
                           unsigned* status) {
    if (!*flag) return;
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const int mi = mol_s[i];
    const double Ax = anchor[i * 3], Ay = anchor[i * 3 + 1], Az = anchor[i * 3 + 2];
    int cnt = 0;
    const int base = FILL ? start[i] : 0;
    for (int jb = 0; jb < N; jb += 32) {
        const int j = jb + lane;
        bool acc = j < N && mol_s[j] != mi;
        if (acc) {
            const double ex = min_image_rn(__dsub_rn(anchor[j * 3], Ax), L);
            const double ey = min_image_rn(__dsub_rn(anchor[j * 3 + 1], Ay), L);
            const double ez = min_image_rn(__dsub_rn(anchor[j * 3 + 2], Az), L);
            acc = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) < r2max;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        if (FILL && acc) {
            const int pos = base + cnt + __popc(bal & ((1u << lane) - 1u));
            if (pos < base + row_cap) {
                const double iL = 1.0 / L;
                const float Dx = (float)min_image_fast(anchor[j * 3] - anchor[i * 3], L, iL);
                const float Dy = (float)min_image_fast(anchor[j * 3 + 1] - anchor[i * 3 + 1], L, iL);
                const float Dz = (float)min_image_fast(anchor[j * 3 + 2] - anchor[i * 3 + 2], L, iL);
                nbr[pos] = make_int4(j | (type_s[j] ? (int)0x80000000u : 0), __float_as_int(Dx), __float_as_int(Dy),
                                     __float_as_int(Dz));
            }
        }
        cnt += __popc(bal);
    }
    if (lane == 0) {
        if (FILL && cnt > row_cap) atomicOr(status, ST_LIST_OVERFLOW);
        count[i] = FILL ? min(cnt, row_cap) : cnt;
    }
}

// Row order for the pair kernel: every row's entries sorted by (partner type, |D|^2 bucket) -
// list_bucket - stably, so that equal keys keep the fill order and the result is a function of
// the row's set of partners alone; also counts each row's O partners.  One block per row, the
// row staged in shared memory: a stable counting sort in which the four warps take contiguous
// quarters of the row, count keys per quarter, and scatter their quarters in order.
constexpr int LS_THREADS = 128;
constexpr int LS_WARPS = LS_THREADS / 32;
constexpr int LS_KEYS = 2 * LIST_BUCKETS;
static_assert(LS_KEYS <= LS_THREADS, "one thread per key in the per-key passes");

__device__ __forceinline__ int list_key(int4 e, float lo, float inv) {
    return (e.x < 0 ? LIST_BUCKETS : 0) + list_bucket(__int_as_float(e.y), __int_as_float(e.z), __int_as_float(e.w), lo, inv);
}

// Persistent grid: a block sorts rows blockIdx.x, + gridDim.x, ... (so a step without a rebuild
// costs one small launch, not one block per row).
__global__ void __launch_bounds__(LS_THREADS) k_list_sort(const int* flag, int N, const int* start, const int* count,
                                                          int4* nbr, int* nO, float lo, float inv,
                                                          const unsigned* status) {
    if (!*flag) return;
    extern __shared__ int4 row[];
    __shared__ int hist[LS_WARPS][LS_KEYS];   // key counts per quarter, then each quarter's first slot per key
    __shared__ int base[LS_KEYS];             // key totals, then their exclusive prefix sums
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        __syncthreads();                          // the previous row is written out
        const int t = threadIdx.x, lane = t & 31, w = t >> 5;
        const int n = count[i];
        int4* g = nbr + start[i];
        for (int k = t; k < n; k += LS_THREADS) row[k] = g[k];
        for (int k = t; k < LS_WARPS * LS_KEYS; k += LS_THREADS) (&hist[0][0])[k] = 0;
        __syncthreads();
        const int q = (n + LS_WARPS - 1) / LS_WARPS;
        const int k0 = min(n, w * q), k1 = min(n, k0 + q);
        const unsigned lt = (1u << lane) - 1u;
        for (int kb = k0; kb < k1; kb += 32) {
            const int k = kb + lane;
            const int key = k < k1 ? list_key(row[k], lo, inv) : -1 - lane;   // idle lanes: distinct dummies
            const unsigned same = __match_any_sync(0xffffffffu, key);
            if (k < k1 && (same & lt) == 0u) hist[w][key] += __popc(same);     // one lane per key
            __syncwarp();
        }
        __syncthreads();
        if (t < LS_KEYS) {
            int sum = 0;
            for (int v = 0; v < LS_WARPS; ++v) sum += hist[v][t];
            base[t] = sum;
        }
        __syncthreads();
        if (w == 0) {   // exclusive prefix over the keys, KPL consecutive keys per lane
            constexpr int KPL = (LS_KEYS + 31) / 32;
            int v[KPL], x = 0;
            for (int k = 0; k < KPL; ++k) {
                const int key = lane * KPL + k;
                v[k] = key < LS_KEYS ? base[key] : 0;
                x += v[k];
            }
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            int run = x;   // inclusive prefix through this lane's keys
            for (int k = KPL - 1; k >= 0; --k) {
                run -= v[k];
                const int key = lane * KPL + k;
                if (key < LS_KEYS) base[key] = run;
            }
        }
        __syncthreads();
        if (t < LS_KEYS) {
            int sum = base[t];
            for (int v = 0; v < LS_WARPS; ++v) {
                const int h = hist[v][t];
                hist[v][t] = sum;
                sum += h;
            }
        }
        __syncthreads();
        for (int kb = k0; kb < k1; kb += 32) {
            const int k = kb + lane;
            const int4 e = k < k1 ? row[k] : make_int4(0, 0, 0, 0);
            const int key = k < k1 ? list_key(e, lo, inv) : -1 - lane;
            const unsigned same = __match_any_sync(0xffffffffu, key);
            if (k < k1) {   // the partner word takes the entry's bucket in bits 26-30
                const int4 out = make_int4((e.x & ~(31 << ENTRY_J_BITS)) | ((key % LIST_BUCKETS) << ENTRY_J_BITS), e.y, e.z, e.w);
                const int dst = hist[w][key] + __popc(same & lt);
                if (QHP_IN_BOUNDS(dst, n, status)) g[dst] = out;
            }
            __syncwarp();
            if (k < k1 && (same & lt) == 0u) hist[w][key] += __popc(same);
            __syncwarp();
        }
        if (t == 0) nO[i] = base[LIST_BUCKETS];
    }
}

}  // namespace

void list_bucket_params(const qhp_system_s* s, float* lo, float* inv) {
    const double l = std::max(0.0, s->ff.rc - 1.0);
    *lo = (float)(l * l);
    *inv = (float)((double)LIST_BUCKETS / (s->r_list * s->r_list - l * l));
}

// The limit is a property of the kernel, shared by every system: it is raised once to the
// longest row the sort handles, so that no system's set-up lowers it below another's rows.
int list_sort_prepare(qhp_system_s* s) {
    if (s->row_cap > LIST_SORT_MAX_ROW) return QHP_ERR_ARG;
    QHP_CUDA(cudaFuncSetAttribute(k_list_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(int4) * (size_t)LIST_SORT_MAX_ROW)));
    int per_sm = 0;
    QHP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_list_sort, LS_THREADS,
                                                           sizeof(int4) * (size_t)s->row_cap));
    s->sort_grid = std::max(1, per_sm) * sm_count();
    return QHP_OK;
}

cudaError_t launch_list_check(qhp_system_s* s, bool force) {
    const float half = (float)(0.5 * s->ff.skin);
    s->launches++;
    k_check<<<1, 1, 0, s->stream>>>(s->dev_max, half * half, s->rebuild_flag, force ? 1 : 0, s->rebuild_count,
                                    s->cond_handle, s->cond_active);
    return cudaGetLastError();
}

cudaError_t launch_cover_check(qhp_system_s* s) {
    const float half = (float)(0.5 * s->ff.skin);
    s->launches++;
    k_check_cover<<<1, 1, 0, s->stream>>>(s->rebuild_flag, s->dev_max, half * half, s->status);
    return cudaGetLastError();
}

cudaError_t launch_rebuild(qhp_system_s* s) {
    const int N = s->N;
    const int tb = 256, gN = (N + tb - 1) / tb;
    const int ncell = s->n_c * s->n_c * s->n_c;
    const int* flag = s->rebuild_flag;
    cudaStream_t st = s->stream;
    if (s->list_mode) {
        k_zero_ints<<<(ncell + tb - 1) / tb, tb, 0, st>>>(flag, s->cell_count, ncell);
        k_zero_ints<<<(ncell + tb - 1) / tb, tb, 0, st>>>(flag, s->cell_fill, ncell);
        k_cells<<<gN, tb, 0, st>>>(flag, N, s->P, s->Q, s->L, s->n_c, 1, s->anchor, s->cell, s->cell_count,
                                   s->keep_anchor);
        k_scan<<<1, 1024, 0, st>>>(flag, s->cell_count, s->cell_start, ncell, -1, nullptr, s->status);
        k_cell_scatter<<<gN, tb, 0, st>>>(flag, N, s->cell, s->cell_start, s->cell_fill, s->tmp_idx, s->status);
        k_cell_sort<<<ncell, 128, 0, st>>>(flag, s->cell_start, s->tmp_idx, s->perm, s->iperm);
        s->launches += 6;
    } else {
        k_cells<<<gN, tb, 0, st>>>(flag, N, s->P, s->Q, s->L, 1, 0, s->anchor, nullptr, nullptr, s->keep_anchor);
        k_identity_order<<<gN, tb, 0, st>>>(flag, N, s->perm, s->iperm);
        s->launches += 2;
    }
    k_sorted_attrs<<<gN, tb, 0, st>>>(flag, N, s->L, s->perm, s->type_d, s->mol_d, s->anchor, (float)s->ff.q_O,
                                      (float)(-0.5 * s->ff.q_O), s->charge_s, s->type_s, s->mol_s, s->cw, s->cwl,
                                      s->precision == QHP_MIXED ? s->dA : nullptr);
    const int wb = 128, gW = (N * 32 + wb - 1) / wb;
    const double r2max = s->r_list * s->r_list;
    const float lo = (float)(s->r_list - 1e-3), hi = (float)(s->r_list + 1e-3);
    // one pass: every atom owns a fixed row of row_cap entries, its length goes to nbr_count
    if (s->list_mode) {
        k_list_cells<true><<<ncell, LC_THREADS, 0, st>>>(flag, N, s->L, s->n_c, r2max, lo * lo, hi * hi, s->perm,
                                                         s->cell_start, s->cw, s->cwl, s->mol_s, s->type_s, s->anchor,
                                                         s->nbr_count, s->nbr_start, s->nbr, s->row_cap, s->status);
    } else {
        k_list_all<true><<<gW, wb, 0, st>>>(flag, N, s->L, r2max, s->mol_s, s->type_s, s->anchor, s->nbr_count, s->nbr_start,
                                            s->nbr, s->row_cap, s->status);
    }
    float blo, binv;
    list_bucket_params(s, &blo, &binv);
    k_list_sort<<<std::min(N, s->sort_grid), LS_THREADS, sizeof(int4) * (size_t)s->row_cap, st>>>(
        flag, N, s->nbr_start, s->nbr_count, s->nbr, s->nbr_nO, blo, binv, s->status);
    s->launches += 3;
    return cudaGetLastError();
}

// Row lengths of the list for the current centroids (synchronous; sizes the rows).
int host_list_size(qhp_system_s* s, int64_t* max_row) {
    int one = 1;
    QHP_CUDA(cudaMemcpyAsync(s->rebuild_flag, &one, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    const int N = s->N;
    const int tb = 256, gN = (N + tb - 1) / tb;
    const int ncell = s->n_c * s->n_c * s->n_c;
    const int* flag = s->rebuild_flag;
    cudaStream_t st = s->stream;
    if (s->list_mode) {
        k_zero_ints<<<(ncell + tb - 1) / tb, tb, 0, st>>>(flag, s->cell_count, ncell);
        k_zero_ints<<<(ncell + tb - 1) / tb, tb, 0, st>>>(flag, s->cell_fill, ncell);
        k_cells<<<gN, tb, 0, st>>>(flag, N, s->P, s->Q, s->L, s->n_c, 1, s->anchor, s->cell, s->cell_count,
                                   s->keep_anchor);
        k_scan<<<1, 1024, 0, st>>>(flag, s->cell_count, s->cell_start, ncell, -1, nullptr, s->status);
        k_cell_scatter<<<gN, tb, 0, st>>>(flag, N, s->cell, s->cell_start, s->cell_fill, s->tmp_idx, s->status);
        k_cell_sort<<<ncell, 128, 0, st>>>(flag, s->cell_start, s->tmp_idx, s->perm, s->iperm);
    } else {
        k_cells<<<gN, tb, 0, st>>>(flag, N, s->P, s->Q, s->L, 1, 0, s->anchor, nullptr, nullptr, s->keep_anchor);
        k_identity_order<<<gN, tb, 0, st>>>(flag, N, s->perm, s->iperm);
    }
    k_sorted_attrs<<<gN, tb, 0, st>>>(flag, N, s->L, s->perm, s->type_d, s->mol_d, s->anchor, (float)s->ff.q_O,
                                      (float)(-0.5 * s->ff.q_O), s->charge_s, s->type_s, s->mol_s, s->cw, s->cwl,
                                      s->precision == QHP_MIXED ? s->dA : nullptr);
    const int wb = 128, gW = (N * 32 + wb - 1) / wb;
    const double r2max = s->r_list * s->r_list;
    const float lo = (float)(s->r_list - 1e-3), hi = (float)(s->r_list + 1e-3);
    if (s->list_mode)
        k_list_cells<false><<<ncell, LC_THREADS, 0, st>>>(flag, N, s->L, s->n_c, r2max, lo * lo, hi * hi, s->perm,
                                                          s->cell_start, s->cw, s->cwl, s->mol_s, s->type_s, s->anchor,
                                                          s->nbr_count, nullptr, nullptr, 0, s->status);
    else
        k_list_all<false><<<gW, wb, 0, st>>>(flag, N, s->L, r2max, s->mol_s, s->type_s, s->anchor, s->nbr_count, nullptr,
                                             nullptr, 0, s->status);
    s->launches += 9;
    QHP_CUDA(cudaGetLastError());
    std::vector<int> cnt(N);
    QHP_CUDA(cudaMemcpyAsync(cnt.data(), s->nbr_count, sizeof(int) * N, cudaMemcpyDeviceToHost, s->stream));
    QHP_CUDA(cudaStreamSynchronize(s->stream));
    int m = 0;
    for (int v : cnt) m = v > m ? v : m;
    *max_row = m;
    return QHP_OK;
}

}  // namespace qhp
