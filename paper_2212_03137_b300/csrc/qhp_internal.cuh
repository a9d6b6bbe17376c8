// Internal declarations of the qhp library: system state, device helpers, kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qhp.h"

namespace qhp {

// Host-side trace range around an entry point (header-only NVTX: a no-op unless a profiler
// is attached), so that timelines show each call and the launches it enqueues.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// ------------------------------------------------------------------ units
// kcal/mol, Angstrom, amu, ps.  ACC converts (kcal/mol)/amu to A^2/ps^2.
constexpr double ACC = 418.4;
constexpr double KB = 8.314462618 / 4184.0;                           // kcal/mol/K
constexpr double HBAR = 1.054571817e-34 * 6.02214076e23 / 4184.0 * 1e12;  // kcal/mol*ps
constexpr double COULOMB = 332.0637133;                                // kcal*A/(mol e^2)
constexpr double CM1 = 2.0 * 3.141592653589793 * 2.99792458e10 * 1e-12;  // cm^-1 -> rad/ps
// Fixed-point scale of mixed-precision bead forces (kcal/mol/A): 2^34.
constexpr double FIX_SCALE = 17179869184.0;
constexpr float FIX_SCALE_F = 17179869184.0f;

// Device status word bits.
enum : unsigned {
    ST_LIST_OVERFLOW = 1u,
    ST_NONFINITE = 2u,
    ST_TIMEOUT = 4u,
    ST_SPREAD = 8u,   // after a rebuild some bead lies farther than skin/2 from its anchor
    ST_BOUNDS = 16u,  // (QHP_CHECK builds) an index read from device data was out of range
};

// Bounds checks of the QHP_CHECK build (-DQHP_CHECK; build(check=True)): an index read from
// device data (a list partner, a permutation, a cell or row position) is tested before use;
// an index out of range sets ST_BOUNDS in the status word and the access is skipped, with no
// trap, so the host reports QHP_ERR_BOUNDS at the next synchronising call.  Plain builds
// compile the test away.
#ifdef QHP_CHECK
__device__ __forceinline__ bool qhp_in_bounds(long long i, long long n, const unsigned* status) {
    if (i >= 0 && i < n) return true;
    atomicOr(const_cast<unsigned*>(status), ST_BOUNDS);
    return false;
}
#define QHP_IN_BOUNDS(i, n, status) ::qhp::qhp_in_bounds((long long)(i), (long long)(n), (status))
#else
#define QHP_IN_BOUNDS(i, n, status) true
#endif

// Philox4x32-10 counter tags (same definition as the oracle, written independently).
enum : uint32_t { TAG_INIT_Q = 1, TAG_INIT_P = 2, TAG_OSTEP = 3, TAG_QTB_WHITE = 4 };

// ------------------------------------------------------------------ Philox
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Salmon et al., SC'11: ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57,
// Weyl key increments 0x9E3779B9 / 0xBB67AE85 between rounds.
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 philox_draw(uint64_t seed, uint32_t elem, uint64_t step, uint32_t tag) {
    return philox10(make_uint4(elem, (uint32_t)step, (uint32_t)(step >> 32), tag), (uint32_t)seed,
                    (uint32_t)(seed >> 32));
}

// 53-bit integer k = (hi >> 5) * 2^26 + (lo >> 6); the uniform is (k + 1/2) 2^-53.
__device__ __forceinline__ uint64_t bits53(uint32_t hi, uint32_t lo) {
    return ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
}

// Box-Muller in FP64: which = 0 -> r cos(2 pi u2), 1 -> r sin(2 pi u2).
__device__ __forceinline__ double normal_f64(uint4 x, int which) {
    const double u1 = ((double)bits53(x.x, x.y) + 0.5) * 0x1p-53;
    const double u2 = ((double)bits53(x.z, x.w) + 0.5) * 0x1p-53;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    return which ? r * s : r * c;
}

// Box-Muller in FP32 on the same 53-bit integers: the uniform keeps 24-bit
// *relative* precision down to 2^-54, so log(u1) stays accurate in the tail.
__device__ __forceinline__ float normal_f32(uint4 x, int which) {
    const float u1 = __fmaf_rn(__ull2float_rn(bits53(x.x, x.y)), 0x1p-53f, 0x1p-54f);
    const float u2 = __fmaf_rn(__ull2float_rn(bits53(x.z, x.w)), 0x1p-53f, 0x1p-54f);
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return which ? r * s : r * c;
}

// ------------------------------------------------------------------ system
struct ModeConsts {           // per-mode constants of one step, FP64
    double omega[64];
    double shear_a[64];       // tan(omega dt/4) / omega   (A(dt/2) shear, / m)
    double shear_b[64];       // sin(omega dt/2) * omega   (A(dt/2) shear, * m)
    double c1[64];            // exp(-gamma_n dt)
    double amp[64];           // sqrt((1 - c1^2) kT ACC)    (* sqrt(m))
};

// Per (atom type, mode) constants of the integrator, mass folded in.
enum : int {
    MT_SA = 0,      // shear a / m (centroid: dt/2 / m drift)
    MT_SB = 1,      // shear b * m
    MT_C1 = 2,      // exp(-gamma_n dt)
    MT_AMP = 3,     // sqrt((1 - c1^2) m kT) (PILE) or sqrt((1 - c1^2) m) (adQTB), A^2/ps^2 units
    MT_INV2M = 4,   // 1 / (2 m)
    MT_N = 8
};

// Mixed-precision bead positions (FP32 offsets from the atom's anchor), sorted atom order.
// With P >= 2 each sorted atom owns a record of bead_stride(P) floats (a multiple of 16 bytes):
// an xy plane of P/2 float4 {x_2k, x_2k+1, y_2k, y_2k+1}, then a z plane of P floats.  The pair
// kernel, whose lanes carry two beads, then reads a partner's beads with one 16-byte and one
// 8-byte load per lane over contiguous bytes (at P = 32 three 128-byte lines per partner,
// against four for one float4 per bead).  P = 1 keeps one {x, y, z, -} record per atom.
__host__ __device__ constexpr int bead_stride(int P) { return P == 1 ? 4 : (3 * P + 3) / 4 * 4; }
// Float offset of component c of bead b of sorted atom s.
__host__ __device__ __forceinline__ size_t bead_word(int s, int b, int c, int P) {
    if (P == 1) return (size_t)s * 4 + c;
    const size_t base = (size_t)s * bead_stride(P);
    return c < 2 ? base + (size_t)(b >> 1) * 4 + 2 * c + (b & 1) : base + 2 * P + b;
}

// Order of the entries within a list row: partners that are O first (their pairs carry the
// LJ term and one charge product), then H; within each group by bucket of the squared anchor
// distance |D|^2: LIST_BUCKETS equal buckets of [lo, r_list^2) with lo = (rc - 1 A)^2, closer
// entries in bucket 0.  The bucket is a monotone function of |D|^2 (each FP32 operation is), so
// an entry in a bucket above bucket(R^2) lies farther than R: the pair kernel skips the tail of
// a group that lies beyond reach, recomputing the same bucket from the same operations.
constexpr int LIST_BUCKETS = 32;
__device__ __forceinline__ int list_bucket_d2(float d2, float lo, float inv) {
    const float b = __fmul_rn(__fsub_rn(d2, lo), inv);
    return b < 1.0f ? 0 : (b < (float)(LIST_BUCKETS - 1) ? (int)b : LIST_BUCKETS - 1);
}
__device__ __forceinline__ int list_bucket(float Dx, float Dy, float Dz, float lo, float inv) {
    return list_bucket_d2(__fadd_rn(__fadd_rn(__fmul_rn(Dx, Dx), __fmul_rn(Dy, Dy)), __fmul_rn(Dz, Dz)), lo, inv);
}
// List entry {partner word, D_x, D_y, D_z}: the partner word holds the partner's sorted index
// in bits 0-25, its distance bucket in bits 26-30 (written by the row sort) and "partner is H"
// in bit 31.
constexpr int ENTRY_J_BITS = 26;
constexpr int MAX_ATOMS = 1 << ENTRY_J_BITS;
static_assert(LIST_BUCKETS <= 32, "the bucket fits the partner word's five bits");
__host__ __device__ __forceinline__ int entry_partner(int x) { return x & (MAX_ATOMS - 1); }
__host__ __device__ __forceinline__ int entry_bucket(int x) { return (x >> ENTRY_J_BITS) & 31; }
__host__ __device__ __forceinline__ bool entry_is_h(int x) { return x < 0; }

// Longest list row the in-place row sort handles (its shared-memory copy of the row).
constexpr int LIST_SORT_MAX_ROW = 12288;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace qhp

namespace qhp {
// Device buffers of the gradient entry points (allocated on first use, freed with the system).
struct GradBuffers {
    bool ready = false;
    double *x = nullptr, *v = nullptr;          // bead positions and tangents, [3][N][P] sorted
    double *F = nullptr, *Ft = nullptr;         // forces and their tangents, [3][N][P] sorted
    double *part = nullptr, *partb = nullptr;   // per (atom, bead) / (molecule, bead) partial sums
    double *x1 = nullptr, *F1 = nullptr;        // one-bead (centroid) configuration, [3][N]
    double *part1 = nullptr, *partb1 = nullptr;
    double *G = nullptr, *parto = nullptr;      // observable gradient [3][N][P], per (molecule, bead) values
    double *lamQ = nullptr, *lamP = nullptr;    // adjoints of the modes and momenta, [N][3][P]
    double* Qbuf = nullptr;                     // modes of one recomputed block, [(block + 1)][N][3][P]
    int qbuf_steps = 0;
    double* sums = nullptr;                     // column sums [16]
    double* acc = nullptr;                      // device accumulators: [0] J, [1..5] dJ/dtheta
};
}  // namespace qhp

struct qhp_system_s {
    // ---- configuration
    int N = 0, n_mol = 0, P = 0, precision = QHP_MIXED;
    double L = 0.0;
    std::vector<int> type, mol;
    std::vector<double> pos0;
    qhp_ff ff{};
    bool ff_set = false, beads_set = false, thermo_set = false;
    qhp_thermo th{};
    double temperature = 300.0;
    uint64_t seed = 0;
    int list_mode = 0;         // 1: centroid Verlet list, 0: all pairs of different molecules
    int n_c = 1;               // cells per edge
    double r_list = 0.0;

    // ---- CUDA
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int64_t launches = 0;

    // ---- device state (original atom order unless marked "sorted")
    double *Q = nullptr, *Pm = nullptr, *fmode = nullptr;    // [N][3][P]
    double *Fd = nullptr;                                    // FP64 bead forces [N][3][P]
    long long* Ffix = nullptr;                               // mixed bead forces, fixed point [N][3][P]
    float4* pos_f4 = nullptr;                                // mixed: sorted, bead_word layout, offsets from anchor
    double* pos_d = nullptr;                                 // fp64: sorted [3][N][P], absolute
    double* anchor = nullptr;                                // [N][3] centroids at the last build
    float* dA = nullptr;                                     // mixed: [n_mol][2][4] min-image A_H - A_O
    double* mass = nullptr;                                  // [N]
    double* sqrtm = nullptr;                                 // [N]
    float* charge_s = nullptr;                               // sorted charges
    int* type_s = nullptr;                                   // sorted types
    int* mol_s = nullptr;                                    // sorted molecule ids
    int* mol_d = nullptr;                                    // [N] molecule id
    int* type_d = nullptr;                                   // [N]
    int *perm = nullptr, *iperm = nullptr;                   // sorted -> atom, atom -> sorted
    int *cell = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cell_fill = nullptr, *tmp_idx = nullptr;
    float4* cw = nullptr;                                    // sorted wrapped centroids (FP32) for the prefilter
    float4* cwl = nullptr;                                   // their low parts: wrapped = cw + cwl (double-float)
    int* nbr_start = nullptr;                                // [N+1], row i starts at i * row_cap
    int* nbr_count = nullptr;                                // [N] row lengths
    int* nbr_nO = nullptr;                                   // [N] leading entries of a row whose partner is O
    int4* nbr = nullptr;                                     // entries {j, Dx, Dy, Dz}
    int64_t nbr_cap = 0;                                     // N * row_cap
    int row_cap = 0;                                         // entries per row
    int sort_grid = 1;                                       // persistent grid of the row sort
    float* e_pair = nullptr;                                 // per (sorted atom, bead) pair energy (mixed)
    double* e_pair_d = nullptr;                              // fp64
    double* e_bond = nullptr;                                // [n_mol][P]
    double* red_tmp = nullptr;                               // reduction scratch
    double* red_out = nullptr;                               // reduction results
    unsigned* status = nullptr;                              // device status word
    unsigned* status_host = nullptr;                         // pinned copy, refreshed after each step call
    cudaEvent_t status_event = nullptr;
    unsigned* dev_max = nullptr;                             // max squared deviation (float bits)
    float* dev_atom = nullptr;     // mixed: per sorted atom, max over beads of |x_ib - A_i|^2 this step
    float* dev_atom_c = nullptr;   // the same over the contracted beads (RESPA)
    int* rebuild_flag = nullptr;
    unsigned long long* step_ctr = nullptr;                  // device copy of the step counter
    int64_t rebuilds_host = 0;
    int keep_anchor = 0;           // 1 while a checkpoint restore rebuilds from stored anchors
    int pair_w = 0;                // warps per atom of the mixed pair kernel (0: default for P)
    int pair_skip = 1;             // 1: the mixed pair kernel skips list entries beyond reach
    // RESPA (Sec. III.A.2): n inner steps per outer step; slow (nonbonded) forces on pc
    // contracted beads; fast (bonded) forces in Ffix / fmode
    int respa_n = 0;               // 0: plain BAOAB
    int pc = 0;
    long long* Ffix_s = nullptr;   // [N][3][pc] slow bead forces (fixed point)
    float4* pos_c = nullptr;       // [sorted N][pc] contracted positions (offsets from anchors)
    double* fmode_s = nullptr;     // [N][3][P] slow mode forces
    float* Cmat_f = nullptr;       // [pc][P] contraction matrix
    int forces_kind = 0;           // what fmode holds: 0 full forces, 1 RESPA fast + slow
    int prof_on = 0;               // per-stage events recorded inside each step
    int use_graphs = 1;            // 0: launch each step's kernels directly
    cudaGraphConditionalHandle cond_handle = 0;   // IF node around the rebuild chain of the step graph
    int cond_active = 0;           // 1 while capturing a step graph that uses it
    cudaStream_t aux_stream = nullptr;            // captures the conditional body
    cudaEvent_t prof_ev[6] = {};
    double* cent_buf = nullptr;    // [N][3] centroid gather buffer
    unsigned* rebuild_count = nullptr;

    // ---- adQTB
    int n_seg = 0;
    float* qtb_u = nullptr;        // [n_seg][3N]
    float* qtb_v = nullptr;        // [n_seg][3N]
    float* qtb_F = nullptr;        // [n_seg][3N]
    double* qtb_gamma = nullptr;   // [2][n_seg+1]
    double* qtb_sqrtS = nullptr;   // [2][n_seg+1] sqrt of the noise power
    double* qtb_h = nullptr;       // [2][2 n_seg] filter taps
    float2* qtb_H = nullptr;       // [2][4 n_seg] filter transform
    float2* qtb_tw4 = nullptr;     // FFT twiddles, 4 n_seg points
    float2* qtb_tw2 = nullptr;     // FFT twiddles, 2 n_seg points
    int* qtb_dof_type = nullptr;   // [3N]
    double* qtb_mdof = nullptr;    // [3N]
    double* qtb_avg = nullptr;     // RATIO running averages [2][2][n_seg+1]
    double* qtb_part = nullptr;    // spectra partial sums
    double* qtb_delta = nullptr;   // last delta bar [2][n_seg+1]
    int qtb_ratio_first = 1;

    // ---- step constants
    qhp::ModeConsts mc{};
    std::vector<double> mode_tab_host;   // [2][P][MT_N]
    double* mode_tab = nullptr;
    double* Tmat = nullptr;        // sqrt(P) T[b][n], FP64 [P][P]
    float* Tmat_f = nullptr;       // same, FP32
    double* Tproj = nullptr;       // T[b][n] / sqrt(P), FP64
    float* Tproj_f = nullptr;

    double* est_part = nullptr;    // estimator partial sums [3][blocks]

    // ---- state bookkeeping
    int64_t kernels_per_step = 0;     // kernels of a captured step outside the rebuild conditional
    int64_t kernels_per_rebuild = 0;  // kernels inside it
    int64_t step = 0;              // host mirror of the device step counter
    bool forces_valid = false;
    bool list_valid = false;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_kind = -1;

    std::vector<qhp::DevBuf> allocs;
    qhp::GradBuffers grad;
};

namespace qhp {

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// Device allocation owned by the system (freed in qhp_destroy_system or on re-initialisation).
template <typename T>
int dalloc(qhp_system_s* s, T** p, size_t count) {
    const size_t bytes = (count > 0 ? count : 1) * sizeof(T);
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return QHP_ERR_NOMEM;
    }
    *p = static_cast<T*>(q);
    s->allocs.push_back({q, bytes});
    return QHP_OK;
}
#define TRY(x)                         \
    do {                               \
        const int rc_ = (x);           \
        if (rc_ != QHP_OK) return rc_; \
    } while (0)

#define QHP_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return ::qhp::cuda_fail(e_, #call);  \
    } while (0)

// Stage timestamp k of the step profile.  Inside a stream capture the record must be an
// external one to become an event-record node of the graph (a plain record would only add
// a capture dependency); outside a capture a plain record is the only valid form.
inline cudaError_t record_stage(qhp_system_s* s, int k) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s->stream, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(s->prof_ev[k], s->stream, cudaEventRecordExternal)
               : cudaEventRecord(s->prof_ev[k], s->stream);
}

// ---- kernels (launchers return cudaError_t of the launch)
struct StepArgs;

cudaError_t launch_init_modes(qhp_system_s* s);
cudaError_t launch_integrate(qhp_system_s* s, bool integrate, bool adqtb);
cudaError_t launch_integrate_gated(qhp_system_s* s);   // positions only, if the rebuild flag is set
int qtb_setup(qhp_system_s* s);
cudaError_t launch_project(qhp_system_s* s, bool kick);
cudaError_t launch_list_check(qhp_system_s* s, bool force);
cudaError_t launch_rebuild(qhp_system_s* s);
cudaError_t launch_cover_check(qhp_system_s* s);   // after a rebuild: every bead within skin/2
cudaError_t launch_integrate_respa(qhp_system_s* s, double ws);   // B (fast + ws x slow) A O A
cudaError_t launch_contract(qhp_system_s* s, bool gated);        // contracted bead positions
cudaError_t launch_project_contracted(qhp_system_s* s, bool kick);
cudaError_t launch_bonded_fast(qhp_system_s* s);
cudaError_t launch_pair_contracted(qhp_system_s* s);
cudaError_t launch_forces(qhp_system_s* s, bool energy);
cudaError_t launch_pair(qhp_system_s* s, bool energy);
cudaError_t launch_bonded(qhp_system_s* s, bool energy);
cudaError_t launch_count_pairs(qhp_system_s* s, unsigned long long* out2);
cudaError_t launch_gather_centroids(qhp_system_s* s, double* out);
cudaError_t launch_step_counter(qhp_system_s* s);
int host_list_size(qhp_system_s* s, int64_t* max_row);
void list_bucket_params(const qhp_system_s* s, float* lo, float* inv);   // the row sort's bucket map
int list_sort_prepare(qhp_system_s* s);         // the row sort's shared-memory limit and grid for s->row_cap
int rebuild_list_now(qhp_system_s* s);   // synchronous; checks the beads are covered
void graph_invalidate(qhp_system_s* s);  // drop the captured step graph (its parameters changed)
int system_sync(qhp_system_s* s);        // synchronise the system's stream, report its status

// One stage of a batched step over many systems: the stage's per-system argument
// records, its (system, block) work items in system order, and the contiguous item
// range of every block of a persistent grid (ranges[g] .. ranges[g + 1]).
struct BatchStage {
    void* args = nullptr;
    int2* items = nullptr;
    int* ranges = nullptr;
    int grid = 0, n_items = 0;
    size_t smem = 0;
    double cost = 0.0;   // estimated work of the whole stage (arbitrary units)
};
// Upload a stage: split the items into `grid` contiguous ranges of about equal cost.
int stage_upload(BatchStage& st, const void* args, size_t args_bytes, const std::vector<int2>& items,
                 const std::vector<double>& cost, int grid);
// Upload a stage whose items run in phases (a phase: items of one kernel specialisation): each
// phase is cut into `grid` chunks of about equal cost and block g runs chunk g of every phase,
// phase by phase, so at any time the blocks of the grid run about the same specialisation.
int stage_upload_phased(BatchStage& st, const void* args, size_t args_bytes, const std::vector<int2>& items,
                        const std::vector<double>& cost, const std::vector<int>& phase, int grid);
void stage_free(BatchStage& st);
int sm_count();
// The one-launch batched step (k_step_batch): integrate and project items per block of the
// step's grid, force items per half block (two halves of 128 threads).
int batch_stage_integrate(const std::vector<qhp_system_s*>& v, BatchStage& st, int grid);
int batch_stage_project(const std::vector<qhp_system_s*>& v, BatchStage& st, int grid);
int batch_integrate_items(const qhp_system_s* s);   // atom groups of 64/P atoms
size_t batch_group_smem(int maxP);                  // integrate / project shared memory
constexpr int BATCH_PAIR_STAGES = 7 * 2 * 3;        // (log2 P, small-box path, W = 1, 2, 4)
constexpr int FORCE_BONDED_VARIANT = BATCH_PAIR_STAGES;   // item kind of the batched bonded terms
int batch_stage_force(const std::vector<qhp_system_s*>& v, BatchStage& st, int* n_pair_items, int halves);
// Per-system record of the batched list check (the single-system k_check), run by the block
// that completes the system's last integrate item.
struct CheckArgs {
    unsigned* dev_max;
    int* flag;
    unsigned* rebuild_count;
    cudaGraphConditionalHandle cond;
    float thr2;
};
// Device state of the step's grid barriers: [0] arrivals, [1] generation, [2] finished blocks.
struct StepBatchState {
    unsigned bar[4];
    unsigned status;               // ST_TIMEOUT when a barrier wait ran out
    unsigned pad;
    unsigned long long ts[4];      // phase boundaries (globaltimer, ns) of the last step
};
int step_batch_config(int maxP, int* grid, size_t* smem);   // co-resident grid and shared memory
cudaError_t launch_step_batch(const BatchStage& integ, const BatchStage& force, const BatchStage& proj,
                              const CheckArgs* checks, int* done, const int* nitems, StepBatchState* state,
                              long long wait_ns, int grid, size_t smem, cudaStream_t stream);

int compute_energy(qhp_system_s* s, qhp_energy* out);
int beads_fp64(qhp_system_s* s, double* dev_out);
cudaError_t launch_estimators(qhp_system_s* s, double* partial, int* nblocks);
cudaError_t launch_sum(qhp_system_s* s, const double* xd, const float* xf, int64_t n, double* out);
cudaError_t launch_qtb_segment_end(qhp_system_s* s);     // spectra, adaptation, next filter
int qtb_generate_segment(qhp_system_s* s, int64_t seg);  // colored noise of segment seg

void mode_constants(qhp_system_s* s);
void transfer_matrix_host(int P, std::vector<double>& T);  // T[b*P + n]

}  // namespace qhp
