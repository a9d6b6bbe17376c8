// Normal-mode kernels: initial state, BAOAB propagation in modes, bead positions,
// force projection and the estimators.
//
// Layout: modes Q, Pm, projected forces fmode and bead forces are [atom][dim][P]
// (mode / bead index innermost, original atom order).  A block holds
// APB = 64/P whole atoms, i.e. 3*P*APB = 192 threads, one per (atom, dim, mode),
// so the P x P bead transform of an atom happens in shared memory.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "qhp_internal.cuh"
#include "step_bodies.cuh"

namespace qhp {

namespace {


// Persistent grid: a block walks atom groups blockIdx.x, + gridDim.x, ... and stages the
// transform in shared memory once.
template <bool MIXED, bool ADQTB, bool INTEGRATE>
__global__ void __launch_bounds__(BLOCK) k_integrate(const __grid_constant__ IntegrateArgs A) {
    extern __shared__ unsigned char smem_raw[];
    if (A.gate && !*A.gate) return;                                   // uniform over the grid
    const int nb = (A.N + A.apb - 1) / A.apb;
    for (int bx = blockIdx.x; bx < nb; bx += gridDim.x) {
        if (bx != (int)blockIdx.x) __syncthreads();                    // previous group done with smem
        integrate_body<MIXED, ADQTB, INTEGRATE>(A, bx, smem_raw, bx == (int)blockIdx.x);
    }
}

template <bool MIXED, bool KICK>
__global__ void __launch_bounds__(BLOCK) k_project(const __grid_constant__ ProjectArgs A) {
    extern __shared__ unsigned char smem_raw[];
    const int nb = (A.N + A.apb - 1) / A.apb;
    for (int bx = blockIdx.x; bx < nb; bx += gridDim.x) {
        if (bx != (int)blockIdx.x) __syncthreads();
        project_body<MIXED, KICK>(A, bx, smem_raw, bx == (int)blockIdx.x);
    }
}

__global__ void k_init_modes(int N, int P, uint64_t seed, double kT_acc, const double* pos0, const double* mass,
                             const double* omega, double* Q, double* Pm) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3 * P) return;
    const int n = idx % P, dof = idx / P, a = dof / 3;
    const double m = mass[a];
    const double zq = normal_f64(philox_draw(seed, (uint32_t)idx, 0ull, TAG_INIT_Q), 0);
    const double zp = normal_f64(philox_draw(seed, (uint32_t)idx, 0ull, TAG_INIT_P), 0);
    Q[idx] = (n == 0) ? pos0[dof] : sqrt(kT_acc / (m * omega[n] * omega[n])) * zq;
    Pm[idx] = sqrt(m * kT_acc) * zp;
}

// Per-block partial sums of: spring, kinetic, centroid-virial sum (x_b - Q_0).F_b.
__global__ void __launch_bounds__(BLOCK) k_estimators(int N, int P, int apb, const double* Q, const double* Pm,
                                                      const double* mass, const double* omega, const double* Tm,
                                                      const double* Fd, const long long* Ffix, double* partial) {
    __shared__ double qs[BLOCK];
    __shared__ double red[3][BLOCK];
    const int t = threadIdx.x;
    const int la = t / (3 * P), d = (t / P) % 3, n = t % P;
    const int a = blockIdx.x * apb + la;
    const bool valid = a < N;
    const int idx = (a * 3 + d) * P + n;
    double q = valid ? Q[idx] : 0.0;
    qs[t] = q;
    __syncthreads();
    double spring = 0.0, kin = 0.0, vir = 0.0;
    if (valid) {
        const double m = mass[a];
        const double p = Pm[idx];
        spring = 0.5 * m * omega[n] * omega[n] * q * q / ACC;
        kin = p * p / (2.0 * m) / ACC;
        const int base = la * 3 * P + d * P;
        double dev = 0.0;     // x_b - Q_0 for bead b = n
        for (int k = 1; k < P; ++k) dev = fma(Tm[n * P + k], qs[base + k], dev);
        const double F = Ffix ? (double)Ffix[idx] / FIX_SCALE : Fd[idx];
        vir = dev * F;
    }
    red[0][t] = spring;
    red[1][t] = kin;
    red[2][t] = vir;
    __syncthreads();
    if (t < 3) {
        double s = 0.0;
        for (int k = 0; k < BLOCK; ++k) s += red[t][k];   // fixed order
        partial[(size_t)t * gridDim.x + blockIdx.x] = s;  // component-major [3][blocks]
    }
}

__global__ void k_beads_fp64(int N, int P, const double* Q, const double* Tm, double* out /*[P][N][3]*/) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * 3 * P) return;
    const int b = idx % P, dof = idx / P;
    const double* q = Q + (size_t)dof * P;
    double acc = 0.0;
    for (int k = 0; k < P; ++k) acc = fma(Tm[b * P + k], q[k], acc);
    out[((size_t)b * N + dof / 3) * 3 + dof % 3] = acc;
}

// Ring-polymer contraction (Sec. III.A.2, Eq. (20)): positions of the Pc contracted beads,
// xc_b = sum_n C[b][n] Q_n with C[b][0] = 1, as FP32 offsets from the atom's anchor
// (FP64 centroid offset + FP32 fluctuation sum, as for the full beads), one thread per
// (atom, contracted bead); their deviations enter the list's displacement maximum.
__global__ void __launch_bounds__(128) k_contract(int N, int P, int Pc, const double* __restrict__ Q,
                                                  const float* __restrict__ Cf, const double* __restrict__ anchor,
                                                  const int* __restrict__ iperm, float4* __restrict__ pos_c,
                                                  unsigned* dev_max, float* dev_atom_c, const int* gate) {
    if (gate && !*gate) return;
    __shared__ unsigned dev_s[128];   // per atom of the block (Pc divides 128): max squared deviation
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    dev_s[threadIdx.x] = 0u;
    __syncthreads();
    float dv = 0.0f;
    if (t < N * Pc) {
        const int a = t / Pc, b = t % Pc;
        float x[3];
        for (int d = 0; d < 3; ++d) {
            const double* q = Q + ((size_t)a * 3 + d) * P;
            float f0 = 0.0f, f1 = 0.0f;
            int n = 1;
            for (; n + 1 < P; n += 2) {
                f0 = fmaf(Cf[b * P + n], (float)q[n], f0);
                f1 = fmaf(Cf[b * P + n + 1], (float)q[n + 1], f1);
            }
            if (n < P) f0 = fmaf(Cf[b * P + n], (float)q[n], f0);
            x[d] = (float)(q[0] - anchor[a * 3 + d]) + (f0 + f1);
        }
        float* pw = reinterpret_cast<float*>(pos_c);
        for (int d = 0; d < 3; ++d) pw[bead_word(iperm[a], b, d, Pc)] = x[d];
        dv = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        atomicMax(&dev_s[threadIdx.x / Pc], __float_as_uint(dv));
    }
    __syncthreads();
    if (t < N * Pc && t % Pc == 0) {
        const int a = t / Pc;
        dev_atom_c[iperm[a]] = __uint_as_float(dev_s[threadIdx.x / Pc]);
    }
    for (int o = 16; o > 0; o >>= 1) dv = fmaxf(dv, __shfl_xor_sync(0xffffffffu, dv, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dev_max, __float_as_uint(dv));
}

// Slow mode forces of the contracted ring polymer, f_n = (1/Pc) sum_b C[b][n] F_b (Eq. (20)),
// f_0 the exact integer sum of the fixed-point forces; with a kick, P_n += scale f_n.
// A warp covers whole dofs (P a power of two): lane b of a dof's first lanes converts its
// bead force b once and the others read it by shuffle.
__global__ void k_project_contracted(int N, int P, int Pc, const long long* __restrict__ Fs,
                                     const float* __restrict__ Cf, double* __restrict__ fmode_s, double* Pm,
                                     double kick_scale, unsigned* status) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = N * 3 * P;
    const bool valid = idx < total;
    const int n = idx % P, dof = idx / P;
    const int lane = threadIdx.x & 31;
    const long long* F = Fs + (size_t)(valid ? dof : 0) * Pc;
    float s0 = 0.0f, s1 = 0.0f;
    if (Pc <= 32) {   // uniform over the grid
        // the dof's bead forces are converted once, by the lanes sub = 0 .. Pc-1 of the warp
        // (P >= 32: a warp holds one dof; P < 32: a group of P lanes per dof)
        const int l0 = P >= 32 ? 0 : lane - n;
        const int sub = P >= 32 ? lane : n;
        const float mine = (valid && sub < Pc) ? __ll2float_rn(F[sub]) * (1.0f / FIX_SCALE_F) : 0.0f;
        for (int b = 0; b < Pc; b += 2) {
            const float f0 = __shfl_sync(0xffffffffu, mine, l0 + b);
            const float f1 = __shfl_sync(0xffffffffu, mine, l0 + (b + 1 < Pc ? b + 1 : b));
            s0 = fmaf(Cf[b * P + n], f0, s0);
            if (b + 1 < Pc) s1 = fmaf(Cf[(b + 1) * P + n], f1, s1);
        }
    } else if (valid) {
        for (int b = 0; b < Pc; ++b) s0 = fmaf(Cf[b * P + n], __ll2float_rn(F[b]) * (1.0f / FIX_SCALE_F), s0);
    }
    if (!valid) return;
    double f;
    if (n == 0) {
        long long sum = 0;
        for (int b = 0; b < Pc; ++b) sum += F[b];
        f = (double)sum * (1.0 / (FIX_SCALE * (double)Pc));   // Pc is a power of two: exact scaling
    } else {
        f = (double)(s0 + s1) / (double)Pc;
    }
    fmode_s[idx] = f;
    if (Pm) {
        const double p = Pm[idx] + kick_scale * f;
        Pm[idx] = p;
        if (!isfinite(p)) atomicOr(status, ST_NONFINITE);
    }
}

size_t integrate_smem(int P, bool mixed) { return BLOCK * 16 + (size_t)P * P * (mixed ? 4 : 8); }

}  // namespace

void transfer_matrix_host(int P, std::vector<double>& T) {
    // Real orthonormal DFT basis: columns are eigenvectors of circ(2,-1,...,-1) (Eq. (2)).
    T.assign((size_t)P * P, 0.0);
    const double pi = 3.141592653589793238462643383279502884;
    for (int b = 0; b < P; ++b)
        for (int n = 0; n < P; ++n) {
            const double ph = 2.0 * pi * (double)((b * n) % P) / (double)P;
            double v;
            if (n == 0) v = 1.0 / sqrt((double)P);
            else if (2 * n < P) v = sqrt(2.0 / P) * cos(ph);
            else if (2 * n == P) v = ((b & 1) ? -1.0 : 1.0) / sqrt((double)P);
            else v = sqrt(2.0 / P) * sin(ph);
            T[(size_t)b * P + n] = v;
        }
}

void mode_constants(qhp_system_s* s) {
    const int P = s->P;
    const double kT = KB * s->temperature;
    const double dt = s->th.dt_fs * 1e-3;
    const double pi = 3.141592653589793238462643383279502884;
    ModeConsts& m = s->mc;
    for (int n = 0; n < 64; ++n) {
        if (n >= P) {
            m.omega[n] = m.shear_a[n] = m.shear_b[n] = m.c1[n] = m.amp[n] = 0.0;
            continue;
        }
        const double w = 2.0 * P * kT / HBAR * sin(pi * n / P);
        m.omega[n] = w;
        // A(dt/2) is the rotation by th = w dt/2 (BAOAB) or, for BCOCB, the Cayley transform,
        // the rotation by 2 atan(th/2); either is applied as the same three shears
        double th = w * 0.5 * dt;
        if (s->th.integrator == QHP_INTEGRATOR_BCOCB) th = 2.0 * atan(0.5 * th);
        m.shear_a[n] = (n == 0) ? 0.0 : tan(0.5 * th) / w;
        m.shear_b[n] = (n == 0) ? 0.0 : sin(th) * w;
        double g = (n == 0) ? s->th.gamma0 : fmax(s->th.gamma0, w);
        if (s->th.kind == QHP_THERMO_NVE) g = 0.0;
        const double c1 = exp(-g * dt);
        m.c1[n] = c1;
        if (s->th.kind == QHP_THERMO_ADQTB) m.amp[n] = sqrt((1.0 - c1 * c1) * ACC);
        else m.amp[n] = sqrt((1.0 - c1 * c1) * kT * ACC);
    }
    // per (atom type, mode) table with the mass folded in: no FP64 division on the device
    s->mode_tab_host.assign((size_t)2 * P * MT_N, 0.0);
    for (int ty = 0; ty < 2; ++ty) {
        const double mass = ty == 0 ? s->ff.m_O : s->ff.m_H;
        for (int n = 0; n < P; ++n) {
            double* c = &s->mode_tab_host[((size_t)ty * P + n) * MT_N];
            c[MT_SA] = (n == 0) ? 0.5 * dt / mass : m.shear_a[n] / mass;
            c[MT_SB] = m.shear_b[n] * mass;
            c[MT_C1] = m.c1[n];
            c[MT_AMP] = m.amp[n] * sqrt(mass);
            c[MT_INV2M] = 0.5 / mass;
        }
    }
}

// Persistent grid size: resident blocks of 192 threads on every SM (at most the work).
static int persistent_grid(const void* kernel, size_t smem, int work_blocks) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BLOCK, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return std::max(1, std::min(work_blocks, per_sm * sm_count()));
}

static IntegrateArgs make_iargs(qhp_system_s* s) {
    IntegrateArgs A;
    A.N = s->N;
    A.P = s->P;
    A.apb = 64 / s->P;
    A.n_seg = s->n_seg > 0 ? s->n_seg : 1;
    const double dt = s->th.dt_fs * 1e-3;
    A.half_dt_acc = 0.5 * dt * ACC;
    A.inv_dt = 1.0 / dt;
    A.seed = s->seed;
    A.step_ctr = s->step_ctr;
    A.Q = s->Q;
    A.Pm = s->Pm;
    A.fmode = s->fmode;
    A.type = s->type_d;
    A.tab = s->mode_tab;
    A.anchor = s->anchor;
    A.iperm = s->iperm;
    A.Tm = s->Tmat;
    A.Tmf = s->Tmat_f;
    A.pos_f4 = s->pos_f4;
    A.pos_d = s->pos_d;
    A.dev_max = s->dev_max;
    A.dev_atom = s->dev_atom;
    A.status = s->status;
    A.qtb_u = s->qtb_u;
    A.qtb_v = s->qtb_v;
    A.qtb_F = s->qtb_F;
    A.gate = nullptr;
    A.fmode_s = nullptr;
    A.ws = 0.0;
    A.fzero = nullptr;
    return A;
}

static IntegrateArgs make_iargs_batch(qhp_system_s* s) {
    IntegrateArgs A = make_iargs(s);
    A.fzero = s->Ffix;
    return A;
}

cudaError_t launch_integrate_gated(qhp_system_s* s) {
    IntegrateArgs A = make_iargs(s);
    A.gate = s->rebuild_flag;
    const int nb = (s->N + A.apb - 1) / A.apb;
    const bool mixed = s->precision == QHP_MIXED;
    const size_t sm = integrate_smem(s->P, mixed);
    s->launches++;
    if (mixed) {
        const int grid = persistent_grid((const void*)k_integrate<true, false, false>, sm, nb);
        k_integrate<true, false, false><<<grid, BLOCK, sm, s->stream>>>(A);
    } else {
        const int grid = persistent_grid((const void*)k_integrate<false, false, false>, sm, nb);
        k_integrate<false, false, false><<<grid, BLOCK, sm, s->stream>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t launch_integrate(qhp_system_s* s, bool integrate, bool adqtb) {
    IntegrateArgs A = make_iargs(s);
    const int nb = (s->N + A.apb - 1) / A.apb;
    const bool mixed = s->precision == QHP_MIXED;
    const size_t sm = integrate_smem(s->P, mixed);
    s->launches++;
#define QHP_INT(M, Q, I)                                                                     \
    do {                                                                                     \
        const int grid = persistent_grid((const void*)k_integrate<M, Q, I>, sm, nb);        \
        k_integrate<M, Q, I><<<grid, BLOCK, sm, s->stream>>>(A);                            \
    } while (0)
    if (mixed) {
        if (!integrate) QHP_INT(true, false, false);
        else if (adqtb) QHP_INT(true, true, true);
        else QHP_INT(true, false, true);
    } else {
        if (!integrate) QHP_INT(false, false, false);
        else if (adqtb) QHP_INT(false, true, true);
        else QHP_INT(false, false, true);
    }
#undef QHP_INT
    return cudaGetLastError();
}

static ProjectArgs make_pargs(qhp_system_s* s) {
    ProjectArgs A;
    A.N = s->N;
    A.P = s->P;
    A.apb = 64 / s->P;
    A.half_dt_acc = 0.5 * s->th.dt_fs * 1e-3 * ACC;
    A.Fd = s->Fd;
    A.Ffix = s->Ffix;
    A.Tp = s->Tproj;
    A.Tpf = s->Tproj_f;
    A.fmode = s->fmode;
    A.Pm = s->Pm;
    A.status = s->status;
    A.step_ctr = s->step_ctr;
    return A;
}

cudaError_t launch_project(qhp_system_s* s, bool kick) {
    const ProjectArgs A = make_pargs(s);
    const int nb = (s->N + A.apb - 1) / A.apb;
    const bool mixed = s->precision == QHP_MIXED;
    const size_t sm = (size_t)s->P * s->P * (mixed ? 4 : 8);
    s->launches++;
#define QHP_PRJ(M, K)                                                                        \
    do {                                                                                     \
        const int grid = persistent_grid((const void*)k_project<M, K>, sm, nb);             \
        k_project<M, K><<<grid, BLOCK, sm, s->stream>>>(A);                                 \
    } while (0)
    if (mixed) {
        if (kick) QHP_PRJ(true, true);
        else QHP_PRJ(true, false);
    } else {
        if (kick) QHP_PRJ(false, true);
        else QHP_PRJ(false, false);
    }
#undef QHP_PRJ
    return cudaGetLastError();
}

// Batched stages of the one-launch step (mixed precision, PILE/NVE): one item per group of
// 64/P atoms, cut into one contiguous range per block of the step's grid.
template <class Args, class Make>
static int integrate_like_stage(const std::vector<qhp_system_s*>& v, BatchStage& st, Make make, int grid) {
    std::vector<Args> a;
    std::vector<int2> items;
    std::vector<double> cost;
    for (size_t k = 0; k < v.size(); ++k) {
        a.push_back(make(v[k]));
        const int nb = batch_integrate_items(v[k]);
        for (int b = 0; b < nb; ++b) {
            items.push_back(make_int2((int)k, b));
            cost.push_back(1.0);
        }
    }
    st.smem = 0;
    return stage_upload(st, a.data(), sizeof(Args) * a.size(), items, cost, grid);
}

// Items (atom groups of 64/P atoms) of one system in the batched integrate and project stages.
int batch_integrate_items(const qhp_system_s* s) { return (s->N + 64 / s->P - 1) / (64 / s->P); }

int batch_stage_integrate(const std::vector<qhp_system_s*>& v, BatchStage& st, int grid) {
    return integrate_like_stage<IntegrateArgs>(v, st, make_iargs_batch, grid);
}

int batch_stage_project(const std::vector<qhp_system_s*>& v, BatchStage& st, int grid) {
    return integrate_like_stage<ProjectArgs>(v, st, make_pargs, grid);
}

// Shared memory of the integrate (BLOCK * 16 + P^2 floats) and project (P^2 floats) bodies.
size_t batch_group_smem(int maxP) { return (size_t)BLOCK * 16 + sizeof(float) * maxP * maxP; }

cudaError_t launch_init_modes(qhp_system_s* s) {
    const int total = s->N * 3 * s->P;
    double* omega_d = s->red_out;   // scratch: the first 64 doubles of red_out hold omega_n
    cudaError_t e = cudaMemcpyAsync(omega_d, s->mc.omega, sizeof(double) * 64, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return e;
    s->launches++;
    // the initial positions are staged in the anchor buffer by the caller
    k_init_modes<<<(total + 255) / 256, 256, 0, s->stream>>>(s->N, s->P, s->seed, KB * s->temperature * ACC,
                                                             s->anchor, s->mass, omega_d, s->Q, s->Pm);
    return cudaGetLastError();
}

cudaError_t launch_integrate_respa(qhp_system_s* s, double ws) {
    IntegrateArgs A = make_iargs(s);
    A.fmode_s = s->fmode_s;
    A.ws = ws;
    const int nb = (s->N + A.apb - 1) / A.apb;
    const size_t sm = integrate_smem(s->P, true);
    const int grid = persistent_grid((const void*)k_integrate<true, false, true>, sm, nb);
    s->launches++;
    k_integrate<true, false, true><<<grid, BLOCK, sm, s->stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_contract(qhp_system_s* s, bool gated) {
    const int total = s->N * s->pc;
    s->launches++;
    k_contract<<<(total + 127) / 128, 128, 0, s->stream>>>(s->N, s->P, s->pc, s->Q, s->Cmat_f, s->anchor, s->iperm,
                                                           s->pos_c, s->dev_max, s->dev_atom_c,
                                                           gated ? s->rebuild_flag : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_project_contracted(qhp_system_s* s, bool kick) {
    const int total = s->N * 3 * s->P;
    const double scale = kick ? s->respa_n * 0.5 * s->th.dt_fs * 1e-3 * ACC : 0.0;
    s->launches++;
    k_project_contracted<<<(total + 255) / 256, 256, 0, s->stream>>>(s->N, s->P, s->pc, s->Ffix_s, s->Cmat_f,
                                                                     s->fmode_s, kick ? s->Pm : nullptr, scale,
                                                                     s->status);
    return cudaGetLastError();
}

int beads_fp64(qhp_system_s* s, double* dev_out) {
    const int total = s->N * 3 * s->P;
    s->launches++;
    k_beads_fp64<<<(total + 255) / 256, 256, 0, s->stream>>>(s->N, s->P, s->Q, s->Tmat, dev_out);
    QHP_CUDA(cudaGetLastError());
    return QHP_OK;
}

cudaError_t launch_estimators(qhp_system_s* s, double* partial, int* nblocks) {
    const int apb = 64 / s->P;
    const int grid = (s->N + apb - 1) / apb;
    *nblocks = grid;
    double* omega_d = s->red_out + 64;
    cudaError_t e = cudaMemcpyAsync(omega_d, s->mc.omega, sizeof(double) * 64, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return e;
    s->launches++;
    k_estimators<<<grid, BLOCK, 0, s->stream>>>(s->N, s->P, apb, s->Q, s->Pm, s->mass, omega_d, s->Tmat, s->Fd,
                                                s->precision == QHP_MIXED ? s->Ffix : nullptr, partial);
    return cudaGetLastError();
}

namespace {
__global__ void k_gather_centroids(int n3, int P, const double* __restrict__ Q, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n3) out[k] = Q[(size_t)k * P];
}
}  // namespace

// Centroids Q_0 into a contiguous [N][3] device buffer.
cudaError_t launch_gather_centroids(qhp_system_s* s, double* out) {
    const int n3 = 3 * s->N;
    s->launches++;
    k_gather_centroids<<<(n3 + 255) / 256, 256, 0, s->stream>>>(n3, s->P, s->Q, out);
    return cudaGetLastError();
}

}  // namespace qhp
