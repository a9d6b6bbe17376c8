// C ABI: system lifecycle, step driver, getters, checkpoints.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "qhp_internal.cuh"

namespace qhp {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), what);
    return QHP_ERR_CUDA;
}

namespace {

void free_all(qhp_system_s* s) {
    if (s->graph_exec) {
        cudaGraphExecDestroy(s->graph_exec);
        s->graph_exec = nullptr;
    }
    s->graph_kind = -1;
    for (auto& b : s->allocs) cudaFree(b.p);
    s->allocs.clear();
    // the adQTB buffers lived in the same pool: forget them so qtb_setup reallocates
    s->qtb_u = s->qtb_v = s->qtb_F = nullptr;
    s->qtb_gamma = s->qtb_sqrtS = s->qtb_h = s->qtb_avg = s->qtb_part = s->qtb_delta = s->qtb_mdof = nullptr;
    s->qtb_H = s->qtb_tw4 = s->qtb_tw2 = nullptr;
    s->qtb_dof_type = nullptr;
    s->n_seg = 0;
    s->grad = GradBuffers{};
    s->respa_n = 0;   // RESPA buffers lived in the same pool
    s->pc = 0;
    s->Ffix_s = nullptr;
    s->pos_c = nullptr;
    s->fmode_s = nullptr;
    s->Cmat_f = nullptr;
    s->nbr = nullptr;
    s->nbr_cap = 0;
}


// ---------------------------------------------------------------- reductions
constexpr int RED_BLOCKS = 256;

template <typename T>
__global__ void k_sum_part(const T* __restrict__ x, int64_t n, double* part) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double* part, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += part[k];
        *out = s;
    }
}

int check_status(qhp_system_s* s, unsigned st) {
    if (st & ST_LIST_OVERFLOW) {
        qhp::set_error("neighbour list overflow (a row exceeds its %d entries)", s->row_cap);
        return QHP_ERR_LIST_OVERFLOW;
    }
    if (st & ST_SPREAD) {
        qhp::set_error("a bead lies farther than skin/2 from its centroid right after a list rebuild: "
                       "increase the skin");
        return QHP_ERR_LIST_OVERFLOW;
    }
    if (st & ST_NONFINITE) {
        qhp::set_error("non-finite momenta detected");
        return QHP_ERR_NONFINITE;
    }
    if (st & ST_TIMEOUT) {
        qhp::set_error("device wait timed out");
        return QHP_ERR_TIMEOUT;
    }
    if (st & ST_BOUNDS) {
        qhp::set_error("an index read from device data was out of range (bounds-checked build); the access was skipped");
        return QHP_ERR_BOUNDS;
    }
    return QHP_OK;
}

int sync_and_check(qhp_system_s* s) {
    QHP_CUDA(cudaStreamSynchronize(s->stream));
    unsigned st = 0;
    QHP_CUDA(cudaMemcpy(&st, s->status, sizeof st, cudaMemcpyDeviceToHost));
    return check_status(s, st);
}

int upload_matrices(qhp_system_s* s) {
    const int P = s->P;
    std::vector<double> T;
    transfer_matrix_host(P, T);
    std::vector<double> Tm(P * P), Tp(P * P);
    std::vector<float> Tmf(P * P), Tpf(P * P);
    for (int b = 0; b < P; ++b)
        for (int n = 0; n < P; ++n) {
            Tm[b * P + n] = sqrt((double)P) * T[b * P + n];
            Tp[b * P + n] = T[b * P + n] / sqrt((double)P);
            Tmf[b * P + n] = (float)Tm[b * P + n];
            Tpf[b * P + n] = (float)Tp[b * P + n];
        }
    QHP_CUDA(cudaMemcpy(s->Tmat, Tm.data(), sizeof(double) * P * P, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(s->Tproj, Tp.data(), sizeof(double) * P * P, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(s->Tmat_f, Tmf.data(), sizeof(float) * P * P, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(s->Tproj_f, Tpf.data(), sizeof(float) * P * P, cudaMemcpyHostToDevice));
    return QHP_OK;
}

void invalidate_graph(qhp_system_s* s) {
    if (s->graph_exec) {
        cudaGraphExecDestroy(s->graph_exec);
        s->graph_exec = nullptr;
    }
    s->graph_kind = -1;
}

// Positions, list check (+ rebuild when due), forces, projection; no time step.
int enqueue_forces(qhp_system_s* s, bool force_rebuild, bool energy) {
    QHP_CUDA(launch_integrate(s, false, false));
    if (s->respa_n) QHP_CUDA(launch_contract(s, false));
    QHP_CUDA(launch_list_check(s, force_rebuild));
    QHP_CUDA(launch_rebuild(s));
    QHP_CUDA(launch_integrate_gated(s));
    if (s->respa_n) QHP_CUDA(launch_contract(s, true));
    QHP_CUDA(launch_cover_check(s));
    QHP_CUDA(launch_forces(s, energy));
    QHP_CUDA(launch_project(s, false));
    s->forces_kind = 0;
    return QHP_OK;
}

// RESPA forces at the current modes, no kick: fast (bonded, all beads) into fmode and
// slow (nonbonded, contracted beads) into fmode_s.
int enqueue_respa_forces(qhp_system_s* s, bool force_rebuild) {
    QHP_CUDA(launch_integrate(s, false, false));
    QHP_CUDA(launch_contract(s, false));
    QHP_CUDA(launch_list_check(s, force_rebuild));
    QHP_CUDA(launch_rebuild(s));
    QHP_CUDA(launch_integrate_gated(s));
    QHP_CUDA(launch_contract(s, true));
    QHP_CUDA(launch_cover_check(s));
    QHP_CUDA(launch_bonded_fast(s));
    QHP_CUDA(launch_project(s, false));
    QHP_CUDA(launch_pair_contracted(s));
    QHP_CUDA(launch_project_contracted(s, false));
    s->forces_kind = 1;
    return QHP_OK;
}

// While a step graph is being captured: add an IF node driven by k_check and capture the
// list rebuild chain (cells, sort, list, positions) into its body on the auxiliary stream,
// so steps without a rebuild launch none of those kernels.
int enqueue_rebuild_conditional(qhp_system_s* s) {
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    QHP_CUDA(cudaStreamGetCaptureInfo(s->stream, &st, nullptr, &cg, &deps, &ed, &nd));
    alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
    memset(pbuf, 0, sizeof pbuf);   // the struct holds a union without a default constructor
    cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(pbuf);
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = s->cond_handle;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    QHP_CUDA(cudaGraphAddNode(&node, cg, deps, ed, nd, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    QHP_CUDA(cudaStreamUpdateCaptureDependencies(s->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    QHP_CUDA(cudaStreamBeginCaptureToGraph(s->aux_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaStream_t main = s->stream;
    s->stream = s->aux_stream;
    const int64_t before = s->launches;
    cudaError_t e = launch_rebuild(s);
    if (e == cudaSuccess) e = launch_integrate_gated(s);
    if (e == cudaSuccess && s->respa_n) e = launch_contract(s, true);
    if (e == cudaSuccess) e = launch_cover_check(s);
    s->kernels_per_rebuild = s->launches - before;
    s->stream = main;
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s->aux_stream, &out);
    if (e != cudaSuccess) return cuda_fail(e, "rebuild chain capture");
    QHP_CUDA(e2);
    return QHP_OK;
}

int enqueue_step(qhp_system_s* s, bool adqtb);

// Capture one whole step into the system's executable graph.
int capture_step_graph(qhp_system_s* s, bool adqtb) {
    invalidate_graph(s);
    if (!s->aux_stream) QHP_CUDA(cudaStreamCreateWithFlags(&s->aux_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    QHP_CUDA(cudaGraphCreate(&g, 0));
    cudaError_t e = cudaGraphConditionalHandleCreate(&s->cond_handle, g, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(s->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "step graph capture start");
    }
    const int64_t before = s->launches;
    s->cond_active = 1;
    s->kernels_per_rebuild = 0;
    const int rc = enqueue_step(s, adqtb);
    s->cond_active = 0;
    cudaGraph_t g2 = nullptr;
    e = cudaStreamEndCapture(s->stream, &g2);
    if (rc != QHP_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return rc != QHP_OK ? rc : cuda_fail(e, "step graph capture end");
    }
    s->kernels_per_step = s->launches - before - s->kernels_per_rebuild;
    s->launches = before;
    e = cudaGraphInstantiate(&s->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph_exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    s->graph_kind = adqtb ? 1 : 0;
    return QHP_OK;
}

// One RESPA outer step (Sec. III.A.2): B_s(n dt/2) [B_f A O A B_f]^n B_s(n dt/2).  The
// first inner integrate applies B_s together with B_f; the list is checked once, right
// before the slow forces, on the displacements of all inner steps and the contracted beads.
// Stage timestamps: inner steps | list | slow pair forces | last bonded | projections.
int enqueue_respa_step(qhp_system_s* s) {
    const bool prof = s->prof_on != 0;
    const int n = s->respa_n;
    if (prof) QHP_CUDA(record_stage(s, 0));
    for (int i = 0; i < n; ++i) {
        QHP_CUDA(launch_integrate_respa(s, i == 0 ? (double)n : 0.0));
        if (i < n - 1) {
            QHP_CUDA(launch_bonded_fast(s));
            QHP_CUDA(launch_project(s, true));
            continue;
        }
        QHP_CUDA(launch_contract(s, false));
        if (prof) QHP_CUDA(record_stage(s, 1));
        QHP_CUDA(launch_list_check(s, false));
        if (s->cond_active) {
            TRY(enqueue_rebuild_conditional(s));
        } else {
            QHP_CUDA(launch_rebuild(s));
            QHP_CUDA(launch_integrate_gated(s));
            QHP_CUDA(launch_contract(s, true));
            QHP_CUDA(launch_cover_check(s));
        }
        if (prof) QHP_CUDA(record_stage(s, 2));
        QHP_CUDA(launch_pair_contracted(s));
        if (prof) QHP_CUDA(record_stage(s, 3));
        QHP_CUDA(launch_bonded_fast(s));
        if (prof) QHP_CUDA(record_stage(s, 4));
        QHP_CUDA(launch_project(s, true));
        QHP_CUDA(launch_project_contracted(s, true));
        if (prof) QHP_CUDA(record_stage(s, 5));
    }
    return QHP_OK;
}

int enqueue_step(qhp_system_s* s, bool adqtb) {
    if (s->respa_n && !adqtb) return enqueue_respa_step(s);
    // Under capture the stage records become event-record nodes, so every replay
    // timestamps its stages.
    const bool prof = s->prof_on != 0;
    if (prof) QHP_CUDA(record_stage(s, 0));
    QHP_CUDA(launch_integrate(s, true, adqtb));
    if (prof) QHP_CUDA(record_stage(s, 1));
    QHP_CUDA(launch_list_check(s, false));
    if (s->cond_active) {
        TRY(enqueue_rebuild_conditional(s));
    } else {
        QHP_CUDA(launch_rebuild(s));
        QHP_CUDA(launch_integrate_gated(s));
        QHP_CUDA(launch_cover_check(s));
    }
    if (prof) QHP_CUDA(record_stage(s, 2));
    QHP_CUDA(launch_forces(s, false));                      // records prof_ev[3] between pair and bonded
    if (prof) QHP_CUDA(record_stage(s, 4));
    QHP_CUDA(launch_project(s, true));
    if (prof) QHP_CUDA(record_stage(s, 5));
    return QHP_OK;
}

// After the step that completes an adQTB segment: spectra, adaptation, next noise segment.
int enqueue_segment_end(qhp_system_s* s, int64_t steps_done) {
    QHP_CUDA(launch_qtb_segment_end(s));
    return qtb_generate_segment(s, steps_done / s->n_seg);
}

// Every (sorted) atom owns a row of row_cap list entries starting at i * row_cap; the
// rebuild writes each row's length to nbr_count.  Rows are sized from the longest row of
// the current centroids with 25% + 64 entries of headroom for density fluctuations; a
// rebuild that would overrun a row raises the list-overflow status instead.
int ensure_capacity(qhp_system_s* s) {
    int64_t longest = 0;
    TRY(host_list_size(s, &longest));
    int64_t row = ((int64_t)(1.25 * (double)longest) + 64 + 7) / 8 * 8;
    if (row > s->N) row = s->N;   // no row is longer than the other atoms
    if (row < 8) row = 8;
    if (row > LIST_SORT_MAX_ROW) {
        qhp::set_error("neighbour rows of %lld entries exceed the %d the row sort handles (reduce the skin)",
                       (long long)row, LIST_SORT_MAX_ROW);
        return QHP_ERR_ARG;
    }
    if (row * (int64_t)s->N > ((int64_t)1 << 31) - 1) {
        qhp::set_error("neighbour list too large (%lld rows of %lld entries)", (long long)s->N, (long long)row);
        return QHP_ERR_NOMEM;
    }
    if (row > s->row_cap) {
        // Grow: the old buffer stays owned by the system until destruction.
        int4* p = nullptr;
        TRY(dalloc(s, &p, (size_t)row * s->N));
        s->nbr = p;
        s->nbr_cap = row * s->N;
        s->row_cap = (int)row;
        TRY(list_sort_prepare(s));
        std::vector<int> start(s->N + 1);
        for (int i = 0; i <= s->N; ++i) start[i] = i * (int)row;
        QHP_CUDA(cudaMemcpy(s->nbr_start, start.data(), sizeof(int) * (s->N + 1), cudaMemcpyHostToDevice));
        invalidate_graph(s);
    }
    return QHP_OK;
}

int post_status(qhp_system_s* s) {
    if (!s->status_host) {
        QHP_CUDA(cudaHostAlloc((void**)&s->status_host, sizeof(unsigned), cudaHostAllocDefault));
        *s->status_host = 0u;
        QHP_CUDA(cudaEventCreateWithFlags(&s->status_event, cudaEventDisableTiming));
    }
    QHP_CUDA(cudaMemcpyAsync(s->status_host, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    QHP_CUDA(cudaEventRecord(s->status_event, s->stream));
    return QHP_OK;
}

int run_steps(qhp_system_s* s, int n, bool adqtb) {
    if (!s->beads_set) {
        set_error("qhp_set_beads must be called before stepping");
        return QHP_ERR_STATE;
    }
    if (n < 0) {
        set_error("negative step count");
        return QHP_ERR_ARG;
    }
    if (adqtb != (s->th.kind == QHP_THERMO_ADQTB)) {
        set_error(adqtb ? "qhp_step_adqtb needs an ADQTB thermostat" : "qhp_step_rpmd needs a PILE thermostat");
        return QHP_ERR_STATE;
    }
    // report a fault found by earlier asynchronous work, without waiting for it
    if (s->status_event && cudaEventQuery(s->status_event) == cudaSuccess) TRY(check_status(s, *s->status_host));
    const int want = s->respa_n ? 1 : 0;
    if (!s->forces_valid || s->forces_kind != want) {
        if (want) TRY(enqueue_respa_forces(s, !s->list_valid));
        else TRY(enqueue_forces(s, !s->list_valid, false));
        s->forces_valid = true;
        s->list_valid = true;
    }
    if (n == 0) return QHP_OK;
    const int kind = adqtb ? 1 : 0;
    const int inner = s->respa_n ? s->respa_n : 1;   // time steps per call unit
    if (!s->use_graphs) {
        for (int k = 0; k < n; ++k) {
            TRY(enqueue_step(s, adqtb));
            s->step += inner;
            if (adqtb && s->step % s->n_seg == 0) TRY(enqueue_segment_end(s, s->step));
        }
        return post_status(s);
    }
    if (adqtb) {
        // step by step through one captured step graph; segment ends are enqueued by the host
        for (int k = 0; k < n; ++k) {
            if (!s->graph_exec || s->graph_kind != kind) TRY(capture_step_graph(s, true));
            QHP_CUDA(cudaGraphLaunch(s->graph_exec, s->stream));
            s->launches += s->kernels_per_step;
            s->step += 1;
            if (s->step % s->n_seg == 0) TRY(enqueue_segment_end(s, s->step));
        }
        return post_status(s);
    }
    if (n >= 1) {
        if (!s->graph_exec || s->graph_kind != kind) TRY(capture_step_graph(s, false));
        for (int k = 0; k < n; ++k) QHP_CUDA(cudaGraphLaunch(s->graph_exec, s->stream));
        s->launches += s->kernels_per_step * n;
    } else {
        TRY(enqueue_step(s, adqtb));
    }
    s->step += (int64_t)n * inner;
    return post_status(s);
}

double self_energy(const qhp_system_s* s) {
    const double a = s->ff.alpha, rc = s->ff.rc;
    double q2 = 0.0;
    for (int i = 0; i < s->N; ++i) {
        const double q = s->type[i] == 0 ? s->ff.q_O : -0.5 * s->ff.q_O;
        q2 += q * q;
    }
    return -(erfc(a * rc) / (2.0 * rc) + a / sqrt(M_PI)) * COULOMB * q2;
}

}  // namespace

void graph_invalidate(qhp_system_s* s) { invalidate_graph(s); }
int system_sync(qhp_system_s* s) { return sync_and_check(s); }

// Rebuild the list around the current modes now (synchronous).  The rebuild chain checks
// that every bead lies within skin/2 of its anchor and reports QHP_ERR_LIST_OVERFLOW if not.
int rebuild_list_now(qhp_system_s* s) {
    TRY(enqueue_forces(s, true, false));
    TRY(sync_and_check(s));
    s->forces_valid = true;
    s->list_valid = true;
    return QHP_OK;
}

cudaError_t launch_sum(qhp_system_s* s, const double* xd, const float* xf, int64_t n, double* out) {
    if (xd) k_sum_part<double><<<RED_BLOCKS, 256, 0, s->stream>>>(xd, n, s->red_tmp);
    else k_sum_part<float><<<RED_BLOCKS, 256, 0, s->stream>>>(xf, n, s->red_tmp);
    k_sum_final<<<1, 32, 0, s->stream>>>(s->red_tmp, RED_BLOCKS, out);
    s->launches += 2;
    return cudaGetLastError();
}

int compute_energy(qhp_system_s* s, qhp_energy* out) {
    TRY(enqueue_forces(s, !s->list_valid, true));
    s->forces_valid = true;
    s->list_valid = true;
    const int P = s->P, N = s->N;
    double* r = s->red_out + 128;   // results: pair, bond, spring, kinetic, virial
    if (s->precision == QHP_MIXED) QHP_CUDA(launch_sum(s, nullptr, s->e_pair, (int64_t)N * P, r + 0));
    else QHP_CUDA(launch_sum(s, s->e_pair_d, nullptr, (int64_t)N * P, r + 0));
    QHP_CUDA(launch_sum(s, s->e_bond, nullptr, (int64_t)s->n_mol * P, r + 1));
    int nb = 0;
    QHP_CUDA(launch_estimators(s, s->est_part, &nb));
    for (int c = 0; c < 3; ++c) QHP_CUDA(launch_sum(s, s->est_part + (size_t)c * nb, nullptr, nb, r + 2 + c));
    double h[5];
    QHP_CUDA(cudaMemcpyAsync(h, r, sizeof h, cudaMemcpyDeviceToHost, s->stream));
    TRY(sync_and_check(s));
    const double kT = KB * s->temperature;
    memset(out, 0, sizeof *out);
    out->nonbonded = h[0] / P;
    out->bonded = h[1] / P;
    out->potential = (h[0] + h[1]) / P + self_energy(s);
    out->spring = h[2];
    out->kinetic_nm = h[3];
    out->kinetic_cv = 1.5 * N * kT - h[4] / (2.0 * P);
    out->fdt_delta = 0.0;
    if (s->qtb_delta && s->n_seg > 0) {   // mean |Delta_bar_FDT,z(w_j)| over both types and all bins
        const size_t nb = 2 * (size_t)(s->n_seg + 1);
        std::vector<double> d(nb);
        QHP_CUDA(cudaMemcpy(d.data(), s->qtb_delta, sizeof(double) * nb, cudaMemcpyDeviceToHost));
        double sum = 0.0;
        for (double v : d) sum += fabs(v);
        out->fdt_delta = sum / (double)nb;
    }
    return QHP_OK;
}

}  // namespace qhp

using namespace qhp;

extern "C" {

const char* qhp_last_error(void) { return g_err.c_str(); }

int qhp_create_system(qhp_sys* out, int n_atoms, const int* type, const int* molecule, const double* pos,
                      double box_L, int precision) {
    if (!out || !type || !molecule || !pos) {
        set_error("null argument");
        return QHP_ERR_ARG;
    }
    *out = nullptr;
    if (n_atoms <= 0 || n_atoms % 3 != 0) {
        set_error("n_atoms must be a positive multiple of 3 (O, H, H molecules)");
        return QHP_ERR_ARG;
    }
    if (n_atoms >= MAX_ATOMS) {
        set_error("n_atoms must be below %d (the neighbour list's partner index)", MAX_ATOMS);
        return QHP_ERR_ARG;
    }
    if (!(box_L > 0.0) || !isfinite(box_L)) {
        set_error("box_L must be positive");
        return QHP_ERR_ARG;
    }
    if (precision != QHP_FP64 && precision != QHP_MIXED) {
        set_error("precision must be QHP_FP64 or QHP_MIXED");
        return QHP_ERR_ARG;
    }
    for (int i = 0; i < n_atoms; ++i) {
        const int want = (i % 3 == 0) ? 0 : 1;
        if (type[i] != want || molecule[i] != i / 3) {
            set_error("atom %d: expected type %d and molecule %d (consecutive O, H, H triples)", i, want, i / 3);
            return QHP_ERR_ARG;
        }
        for (int d = 0; d < 3; ++d)
            if (!isfinite(pos[3 * i + d])) {
                set_error("non-finite position of atom %d", i);
                return QHP_ERR_ARG;
            }
    }
    qhp_system_s* s = new qhp_system_s();
    s->N = n_atoms;
    s->n_mol = n_atoms / 3;
    s->L = box_L;
    s->precision = precision;
    s->type.assign(type, type + n_atoms);
    s->mol.assign(molecule, molecule + n_atoms);
    s->pos0.assign(pos, pos + 3 * (size_t)n_atoms);
    s->th.kind = QHP_THERMO_PILE;
    s->th.gamma0 = 1.0;
    s->th.dt_fs = 0.5;
    s->th.n_seg = 1024;
    s->th.a_gamma = 10.0;
    s->th.gamma_min_frac = 0.01;
    s->th.adapt = QHP_ADAPT_SIMPLE;
    s->th.tau_ratio_ps = 1.0;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "stream creation");
    }
    s->stream = s->own_stream;
    *out = s;
    return QHP_OK;
}

int qhp_destroy_system(qhp_sys s) {
    if (!s) return QHP_OK;
    cudaStreamSynchronize(s->stream);
    free_all(s);
    if (s->status_event) cudaEventDestroy(s->status_event);
    if (s->aux_stream) cudaStreamDestroy(s->aux_stream);
    for (int k = 0; k < 6; ++k)
        if (s->prof_ev[k]) cudaEventDestroy(s->prof_ev[k]);
    if (s->status_host) cudaFreeHost(s->status_host);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    delete s;
    return QHP_OK;
}

int qhp_set_forcefield(qhp_sys s, const qhp_ff* ff) {
    if (!s || !ff) {
        set_error("null argument");
        return QHP_ERR_ARG;
    }
    if (!(ff->rc > 0.0) || !(ff->rc < 0.5 * s->L) || ff->skin < 0.0 || !(ff->m_O > 0.0) || !(ff->m_H > 0.0) ||
        ff->alpha < 0.0 || ff->sigma <= 0.0) {
        set_error("force field: need 0 < rc < box/2, skin >= 0, positive masses and sigma, alpha >= 0");
        return QHP_ERR_ARG;
    }
    if (s->beads_set && (ff->rc != s->ff.rc || ff->skin != s->ff.skin || ff->m_O != s->ff.m_O || ff->m_H != s->ff.m_H)) {
        set_error("after qhp_set_beads only eps, sigma, q_O, k_b, r0, k_theta, theta0 and alpha may change");
        return QHP_ERR_STATE;
    }
    s->ff = *ff;
    s->ff_set = true;
    s->r_list = ff->rc + ff->skin;
    // cells at least r_list/2 wide: every list partner lies within a 5 x 5 x 5 stencil
    s->n_c = std::max(1, (int)floor(2.0 * s->L / s->r_list));
    s->list_mode = (s->n_c >= 5 && s->r_list < 0.5 * s->L) ? 1 : 0;
    if (!s->list_mode) s->n_c = 1;
    s->forces_valid = false;
    s->list_valid = false;
    invalidate_graph(s);
    return QHP_OK;
}

int qhp_set_beads(qhp_sys s, int P, double temperature, uint64_t seed) {
    if (!s) {
        set_error("null system");
        return QHP_ERR_ARG;
    }
    if (!s->ff_set) {
        set_error("qhp_set_forcefield must come first");
        return QHP_ERR_STATE;
    }
    if (P < 1 || P > 64 || (P & (P - 1))) {
        set_error("P must be a power of two in [1, 64]");
        return QHP_ERR_ARG;
    }
    if (!(temperature > 0.0)) {
        set_error("temperature must be positive");
        return QHP_ERR_ARG;
    }
    if ((int64_t)s->N * P >= (int64_t)1 << 30) {   // kernels use 32-bit (atom, bead) offsets
        set_error("n_atoms * P must stay below 2^30");
        return QHP_ERR_ARG;
    }
    QHP_CUDA(cudaStreamSynchronize(s->stream));
    free_all(s);
    s->P = P;
    s->temperature = temperature;
    s->seed = seed;
    const int N = s->N;
    const size_t NP3 = (size_t)N * 3 * P;
    TRY(dalloc(s, &s->Q, NP3));
    TRY(dalloc(s, &s->Pm, NP3));
    TRY(dalloc(s, &s->fmode, NP3));
    if (s->precision == QHP_MIXED) {
        TRY(dalloc(s, &s->Ffix, NP3));
        TRY(dalloc(s, &s->pos_f4, (size_t)N * P));
        TRY(dalloc(s, &s->dev_atom, (size_t)N));
        TRY(dalloc(s, &s->e_pair, (size_t)N * P));
        TRY(dalloc(s, &s->dA, (size_t)s->n_mol * 8));
    } else {
        TRY(dalloc(s, &s->Fd, NP3));
        TRY(dalloc(s, &s->pos_d, NP3));
        TRY(dalloc(s, &s->e_pair_d, (size_t)N * P));
    }
    TRY(dalloc(s, &s->anchor, (size_t)N * 3));
    TRY(dalloc(s, &s->mass, N));
    TRY(dalloc(s, &s->sqrtm, N));
    TRY(dalloc(s, &s->charge_s, N));
    TRY(dalloc(s, &s->type_s, N));
    TRY(dalloc(s, &s->mol_s, N));
    TRY(dalloc(s, &s->mol_d, N));
    TRY(dalloc(s, &s->type_d, N));
    TRY(dalloc(s, &s->perm, N));
    TRY(dalloc(s, &s->iperm, N));
    TRY(dalloc(s, &s->cell, N));
    TRY(dalloc(s, &s->tmp_idx, N));
    const int ncell = s->n_c * s->n_c * s->n_c;
    TRY(dalloc(s, &s->cell_count, ncell));
    TRY(dalloc(s, &s->cell_fill, ncell));
    TRY(dalloc(s, &s->cell_start, ncell + 1));
    TRY(dalloc(s, &s->cw, N));
    TRY(dalloc(s, &s->cwl, N));
    TRY(dalloc(s, &s->nbr_start, N + 1));
    TRY(dalloc(s, &s->nbr_count, N));
    TRY(dalloc(s, &s->nbr_nO, N));
    TRY(dalloc(s, &s->e_bond, (size_t)s->n_mol * P));
    TRY(dalloc(s, &s->red_tmp, 1024));
    TRY(dalloc(s, &s->red_out, 256));
    TRY(dalloc(s, &s->est_part, (size_t)3 * (N + 1)));
    TRY(dalloc(s, &s->status, 1));
    TRY(dalloc(s, &s->dev_max, 1));
    TRY(dalloc(s, &s->rebuild_flag, 1));
    TRY(dalloc(s, &s->step_ctr, 1));
    TRY(dalloc(s, &s->rebuild_count, 2));   // [0] all rebuilds, [1] those run inside step graphs
    TRY(dalloc(s, &s->Tmat, (size_t)P * P));
    TRY(dalloc(s, &s->Tproj, (size_t)P * P));
    TRY(dalloc(s, &s->Tmat_f, (size_t)P * P));
    TRY(dalloc(s, &s->Tproj_f, (size_t)P * P));
    TRY(dalloc(s, &s->cent_buf, (size_t)N * 3));
    s->nbr = nullptr;
    s->nbr_cap = 0;
    s->row_cap = 0;

    std::vector<double> m(N), sm(N);
    for (int i = 0; i < N; ++i) {
        m[i] = s->type[i] == 0 ? s->ff.m_O : s->ff.m_H;
        sm[i] = sqrt(m[i]);
    }
    QHP_CUDA(cudaMemcpy(s->mass, m.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(s->sqrtm, sm.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(s->mol_d, s->mol.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(s->type_d, s->type.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(s->anchor, s->pos0.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemset(s->status, 0, sizeof(unsigned)));
    QHP_CUDA(cudaMemset(s->dev_max, 0, sizeof(unsigned)));
    QHP_CUDA(cudaMemset(s->step_ctr, 0, sizeof(unsigned long long)));
    QHP_CUDA(cudaMemset(s->rebuild_count, 0, 2 * sizeof(unsigned)));
    QHP_CUDA(cudaMemset(s->fmode, 0, sizeof(double) * NP3));
    TRY(upload_matrices(s));
    if (s->th.kind == QHP_THERMO_ADQTB && P != 1) s->th.kind = QHP_THERMO_PILE;
    TRY(dalloc(s, &s->mode_tab, (size_t)2 * P * MT_N));
    mode_constants(s);
    QHP_CUDA(cudaMemcpy(s->mode_tab, s->mode_tab_host.data(), sizeof(double) * s->mode_tab_host.size(),
                        cudaMemcpyHostToDevice));
    QHP_CUDA(launch_init_modes(s));
    s->step = 0;
    s->beads_set = true;
    s->forces_valid = false;
    s->list_valid = false;
    TRY(ensure_capacity(s));
    if (s->th.kind == QHP_THERMO_ADQTB) TRY(qtb_setup(s));
    return sync_and_check(s);
}

int qhp_set_respa(qhp_sys s, int n_alt, int contracted_beads) {
    if (!s || !s->beads_set) {
        set_error("qhp_set_respa: system not initialised");
        return QHP_ERR_STATE;
    }
    if (n_alt < 0 || n_alt > 1024) {
        set_error("qhp_set_respa: n_alt must be in [0, 1024] (0 turns RESPA off)");
        return QHP_ERR_ARG;
    }
    if (n_alt == 0) {
        if (s->respa_n) {
            s->respa_n = 0;
            s->forces_valid = false;
            invalidate_graph(s);
        }
        return QHP_OK;
    }
    if (s->precision != QHP_MIXED || s->th.kind == QHP_THERMO_ADQTB) {
        set_error("qhp_set_respa: needs a mixed-precision system with the PILE or NVE thermostat");
        return QHP_ERR_STATE;
    }
    const int P = s->P;
    const int pc = contracted_beads == 0 ? P : contracted_beads;
    if (pc < 1 || pc > P || (pc & (pc - 1)) || P % pc) {
        set_error("qhp_set_respa: contracted beads must be a power of two dividing P");
        return QHP_ERR_ARG;
    }
    if (pc != s->pc || !s->Ffix_s) {
        TRY(dalloc(s, &s->Ffix_s, (size_t)s->N * 3 * pc));
        TRY(dalloc(s, &s->pos_c, (size_t)s->N * pc));
        if (!s->dev_atom_c) TRY(dalloc(s, &s->dev_atom_c, (size_t)s->N));
        if (!s->fmode_s) TRY(dalloc(s, &s->fmode_s, (size_t)s->N * 3 * P));
        TRY(dalloc(s, &s->Cmat_f, (size_t)pc * P));
        // C[b][n] = sqrt(P) T[b P/pc][n] on the pc lowest-frequency modes (centroid, cos/sin of
        // frequencies 1 .. pc/2 - 1, cos of frequency pc/2), 0 on the others (Eq. (20))
        std::vector<double> T;
        transfer_matrix_host(P, T);
        std::vector<char> keep(P, 0);
        keep[0] = 1;
        if (pc == P) {
            std::fill(keep.begin(), keep.end(), 1);
        } else {
            for (int k = 1; k < pc / 2; ++k) keep[k] = keep[P - k] = 1;
            if (pc >= 2) keep[pc / 2] = 1;
        }
        std::vector<float> C((size_t)pc * P, 0.0f);
        for (int b = 0; b < pc; ++b)
            for (int n = 0; n < P; ++n)
                if (keep[n]) C[(size_t)b * P + n] = (float)(sqrt((double)P) * T[(size_t)(b * (P / pc)) * P + n]);
        for (int b = 0; b < pc; ++b) C[(size_t)b * P] = 1.0f;   // the centroid enters every bead with weight one
        QHP_CUDA(cudaMemcpy(s->Cmat_f, C.data(), sizeof(float) * C.size(), cudaMemcpyHostToDevice));
    }
    s->respa_n = n_alt;
    s->pc = pc;
    s->forces_valid = false;
    invalidate_graph(s);
    return QHP_OK;
}

int qhp_set_thermostat(qhp_sys s, const qhp_thermo* th) {
    if (!s || !th) {
        set_error("null argument");
        return QHP_ERR_ARG;
    }
    if (!(th->dt_fs > 0.0) || th->gamma0 < 0.0 ||
        (th->kind != QHP_THERMO_PILE && th->kind != QHP_THERMO_ADQTB && th->kind != QHP_THERMO_NVE) ||
        (th->integrator != QHP_INTEGRATOR_BAOAB && th->integrator != QHP_INTEGRATOR_BCOCB)) {
        set_error("thermostat: need dt_fs > 0, gamma0 >= 0, kind PILE, ADQTB or NVE, integrator BAOAB or BCOCB");
        return QHP_ERR_ARG;
    }
    if (th->kind == QHP_THERMO_ADQTB) {
        if (!(th->gamma0 > 0.0) || th->n_seg < 4 || th->n_seg > 2048 || (th->n_seg & (th->n_seg - 1)) ||
            (th->adapt != QHP_ADAPT_NONE && th->adapt != QHP_ADAPT_SIMPLE && th->adapt != QHP_ADAPT_RATIO)) {
            set_error("adQTB: need gamma0 > 0, n_seg a power of two in [4, 2048], a valid adapt mode");
            return QHP_ERR_ARG;
        }
        if (s->beads_set && s->P != 1) {
            set_error("adQTB runs on a single bead (P = 1)");
            return QHP_ERR_STATE;
        }
    }
    s->th = *th;
    invalidate_graph(s);
    if (s->beads_set) {
        QHP_CUDA(cudaStreamSynchronize(s->stream));
        mode_constants(s);
        QHP_CUDA(cudaMemcpy(s->mode_tab, s->mode_tab_host.data(), sizeof(double) * s->mode_tab_host.size(),
                            cudaMemcpyHostToDevice));
        if (th->kind == QHP_THERMO_ADQTB) TRY(qtb_setup(s));
    }
    return QHP_OK;
}

int qhp_step_rpmd(qhp_sys s, int n) {
    if (!s) return QHP_ERR_ARG;
    TraceRange tr("qhp_step_rpmd");
    return run_steps(s, n, false);
}

int qhp_step_adqtb(qhp_sys s, int n) {
    if (!s) return QHP_ERR_ARG;
    TraceRange tr("qhp_step_adqtb");
    return run_steps(s, n, true);
}

int qhp_compute_forces(qhp_sys s) {
    if (!s || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    TraceRange tr("qhp_compute_forces");
    TRY(enqueue_forces(s, !s->list_valid, false));
    s->forces_valid = true;
    s->list_valid = true;
    return QHP_OK;
}

int qhp_sync(qhp_sys s) {
    if (!s) return QHP_ERR_ARG;
    return sync_and_check(s);
}

int qhp_get_energy(qhp_sys s, qhp_energy* out) {
    if (!s || !out || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    return compute_energy(s, out);
}

static int get_forces_to(qhp_system_s* s, double* out, bool device_out) {
    if (!s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    if (!s->forces_valid) TRY(qhp_compute_forces(s));
    TRY(sync_and_check(s));
    const int N = s->N, P = s->P;
    const size_t NP3 = (size_t)N * 3 * P;
    std::vector<double> F(NP3);
    if (s->precision == QHP_MIXED) {
        std::vector<long long> Fi(NP3);
        QHP_CUDA(cudaMemcpy(Fi.data(), s->Ffix, sizeof(long long) * NP3, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < NP3; ++k) F[k] = (double)Fi[k] / FIX_SCALE;
    } else {
        QHP_CUDA(cudaMemcpy(F.data(), s->Fd, sizeof(double) * NP3, cudaMemcpyDeviceToHost));
    }
    std::vector<double> o(NP3);
    for (int a = 0; a < N; ++a)
        for (int d = 0; d < 3; ++d)
            for (int b = 0; b < P; ++b) o[((size_t)b * N + a) * 3 + d] = F[((size_t)a * 3 + d) * P + b];
    if (device_out) QHP_CUDA(cudaMemcpy(out, o.data(), sizeof(double) * NP3, cudaMemcpyHostToDevice));
    else memcpy(out, o.data(), sizeof(double) * NP3);
    return QHP_OK;
}

int qhp_get_forces(qhp_sys s, double* out) {
    if (!s || !out) return QHP_ERR_ARG;
    return get_forces_to(s, out, false);
}

int qhp_get_forces_device(qhp_sys s, double* out) {
    if (!s || !out) return QHP_ERR_ARG;
    return get_forces_to(s, out, true);
}

int qhp_get_centroid(qhp_sys s, double* out) {
    if (!s || !out || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    QHP_CUDA(launch_gather_centroids(s, s->cent_buf));
    QHP_CUDA(cudaMemcpyAsync(out, s->cent_buf, sizeof(double) * 3 * s->N, cudaMemcpyDeviceToHost, s->stream));
    return sync_and_check(s);
}

int qhp_get_beads(qhp_sys s, double* out) {
    if (!s || !out || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    double* tmp = nullptr;
    QHP_CUDA(cudaMalloc(&tmp, sizeof(double) * NP3));
    int rc = beads_fp64(s, tmp);
    if (rc == QHP_OK) rc = sync_and_check(s);
    if (rc == QHP_OK) {
        cudaError_t e = cudaMemcpy(out, tmp, sizeof(double) * NP3, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy beads");
    }
    cudaFree(tmp);
    return rc;
}

int qhp_get_modes(qhp_sys s, double* Q, double* Pm) {
    if (!s || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    TRY(sync_and_check(s));
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    if (Q) QHP_CUDA(cudaMemcpy(Q, s->Q, sizeof(double) * NP3, cudaMemcpyDeviceToHost));
    if (Pm) QHP_CUDA(cudaMemcpy(Pm, s->Pm, sizeof(double) * NP3, cudaMemcpyDeviceToHost));
    return QHP_OK;
}

static int set_modes_kind(qhp_system_s* s, const double* Q, const double* Pm, cudaMemcpyKind kind) {
    if (!s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    if (Q) QHP_CUDA(cudaMemcpyAsync(s->Q, Q, sizeof(double) * NP3, kind, s->stream));
    if (Pm) QHP_CUDA(cudaMemcpyAsync(s->Pm, Pm, sizeof(double) * NP3, kind, s->stream));
    if (kind == cudaMemcpyHostToDevice) QHP_CUDA(cudaStreamSynchronize(s->stream));
    if (Q) {
        s->forces_valid = false;
        s->list_valid = false;
    }
    return QHP_OK;
}

int qhp_set_modes(qhp_sys s, const double* Q, const double* Pm) {
    if (!s) return QHP_ERR_ARG;
    return set_modes_kind(s, Q, Pm, cudaMemcpyHostToDevice);
}

int qhp_set_modes_device(qhp_sys s, const double* Q, const double* Pm) {
    if (!s) return QHP_ERR_ARG;
    return set_modes_kind(s, Q, Pm, cudaMemcpyDeviceToDevice);
}

int qhp_get_modes_device(qhp_sys s, double* Q, double* Pm) {
    if (!s || !s->beads_set) return QHP_ERR_STATE;
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    if (Q) QHP_CUDA(cudaMemcpyAsync(Q, s->Q, sizeof(double) * NP3, cudaMemcpyDeviceToDevice, s->stream));
    if (Pm) QHP_CUDA(cudaMemcpyAsync(Pm, s->Pm, sizeof(double) * NP3, cudaMemcpyDeviceToDevice, s->stream));
    return QHP_OK;
}

int qhp_build_list(qhp_sys s) {
    if (!s || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    TRY(ensure_capacity(s));
    TRY(enqueue_forces(s, true, false));
    s->forces_valid = true;
    s->list_valid = true;
    return sync_and_check(s);
}

int qhp_get_cells(qhp_sys s, int* cell, int* order) {
    if (!s || !s->beads_set) return QHP_ERR_STATE;
    TRY(sync_and_check(s));
    if (cell) {
        if (s->list_mode) QHP_CUDA(cudaMemcpy(cell, s->cell, sizeof(int) * s->N, cudaMemcpyDeviceToHost));
        else std::fill(cell, cell + s->N, 0);
    }
    if (order) QHP_CUDA(cudaMemcpy(order, s->perm, sizeof(int) * s->N, cudaMemcpyDeviceToHost));
    return QHP_OK;
}

int qhp_get_list_pairs(qhp_sys s, int64_t* pairs, int64_t cap, int64_t* count) {
    if (!s || !count || !s->beads_set) return QHP_ERR_STATE;
    if (!s->list_valid) TRY(qhp_build_list(s));
    TRY(sync_and_check(s));
    const int N = s->N;
    std::vector<int> cnt(N), perm(N);
    QHP_CUDA(cudaMemcpy(cnt.data(), s->nbr_count, sizeof(int) * N, cudaMemcpyDeviceToHost));
    QHP_CUDA(cudaMemcpy(perm.data(), s->perm, sizeof(int) * N, cudaMemcpyDeviceToHost));
    std::vector<int4> e((size_t)s->nbr_cap);
    QHP_CUDA(cudaMemcpy(e.data(), s->nbr, sizeof(int4) * e.size(), cudaMemcpyDeviceToHost));
    int64_t c = 0;
    for (int i = 0; i < N; ++i)
        for (int64_t k = (int64_t)i * s->row_cap; k < (int64_t)i * s->row_cap + cnt[i]; ++k) {
            const int a = perm[i], b = perm[entry_partner(e[k].x)];
            if (a < b) {
                if (pairs && c < cap) {
                    pairs[2 * c] = a;
                    pairs[2 * c + 1] = b;
                }
                ++c;
            }
        }
    *count = c;
    return QHP_OK;
}

int qhp_get_info(qhp_sys s, qhp_info* out) {
    if (!s || !out) return QHP_ERR_ARG;
    memset(out, 0, sizeof *out);
    out->n_atoms = s->N;
    out->P = s->P;
    out->precision = s->precision;
    out->list_mode = s->list_mode;
    out->step = s->step;
    out->list_capacity = s->nbr_cap;
    out->kernel_launches = s->launches;
    out->n_cells_per_edge = s->n_c;
    if (s->beads_set) {
        cudaStreamSynchronize(s->stream);
        unsigned rb[2] = {0u, 0u};
        std::vector<int> cnt(s->N);
        cudaMemcpy(rb, s->rebuild_count, sizeof rb, cudaMemcpyDeviceToHost);
        cudaMemcpy(cnt.data(), s->nbr_count, sizeof(int) * s->N, cudaMemcpyDeviceToHost);
        int64_t tot = 0;
        for (int v : cnt) tot += v;
        out->rebuilds = rb[0];
        out->list_entries = tot;
        // kernels run inside step-graph conditionals are counted by the device
        out->kernel_launches = s->launches + (int64_t)rb[1] * s->kernels_per_rebuild;
    }
    return QHP_OK;
}

int qhp_set_stream(qhp_sys s, void* stream) {
    if (!s) return QHP_ERR_ARG;
    cudaStream_t ns = stream ? (cudaStream_t)stream : s->own_stream;
    if (ns != s->stream) {
        QHP_CUDA(cudaStreamSynchronize(s->stream));
        s->stream = ns;
    }
    return QHP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- adQTB access, checkpoints
extern "C" {

int qhp_get_gamma(qhp_sys s, double* out) {
    if (!s || !out || !s->qtb_gamma) {
        set_error("no adQTB thermostat");
        return QHP_ERR_STATE;
    }
    TRY(sync_and_check(s));
    QHP_CUDA(cudaMemcpy(out, s->qtb_gamma, sizeof(double) * 2 * (s->n_seg + 1), cudaMemcpyDeviceToHost));
    return QHP_OK;
}

int qhp_set_gamma(qhp_sys s, const double* in) {
    if (!s || !in || !s->qtb_gamma) {
        set_error("no adQTB thermostat");
        return QHP_ERR_STATE;
    }
    QHP_CUDA(cudaStreamSynchronize(s->stream));
    QHP_CUDA(cudaMemcpy(s->qtb_gamma, in, sizeof(double) * 2 * (s->n_seg + 1), cudaMemcpyHostToDevice));
    return QHP_OK;
}

int qhp_get_qtb_noise(qhp_sys s, float* u) {
    if (!s || !u || !s->qtb_u) {
        set_error("no adQTB thermostat");
        return QHP_ERR_STATE;
    }
    TRY(sync_and_check(s));
    QHP_CUDA(cudaMemcpy(u, s->qtb_u, sizeof(float) * (size_t)s->n_seg * 3 * s->N, cudaMemcpyDeviceToHost));
    return QHP_OK;
}

int qhp_get_qtb_records(qhp_sys s, float* v, float* F) {
    if (!s || !s->qtb_v) {
        set_error("no adQTB thermostat");
        return QHP_ERR_STATE;
    }
    TRY(sync_and_check(s));
    const size_t n = (size_t)s->n_seg * 3 * s->N;
    if (v) QHP_CUDA(cudaMemcpy(v, s->qtb_v, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (F) QHP_CUDA(cudaMemcpy(F, s->qtb_F, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return QHP_OK;
}

// Blob: header, Q, Pm, list anchors, [adQTB: gamma, RATIO averages, u, v, F].  The
// anchors (centroids at the last list build) and the running deviation maximum are
// part of the state: the mixed path rounds positions relative to the anchors and the
// next rebuild depends on the maximum, so a restore that rebuilt from fresh anchors
// would not continue bit for bit.
struct StateHeader {
    uint64_t magic, N, P, step, n_seg, ratio_first, precision, dev_max_bits;
};
static const uint64_t STATE_MAGIC = 0x3250485153544154ull;

static size_t state_bytes(const qhp_system_s* s) {
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    const size_t nq = s->qtb_u ? (size_t)s->n_seg * 3 * s->N : 0;
    const size_t ng = s->qtb_u ? 2 * (size_t)(s->n_seg + 1) : 0;
    return sizeof(StateHeader) + (2 * NP3 + 3 * (size_t)s->N) * sizeof(double) + 3 * ng * sizeof(double) +
           3 * nq * sizeof(float);
}

int qhp_get_state(qhp_sys s, void* buf, size_t* size) {
    if (!s || !size || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    const size_t nq = s->qtb_u ? (size_t)s->n_seg * 3 * s->N : 0;
    const size_t ng = s->qtb_u ? 2 * (size_t)(s->n_seg + 1) : 0;
    const size_t need = state_bytes(s);
    if (!buf) {
        *size = need;
        return QHP_OK;
    }
    if (*size < need) {
        set_error("state buffer too small (%zu < %zu)", *size, need);
        return QHP_ERR_ARG;
    }
    if (!s->forces_valid) TRY(qhp_compute_forces(s));
    TRY(sync_and_check(s));
    unsigned dm = 0;
    QHP_CUDA(cudaMemcpy(&dm, s->dev_max, sizeof dm, cudaMemcpyDeviceToHost));
    char* p = static_cast<char*>(buf);
    StateHeader h{STATE_MAGIC, (uint64_t)s->N, (uint64_t)s->P, (uint64_t)s->step, (uint64_t)(s->qtb_u ? s->n_seg : 0),
                  (uint64_t)s->qtb_ratio_first, (uint64_t)s->precision, (uint64_t)dm};
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    QHP_CUDA(cudaMemcpy(p, s->Q, NP3 * sizeof(double), cudaMemcpyDeviceToHost));
    p += NP3 * sizeof(double);
    QHP_CUDA(cudaMemcpy(p, s->Pm, NP3 * sizeof(double), cudaMemcpyDeviceToHost));
    p += NP3 * sizeof(double);
    QHP_CUDA(cudaMemcpy(p, s->anchor, 3 * (size_t)s->N * sizeof(double), cudaMemcpyDeviceToHost));
    p += 3 * (size_t)s->N * sizeof(double);
    if (nq) {
        QHP_CUDA(cudaMemcpy(p, s->qtb_gamma, ng * sizeof(double), cudaMemcpyDeviceToHost));
        p += ng * sizeof(double);
        QHP_CUDA(cudaMemcpy(p, s->qtb_avg, 2 * ng * sizeof(double), cudaMemcpyDeviceToHost));
        p += 2 * ng * sizeof(double);
        QHP_CUDA(cudaMemcpy(p, s->qtb_u, nq * sizeof(float), cudaMemcpyDeviceToHost));
        p += nq * sizeof(float);
        QHP_CUDA(cudaMemcpy(p, s->qtb_v, nq * sizeof(float), cudaMemcpyDeviceToHost));
        p += nq * sizeof(float);
        QHP_CUDA(cudaMemcpy(p, s->qtb_F, nq * sizeof(float), cudaMemcpyDeviceToHost));
    }
    *size = need;
    return QHP_OK;
}

int qhp_set_state(qhp_sys s, const void* buf, size_t size) {
    if (!s || !buf || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    StateHeader h;
    if (size < sizeof h) {
        set_error("state blob too small");
        return QHP_ERR_ARG;
    }
    memcpy(&h, buf, sizeof h);
    const size_t NP3 = (size_t)s->N * 3 * s->P;
    const size_t nq = s->qtb_u ? (size_t)s->n_seg * 3 * s->N : 0;
    const size_t ng = s->qtb_u ? 2 * (size_t)(s->n_seg + 1) : 0;
    if (h.magic != STATE_MAGIC || h.N != (uint64_t)s->N || h.P != (uint64_t)s->P ||
        h.n_seg != (uint64_t)(s->qtb_u ? s->n_seg : 0) || h.precision != (uint64_t)s->precision ||
        size < state_bytes(s)) {
        set_error("state blob does not match this system");
        return QHP_ERR_ARG;
    }
    QHP_CUDA(cudaStreamSynchronize(s->stream));
    const char* p = static_cast<const char*>(buf) + sizeof h;
    QHP_CUDA(cudaMemcpy(s->Q, p, NP3 * sizeof(double), cudaMemcpyHostToDevice));
    p += NP3 * sizeof(double);
    QHP_CUDA(cudaMemcpy(s->Pm, p, NP3 * sizeof(double), cudaMemcpyHostToDevice));
    p += NP3 * sizeof(double);
    QHP_CUDA(cudaMemcpy(s->anchor, p, 3 * (size_t)s->N * sizeof(double), cudaMemcpyHostToDevice));
    p += 3 * (size_t)s->N * sizeof(double);
    if (nq) {
        QHP_CUDA(cudaMemcpy(s->qtb_gamma, p, ng * sizeof(double), cudaMemcpyHostToDevice));
        p += ng * sizeof(double);
        QHP_CUDA(cudaMemcpy(s->qtb_avg, p, 2 * ng * sizeof(double), cudaMemcpyHostToDevice));
        p += 2 * ng * sizeof(double);
        QHP_CUDA(cudaMemcpy(s->qtb_u, p, nq * sizeof(float), cudaMemcpyHostToDevice));
        p += nq * sizeof(float);
        QHP_CUDA(cudaMemcpy(s->qtb_v, p, nq * sizeof(float), cudaMemcpyHostToDevice));
        p += nq * sizeof(float);
        QHP_CUDA(cudaMemcpy(s->qtb_F, p, nq * sizeof(float), cudaMemcpyHostToDevice));
        s->qtb_ratio_first = (int)h.ratio_first;
    }
    s->step = (int64_t)h.step;
    unsigned long long st = h.step;
    QHP_CUDA(cudaMemcpy(s->step_ctr, &st, sizeof st, cudaMemcpyHostToDevice));
    // rebuild the list from the stored anchors, then the forces at the restored modes
    s->keep_anchor = 1;
    int rc = ensure_capacity(s);
    if (rc == QHP_OK) rc = enqueue_forces(s, true, false);
    s->keep_anchor = 0;
    TRY(rc);
    const unsigned dm = (unsigned)h.dev_max_bits;
    QHP_CUDA(cudaMemcpyAsync(s->dev_max, &dm, sizeof dm, cudaMemcpyHostToDevice, s->stream));
    s->forces_valid = true;
    s->list_valid = true;
    return sync_and_check(s);
}

}  // extern "C"

// ---------------------------------------------------------------- measurement hooks
extern "C" {

int qhp_set_profiling(qhp_sys s, int on) {
    if (!s) return QHP_ERR_ARG;
    if (on && !s->prof_ev[0])
        for (int k = 0; k < 6; ++k) QHP_CUDA(cudaEventCreate(&s->prof_ev[k]));
    if ((on != 0) != (s->prof_on != 0)) invalidate_graph(s);   // events are captured into the step graph
    s->prof_on = on ? 1 : 0;
    return QHP_OK;
}

int qhp_set_graph_mode(qhp_sys s, int use_graphs) {
    if (!s || (use_graphs != 0 && use_graphs != 1)) {
        set_error("qhp_set_graph_mode: need a system and use_graphs 0 or 1");
        return QHP_ERR_ARG;
    }
    if (use_graphs != s->use_graphs) invalidate_graph(s);
    s->use_graphs = use_graphs;
    return QHP_OK;
}

int qhp_get_profile(qhp_sys s, qhp_profile* out) {
    if (!s || !out) return QHP_ERR_ARG;
    if (!s->prof_on) {
        set_error("profiling is off");
        return QHP_ERR_STATE;
    }
    TRY(sync_and_check(s));
    float t[5];
    for (int k = 0; k < 5; ++k) QHP_CUDA(cudaEventElapsedTime(&t[k], s->prof_ev[k], s->prof_ev[k + 1]));
    out->integrate_ms = t[0];
    out->list_ms = t[1];
    out->pair_ms = t[2];
    out->bonded_ms = t[3];
    out->project_ms = t[4];
    float tot = 0.f;
    QHP_CUDA(cudaEventElapsedTime(&tot, s->prof_ev[0], s->prof_ev[5]));
    out->step_ms = tot;
    return QHP_OK;
}

int qhp_count_pairs(qhp_sys s, int64_t* pairs, int64_t* oo_pairs) {
    if (!s || !pairs || !s->beads_set) {
        set_error("system not initialised");
        return QHP_ERR_STATE;
    }
    if (!s->forces_valid) TRY(qhp_compute_forces(s));
    unsigned long long* d = reinterpret_cast<unsigned long long*>(s->red_out + 192);
    QHP_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s->stream));
    QHP_CUDA(launch_count_pairs(s, d));
    unsigned long long h[2];
    QHP_CUDA(cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s->stream));
    TRY(sync_and_check(s));
    *pairs = (int64_t)h[0];
    if (oo_pairs) *oo_pairs = (int64_t)h[1];
    return QHP_OK;
}

}  // extern "C"
