// Many independent systems stepped together (the paper's bead parallelism taken one level
// further: systems of uneven size and bead count share every launch).
//
// One batched step is one CUDA graph: one cooperative launch of k_step_batch over every
// system (integrate with each system's list check, forces, projection: three phases between
// grid barriers, persistent blocks walking (system, group) items), then one conditional node
// per system that runs only when that system's check fired in this step: the list rebuild and
// that system's forces and projection with the single-system kernels.  A block walks its item
// ranges in system order; the host scheduler cuts the item lists into one contiguous range per
// block (per half block for the forces, one specialisation after another) with about equal
// estimated work, so uneven systems balance and a block keeps its system's transform in shared
// memory across items.
//
// The autotuner times the pair kernel of one system per bead count with 1, 2 and 4 warps
// per atom and keeps the fastest for every system with that bead count.
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "qhp_internal.cuh"

struct qhp_batch_s {
    std::vector<qhp_sys> sys;
    std::vector<cudaStream_t> sys_streams;   // the members' streams before they joined
    cudaStream_t own_stream = nullptr, stream = nullptr, aux = nullptr;
    qhp::BatchStage integrate, force, project;
    qhp::CheckArgs* check_args = nullptr;   // device [n_sys]
    int* done = nullptr;                    // device [n_sys]: integrate items finished this step
    int* nitems = nullptr;                  // device [n_sys]: integrate items per system
    qhp::StepBatchState* state = nullptr;   // device: grid barriers, timeout status, phase stamps
    int items_pair = 0;
    int grid = 0;                           // co-resident blocks of the step kernel
    size_t smem = 0;
    long long wait_ns = 2000000000LL;       // a grid barrier gives up after this long
    cudaGraphExec_t exec = nullptr;
    std::vector<int4*> nbr_seen;            // list buffers the stages were built for
    std::vector<int> rowcap_seen;
    std::vector<int> pairw_seen;            // and the warps-per-atom settings
    int64_t steps = 0;
    int64_t launches = 0;
    int kernels_per_step = 0;
    std::vector<int> kernels_per_rebuild;
    cudaEvent_t ev[3] = {};                 // step kernel start / end, rebuild bodies end
};

namespace qhp {

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

void stage_free(BatchStage& st) {
    cudaFree(st.args);
    cudaFree(st.items);
    cudaFree(st.ranges);
    st = BatchStage{};
}

int stage_upload(BatchStage& st, const void* args, size_t args_bytes, const std::vector<int2>& items,
                 const std::vector<double>& cost, int grid) {
    const size_t smem = st.smem;
    stage_free(st);
    st.smem = smem;
    const int n = (int)items.size();
    grid = std::max(1, grid);   // blocks past the items get empty ranges
    double total = 0.0;
    for (double c : cost) total += c;
    // contiguous ranges: block g starts where the running cost first reaches g/grid of the total
    std::vector<int> r(grid + 1, n);
    r[0] = 0;
    double acc = 0.0;
    int g = 1;
    for (int i = 0; i < n && g < grid; ++i) {
        acc += cost[i];
        while (g < grid && acc >= total * (double)g / (double)grid) r[g++] = i + 1;
    }
    st.grid = grid;
    st.n_items = n;
    st.cost = total;
    QHP_CUDA(cudaMalloc(&st.args, std::max<size_t>(args_bytes, 1)));
    QHP_CUDA(cudaMalloc(&st.items, sizeof(int2) * std::max(n, 1)));
    QHP_CUDA(cudaMalloc(&st.ranges, sizeof(int) * (grid + 1)));
    QHP_CUDA(cudaMemcpy(st.args, args, args_bytes, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(st.items, items.data(), sizeof(int2) * n, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(st.ranges, r.data(), sizeof(int) * (grid + 1), cudaMemcpyHostToDevice));
    return QHP_OK;
}

int stage_upload_phased(BatchStage& st, const void* args, size_t args_bytes, const std::vector<int2>& items,
                        const std::vector<double>& cost, const std::vector<int>& phase, int grid) {
    const int n = (int)items.size();
    grid = std::max(1, grid);   // blocks past the items get empty ranges
    int n_phase = 0;
    for (int p : phase) n_phase = std::max(n_phase, p + 1);
    // per phase, its items in order and the cut into `grid` chunks of about equal cost
    std::vector<std::vector<int>> idx(n_phase);
    for (int i = 0; i < n; ++i) idx[phase[i]].push_back(i);
    std::vector<std::vector<int>> cut(n_phase);
    for (int p = 0; p < n_phase; ++p) {
        const std::vector<int>& ix = idx[p];
        double total = 0.0;
        for (int i : ix) total += cost[i];
        std::vector<int>& r = cut[p];
        r.assign(grid + 1, (int)ix.size());
        r[0] = 0;
        double acc = 0.0;
        int g = 1;
        for (int k = 0; k < (int)ix.size() && g < grid; ++k) {
            acc += cost[ix[k]];
            while (g < grid && acc >= total * (double)g / (double)grid) r[g++] = k + 1;
        }
    }
    // block g runs chunk g of every phase, phase by phase
    std::vector<int2> out;
    out.reserve(n);
    std::vector<int> ranges(grid + 1, 0);
    double total = 0.0;
    for (int g = 0; g < grid; ++g) {
        for (int p = 0; p < n_phase; ++p)
            for (int k = cut[p][g]; k < cut[p][g + 1]; ++k) {
                out.push_back(items[idx[p][k]]);
                total += cost[idx[p][k]];
            }
        ranges[g + 1] = (int)out.size();
    }
    const size_t smem = st.smem;
    stage_free(st);
    st.smem = smem;
    st.grid = grid;
    st.n_items = n;
    st.cost = total;
    QHP_CUDA(cudaMalloc(&st.args, std::max<size_t>(args_bytes, 1)));
    QHP_CUDA(cudaMalloc(&st.items, sizeof(int2) * std::max(n, 1)));
    QHP_CUDA(cudaMalloc(&st.ranges, sizeof(int) * (grid + 1)));
    QHP_CUDA(cudaMemcpy(st.args, args, args_bytes, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(st.items, out.data(), sizeof(int2) * n, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(st.ranges, ranges.data(), sizeof(int) * (grid + 1), cudaMemcpyHostToDevice));
    return QHP_OK;
}

namespace {

void drop_graph(qhp_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

std::vector<qhp_system_s*> members(qhp_batch_s* b) { return std::vector<qhp_system_s*>(b->sys.begin(), b->sys.end()); }

int build_stages(qhp_batch_s* b) {
    const std::vector<qhp_system_s*> v = members(b);
    int maxP = 1;
    for (qhp_system_s* s : v) maxP = std::max(maxP, s->P);
    TRY(step_batch_config(maxP, &b->grid, &b->smem));
    TRY(batch_stage_integrate(v, b->integrate, b->grid));
    TRY(batch_stage_force(v, b->force, &b->items_pair, 2 * b->grid));
    TRY(batch_stage_project(v, b->project, b->grid));
    b->nbr_seen.clear();
    b->rowcap_seen.clear();
    b->pairw_seen.clear();
    for (qhp_system_s* s : v) {
        b->nbr_seen.push_back(s->nbr);
        b->rowcap_seen.push_back(s->row_cap);
        b->pairw_seen.push_back(s->pair_w);
    }
    drop_graph(b);
    return QHP_OK;
}

// Capture one batched step into b->exec.
int capture(qhp_batch_s* b) {
    drop_graph(b);
    const int n = (int)b->sys.size();
    cudaGraph_t g = nullptr;
    QHP_CUDA(cudaGraphCreate(&g, 0));
    std::vector<cudaGraphConditionalHandle> handles(n);
    std::vector<CheckArgs> ca(n);
    for (int k = 0; k < n; ++k) {
        qhp_system_s* s = b->sys[k];
        cudaError_t e = cudaGraphConditionalHandleCreate(&handles[k], g, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "batch conditional handle");
        }
        const float half = (float)(0.5 * s->ff.skin);
        ca[k] = CheckArgs{s->dev_max, s->rebuild_flag, s->rebuild_count, handles[k], half * half};
    }
    if (!b->check_args) QHP_CUDA(cudaMalloc(&b->check_args, sizeof(CheckArgs) * n));
    if (!b->done) QHP_CUDA(cudaMalloc(&b->done, sizeof(int) * n));
    if (!b->nitems) QHP_CUDA(cudaMalloc(&b->nitems, sizeof(int) * n));
    std::vector<int> ni(n);
    for (int k = 0; k < n; ++k) ni[k] = batch_integrate_items(b->sys[k]);
    if (!b->state) QHP_CUDA(cudaMalloc(&b->state, sizeof(StepBatchState)));
    QHP_CUDA(cudaMemcpy(b->check_args, ca.data(), sizeof(CheckArgs) * n, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemcpy(b->nitems, ni.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    QHP_CUDA(cudaMemset(b->done, 0, sizeof(int) * n));
    QHP_CUDA(cudaMemset(b->state, 0, sizeof(StepBatchState)));

    cudaError_t e = cudaStreamBeginCaptureToGraph(b->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "batch capture start");
    }
    int rc = QHP_OK;
    b->kernels_per_rebuild.assign(n, 0);
    auto fail = [&](cudaError_t err, const char* what) {
        if (rc == QHP_OK && err != cudaSuccess) rc = cuda_fail(err, what);
    };
    // event-record nodes around the launch and the rebuild bodies: every replay timestamps them
    auto mark = [&](int k) { fail(cudaEventRecordWithFlags(b->ev[k], b->stream, cudaEventRecordExternal), "batch event"); };
    mark(0);
    fail(launch_step_batch(b->integrate, b->force, b->project, b->check_args, b->done, b->nitems, b->state, b->wait_ns,
                           b->grid, b->smem, b->stream),
         "batched step launch");
    mark(1);
    std::vector<cudaGraphNode_t> conds(n);
    if (rc == QHP_OK) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* ed = nullptr;
        size_t nd = 0;
        fail(cudaStreamGetCaptureInfo(b->stream, &cs, nullptr, &cg, &deps, &ed, &nd), "batch capture info");
        std::vector<cudaGraphNode_t> dep(deps, deps + nd);
        for (int k = 0; k < n && rc == QHP_OK; ++k) {
            alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
            memset(pbuf, 0, sizeof pbuf);
            cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(pbuf);
            p.type = cudaGraphNodeTypeConditional;
            p.conditional.handle = handles[k];
            p.conditional.type = cudaGraphCondTypeIf;
            p.conditional.size = 1;
            fail(cudaGraphAddNode(&conds[k], cg, dep.data(), nullptr, dep.size(), &p), "batch conditional node");
            if (rc != QHP_OK) break;
            cudaGraph_t body = p.conditional.phGraph_out[0];
            fail(cudaStreamBeginCaptureToGraph(b->aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                 "batch body capture");
            if (rc != QHP_OK) break;
            // the rebuilt system's step from its list check on, as stepping it alone does
            qhp_system_s* s = b->sys[k];
            cudaStream_t keep = s->stream;
            const int prof = s->prof_on;
            s->stream = b->aux;
            s->prof_on = 0;
            const int64_t before = s->launches;
            cudaError_t e1 = launch_rebuild(s);
            if (e1 == cudaSuccess) e1 = launch_integrate_gated(s);
            if (e1 == cudaSuccess) e1 = launch_cover_check(s);
            if (e1 == cudaSuccess) e1 = launch_forces(s, false);
            if (e1 == cudaSuccess) e1 = launch_project(s, true);
            b->kernels_per_rebuild[k] = (int)(s->launches - before);
            s->launches = before;
            s->stream = keep;
            s->prof_on = prof;
            cudaGraph_t out = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(b->aux, &out);
            fail(e1, "batch rebuild chain");
            fail(e2, "batch body capture end");
        }
        if (rc == QHP_OK)
            fail(cudaStreamUpdateCaptureDependencies(b->stream, conds.data(), nullptr, n,
                                                     cudaStreamSetCaptureDependencies),
                 "batch join");
    }
    mark(2);
    cudaGraph_t g2 = nullptr;
    e = cudaStreamEndCapture(b->stream, &g2);
    if (rc == QHP_OK && e != cudaSuccess) rc = cuda_fail(e, "batch capture end");
    if (rc == QHP_OK) {
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            rc = cuda_fail(e, "batch graph instantiate");
        }
    }
    cudaGraphDestroy(g);
    b->kernels_per_step = 1;
    return rc;
}

bool stale(qhp_batch_s* b) {
    for (size_t k = 0; k < b->sys.size(); ++k)
        if (b->sys[k]->nbr != b->nbr_seen[k] || b->sys[k]->row_cap != b->rowcap_seen[k] ||
            b->sys[k]->pair_w != b->pairw_seen[k])
            return true;
    return false;
}

// Time the mixed pair kernel of one system for W = 1, 2, 4 warps per atom (CUDA events,
// after warm-up launches) and keep the fastest.
int tune_pair(qhp_system_s* s, int reps, int* best_out, float* ms_out) {
    cudaEvent_t e0, e1;
    QHP_CUDA(cudaEventCreate(&e0));
    QHP_CUDA(cudaEventCreate(&e1));
    const int keep = s->pair_w;
    int best = 0;
    float best_ms = 0.0f;
    int rc = QHP_OK;
    const int cand[3] = {1, 2, 4};
    for (int W : cand) {
        s->pair_w = W;
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch_pair(s, false);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_pair(s, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "pair autotune");
            break;
        }
        if (best == 0 || ms < best_ms) {
            best = W;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->pair_w = rc == QHP_OK ? best : keep;
    if (rc == QHP_OK) {
        // the W variants sum in different orders: recompute the forces with the chosen one
        graph_invalidate(s);
        TRY(qhp_compute_forces(s));
        TRY(system_sync(s));
        if (best_out) *best_out = best;
        if (ms_out) *ms_out = best_ms / (float)reps;
    }
    return rc;
}

}  // namespace

}  // namespace qhp

using namespace qhp;

extern "C" {

int qhp_autotune(qhp_sys s, int reps, int* warps_per_atom) {
    if (!s || !s->beads_set || s->precision != QHP_MIXED || reps < 1) {
        set_error("qhp_autotune: needs an initialised mixed-precision system and reps >= 1");
        return QHP_ERR_STATE;
    }
    if (!s->forces_valid) TRY(qhp_compute_forces(s));
    TRY(system_sync(s));
    return tune_pair(s, reps, warps_per_atom, nullptr);
}

int qhp_set_pair_warps(qhp_sys s, int warps_per_atom) {
    if (!s || (warps_per_atom != 0 && warps_per_atom != 1 && warps_per_atom != 2 && warps_per_atom != 4)) {
        set_error("qhp_set_pair_warps: warps_per_atom must be 0 (default), 1, 2 or 4");
        return QHP_ERR_ARG;
    }
    if (s->pair_w != warps_per_atom) {
        s->pair_w = warps_per_atom;
        s->forces_valid = false;   // the next step recomputes the forces with this setting
        graph_invalidate(s);
    }
    return QHP_OK;
}

int qhp_set_pair_skip(qhp_sys s, int enabled) {
    if (!s || (enabled != 0 && enabled != 1)) {
        set_error("qhp_set_pair_skip: enabled must be 0 or 1");
        return QHP_ERR_ARG;
    }
    if (s->pair_skip != enabled) {
        s->pair_skip = enabled;
        graph_invalidate(s);
    }
    return QHP_OK;
}

int qhp_create_batch(qhp_batch* out, int n_sys, const qhp_sys* systems) {
    if (!out || n_sys < 1 || !systems) {
        set_error("qhp_create_batch: need n_sys >= 1 systems");
        return QHP_ERR_ARG;
    }
    *out = nullptr;
    for (int k = 0; k < n_sys; ++k) {
        qhp_system_s* s = systems[k];
        if (!s || !s->beads_set || s->precision != QHP_MIXED ||
            (s->th.kind != QHP_THERMO_PILE && s->th.kind != QHP_THERMO_NVE) || s->respa_n) {
            set_error("qhp_create_batch: system %d must be initialised, mixed precision, PILE or NVE, without RESPA", k);
            return QHP_ERR_STATE;
        }
        for (int j = 0; j < k; ++j)
            if (systems[j] == s) {
                set_error("qhp_create_batch: system %d appears twice", k);
                return QHP_ERR_ARG;
            }
    }
    qhp_batch_s* b = new qhp_batch_s();
    b->sys.assign(systems, systems + n_sys);
    int rc = QHP_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&b->ev[k]);
    if (e != cudaSuccess) rc = cuda_fail(e, "batch streams");
    b->stream = b->own_stream;
    // every member starts with valid forces and list; from now on its work is queued on
    // the batch's stream, so member calls and batch steps stay in order
    for (int k = 0; k < n_sys && rc == QHP_OK; ++k) {
        qhp_system_s* s = b->sys[k];
        if (!s->forces_valid) rc = qhp_compute_forces(s);
        if (rc == QHP_OK) rc = system_sync(s);
        b->sys_streams.push_back(s->stream);
        s->stream = b->stream;
    }
    if (rc == QHP_OK) rc = build_stages(b);
    if (rc != QHP_OK) {
        qhp_destroy_batch(b);
        return rc;
    }
    *out = b;
    return QHP_OK;
}

int qhp_destroy_batch(qhp_batch b) {
    if (!b) return QHP_ERR_ARG;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (size_t k = 0; k < b->sys_streams.size(); ++k) {
        b->sys[k]->stream = b->sys_streams[k];
        graph_invalidate(b->sys[k]);
    }
    drop_graph(b);
    stage_free(b->integrate);
    stage_free(b->force);
    stage_free(b->project);
    cudaFree(b->check_args);
    cudaFree(b->done);
    cudaFree(b->nitems);
    cudaFree(b->state);
    for (int k = 0; k < 3; ++k)
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    if (b->aux) cudaStreamDestroy(b->aux);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return QHP_OK;
}

int qhp_batch_set_stream(qhp_batch b, void* stream) {
    if (!b) return QHP_ERR_ARG;
    QHP_CUDA(cudaStreamSynchronize(b->stream));
    b->stream = stream ? (cudaStream_t)stream : b->own_stream;
    for (qhp_system_s* s : b->sys) {
        s->stream = b->stream;
        graph_invalidate(s);
    }
    drop_graph(b);
    return QHP_OK;
}

int qhp_batch_step(qhp_batch b, int n) {
    if (!b || n < 0) {
        set_error("qhp_batch_step: need a batch and n >= 0");
        return QHP_ERR_ARG;
    }
    if (n == 0) return QHP_OK;
    TraceRange tr("qhp_batch_step");
    // report a fault of an earlier batched step found by a member's last synchronising call
    if (stale(b)) TRY(build_stages(b));
    if (!b->exec) TRY(capture(b));
    for (int k = 0; k < n; ++k) QHP_CUDA(cudaGraphLaunch(b->exec, b->stream));
    b->steps += n;
    b->launches += (int64_t)b->kernels_per_step * n;
    for (qhp_system_s* s : b->sys) {
        s->step += n;
        s->forces_valid = true;
        s->list_valid = true;
    }
    return QHP_OK;
}

int qhp_batch_sync(qhp_batch b) {
    if (!b) return QHP_ERR_ARG;
    QHP_CUDA(cudaStreamSynchronize(b->stream));
    if (b->state) {
        unsigned st = 0;
        QHP_CUDA(cudaMemcpy(&st, &b->state->status, sizeof st, cudaMemcpyDeviceToHost));
        if (st & ST_TIMEOUT) {
            // the barrier words may be mid-count: start the next step from a clean state
            QHP_CUDA(cudaMemset(b->state, 0, sizeof(StepBatchState)));
            set_error("qhp_batch_sync: a grid barrier of the batched step waited longer than %lld ns", b->wait_ns);
            return QHP_ERR_TIMEOUT;
        }
    }
    for (qhp_system_s* s : b->sys) TRY(system_sync(s));
    return QHP_OK;
}

int qhp_batch_set_wait_limit(qhp_batch b, long long wait_ns) {
    if (!b || wait_ns < 1000 || wait_ns > 100000000000LL) {
        set_error("qhp_batch_set_wait_limit: wait_ns must lie in [1e3, 1e11]");
        return QHP_ERR_ARG;
    }
    if (wait_ns != b->wait_ns) {
        b->wait_ns = wait_ns;
        drop_graph(b);
    }
    return QHP_OK;
}

int qhp_batch_autotune(qhp_batch b, int reps, int* tuned /*[7]: W for P = 1, 2, 4, ..., 64; 0 if absent*/) {
    if (!b || reps < 1) return QHP_ERR_ARG;
    TRY(qhp_batch_sync(b));
    std::map<int, qhp_system_s*> largest;   // per bead count, the member with most atoms
    for (qhp_system_s* s : b->sys) {
        auto it = largest.find(s->P);
        if (it == largest.end() || s->N > it->second->N) largest[s->P] = s;
    }
    std::map<int, int> W;
    for (auto& kv : largest) {
        int best = 0;
        TRY(tune_pair(kv.second, reps, &best, nullptr));
        W[kv.first] = best;
    }
    for (qhp_system_s* s : b->sys) {
        if (s->pair_w != W[s->P]) {
            // forces of the current state are recomputed in the tuned summation order
            s->pair_w = W[s->P];
            graph_invalidate(s);
            TRY(qhp_compute_forces(s));
        }
    }
    TRY(qhp_batch_sync(b));
    if (tuned)
        for (int k = 0; k < 7; ++k) {
            auto it = W.find(1 << k);
            tuned[k] = it == W.end() ? 0 : it->second;
        }
    return build_stages(b);
}

int qhp_batch_get_profile(qhp_batch b, qhp_profile* out) {
    if (!b || !out) return QHP_ERR_ARG;
    if (!b->exec || b->steps == 0) {
        set_error("qhp_batch_get_profile: no batched step has run");
        return QHP_ERR_STATE;
    }
    QHP_CUDA(cudaStreamSynchronize(b->stream));
    // phases of the step kernel from its device clock stamps; the rebuild bodies by events
    StepBatchState h;
    QHP_CUDA(cudaMemcpy(&h, b->state, sizeof h, cudaMemcpyDeviceToHost));
    float launch_ms = 0.0f, bodies_ms = 0.0f;
    QHP_CUDA(cudaEventElapsedTime(&launch_ms, b->ev[0], b->ev[1]));
    QHP_CUDA(cudaEventElapsedTime(&bodies_ms, b->ev[1], b->ev[2]));
    auto span = [&](int a, int c) { return h.ts[c] > h.ts[a] ? (float)((double)(h.ts[c] - h.ts[a]) * 1e-6) : 0.0f; };
    out->integrate_ms = span(0, 1);   // with the list checks
    out->pair_ms = span(1, 2);        // pair and bonded items
    out->bonded_ms = 0.0f;
    out->project_ms = span(2, 3);
    out->list_ms = bodies_ms;         // conditional bodies: rebuilds and the rebuilt systems' forces
    out->step_ms = launch_ms + bodies_ms;
    return QHP_OK;
}

int qhp_batch_get_info(qhp_batch b, qhp_batch_info* out) {
    if (!b || !out) return QHP_ERR_ARG;
    memset(out, 0, sizeof *out);
    out->n_sys = (int)b->sys.size();
    for (qhp_system_s* s : b->sys) out->atom_beads += (int64_t)s->N * s->P;
    out->steps = b->steps;
    out->kernels_per_step = b->kernels_per_step;
    out->grid_integrate = b->integrate.grid;
    out->grid_pair = b->force.grid;   // half blocks of the step kernel: pair and bonded items
    out->grid_bonded = 0;
    out->grid_project = b->project.grid;
    out->items_pair = b->items_pair;
    // kernels run inside the conditional rebuild bodies, counted on the device
    cudaStreamSynchronize(b->stream);
    int64_t extra = 0;
    for (size_t k = 0; k < b->sys.size() && k < b->kernels_per_rebuild.size(); ++k) {
        unsigned rb[2] = {0u, 0u};
        cudaMemcpy(rb, b->sys[k]->rebuild_count, sizeof rb, cudaMemcpyDeviceToHost);
        out->rebuilds += rb[0];
        extra += (int64_t)rb[1] * b->kernels_per_rebuild[k];
    }
    out->kernel_launches = b->launches + extra;
    return QHP_OK;
}

}  // extern "C"
