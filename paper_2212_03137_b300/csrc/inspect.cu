// Inspection of the centroid list one atom at a time (for large boxes, where exporting
// every pair is impractical).
#include <vector>

#include "qhp_internal.cuh"

using namespace qhp;

extern "C" int qhp_get_list_row(qhp_sys s, int atom, int* partners, int cap, int* count) {
    if (!s || !count || !s->beads_set || atom < 0 || atom >= s->N || cap < 0) {
        set_error("qhp_get_list_row: bad system, atom index or capacity");
        return QHP_ERR_ARG;
    }
    if (!s->list_valid) {
        const int rc = qhp_build_list(s);
        if (rc != QHP_OK) return rc;
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qhp_get_list_row sync");
    int sorted = 0, n = 0, k0 = 0;
    e = cudaMemcpy(&sorted, s->iperm + atom, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&n, s->nbr_count + sorted, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&k0, s->nbr_start + sorted, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "qhp_get_list_row copy");
    std::vector<int4> ent(n > 0 ? n : 1);
    std::vector<int> perm(s->N);
    if (n > 0) e = cudaMemcpy(ent.data(), s->nbr + k0, sizeof(int4) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(perm.data(), s->perm, sizeof(int) * s->N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "qhp_get_list_row copy");
    for (int k = 0; k < n && k < cap; ++k) partners[k] = perm[entry_partner(ent[k].x)];
    *count = n;
    return QHP_OK;
}
