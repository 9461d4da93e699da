// api_cable.cu -- C ABI of the cable coupling: cells of compartments with a
// per-cell tree (Hines) solve in place of the diagonal voltage update.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "runtime.cuh"

using namespace nmodl;

extern "C" {

NMODL_API int nmodl_cable_create(nmodl_ctx* c, int64_t n_nodes, const int32_t* parent,
                                 const double* ga, const double* gb, nmodl_cable** out) {
    if (!out) return NMODL_ERR_ARG;
    *out = nullptr;
    if (!c || n_nodes < 1 || !parent || !ga || !gb || n_nodes > INT32_MAX) return NMODL_ERR_ARG;
    DeviceGuard dg(c->device);
    std::vector<int32_t> hp(n_nodes);
    std::vector<double> ha(n_nodes), hb(n_nodes);
    cudaError_t e = cudaMemcpy(hp.data(), parent, n_nodes * sizeof(int32_t), cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(ha.data(), ga, n_nodes * sizeof(double), cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(hb.data(), gb, n_nodes * sizeof(double), cudaMemcpyDefault);
    if (e != cudaSuccess) return nmodl_cuda_status(e);
    // cells: contiguous ranges starting at a root; parents precede children
    std::vector<int64_t> off;
    int64_t start = 0;
    for (int64_t i = 0; i < n_nodes; ++i) {
        if (hp[i] < 0) {
            if (hp[i] != -1) return NMODL_ERR_ARG;
            start = i;
            off.push_back(i);
        } else if (i == 0 || hp[i] >= i || hp[i] < start) {
            return NMODL_ERR_ARG;
        }
        if (!(ha[i] >= 0.0) || !(hb[i] >= 0.0)) return NMODL_ERR_ARG;
    }
    off.push_back(n_nodes);
    nmodl_cable* cb = new (std::nothrow) nmodl_cable();
    if (!cb) return NMODL_ERR_OOM;
    cb->ctx = c;
    cb->n_nodes = n_nodes;
    cb->n_cells = (int64_t)off.size() - 1;
    cb->cell_off = off;
    cb->parent = hp;
    do {
        if ((e = dalloc(&cb->d_parent, n_nodes)) != cudaSuccess) break;
        if ((e = dalloc(&cb->d_ga, n_nodes)) != cudaSuccess) break;
        if ((e = dalloc(&cb->d_gb, n_nodes)) != cudaSuccess) break;
        if ((e = dalloc(&cb->d_cell_off, off.size())) != cudaSuccess) break;
        if ((e = dalloc(&cb->d_d2, n_nodes)) != cudaSuccess) break;
        if ((e = dalloc(&cb->d_r2, n_nodes)) != cudaSuccess) break;
        cudaMemcpyAsync(cb->d_parent, hp.data(), n_nodes * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(cb->d_ga, ha.data(), n_nodes * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(cb->d_gb, hb.data(), n_nodes * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(cb->d_cell_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
        e = cudaStreamSynchronize(c->stream);
    } while (false);
    if (e != cudaSuccess) {
        void* ptrs[] = {cb->d_parent, cb->d_ga, cb->d_gb, cb->d_cell_off, cb->d_d2, cb->d_r2};
        for (void* q : ptrs) cudaFree(q);
        delete cb;
        return nmodl_cuda_status(e);
    }
    *out = cb;
    return NMODL_OK;
}

NMODL_API void nmodl_cable_destroy(nmodl_cable* cb) {
    if (!cb) return;
    DeviceGuard dg(cb->ctx->device);
    cudaStreamSynchronize(cb->ctx->stream);
    auto& P = cb->ctx->plans;  // fused cable plans of this cable
    P.erase(std::remove_if(P.begin(), P.end(),
                           [cb](const std::unique_ptr<Plan>& p) { return p->cable == cb; }),
            P.end());
    for (auto& g : cb->graphs) cudaGraphExecDestroy(g.exec);
    void* ptrs[] = {cb->d_parent, cb->d_ga, cb->d_gb, cb->d_cell_off, cb->d_d2, cb->d_r2};
    for (void* q : ptrs) cudaFree(q);
    delete cb;
}

NMODL_API int nmodl_cable_n_cells(const nmodl_cable* cb) {
    return cb ? (int)cb->n_cells : NMODL_ERR_ARG;
}

}  // extern "C"

static cudaError_t enqueue_cable_steps(nmodl_ctx* c, nmodl_cable* cb, nmodl_mech* const* mechs,
                                       int n_mechs, double dt, double cm, double* v,
                                       double* rhs, double* d, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        cudaMemsetAsync(rhs, 0, cb->n_nodes * sizeof(double), c->stream);
        cudaMemsetAsync(d, 0, cb->n_nodes * sizeof(double), c->stream);
        nmodl_zero_ions(c, cb->n_nodes);
        for (int i = 0; i < n_mechs; ++i) nmodl_enqueue_cur(mechs[i], v, rhs, d);
        launch_cable_solve(cb->n_cells, cb->d_cell_off, cb->d_parent, cb->d_ga, cb->d_gb,
                           1e-3 * cm / dt, v, rhs, d, cb->d_d2, cb->d_r2, c->opt.clamp_v,
                           c->d_err, c->stream);
        for (int i = 0; i < n_mechs; ++i) nmodl_enqueue_state(mechs[i], dt, v);
    }
    return cudaGetLastError();
}

extern "C" NMODL_API int nmodl_step_cable(nmodl_ctx* c, nmodl_cable* cb,
                                          nmodl_mech* const* mechs, int n_mechs, double dt,
                                          double cm, double* v, double* rhs, double* d,
                                          int nsteps) {
    if (!c || !cb || cb->ctx != c || !mechs || n_mechs < 1 || nsteps < 0 || !(dt > 0.0) ||
        !(cm > 0.0))
        return NMODL_ERR_ARG;
    for (int i = 0; i < n_mechs; ++i)
        if (!mechs[i] || mechs[i]->ctx != c || mechs[i]->n_nodes != cb->n_nodes)
            return NMODL_ERR_ARG;
    if (nsteps == 0) return NMODL_OK;
    if (!v || !rhs || !d) return NMODL_ERR_ARG;
    if (c->has_ions() && c->ion_nodes != cb->n_nodes) return NMODL_ERR_ARG;
    if (nmodl_check_ion_reads(c, mechs, n_mechs)) return NMODL_ERR_ARG;
    DeviceGuard dg(c->device);
    // fused form: tiles of whole cells, the tree solve inside the tile kernel
    int rc = NMODL_OK;
    Plan* p = nmodl_get_plan(c, mechs, n_mechs, v, &rc, cb);
    if (!p) return rc;
    for (int i = 0; i < n_mechs; ++i) nmodl_count_states(mechs[i], nsteps);
    if (p->fused) {
        const int W = c->opt.window;
        for (int s0 = 0; s0 < nsteps; s0 += W) {
            cudaError_t e = nmodl_run_window(c, p, mechs, n_mechs, dt, cm, v, rhs, d,
                                             std::min(W, nsteps - s0));
            if (e != cudaSuccess) return nmodl_cuda_status(e);
        }
        return NMODL_OK;
    }
    std::vector<nmodl_mech*> list(mechs, mechs + n_mechs);
    if (list != cb->graph_mechs || cb->graph_epoch != c->epoch) {  // stale graphs
        for (auto& g : cb->graphs) cudaGraphExecDestroy(g.exec);
        cb->graphs.clear();
        cb->graph_mechs = list;
        cb->graph_epoch = c->epoch;
    }
    const int W = c->opt.window;
    for (int s0 = 0; s0 < nsteps; s0 += W) {
        const int w = std::min(W, nsteps - s0);
        cudaError_t e;
        if (!c->opt.use_graph || c->stream == nullptr) {
            e = enqueue_cable_steps(c, cb, mechs, n_mechs, dt, cm, v, rhs, d, w);
        } else {
            cudaGraphExec_t exec = nullptr;
            for (auto& ge : cb->graphs)
                if (ge.v == v && ge.rhs == rhs && ge.d == d && ge.dt == dt && ge.cm == cm &&
                    ge.nsteps == w)
                    exec = ge.exec;
            if (!exec) {
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) return nmodl_cuda_status(e);
                cudaError_t le = enqueue_cable_steps(c, cb, mechs, n_mechs, dt, cm, v, rhs, d, w);
                e = cudaStreamEndCapture(c->stream, &graph);
                if (le != cudaSuccess || e != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    return nmodl_cuda_status(le != cudaSuccess ? le : e);
                }
                e = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) return nmodl_cuda_status(e);
                cb->graphs.push_back(GraphEntry{v, rhs, d, dt, cm, w, 0, exec});
            }
            e = cudaGraphLaunch(exec, c->stream);
        }
        if (e != cudaSuccess) return nmodl_cuda_status(e);
    }
    return NMODL_OK;
}
