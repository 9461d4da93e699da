// api.cu -- C ABI of libnmodl_b300.so: contexts, mechanisms, validation,
// the fused-step tile planner / autotuner and CUDA-graph windows.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "runtime.cuh"

using namespace nmodl;

namespace nmodl {
// api_surrogate.cu: surrogate state update of a NMODL_KIN9 mechanism
cudaError_t enqueue_surrogate_state(nmodl_mech* m, double dt, const double* v);
cudaError_t enqueue_surrogate_network_step(nmodl_mech* m, double dt, double cm, double* v,
                                           double* rhs, double* d, int clamp);
}  // namespace nmodl

// Drop the cached step plans (and their graphs) that involve mechanism m
// (all of them for m == nullptr).
void nmodl_invalidate_plans(nmodl_ctx* c, nmodl_mech* m) {
    c->epoch++;
    auto& P = c->plans;
    P.erase(std::remove_if(P.begin(), P.end(),
                           [m](const std::unique_ptr<Plan>& p) {
                               return !m || std::find(p->mechs.begin(), p->mechs.end(), m) !=
                                                p->mechs.end();
                           }),
            P.end());
}

int nmodl_cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return NMODL_OK;
    if (e == cudaErrorMemoryAllocation) return NMODL_ERR_OOM;
    return NMODL_ERR_CUDA;
}

namespace {
int cuda_status(cudaError_t e) { return nmodl_cuda_status(e); }
}  // namespace

// ------------------------------------------------------------ parameters

static bool is_int(double x, double lo, double hi) {
    return std::isfinite(x) && x == std::floor(x) && x >= lo && x <= hi;
}

static GateD make_gate(int af, double aA, double avh, double ak, int bf, double bA,
                       double bvh, double bk, int power) {
    GateD g{};
    g.aform = af; g.aA = aA; g.avh = avh; g.ark = 1.0 / ak;
    g.bform = bf; g.bA = bA; g.bvh = bvh; g.brk = 1.0 / bk;
    g.power = power;
    return g;
}

static int build_desc(nmodl_mech* m) {
    const std::vector<double>& p = m->params;
    for (double x : p)
        if (!std::isfinite(x)) return NMODL_ERR_ARG;
    if (m->type == NMODL_HH) {
        if (p.size() != NMODL_HH_NPARAM) return NMODL_ERR_ARG;
        MechD& d = m->md;
        d = MechD{};
        d.kind = NMODL_HH;
        d.n_gates = 3;
        d.phi = std::pow(3.0, (p[6] - 6.3) / 10.0);
        d.hh_g[0] = p[0]; d.hh_g[1] = p[1]; d.hh_g[2] = p[2];
        d.hh_e[0] = p[3]; d.hh_e[1] = p[4]; d.hh_e[2] = p[5];
        // HH rates rewritten in the shapes of u = (v - vh)/k:
        // alpha_m = 0.1 vtrap(-(v+40),10) = 1.0 u/(1-exp(-u)), u=(v+40)/10
        d.gate[0] = make_gate(kLinoid, 1.0, -40.0, 10.0, kExp, 4.0, -65.0, -18.0, 3);
        d.gate[1] = make_gate(kExp, 0.07, -65.0, -20.0, kSigmoid, 1.0, -35.0, 10.0, 1);
        d.gate[2] = make_gate(kLinoid, 0.1, -55.0, 10.0, kExp, 0.125, -65.0, -80.0, 4);
        m->n_states = 3;
        return NMODL_OK;
    }
    if (m->type == NMODL_CNEXP) {
        if (p.size() != NMODL_CNEXP_NPARAM) return NMODL_ERR_ARG;
        if (!is_int(p[0], 0, kMaxGates) || !(p[3] > 0.0)) return NMODL_ERR_ARG;
        MechD& d = m->md;
        d = MechD{};
        d.kind = NMODL_CNEXP;
        d.n_gates = (int)p[0];
        d.gbar = p[1];
        d.e = p[2];
        d.phi = std::pow(p[3], (p[4] - p[5]) / 10.0);
        for (int g = 0; g < d.n_gates; ++g) {
            const double* q = &p[6 + 9 * g];
            if (!is_int(q[0], 0, 8) || !is_int(q[1], 0, 2) || !is_int(q[5], 0, 2))
                return NMODL_ERR_ARG;
            if (q[4] == 0.0 || q[8] == 0.0) return NMODL_ERR_ARG;
            d.gate[g] = make_gate((int)q[1], q[2], q[3], q[4], (int)q[5], q[6], q[7],
                                  q[8], (int)q[0]);
        }
        m->n_states = d.n_gates;
        return NMODL_OK;
    }
    if (m->type == NMODL_KIN3) {
        if (p.size() != NMODL_KIN3_NPARAM) return NMODL_ERR_ARG;
        if (!is_int(p[2], 0, 2)) return NMODL_ERR_ARG;
        Kin3D& k = m->k3;
        k = Kin3D{};
        k.gbar = p[0];
        k.e = p[1];
        k.open = (int)p[2];
        for (int e = 0; e < 3; ++e) {
            k.af[e] = p[3 + 4 * e];
            k.bf[e] = p[4 + 4 * e];
            k.ab[e] = p[5 + 4 * e];
            k.bb[e] = p[6 + 4 * e];
            if (k.af[e] < 0.0 || k.ab[e] < 0.0) return NMODL_ERR_ARG;
        }
        m->n_states = 3;
        m->md = MechD{};
        m->md.kind = NMODL_KIN3;
        m->md.n_gates = 3;
        m->md.k3 = k;
        return NMODL_OK;
    }
    if (m->type == NMODL_CACUM) {
        if (p.size() != NMODL_CACUM_NPARAM) return NMODL_ERR_ARG;
        for (double x : p)
            if (x < 0.0) return NMODL_ERR_ARG;
        if (!(p[1] > 0.0) || !(p[3] * p[2] + p[4] > 0.0)) return NMODL_ERR_ARG;
        CacumD& c = m->cd;
        c.k = p[0];
        c.rtau = 1.0 / p[1];
        c.cai0 = p[2];
        c.kf = p[3];
        c.kb = p[4];
        c.btot = p[5];
        m->n_states = 2;
        m->md = MechD{};
        m->md.kind = NMODL_CACUM;
        m->md.n_gates = 2;
        m->md.cd = c;
        return NMODL_OK;
    }
    if (m->type == NMODL_KIN9) {
        if (p.size() != NMODL_KIN9_NPARAM) return NMODL_ERR_ARG;
        if (!is_int(p[2], 0, 8)) return NMODL_ERR_ARG;
        Kin9D& k = m->kd;
        k = Kin9D{};
        k.gbar = p[0];
        k.e = p[1];
        k.open = (int)p[2];
        for (int e = 0; e < kKinEdges; ++e) {
            k.af[e] = p[3 + 4 * e];
            k.bf[e] = p[4 + 4 * e];
            k.ab[e] = p[5 + 4 * e];
            k.bb[e] = p[6 + 4 * e];
            if (k.af[e] < 0.0 || k.ab[e] < 0.0) return NMODL_ERR_ARG;
        }
        m->n_states = kKinStates;
        // the fused kernel's view: kind, state count and the current
        m->md = MechD{};
        m->md.kind = NMODL_KIN9;
        m->md.n_gates = kKinStates;
        m->md.gbar = k.gbar;
        m->md.e = k.e;
        m->md.open = k.open;
        m->md.ion = m->ion;
        return NMODL_OK;
    }
    return NMODL_ERR_ARG;
}

namespace nmodl {
// Parameter block -> device descriptor, for entry points without a
// nmodl_mech object.
int build_desc_for(int type, const double* params, int64_t n_params, MechD* md,
                   Kin9D* kd, int* n_states) {
    if (n_params < 0 || n_params > 64 || (n_params > 0 && !params)) return NMODL_ERR_ARG;
    // one scratch object per host thread; its parameter buffer is reserved
    // on the thread's first call, so later calls allocate nothing
    thread_local nmodl_mech tmp;
    if (tmp.params.capacity() < 64) tmp.params.reserve(64);
    tmp.type = type;
    tmp.params.assign(params, params + n_params);
    const int rc = build_desc(&tmp);
    if (rc) return rc;
    *md = tmp.md;
    *kd = tmp.kd;
    *n_states = tmp.n_states;
    return NMODL_OK;
}
}  // namespace nmodl

// ---------------------------------------------------------------- ABI

extern "C" {

int nmodl_version(void) { return 100; }

const char* nmodl_strerror(int s) {
    switch (s) {
    case NMODL_OK: return "ok";
    case NMODL_ERR_ARG: return "invalid argument or parameter block";
    case NMODL_ERR_UNSORTED: return "node_index is not non-decreasing";
    case NMODL_ERR_OOM: return "device allocation failed";
    case NMODL_ERR_CUDA: return "CUDA runtime error";
    case NMODL_ERR_NONFINITE: return "non-finite value in results";
    case NMODL_ERR_NOCONV: return "Newton iteration did not converge";
    case NMODL_ERR_TIMEOUT: return "bounded device wait ran out";
    case NMODL_ERR_RANGE: return "node_index outside [0, n_nodes)";
    case NMODL_ERR_UNSUPPORTED: return "unsupported combination";
    case NMODL_ERR_TOO_LARGE: return "size exceeds the fixed scratch capacity";
    default: return "unknown status";
    }
}

int nmodl_options_default(nmodl_options* o) {
    if (!o) return NMODL_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->precision = NMODL_FP64;
    o->newton_max_iter = 8;
    o->newton_tol = 1e-14;
    o->ir_max = 4;
    o->window = 40;
    o->use_graph = 1;
    o->autotune = 1;
    o->clamp_v = 0;
    return NMODL_OK;
}

static int check_options(const nmodl_options* o) {
    if (o->precision != NMODL_FP64 && o->precision != NMODL_MIXED) return NMODL_ERR_ARG;
    if (o->newton_max_iter < 1 || o->newton_max_iter > 64) return NMODL_ERR_ARG;
    if (!(o->newton_tol >= 0.0)) return NMODL_ERR_ARG;
    if (o->ir_max < 0 || o->ir_max > 64) return NMODL_ERR_ARG;
    if (o->window < 1) return NMODL_ERR_ARG;
    if (o->cnexp_pade != 0 && o->cnexp_pade != 1) return NMODL_ERR_ARG;
    if (o->no_fuse != 0 && o->no_fuse != 1) return NMODL_ERR_ARG;
    if (o->tile_smem < 0 || o->block < 0 || o->block > kFusedMaxBlock || (o->block % 32))
        return NMODL_ERR_ARG;
    return NMODL_OK;
}

int nmodl_ctx_create(int device, void* cuda_stream, const nmodl_options* opt,
                     nmodl_ctx** out) {
    if (!out) return NMODL_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return NMODL_ERR_CUDA;
    nmodl_options o;
    nmodl_options_default(&o);
    if (opt) o = *opt;
    int rc = check_options(&o);
    if (rc) return rc;
    DeviceGuard g(device);
    nmodl_ctx* c = new (std::nothrow) nmodl_ctx();
    if (!c) return NMODL_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->opt = o;
    if (dalloc(&c->d_err, 1) != cudaSuccess) {
        delete c;
        return NMODL_ERR_OOM;
    }
    cudaMemset(c->d_err, 0, sizeof(int32_t));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(c->d_err);
        delete c;
        return NMODL_ERR_CUDA;
    }
    *out = c;
    return NMODL_OK;
}

int nmodl_ctx_set_options(nmodl_ctx* c, const nmodl_options* opt) {
    if (!c || !opt) return NMODL_ERR_ARG;
    int rc = check_options(opt);
    if (rc) return rc;
    c->opt = *opt;
    c->plans.clear();  // plans depend on precision / tile options
    c->epoch++;
    return NMODL_OK;
}

int nmodl_sync(nmodl_ctx* c) {
    if (!c) return NMODL_ERR_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return NMODL_ERR_CUDA;
    int32_t h = 0;
    e = cudaMemcpy(&h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return NMODL_ERR_CUDA;
    if (h) cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream);
    return h;
}

void nmodl_ctx_destroy(nmodl_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    c->plans.clear();
    cudaFree(c->d_err);
    delete c;
}

static void free_mech(nmodl_mech* m) {
    cudaFree(m->d_fb_list);
    cudaFree(m->d_fb_count);
    cudaFree(m->d_ni);
    cudaFree(m->d_states);
    cudaFree(m->d_chunk);
    cudaFree(m->d_md);
    cudaFree(m->d_kd);
    cudaFree(m->d_cnt);
    cudaFree(m->d_k3);
    cudaFree(m->d_cd);
    delete m;
}

int nmodl_mech_create(nmodl_ctx* c, int type, int64_t n, const int32_t* node_index,
                      int64_t n_nodes, const double* params, int64_t n_params,
                      nmodl_mech** out) {
    if (!out) return NMODL_ERR_ARG;
    *out = nullptr;
    if (!c || n < 0 || n_nodes < 0 || n_params < 0 || (n > 0 && !node_index) ||
        (n_params > 0 && !params))
        return NMODL_ERR_ARG;
    if (n > INT32_MAX - 64 || n_nodes > INT32_MAX) return NMODL_ERR_ARG;
    DeviceGuard g(c->device);
    nmodl_mech* m = new (std::nothrow) nmodl_mech();
    if (!m) return NMODL_ERR_OOM;
    m->ctx = c;
    m->type = type;
    m->n = n;
    m->n_nodes = n_nodes;
    m->params.assign(params, params + n_params);
    int rc = build_desc(m);
    if (rc) {
        delete m;
        return rc;
    }
    m->stride = (n + 31) / 32 * 32;
    m->n_chunks = (n + 31) / 32;
    cudaError_t e = cudaSuccess;
    int32_t* d_flags = nullptr;
    do {
        if ((e = dalloc(&m->d_ni, (size_t)n)) != cudaSuccess) break;
        if ((e = dalloc(&m->d_states, (size_t)m->n_states * m->stride)) != cudaSuccess) break;
        if ((e = dalloc(&m->d_chunk, (size_t)m->n_chunks + 1)) != cudaSuccess) break;
        if ((e = dalloc(&m->d_md, 1)) != cudaSuccess) break;
        if ((e = dalloc(&m->d_kd, 1)) != cudaSuccess) break;
        if ((e = dalloc(&m->d_cnt, 1)) != cudaSuccess) break;
        if ((e = dalloc(&m->d_k3, 1)) != cudaSuccess) break;
        if ((e = dalloc(&m->d_cd, 1)) != cudaSuccess) break;
        if ((e = dalloc(&d_flags, 1)) != cudaSuccess) break;
        // every copy and fill below is ordered on the context stream, which
        // need not synchronise with the legacy default stream
        if (n > 0 && (e = cudaMemcpyAsync(m->d_ni, node_index, n * sizeof(int32_t),
                                          cudaMemcpyDefault, c->stream)) != cudaSuccess)
            break;
        if (m->n_states && m->stride &&
            (e = cudaMemsetAsync(m->d_states, 0, m->n_states * m->stride * sizeof(double), c->stream)) != cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(m->d_md, &m->md, sizeof(MechD), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(m->d_kd, &m->kd, sizeof(Kin9D), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(m->d_k3, &m->k3, sizeof(Kin3D), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(m->d_cd, &m->cd, sizeof(CacumD), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(m->d_cnt, 0, sizeof(KinCounters), c->stream)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(d_flags, 0, sizeof(int32_t), c->stream)) != cudaSuccess) break;
        launch_validate_index(m->d_ni, n, n_nodes, d_flags, c->stream);
        launch_chunk_starts(m->d_ni, n, m->n_chunks, m->d_chunk, c->stream);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) break;
        int32_t flags = 0;
        if ((e = cudaMemcpy(&flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
        cudaFree(d_flags);
        d_flags = nullptr;
        if (flags & 2) rc = NMODL_ERR_RANGE;
        else if (flags & 1) rc = NMODL_ERR_UNSORTED;
    } while (false);
    if (d_flags) cudaFree(d_flags);
    if (e != cudaSuccess) rc = cuda_status(e);
    if (rc) {
        free_mech(m);
        return rc;
    }
    c->live_mechs++;
    *out = m;
    return NMODL_OK;
}

void nmodl_mech_destroy(nmodl_mech* m) {
    if (!m) return;
    nmodl_ctx* c = m->ctx;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    nmodl_invalidate_plans(c, m);
    c->live_mechs--;
    free_mech(m);
}

int nmodl_mech_n_states(const nmodl_mech* m) { return m ? m->n_states : NMODL_ERR_ARG; }

int nmodl_init(nmodl_mech* m, const double* v) {
    if (!m || (m->n > 0 && !v)) return NMODL_ERR_ARG;
    nmodl_ctx* c = m->ctx;
    DeviceGuard g(c->device);
    if (m->type == NMODL_KIN9)
        launch_kin9_init(m->d_kd, m->n, m->d_ni, v, m->d_states, m->stride, c->d_err, c->stream);
    else if (m->type == NMODL_KIN3)
        launch_kin3_init(m->d_k3, m->n, m->d_ni, v, m->d_states, m->stride, c->d_err, c->stream);
    else if (m->type == NMODL_CACUM)
        launch_cacum_init(m->d_cd, m->n, m->d_states, m->stride, c->stream);
    else
        launch_init_gates(m->d_md, m->n_states, m->n, m->d_ni, v, m->d_states, m->stride,
                          c->d_err, c->stream);
    return cuda_status(cudaGetLastError());
}

void nmodl_enqueue_state(nmodl_mech* m, double dt, const double* v) {
    nmodl_ctx* c = m->ctx;
    const nmodl_options& o = c->opt;
    if (m->type == NMODL_KIN9 && m->sur) {
        nmodl::enqueue_surrogate_state(m, dt, v);
    } else if (m->type == NMODL_KIN9)
        launch_kin9_state(o.precision, m->d_kd, m->kd, m->n, m->d_ni, v, m->d_states, m->stride,
                          dt, nullptr, o.newton_tol, o.newton_max_iter, o.ir_max, nullptr, 0,
                          nullptr, m->d_cnt, c->d_err, c->stream);
    else if (m->type == NMODL_KIN3)
        launch_kin3_state(o.precision, m->d_k3, m->k3, m->n, m->d_ni, v, m->d_states, m->stride,
                          dt, o.newton_tol, o.ir_max, m->d_cnt, c->d_err, c->stream);
    else if (m->type == NMODL_CACUM)
        launch_cacum_state(o.precision, m->d_cd, m->cd, m->n, m->d_ni, c->ion[NMODL_ION_CA],
                           m->d_states, m->stride, dt, o.newton_tol, o.newton_max_iter, o.ir_max,
                           m->d_cnt, c->d_err, c->stream);
    else
        launch_state_gates(o.precision, m->d_md, m->n_states, m->n, m->d_ni, v,
                           m->d_states, m->stride, dt, o.cnexp_pade, c->d_err, c->stream);
}

// host-side counters of state updates (kept here, not at enqueue time, so
// that graph replays are counted)
void nmodl_count_states(nmodl_mech* m, int64_t k) {
    m->calls += k;
    if (m->type == NMODL_KIN9 && m->sur) m->sur_calls += k;
}

void nmodl_enqueue_cur(nmodl_mech* m, const double* v, double* rhs, double* d) {
    nmodl_ctx* c = m->ctx;
    if (m->type == NMODL_CACUM) return;  // no membrane current
    const void* desc = (m->type == NMODL_KIN9)   ? (const void*)m->d_kd
                       : (m->type == NMODL_KIN3) ? (const void*)m->d_k3
                                                 : (const void*)m->d_md;
    const int kind = (m->type == NMODL_KIN9 || m->type == NMODL_KIN3) ? m->type : NMODL_CNEXP;
    double* ion_a = nullptr;
    double* ion_b = nullptr;
    if (m->type == NMODL_HH) {
        ion_a = c->ion[NMODL_ION_NA];
        ion_b = c->ion[NMODL_ION_K];
    } else if (m->ion != NMODL_ION_NONE) {
        ion_a = c->ion[m->ion];
    }
    launch_cur_seg(kind, desc, m->n_chunks, m->d_chunk, m->d_ni, v, m->d_states, m->stride,
                   rhs, d, ion_a, ion_b, c->d_err, c->stream);
}

void nmodl_zero_ions(nmodl_ctx* c, int64_t n_nodes) {
    for (int q = 1; q < 4; ++q)
        if (c->ion[q] && n_nodes > 0)
            cudaMemsetAsync(c->ion[q], 0, n_nodes * sizeof(double), c->stream);
}

int nmodl_check_ion_reads(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs) {
    for (int i = 0; i < n_mechs; ++i)
        if (mechs[i]->type == NMODL_CACUM && mechs[i]->n > 0 &&
            (!c->ion[NMODL_ION_CA] || c->ion_nodes != mechs[i]->n_nodes))
            return NMODL_ERR_ARG;
    return NMODL_OK;
}

int nmodl_state(nmodl_mech* m, double dt, const double* v) {
    if (!m || !(dt > 0.0) || !std::isfinite(dt) || (m->n > 0 && !v)) return NMODL_ERR_ARG;
    if (nmodl_check_ion_reads(m->ctx, &m, 1)) return NMODL_ERR_ARG;
    DeviceGuard g(m->ctx->device);
    nmodl_enqueue_state(m, dt, v);
    nmodl_count_states(m, 1);
    return cuda_status(cudaGetLastError());
}

int nmodl_cur(nmodl_mech* m, const double* v, double* rhs, double* d) {
    if (!m || (m->n > 0 && (!v || !rhs || !d))) return NMODL_ERR_ARG;
    if (m->ctx->has_ions() && m->ctx->ion_nodes != m->n_nodes) return NMODL_ERR_ARG;
    DeviceGuard g(m->ctx->device);
    nmodl_enqueue_cur(m, v, rhs, d);
    return cuda_status(cudaGetLastError());
}

// -------------------------------------------------------------- planning

// Shared memory of one tile, matching the layout in k_fused_tiles (tables:
// per-type segment tables, the cable form, which computes conductances in
// its owner loop; otherwise flat node-major slots of 16 bytes, slots[t] per
// instance).
static size_t tile_smem_bytes(int prec, int T, const int* gates, const int* slots, int64_t NT,
                              const int64_t* cnt, bool cable, bool ions, bool tables, bool ext) {
    size_t b = 8 * (size_t)NT;
    size_t inst = 0, items = 0, nslot = 0;
    for (int t = 0; t < T; ++t) {
        inst += cnt[t];
        items += (size_t)gates[t] * cnt[t];
        nslot += (size_t)slots[t] * cnt[t];
    }
    b += 8 * items + 2 * inst;
    b += tables ? 2 * (size_t)T * (NT + 1) : 2 * inst + 2 * (size_t)(NT + 1) + 2 * (size_t)NT;
    if (!tables && ions) b += nslot;  // the ion of each slot
    if (prec == NMODL_MIXED) b = (b + 15) / 16 * 16 + 4 * (size_t)NT;
    if (ions) b = (b + 15) / 16 * 16 + 8 * (size_t)NT;  // the step's ica per node
    // d, rhs, ga, gb, parent, and the level schedule (at most 6 NT + 5 uint16)
    if (cable) b = (b + 15) / 16 * 16 + 34 * (size_t)NT + 2 * (6 * (size_t)NT + 5);
    // the node-major slots of the step: (e, g) doubles; MIXED without the
    // small systems: three FP32 conductance factors and the current's id
    if (!tables) b = (b + 15) / 16 * 16 + 16 * nslot;
    return (b + 15) / 16 * 16;
}

// Greedy tiling: fine blocks (node ranges [bounds[k], bounds[k+1]): groups
// of 32 nodes, or whole cells in the cable form) are merged while the
// tile's shared memory stays within budget; returns false if one fine block
// does not fit.
static bool make_tiles(int prec, const std::vector<std::vector<int32_t>>& off, int T,
                       const int* gates, const int* slots,
                       const std::vector<int64_t>& bounds, bool cable, bool ions, bool ext,
                       size_t budget,
                       std::vector<int32_t>& recs, size_t& max_smem) {
    const bool tables = cable;
    recs.clear();
    max_smem = 0;
    const int64_t K = (int64_t)off[0].size() - 1;  // fine blocks
    int64_t k0 = 0;
    std::vector<int64_t> cnt(T);
    while (k0 < K) {
        int64_t k1 = k0 + 1;
        auto fits = [&](int64_t a, int64_t b) -> bool {
            const int64_t NT = bounds[b] - bounds[a];
            if (NT > 65535) return false;
            int64_t nslot = 0;
            for (int t = 0; t < T; ++t) {
                cnt[t] = off[t][b] - off[t][a];
                nslot += slots[t] * cnt[t];
                if (cnt[t] > 65535) return false;
            }
            if (!tables && nslot > 65535) return false;  // uint16 node-major slots
            return tile_smem_bytes(prec, T, gates, slots, NT, cnt.data(), cable, ions, tables, ext) <=
                   budget;
        };
        if (!fits(k0, k1)) return false;
        while (k1 < K && fits(k0, k1 + 1)) ++k1;
        const int64_t n0 = bounds[k0], n1 = bounds[k1];
        recs.push_back((int32_t)n0);
        recs.push_back((int32_t)n1);
        for (int t = 0; t < T; ++t) {
            recs.push_back(off[t][k0]);
            recs.push_back(off[t][k1]);
            cnt[t] = off[t][k1] - off[t][k0];
        }
        max_smem = std::max(max_smem,
                            tile_smem_bytes(prec, T, gates, slots, n1 - n0, cnt.data(), cable,
                                            ions, tables, ext));
        k0 = k1;
    }
    return true;
}

// Largest-first order of tile records (cost = gate items + instances), the
// work list of the fused kernel.
static void lpt_order(std::vector<int32_t>& recs, int T, const int* gates, int stride) {
    const size_t n = recs.size() / stride;
    std::vector<std::pair<int64_t, size_t>> cost(n);
    for (size_t k = 0; k < n; ++k) {
        int64_t c = 0;
        for (int t = 0; t < T; ++t)
            c += (int64_t)(gates[t] + 1) * (recs[k * stride + 3 + 2 * t] - recs[k * stride + 2 + 2 * t]);
        cost[k] = {-c, k};
    }
    std::stable_sort(cost.begin(), cost.end());
    std::vector<int32_t> out(recs.size());
    for (size_t k = 0; k < n; ++k)
        std::copy(recs.begin() + cost[k].second * stride,
                  recs.begin() + (cost[k].second + 1) * stride, out.begin() + k * stride);
    recs.swap(out);
}

// Level schedule of the tree solve of one tile (local node ids, uint16):
// [H, D, EL[H+1], SL[D+1], E[NT], S[NT], coff[NT+1], clist[...]] with E the
// nodes by height above the leaves (a node's children all have lower
// height), EL its level offsets, S the nodes by depth below the root, SL
// its offsets, and the children of node i at clist[coff[i] .. coff[i+1])
// in increasing order.  Nodes of one level are independent.
static void cable_sched(const nmodl_cable* cb, int64_t n0, int64_t n1,
                        std::vector<uint16_t>& out) {
    const int NT = (int)(n1 - n0);
    std::vector<int> par(NT), h(NT, 0), dep(NT, 0), nch(NT, 0);
    int roots = 0;
    for (int i = 0; i < NT; ++i) {
        const int32_t p = cb->parent[n0 + i];
        par[i] = p < 0 ? -1 : (int)(p - n0);
        roots += p < 0;
    }
    for (int i = NT - 1; i >= 0; --i)
        if (par[i] >= 0) {
            h[par[i]] = std::max(h[par[i]], h[i] + 1);
            nch[par[i]]++;
        }
    int H = 0, D = 0;
    for (int i = 0; i < NT; ++i) {
        dep[i] = par[i] < 0 ? 0 : dep[par[i]] + 1;
        H = std::max(H, h[i] + 1);
        D = std::max(D, dep[i] + 1);
    }
    std::vector<int> EL(H + 1, 0), SL(D + 1, 0);
    for (int i = 0; i < NT; ++i) {
        EL[h[i] + 1]++;
        SL[dep[i] + 1]++;
    }
    for (int k = 0; k < H; ++k) EL[k + 1] += EL[k];
    for (int k = 0; k < D; ++k) SL[k + 1] += SL[k];
    std::vector<int> E(NT), S(NT), pe(EL.begin(), EL.end() - 1), ps(SL.begin(), SL.end() - 1);
    for (int i = 0; i < NT; ++i) {
        E[pe[h[i]]++] = i;
        S[ps[dep[i]]++] = i;
    }
    std::vector<int> coff(NT + 1, 0);
    for (int i = 0; i < NT; ++i) coff[i + 1] = coff[i] + nch[i];
    std::vector<int> clist(NT - roots), pc(coff.begin(), coff.end() - 1);
    for (int i = 0; i < NT; ++i)
        if (par[i] >= 0) clist[pc[par[i]]++] = i;
    out.clear();
    out.push_back((uint16_t)H);
    out.push_back((uint16_t)D);
    for (int x : EL) out.push_back((uint16_t)x);
    for (int x : SL) out.push_back((uint16_t)x);
    for (int x : E) out.push_back((uint16_t)x);
    for (int x : S) out.push_back((uint16_t)x);
    for (int x : coff) out.push_back((uint16_t)x);
    for (int x : clist) out.push_back((uint16_t)x);
}

// Append (schedule offset, length) to every tile record of a cable plan and
// the schedules to `sched`.
static void add_cable_sched(const nmodl_cable* cb, int T, std::vector<int32_t>& recs,
                            std::vector<uint16_t>& sched) {
    const int in = 2 + 2 * T, outs = in + 2;
    const size_t n = recs.size() / in;
    std::vector<int32_t> r2(n * outs);
    std::vector<uint16_t> one;
    sched.clear();
    for (size_t k = 0; k < n; ++k) {
        std::copy(recs.begin() + k * in, recs.begin() + (k + 1) * in, r2.begin() + k * outs);
        cable_sched(cb, recs[k * in], recs[k * in + 1], one);
        r2[k * outs + in] = (int32_t)sched.size();
        r2[k * outs + in + 1] = (int32_t)one.size();
        sched.insert(sched.end(), one.begin(), one.end());
    }
    recs.swap(r2);
}

// The plan's device descriptors (once): MechD of every mechanism, and the
// Kin9D rate constants of the 9-state ones (zero for the others).
static cudaError_t upload_descriptors(nmodl_ctx* c, Plan* p, nmodl_mech* const* mechs, int T) {
    if (p->d_md) return cudaSuccess;
    cudaError_t e = dalloc(&p->d_md, T);
    if (e == cudaSuccess) e = dalloc(&p->d_k9, T);
    if (e != cudaSuccess) return e;
    std::vector<MechD> mds(T);
    std::vector<Kin9D> k9s(T, Kin9D{});
    for (int t = 0; t < T; ++t) {
        mds[t] = mechs[t]->md;
        if (mechs[t]->type == NMODL_KIN9) k9s[t] = mechs[t]->kd;
    }
    e = cudaMemcpyAsync(p->d_md, mds.data(), T * sizeof(MechD), cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_k9, k9s.data(), T * sizeof(Kin9D), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

static cudaError_t enqueue_generic_steps(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs,
                                         double dt, double cm, double* v, double* rhs,
                                         double* d, int nsteps, int64_t n_nodes);

struct Candidate {
    size_t budget;
    int block;
    bool persistent;
    std::vector<int32_t> recs;
    size_t smem;
    double ms = 0.0;
    std::shared_ptr<std::vector<uint16_t>> sched;  // cable level schedules
};

// The gate-warp form of k_hh.cu: one HH mechanism with one instance on
// each node (node_index = 0, 1, ..., n - 1), FP64, isolated compartments,
// no ion arrays, the exponential cnexp factor, and at most 32 nodes per SM
// (a network too small for the tile kernel to fill the GPU).  Returns the
// nodes per block, 0 where the form does not apply.
// Instance i of m sits on node i for every i (node_index = 0, 1, ...,
// n_nodes - 1).  Reads node_index back once, at plan time.
static bool identity_nodes(nmodl_ctx* c, const nmodl_mech* m) {
    if (m->n != m->n_nodes || m->n == 0) return false;
    std::vector<int32_t> ni((size_t)m->n);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(ni.data(), m->d_ni, ni.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return false;
    for (int64_t i = 0; i < m->n; ++i)
        if (ni[(size_t)i] != i) return false;
    return true;
}

static int hh_warps_shape(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs,
                          nmodl_cable* cb) {
    if (n_mechs != 1 || cb || c->opt.no_fuse || c->opt.precision != NMODL_FP64 ||
        c->opt.cnexp_pade || c->has_ions())
        return 0;
    const nmodl_mech* m = mechs[0];
    if (m->type != NMODL_HH) return 0;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        sms <= 0 || m->n > 32 * (int64_t)sms || !identity_nodes(c, m))
        return 0;
    return hh_warps_per_block(m->n, sms);
}

// One NMODL_KIN9 mechanism with an attached surrogate, instance i on node i,
// isolated compartments, no ion arrays: the surrogate kernel forms each
// node's current, rhs and d and its v update itself before the state update
// (one kernel and the fallback per step instead of the zeroing, current and
// v-update launches in front of them).
static bool sur_step_fits(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs,
                          nmodl_cable* cb) {
    if (n_mechs != 1 || cb || c->opt.no_fuse || c->has_ions()) return false;
    const nmodl_mech* m = mechs[0];
    return m->type == NMODL_KIN9 && m->sur && identity_nodes(c, m);
}

static int build_plan(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs, Plan* p,
                      const double* v_user, nmodl_cable* cb) {
    p->mechs.assign(mechs, mechs + n_mechs);
    p->cable = cb;
    p->precision = c->opt.precision;
    p->n_nodes = mechs[0]->n_nodes;
    // the fused tile kernel covers HH, CNEXP, the small systems (KIN3,
    // CACUM) and the 9-state scheme (without an attached surrogate, whose
    // inference runs on the tensor cores), with or without ion arrays, as
    // long as the tile's per-state bookkeeping fits
    bool cnexp = n_mechs <= kMaxMechsFused && !c->opt.no_fuse;
    int state_rows = 0;
    for (int i = 0; i < n_mechs; ++i) {
        const int ty = mechs[i]->type;
        if (ty != NMODL_HH && ty != NMODL_CNEXP && ty != NMODL_KIN3 && ty != NMODL_CACUM &&
            !(ty == NMODL_KIN9 && !mechs[i]->sur))
            cnexp = false;
        state_rows += mechs[i]->n_states;
    }
    if (state_rows > kMaxMechsFused * kMaxGates) cnexp = false;
    // A list of 9-state schemes alone gains nothing from the tile kernel in
    // MIXED (measured on 1M instances: 0.9x the standalone Newton kernel,
    // whose smaller FP32 factorisation keeps more blocks per SM; FP64 1.09x):
    // it keeps the per-mechanism launches there.
    bool only_kin9 = true;
    for (int i = 0; i < n_mechs; ++i) only_kin9 = only_kin9 && mechs[i]->type == NMODL_KIN9;
    if (only_kin9 && c->opt.precision == NMODL_MIXED) cnexp = false;
    const bool ions = c->has_ions();
    bool ext = ions;  // the kernel variant with the small systems and ion sums
    bool kin = false;  // ... and the 9-state scheme
    for (int i = 0; i < n_mechs; ++i) {
        if (mechs[i]->type == NMODL_KIN3 || mechs[i]->type == NMODL_CACUM) ext = true;
        if (mechs[i]->type == NMODL_KIN9) ext = kin = true;
    }
    p->variant = p->precision + (ext ? 2 : 0) + (kin ? 2 : 0);
    p->fused = false;
    const bool dbg = std::getenv("NMODL_PLAN_DEBUG") != nullptr;
    if ((p->sur_step = sur_step_fits(c, mechs, n_mechs, cb))) {
        p->fused = true;
        if (dbg) std::fprintf(stderr, "[nmodl plan] surrogate network step\n");
        return NMODL_OK;
    }
    if ((p->hh_per_block = hh_warps_shape(c, mechs, n_mechs, cb)) > 0) {
        p->fused = true;
        if (dbg) std::fprintf(stderr, "[nmodl plan] HH gate warps, %d nodes per block\n",
                              p->hh_per_block);
        return NMODL_OK;
    }
    if (!cnexp || p->n_nodes == 0) {
        if (dbg) std::fprintf(stderr, "[nmodl plan] not fusable\n");
        return NMODL_OK;
    }

    const int T = n_mechs;
    std::vector<int64_t> bounds;
    if (cb) {
        bounds = cb->cell_off;  // whole cells
    } else {
        const int G = 32;
        for (int64_t k = 0; k * G < p->n_nodes; ++k) bounds.push_back(k * G);
        bounds.push_back(p->n_nodes);
    }
    const int64_t K = (int64_t)bounds.size() - 1;
    int64_t* d_bounds = nullptr;
    int32_t* d_off = nullptr;
    cudaError_t e;
    if ((e = dalloc(&d_bounds, K + 1)) != cudaSuccess) return cuda_status(e);
    if ((e = dalloc(&d_off, (size_t)T * (K + 1))) != cudaSuccess) {
        cudaFree(d_bounds);
        return cuda_status(e);
    }
    cudaMemcpyAsync(d_bounds, bounds.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                    c->stream);
    for (int t = 0; t < T; ++t)
        launch_tile_bounds(mechs[t]->d_ni, mechs[t]->n, d_bounds, K + 1, d_off + t * (K + 1),
                           c->stream);
    std::vector<int32_t> hoff((size_t)T * (K + 1));
    e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(hoff.data(), d_off, hoff.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d_bounds);
    cudaFree(d_off);
    if (e != cudaSuccess) return cuda_status(e);
    std::vector<std::vector<int32_t>> off(T);
    for (int t = 0; t < T; ++t)
        off[t].assign(hoff.begin() + t * (K + 1), hoff.begin() + (t + 1) * (K + 1));
    int gates[kMaxMechsFused], slots[kMaxMechsFused];
    for (int t = 0; t < T; ++t) {
        gates[t] = mechs[t]->n_states;
        slots[t] = flat_slots(mechs[t]->type);
    }

    int dev_smem_optin = 0;
    cudaDeviceGetAttribute(&dev_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    const size_t stat = fused_static_smem(p->variant);
    const size_t cap = dev_smem_optin > (int)stat ? dev_smem_optin - stat : 0;
    e = fused_prepare(p->variant, cap);
    if (e != cudaSuccess) return cuda_status(e);
    p->tile_stride = 2 + 2 * T + (cb ? 2 : 0);
    const int stride = p->tile_stride;

    // ---- candidate shapes
    std::vector<size_t> budgets;
    std::vector<int> blocks;
    std::vector<bool> pers;
    const bool tune = c->opt.autotune != 0;
    if (c->opt.tile_smem > 0) budgets = {std::min<size_t>(c->opt.tile_smem, cap)};
    else if (tune) {
        budgets = {16 * 1024, 24 * 1024, 32 * 1024, 48 * 1024, 64 * 1024, 96 * 1024, 150 * 1024,
                   cap};
        // and the largest tile with which k blocks fit on an SM, k = 1..4
        int sm_smem = 0, reserved = 0;
        cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, c->device);
        for (int k = 1; k <= 4; ++k) {
            const int64_t per = (int64_t)sm_smem / k - (int64_t)stat - reserved;
            if (per >= 16 * 1024) budgets.push_back((size_t)(per / 1024 * 1024));
        }
        // networks too small to give every SM a 16 KB tile: smaller tiles
        // spread them over more SMs (a 32-node group is the smallest tile)
        if (p->n_nodes <= 148 * 256) {
            budgets.push_back(4 * 1024);
            budgets.push_back(8 * 1024);
        }
        std::sort(budgets.begin(), budgets.end());
        budgets.erase(std::unique(budgets.begin(), budgets.end()), budgets.end());
    }
    else budgets = {std::min<size_t>(cap, 96 * 1024)};
    size_t items = 0;
    for (int t = 0; t < T; ++t) items += (size_t)gates[t] * mechs[t]->n;
    // (the 9-state variant: blocks up to 256 run its register-rich build,
    // larger ones its wide build: FP64 up to 768 threads, MIXED up to 512)
    const int max_block = kin ? fused_kin_wide_block(p->precision) : kFusedMaxBlock;
    if (c->opt.block > 0) blocks = {std::min(c->opt.block, max_block)};
    else if (tune && kin) blocks = {128, 256, max_block == 768 ? 512 : 384, max_block};
    else if (tune) blocks = {128, 256, 512, 1024};
    else blocks = {256};
    pers = tune ? std::vector<bool>{false, true} : std::vector<bool>{false};

    std::vector<Candidate> cands;
    for (size_t b : budgets) {
        std::vector<int32_t> recs;
        auto sched_p = std::make_shared<std::vector<uint16_t>>();
        std::vector<uint16_t>& sched = *sched_p;
        size_t max_smem = 0;
        if (b > cap || !make_tiles(p->precision, off, T, gates, slots, bounds, cb != nullptr, ions,
                                   ext, b, recs, max_smem)) {
            if (dbg) std::fprintf(stderr, "[nmodl plan] budget %zu: no tiling\n", b);
            continue;
        }
        if (cb) add_cable_sched(cb, T, recs, sched);
        lpt_order(recs, T, gates, stride);
        for (int blk : blocks)
            for (bool ps : pers)
                cands.push_back(Candidate{b, blk, ps, recs, std::max<size_t>(max_smem, 16), 0.0,
                                          sched_p});
    }
    if (dbg)
        std::fprintf(stderr, "[nmodl plan] prec %d types %d nodes %lld cap %zu stat %zu cands %zu\n",
                     p->precision, T, (long long)p->n_nodes, cap, stat, cands.size());
    if (cands.empty()) return NMODL_OK;  // no tile fits: generic step
    int32_t* d_counter = nullptr;
    if ((e = dalloc(&d_counter, 1)) != cudaSuccess) return cuda_status(e);
    p->d_counter = d_counter;

    size_t best = 0;
    bool generic_wins = false;
    if (cands.size() > 1) {
        // time each candidate on a scratch copy: a prefix of the network of
        // up to 16M instances (several waves of even the largest tiles),
        // min(window, 8) steps, best of 2
        std::vector<double*> sst(T, nullptr);
        double *sv = nullptr, *srhs = nullptr, *sd = nullptr;
        int32_t* d_trial = nullptr;
        bool ok = true;
        for (int t = 0; t < T && ok; ++t) {
            const size_t cnt = (size_t)mechs[t]->n_states * mechs[t]->stride;
            ok = dalloc(&sst[t], cnt) == cudaSuccess &&
                 (cnt == 0 || cudaMemcpyAsync(sst[t], mechs[t]->d_states, cnt * sizeof(double),
                                              cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess);
        }
        ok = ok && dalloc(&sv, p->n_nodes) == cudaSuccess && dalloc(&srhs, p->n_nodes) == cudaSuccess &&
             dalloc(&sd, p->n_nodes) == cudaSuccess;
        if (ok && v_user)
            ok = cudaMemcpyAsync(sv, v_user, p->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream) == cudaSuccess;
        else if (ok)
            ok = cudaMemsetAsync(sv, 0, p->n_nodes * sizeof(double), c->stream) == cudaSuccess;
        size_t max_recs = 0, max_sched = 0;
        for (auto& cd : cands) {
            max_recs = std::max(max_recs, cd.recs.size());
            max_sched = std::max(max_sched, cd.sched->size());
        }
        ok = ok && dalloc(&d_trial, max_recs) == cudaSuccess;
        uint16_t* d_sched_trial = nullptr;
        ok = ok && dalloc(&d_sched_trial, max_sched) == cudaSuccess;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
        // ms per instance of one candidate over nsteps steps (best of 2), or
        // a negative value if a launch failed
        auto time_cand = [&](Candidate& cd, int nsteps) -> double {
            // prefix of the tiles in node order: re-sort the (LPT) list by n0
            const int st = p->tile_stride;
            const size_t nt = cd.recs.size() / st;
            std::vector<size_t> idx(nt);
            for (size_t k = 0; k < nt; ++k) idx[k] = k;
            std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
                return cd.recs[a * st] < cd.recs[b * st];
            });
            std::vector<int32_t> sub;
            int64_t inst = 0;
            for (size_t k : idx) {
                if (inst > 16000000) break;
                for (int tt = 0; tt < T; ++tt)
                    inst += cd.recs[k * st + 3 + 2 * tt] - cd.recs[k * st + 2 + 2 * tt];
                sub.insert(sub.end(), cd.recs.begin() + k * st, cd.recs.begin() + (k + 1) * st);
            }
            lpt_order(sub, T, gates, st);
            cudaMemcpyAsync(d_trial, sub.data(), sub.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, c->stream);
            if (!cd.sched->empty())
                cudaMemcpyAsync(d_sched_trial, cd.sched->data(), cd.sched->size() * sizeof(uint16_t),
                                cudaMemcpyHostToDevice, c->stream);
            FusedArgs a{};
            a.md = nullptr;
            a.n_types = T;
            for (int t = 0; t < T; ++t) {
                a.n_gates[t] = mechs[t]->n_states;
                a.states[t] = sst[t];
                a.stride[t] = mechs[t]->stride;
                a.ni[t] = mechs[t]->d_ni;
            }
            a.tiles = d_trial;
            a.tile_stride = st;
            a.n_tiles = (int)(sub.size() / st);
            a.tile_counter = cd.persistent ? d_counter : nullptr;
            a.nsteps = nsteps;
            a.clamp_v = c->opt.clamp_v;
            a.pade = c->opt.cnexp_pade;
            a.v = sv;
            a.rhs = srhs;
            a.d = sd;
            a.dt = 0.025;
            a.cm = 1.0;
            a.err = nullptr;
            if (cb) {
                a.cable = 1;
                a.parent = cb->d_parent;
                a.ga = cb->d_ga;
                a.gb = cb->d_gb;
                a.sched = d_sched_trial;
            }
            a.ions = ions;  // sums and ica kept, no ion array written
            a.newton_tol = c->opt.newton_tol;
            a.newton_max_iter = c->opt.newton_max_iter;
            a.ir_max = c->opt.ir_max;
            // descriptors
            if (upload_descriptors(c, p, mechs, T) != cudaSuccess) return -1.0;
            a.md = p->d_md;
            a.k9d = p->d_k9;
            double best_ms = 1e30;
            for (int rep = 0; rep < 2 && ok; ++rep) {
                if (cd.persistent) cudaMemsetAsync(d_counter, 0, sizeof(int32_t), c->stream);
                cudaEventRecord(e0, c->stream);
                const int grid = cd.persistent
                                     ? fused_resident_grid(p->variant, a.n_tiles, cd.block, cd.smem)
                                     : a.n_tiles;
                ok = launch_fused(p->variant, a, grid, cd.block, cd.smem, c->stream) ==
                     cudaSuccess;
                cudaEventRecord(e1, c->stream);
                ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best_ms = std::min(best_ms, (double)ms);
            }
            if (!ok) return -1.0;
            return best_ms / std::max<int64_t>(1, inst);
        };
        // stage 1: every candidate over min(window, 8) steps; stage 2: the
        // four fastest again over the window (at most 64 steps), where the
        // load and store of each tile weigh as little as in the real launch
        // (over 8 steps they favoured shapes that lose at full length)
        const int trial_steps = std::min(c->opt.window, 8);
        const int full_steps = std::min(c->opt.window, 64);
        for (size_t ci = 0; ok && ci < cands.size(); ++ci) {
            const double ms = time_cand(cands[ci], trial_steps);
            if (ms < 0.0) ok = false;
            cands[ci].ms = ms;
            if (cands[ci].ms < cands[best].ms || ci == 0) best = ci;
        }
        double best_ms = ok ? cands[best].ms : 0.0;  // of the chosen shape, per instance
        int best_steps = trial_steps;                // ... over this many steps
        if (ok && full_steps > trial_steps && cands.size() > 1) {
            std::vector<size_t> order(cands.size());
            for (size_t k = 0; k < order.size(); ++k) order[k] = k;
            std::stable_sort(order.begin(), order.end(),
                             [&](size_t x, size_t y) { return cands[x].ms < cands[y].ms; });
            double best_full = 1e30;
            for (size_t r = 0; ok && r < std::min<size_t>(4, order.size()); ++r) {
                const double ms = time_cand(cands[order[r]], full_steps);
                if (ms < 0.0) {
                    ok = false;
                } else {
                    if (dbg)
                        std::fprintf(stderr, "[nmodl plan] window trial budget %zu block %d persistent %d ns/inst (per %d steps) %.4f\n",
                                     cands[order[r]].budget, cands[order[r]].block,
                                     (int)cands[order[r]].persistent, trial_steps,
                                     ms * 1e6 * trial_steps / full_steps);
                    if (ms < best_full) {
                        best_full = ms;
                        best = order[r];
                        best_ms = ms;
                        best_steps = full_steps;
                    }
                }
            }
        }
        // FP64 lists with the 9-state scheme: the fused variant runs one
        // block per SM (the FP64 solve holds ~245 registers per thread), so
        // its cnexp items run at 8 warps per SM and the per-mechanism
        // launches can be faster.  Time them too, over the whole network on
        // the same scratch copies (each mechanism's state array swapped for
        // its copy during the trial, its Newton counters restored after),
        // and keep the faster form.  Not with a fixed tile budget or block.
        if (ok && kin && p->precision == NMODL_FP64 && !cb && c->opt.tile_smem == 0 &&
            c->opt.block == 0) {
            std::vector<KinCounters> saved(T);
            ok = cudaStreamSynchronize(c->stream) == cudaSuccess;
            for (int t = 0; t < T && ok; ++t)
                if (mechs[t]->d_cnt)
                    ok = cudaMemcpy(&saved[t], mechs[t]->d_cnt, sizeof(KinCounters),
                                    cudaMemcpyDeviceToHost) == cudaSuccess;
            int64_t total = 0;
            for (int t = 0; t < T; ++t) total += mechs[t]->n;
            double gbest = 1e30;
            if (ok) {
                for (int t = 0; t < T; ++t) std::swap(mechs[t]->d_states, sst[t]);
                for (int rep = 0; rep < 2 && ok; ++rep) {
                    cudaEventRecord(e0, c->stream);
                    ok = enqueue_generic_steps(c, mechs, n_mechs, 0.025, 1.0, sv, srhs, sd,
                                               best_steps, p->n_nodes) == cudaSuccess;
                    cudaEventRecord(e1, c->stream);
                    ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    gbest = std::min(gbest, (double)ms);
                }
                cudaStreamSynchronize(c->stream);
                for (int t = 0; t < T; ++t) std::swap(mechs[t]->d_states, sst[t]);
                for (int t = 0; t < T; ++t)
                    if (mechs[t]->d_cnt)
                        cudaMemcpy(mechs[t]->d_cnt, &saved[t], sizeof(KinCounters),
                                   cudaMemcpyHostToDevice);
            }
            const double gms = gbest / std::max<int64_t>(1, total);
            if (dbg)
                std::fprintf(stderr, "[nmodl plan] per-mechanism launches ns/inst (per %d steps) %.4f vs fused %.4f\n",
                             best_steps, gms * 1e6, best_ms * 1e6);
            generic_wins = ok && gms < best_ms;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        for (double* q : sst) cudaFree(q);
        cudaFree(sv);
        cudaFree(srhs);
        cudaFree(sd);
        cudaFree(d_trial);
        cudaFree(d_sched_trial);
        cudaGetLastError();
        if (!ok) best = 0;
    }
    if (dbg)
        for (size_t ci = 0; ci < cands.size(); ++ci)
            std::fprintf(stderr, "[nmodl plan] budget %zu block %d persistent %d tiles %zu smem %zu ns/inst %.4g%s\n",
                         cands[ci].budget, cands[ci].block, (int)cands[ci].persistent,
                         cands[ci].recs.size() / p->tile_stride, cands[ci].smem, cands[ci].ms * 1e6,
                         ci == best ? "  <- chosen" : "");
    if (generic_wins) {
        if (dbg) std::fprintf(stderr, "[nmodl plan] per-mechanism launches chosen\n");
        return NMODL_OK;  // p->fused stays false
    }
    Candidate& ch = cands[best];
    p->budget = ch.budget;
    p->block = ch.block;
    p->persistent = ch.persistent;
    p->smem = ch.smem;
    p->n_tiles = (int)(ch.recs.size() / p->tile_stride);
    p->grid = ch.persistent ? fused_resident_grid(p->variant, p->n_tiles, ch.block, ch.smem)
                            : p->n_tiles;
    if ((e = dalloc(&p->d_tiles, ch.recs.size())) != cudaSuccess) return cuda_status(e);
    cudaMemcpyAsync(p->d_tiles, ch.recs.data(), ch.recs.size() * sizeof(int32_t),
                    cudaMemcpyHostToDevice, c->stream);
    if (!ch.sched->empty()) {
        if ((e = dalloc(&p->d_sched, ch.sched->size())) != cudaSuccess) return cuda_status(e);
        cudaMemcpyAsync(p->d_sched, ch.sched->data(), ch.sched->size() * sizeof(uint16_t),
                        cudaMemcpyHostToDevice, c->stream);
    }
    if ((e = upload_descriptors(c, p, mechs, T)) != cudaSuccess) return cuda_status(e);
    cudaStreamSynchronize(c->stream);  // host buffers above go out of scope
    p->fused = true;
    return NMODL_OK;
}

Plan* nmodl_get_plan(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs, const double* v,
                     int* rc, nmodl_cable* cb) {
    for (auto& p : c->plans) {
        if ((int)p->mechs.size() == n_mechs && p->precision == c->opt.precision &&
            p->cable == cb && std::equal(p->mechs.begin(), p->mechs.end(), mechs))
            return p.get();
    }
    std::unique_ptr<Plan> p(new (std::nothrow) Plan());
    if (!p) {
        *rc = NMODL_ERR_OOM;
        return nullptr;
    }
    *rc = build_plan(c, mechs, n_mechs, p.get(), v, cb);
    if (*rc) return nullptr;
    c->plans.push_back(std::move(p));
    return c->plans.back().get();
}

static FusedArgs fused_args(nmodl_ctx* c, Plan* p, double dt, double cm, double* v,
                            double* rhs, double* d, int nsteps) {
    FusedArgs a{};
    a.md = p->d_md;
    a.k9d = p->d_k9;
    a.n_types = (int)p->mechs.size();
    for (int t = 0; t < a.n_types; ++t) {
        nmodl_mech* m = p->mechs[t];
        a.n_gates[t] = m->n_states;
        a.states[t] = m->d_states;
        a.stride[t] = m->stride;
        a.ni[t] = m->d_ni;
        if (m->type == NMODL_KIN9 || m->type == NMODL_KIN3 || m->type == NMODL_CACUM)
            a.cnt[t] = m->d_cnt;
    }
    a.tiles = p->d_tiles;
    a.tile_stride = p->tile_stride;
    a.n_tiles = p->n_tiles;
    a.tile_counter = p->persistent ? p->d_counter : nullptr;
    a.nsteps = nsteps;
    a.clamp_v = c->opt.clamp_v;
    a.pade = c->opt.cnexp_pade;
    a.v = v;
    a.rhs = rhs;
    a.d = d;
    a.dt = dt;
    a.cm = cm;
    a.err = c->d_err;
    a.ions = c->has_ions();
    for (int q = 1; q < 4; ++q) a.ion[q] = c->ion[q];
    a.newton_tol = c->opt.newton_tol;
    a.newton_max_iter = c->opt.newton_max_iter;
    a.ir_max = c->opt.ir_max;
    if (nmodl_cable* cb = p->cable) {
        a.cable = 1;
        a.parent = cb->d_parent;
        a.ga = cb->d_ga;
        a.gb = cb->d_gb;
        a.sched = p->d_sched;
    }
    return a;
}

static cudaError_t enqueue_generic_steps(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs,
                                         double dt, double cm, double* v, double* rhs,
                                         double* d, int nsteps, int64_t n_nodes) {
    for (int s = 0; s < nsteps; ++s) {
        cudaMemsetAsync(rhs, 0, n_nodes * sizeof(double), c->stream);
        cudaMemsetAsync(d, 0, n_nodes * sizeof(double), c->stream);
        nmodl_zero_ions(c, n_nodes);
        for (int i = 0; i < n_mechs; ++i) nmodl_enqueue_cur(mechs[i], v, rhs, d);
        launch_vupdate(n_nodes, v, rhs, d, 1e-3 * cm / dt, c->opt.clamp_v, c->d_err, c->stream);
        for (int i = 0; i < n_mechs; ++i) nmodl_enqueue_state(mechs[i], dt, v);
    }
    return cudaGetLastError();
}

// Enqueue one window either directly or by replaying its cached graph.
cudaError_t nmodl_run_window(nmodl_ctx* c, Plan* p, nmodl_mech* const* mechs, int n_mechs,
                              double dt, double cm, double* v, double* rhs, double* d,
                              int w) {
    auto direct = [&]() -> cudaError_t {
        if (p->sur_step) {
            for (int s = 0; s < w; ++s) {
                const cudaError_t se = enqueue_surrogate_network_step(
                    mechs[0], dt, cm, v, rhs, d, c->opt.clamp_v);
                if (se != cudaSuccess) return se;
            }
            return cudaSuccess;
        }
        if (p->hh_per_block > 0) {
            nmodl_mech* m = mechs[0];
            HhArgs a{};
            for (int q = 0; q < 3; ++q) {
                a.gate[q] = m->md.gate[q];
                fold_gate(a.gate[q], m->md.phi * dt);
                a.g[q] = m->md.hh_g[q];
                a.e[q] = m->md.hh_e[q];
            }
            a.n = p->n_nodes;
            a.per_block = p->hh_per_block;
            a.nsteps = w;
            a.clamp_v = c->opt.clamp_v;
            a.dt = dt;
            a.cm = cm;
            a.v = v;
            a.states = m->d_states;
            a.stride = m->stride;
            a.rhs = rhs;
            a.d = d;
            a.err = c->d_err;
            return launch_hh_gate_warps(a, c->stream);
        }
        if (p->fused) {
            FusedArgs a = fused_args(c, p, dt, cm, v, rhs, d, w);
            if (p->persistent) {
                cudaError_t me = cudaMemsetAsync(p->d_counter, 0, sizeof(int32_t), c->stream);
                if (me != cudaSuccess) return me;
            }
            return launch_fused(p->variant, a, p->grid, p->block, p->smem, c->stream);
        }
        return enqueue_generic_steps(c, mechs, n_mechs, dt, cm, v, rhs, d, w, p->n_nodes);
    };
    if (!c->opt.use_graph || c->stream == nullptr) return direct();
    for (auto& ge : p->graphs)
        if (ge.v == v && ge.rhs == rhs && ge.d == d && ge.dt == dt && ge.cm == cm &&
            ge.nsteps == w && ge.clamp == c->opt.clamp_v)
            return cudaGraphLaunch(ge.exec, c->stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return direct();
    cudaError_t le = direct();
    e = cudaStreamEndCapture(c->stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return le != cudaSuccess ? le : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    p->graphs.push_back(GraphEntry{v, rhs, d, dt, cm, w, c->opt.clamp_v, exec});
    if (p->graphs.size() > 16) {
        cudaGraphExecDestroy(p->graphs.front().exec);
        p->graphs.erase(p->graphs.begin());
    }
    return cudaGraphLaunch(exec, c->stream);
}

int nmodl_step(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs, double dt, double cm,
               double* v, double* rhs, double* d, int nsteps) {
    if (!c || !mechs || n_mechs < 1 || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt) ||
        !(cm > 0.0) || !std::isfinite(cm))
        return NMODL_ERR_ARG;
    const int64_t n_nodes = mechs[0]->n_nodes;
    for (int i = 0; i < n_mechs; ++i)
        if (!mechs[i] || mechs[i]->ctx != c || mechs[i]->n_nodes != n_nodes) return NMODL_ERR_ARG;
    if (nsteps == 0 || n_nodes == 0) return NMODL_OK;
    if (!v || !rhs || !d) return NMODL_ERR_ARG;
    if (c->has_ions() && c->ion_nodes != n_nodes) return NMODL_ERR_ARG;
    if (nmodl_check_ion_reads(c, mechs, n_mechs)) return NMODL_ERR_ARG;
    DeviceGuard g(c->device);
    int rc = NMODL_OK;
    Plan* p = nmodl_get_plan(c, mechs, n_mechs, v, &rc, nullptr);
    if (!p) return rc;
    for (int i = 0; i < n_mechs; ++i) nmodl_count_states(mechs[i], nsteps);
    const int W = c->opt.window;
    for (int s = 0; s < nsteps; s += W) {
        const int w = std::min(W, nsteps - s);
        cudaError_t e = nmodl_run_window(c, p, mechs, n_mechs, dt, cm, v, rhs, d, w);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return NMODL_OK;
}

int nmodl_plan_describe(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs, int64_t* out) {
    if (!c || !mechs || n_mechs < 1 || !out) return NMODL_ERR_ARG;
    // the most recently built plan of this mechanism list (isolated or cable)
    for (auto it = c->plans.rbegin(); it != c->plans.rend(); ++it) {
        auto& p = *it;
        if ((int)p->mechs.size() == n_mechs && p->precision == c->opt.precision &&
            std::equal(p->mechs.begin(), p->mechs.end(), mechs)) {
            if (p->sur_step) {
                out[0] = 3;
                out[1] = out[3] = out[4] = out[5] = 0;
                out[2] = 512;
                return NMODL_OK;
            }
            if (p->hh_per_block > 0) {
                out[0] = 2;
                out[1] = (p->n_nodes + p->hh_per_block - 1) / p->hh_per_block;
                out[2] = 96;
                out[3] = 0;
                out[4] = 0;
                out[5] = p->hh_per_block;
                return NMODL_OK;
            }
            out[0] = p->fused ? 1 : 0;
            out[1] = p->n_tiles;
            out[2] = p->block;
            out[3] = (int64_t)p->smem;
            out[4] = p->persistent ? 1 : 0;
            out[5] = (int64_t)p->budget;
            return NMODL_OK;
        }
    }
    return NMODL_ERR_ARG;
}

int nmodl_ctx_set_ions(nmodl_ctx* c, int64_t n_nodes, double* ina, double* ik, double* ica) {
    if (!c || n_nodes < 0 || ((ina || ik || ica) && n_nodes == 0)) return NMODL_ERR_ARG;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    // plans and graphs hold the previous arrays (and the fused/unfused choice)
    nmodl_invalidate_plans(c, nullptr);
    c->ion[NMODL_ION_NA] = ina;
    c->ion[NMODL_ION_K] = ik;
    c->ion[NMODL_ION_CA] = ica;
    c->ion_nodes = (ina || ik || ica) ? n_nodes : 0;
    return NMODL_OK;
}

int nmodl_mech_set_ion(nmodl_mech* m, int ion) {
    if (!m || ion < NMODL_ION_NONE || ion > NMODL_ION_CA) return NMODL_ERR_ARG;
    if ((m->type == NMODL_HH || m->type == NMODL_CACUM) && ion != NMODL_ION_NONE)
        return NMODL_ERR_ARG;
    if (m->ion == ion) return NMODL_OK;
    DeviceGuard g(m->ctx->device);
    cudaError_t e = cudaStreamSynchronize(m->ctx->stream);
    if (e != cudaSuccess) return cuda_status(e);
    nmodl_invalidate_plans(m->ctx, m);
    m->ion = ion;
    m->md.ion = ion;
    return NMODL_OK;
}

int nmodl_get_state(nmodl_mech* m, int k, double* out) {
    if (!m || k < 0 || k >= m->n_states || (m->n > 0 && !out)) return NMODL_ERR_ARG;
    if (m->n == 0) return NMODL_OK;
    DeviceGuard g(m->ctx->device);
    cudaError_t e = cudaMemcpyAsync(out, m->d_states + (int64_t)k * m->stride,
                                    m->n * sizeof(double), cudaMemcpyDefault, m->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->ctx->stream);
    return cuda_status(e);
}

int nmodl_set_state(nmodl_mech* m, int k, const double* in) {
    if (!m || k < 0 || k >= m->n_states || (m->n > 0 && !in)) return NMODL_ERR_ARG;
    if (m->n == 0) return NMODL_OK;
    DeviceGuard g(m->ctx->device);
    cudaError_t e = cudaMemcpyAsync(m->d_states + (int64_t)k * m->stride, in,
                                    m->n * sizeof(double), cudaMemcpyDefault, m->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->ctx->stream);
    return cuda_status(e);
}

int nmodl_stats(nmodl_mech* m, nmodl_stats_t* out) {
    if (!m || !out) return NMODL_ERR_ARG;
    DeviceGuard g(m->ctx->device);
    std::memset(out, 0, sizeof(*out));
    KinCounters k{};
    cudaError_t e = cudaStreamSynchronize(m->ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&k, m->d_cnt, sizeof(k), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    out->calls = m->calls;
    out->newton_iters = (int64_t)k.iters;
    out->newton_max = k.max_iter_seen;
    out->nonconverged = (int64_t)k.nonconv;
    out->fallback = (int64_t)k.fallback;
    out->surrogate_calls = m->sur_calls;
    return NMODL_OK;
}

}  // extern "C"
