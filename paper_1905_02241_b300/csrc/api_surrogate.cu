// api_surrogate.cu -- C ABI of the kinetic surrogate: creation, weights,
// forward, loss/gradients, Adam training step, Newton-generated training
// pairs, and attaching the surrogate to a NMODL_KIN9 mechanism.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "mlp.cuh"
#include "runtime.cuh"

using namespace nmodl;

namespace {

// public (unpadded) <-> padded FP32 parameter layouts
void pub_to_pad(const float* in, float* out) {
    std::memset(out, 0, sizeof(float) * kParamsPadded);
    const float* p = in;
    for (int o = 0; o < kHid; ++o)
        for (int i = 0; i < kInRaw; ++i) out[kOffW1 + o * kIn + i] = *p++;
    for (int o = 0; o < kHid; ++o) out[kOffB1 + o] = *p++;
    for (int k = 0; k < kHid * kHid; ++k) out[kOffW2 + k] = *p++;
    for (int o = 0; o < kHid; ++o) out[kOffB2 + o] = *p++;
    for (int k = 0; k < kHid * kHid; ++k) out[kOffW3 + k] = *p++;
    for (int o = 0; o < kHid; ++o) out[kOffB3 + o] = *p++;
    for (int o = 0; o < kOutRaw; ++o)
        for (int i = 0; i < kHid; ++i) out[kOffW4 + o * kHid + i] = *p++;
    for (int o = 0; o < kOutRaw; ++o) out[kOffB4 + o] = *p++;
}

void pad_to_pub(const float* in, float* out) {
    float* p = out;
    for (int o = 0; o < kHid; ++o)
        for (int i = 0; i < kInRaw; ++i) *p++ = in[kOffW1 + o * kIn + i];
    for (int o = 0; o < kHid; ++o) *p++ = in[kOffB1 + o];
    for (int k = 0; k < kHid * kHid; ++k) *p++ = in[kOffW2 + k];
    for (int o = 0; o < kHid; ++o) *p++ = in[kOffB2 + o];
    for (int k = 0; k < kHid * kHid; ++k) *p++ = in[kOffW3 + k];
    for (int o = 0; o < kHid; ++o) *p++ = in[kOffB3 + o];
    for (int o = 0; o < kOutRaw; ++o)
        for (int i = 0; i < kHid; ++i) *p++ = in[kOffW4 + o * kHid + i];
    for (int o = 0; o < kOutRaw; ++o) *p++ = in[kOffB4 + o];
}

void refresh_bf16(nmodl_surrogate* s) {
    cudaStream_t st = s->ctx->stream;
    launch_to_bf16(s->params + kOffW1, kHid * kIn, s->wbf + kBfW1, st);
    launch_to_bf16(s->params + kOffW2, kHid * kHid, s->wbf + kBfW2, st);
    launch_to_bf16(s->params + kOffW3, kHid * kHid, s->wbf + kBfW3, st);
    launch_to_bf16(s->params + kOffW4, kOut * kHid, s->wbf + kBfW4, st);
    launch_train_image(s->params, s->img, st);
}

void free_sur(nmodl_surrogate* s) {
    void* ptrs[] = {s->params, s->wbf, s->img, s->grad, s->m, s->v, s->ds1, s->ds2, s->ds3, s->part,
                    s->loss_part, s->loss};
    for (void* p : ptrs) cudaFree(p);
    delete s;
}

TrainArgs train_args(nmodl_surrogate* s, int64_t n, const float* X, int* grid) {
    TrainArgs a{};
    a.X = X;
    a.n = n;
    a.img = s->img;
    a.ds1 = s->ds1;
    a.ds2 = s->ds2;
    a.ds3 = s->ds3;
    a.part = s->part;
    a.loss_part = s->loss_part;
    a.err = s->ctx->d_err;
    *grid = train_grid(n, &a.tiles_per_cta);
    return a;
}

// Loss and gradient partials of one batch (the fused tensor-core kernel),
// then their sum into s->grad (adam = 0) or the Adam step on the master
// parameters, their bf16 copies and the weight image (adam = 1); s->loss
// receives the loss (in a replayed run also loss_steps[step], and the step
// index advances: done is the zeroed arrival counter of that).
cudaError_t loss_and_grad(nmodl_surrogate* s, int64_t n, const float* X, const float* T,
                          int adam, float lr, FitSched fs = FitSched{},
                          float* loss_steps = nullptr, unsigned int* done = nullptr) {
    cudaStream_t st = s->ctx->stream;
    int grid = 0;
    TrainArgs a = train_args(s, n, X, &grid);
    a.T = T;
    a.mode = 1;
    a.fs = fs;
    cudaError_t e = launch_train_tiles(a, grid, st);
    if (e != cudaSuccess) return e;
    launch_grad_adam(s->part, grid, s->loss_part, s->loss, s->grad, adam, s->params, s->m, s->v,
                     s->wbf, s->img, lr, 0.9f, 0.999f, 1e-8f, s->step, fs, loss_steps, done, st);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

NMODL_API int nmodl_surrogate_n_params(void) { return kParamsPublic; }

NMODL_API int nmodl_surrogate_create(nmodl_ctx* c, int64_t max_batch, const float* weights,
                                     int scaled, nmodl_surrogate** out) {
    if (!c || !out || max_batch < 16 || max_batch > (1 << 24) || (max_batch % 16))
        return NMODL_ERR_ARG;
    *out = nullptr;
    DeviceGuard dg(c->device);
    nmodl_surrogate* s = new (std::nothrow) nmodl_surrogate();
    if (!s) return NMODL_ERR_OOM;
    s->ctx = c;
    s->scaled = scaled ? 1 : 0;
    s->max_batch = max_batch;
    const int64_t B = max_batch;
    s->n_part_max = train_max_grid(B);
    cudaError_t e = cudaSuccess;
    do {
        if ((e = dalloc(&s->params, kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->wbf, kBfCount)) != cudaSuccess) break;
        if ((e = dalloc(&s->img, kTrImgBytes)) != cudaSuccess) break;
        if ((e = dalloc(&s->grad, kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->m, kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->v, kParamsPadded)) != cudaSuccess) break;
        // whole 128-row tiles: the training kernel stores each tile's block
        // (FP16 column pairs), a partial last tile included
        const int64_t Bt = (B + 127) / 128 * 128;
        if ((e = dalloc(&s->ds1, Bt * kHid / 2)) != cudaSuccess) break;
        if ((e = dalloc(&s->ds2, Bt * kHid / 2)) != cudaSuccess) break;
        if ((e = dalloc(&s->ds3, Bt * kHid / 2)) != cudaSuccess) break;
        if ((e = dalloc(&s->part, (int64_t)s->n_part_max * kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->loss_part, s->n_part_max)) != cudaSuccess) break;
        if ((e = dalloc(&s->loss, 1)) != cudaSuccess) break;
        std::vector<float> pad(kParamsPadded, 0.f);
        if (weights) pub_to_pad(weights, pad.data());
        if ((e = cudaMemcpyAsync(s->params, pad.data(), sizeof(float) * kParamsPadded,
                                 cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) break;
        cudaMemsetAsync(s->m, 0, sizeof(float) * kParamsPadded, c->stream);
        cudaMemsetAsync(s->v, 0, sizeof(float) * kParamsPadded, c->stream);
        cudaMemsetAsync(s->grad, 0, sizeof(float) * kParamsPadded, c->stream);
        refresh_bf16(s);
        e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = surrogate_prepare();
        if (e == cudaSuccess) e = train_prepare();
    } while (false);
    if (e != cudaSuccess) {
        free_sur(s);
        return nmodl_cuda_status(e);
    }
    *out = s;
    return NMODL_OK;
}

NMODL_API void nmodl_surrogate_destroy(nmodl_surrogate* s) {
    if (!s) return;
    DeviceGuard dg(s->ctx->device);
    cudaStreamSynchronize(s->ctx->stream);
    free_sur(s);
}

NMODL_API int nmodl_surrogate_set_weights(nmodl_surrogate* s, const float* w) {
    if (!s || !w) return NMODL_ERR_ARG;
    DeviceGuard dg(s->ctx->device);
    std::vector<float> pad(kParamsPadded);
    pub_to_pad(w, pad.data());
    cudaError_t e = cudaMemcpyAsync(s->params, pad.data(), sizeof(float) * kParamsPadded,
                                    cudaMemcpyHostToDevice, s->ctx->stream);
    if (e == cudaSuccess) {
        refresh_bf16(s);
        e = cudaStreamSynchronize(s->ctx->stream);
    }
    s->step = 0;
    cudaMemsetAsync(s->m, 0, sizeof(float) * kParamsPadded, s->ctx->stream);
    cudaMemsetAsync(s->v, 0, sizeof(float) * kParamsPadded, s->ctx->stream);
    return nmodl_cuda_status(e);
}

NMODL_API int nmodl_surrogate_get_weights(nmodl_surrogate* s, float* w) {
    if (!s || !w) return NMODL_ERR_ARG;
    DeviceGuard dg(s->ctx->device);
    std::vector<float> pad(kParamsPadded);
    cudaError_t e = cudaStreamSynchronize(s->ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(pad.data(), s->params, sizeof(float) * kParamsPadded,
                       cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) pad_to_pub(pad.data(), w);
    return nmodl_cuda_status(e);
}

NMODL_API int nmodl_surrogate_forward(nmodl_surrogate* s, int64_t n, const float* X, float* Y) {
    if (!s || n < 0 || n > s->max_batch || (n > 0 && (!X || !Y))) return NMODL_ERR_ARG;
    if (n == 0) return NMODL_OK;
    DeviceGuard dg(s->ctx->device);
    int grid = 0;
    TrainArgs a = train_args(s, n, X, &grid);
    a.Y = Y;
    a.mode = 0;
    return nmodl_cuda_status(launch_train_tiles(a, grid, s->ctx->stream));
}

NMODL_API int nmodl_surrogate_loss_grad(nmodl_surrogate* s, int64_t n, const float* X,
                                        const float* T, float* grad_host, float* loss_host) {
    if (!s || n < 16 || n > s->max_batch || !X || !T) return NMODL_ERR_ARG;
    DeviceGuard dg(s->ctx->device);
    cudaError_t e = loss_and_grad(s, n, X, T, 0, 0.f);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->ctx->stream);
    if (e == cudaSuccess && loss_host)
        e = cudaMemcpy(loss_host, s->loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && grad_host) {
        std::vector<float> pad(kParamsPadded);
        e = cudaMemcpy(pad.data(), s->grad, sizeof(float) * kParamsPadded,
                       cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) pad_to_pub(pad.data(), grad_host);
    }
    return nmodl_cuda_status(e);
}

NMODL_API int nmodl_surrogate_train_step(nmodl_surrogate* s, int64_t n, const float* X,
                                         const float* T, float lr, float* loss_dev) {
    if (!s || n < 16 || n > s->max_batch || !X || !T || !(lr > 0.f)) return NMODL_ERR_ARG;
    DeviceGuard dg(s->ctx->device);
    cudaStream_t st = s->ctx->stream;
    s->step += 1;
    cudaError_t e = loss_and_grad(s, n, X, T, 1, lr);
    if (e == cudaSuccess && loss_dev)
        e = cudaMemcpyAsync(loss_dev, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return nmodl_cuda_status(e);
}

// A whole training run: one optimiser step (loss and gradients, Adam with
// the scheduled learning rate, bf16 refresh, loss record) is captured as a
// CUDA graph of 16 steps whose kernels read the step index from device
// memory, replayed once per 16 steps.
NMODL_API int nmodl_surrogate_fit(nmodl_surrogate* s, int64_t n, const float* X, const float* T,
                                  int64_t batch, int epochs, float lr, float lr_min,
                                  float* loss_steps) {
    if (!s || batch < 16 || batch > s->max_batch || (batch % 16) || n < batch || epochs < 1 ||
        !X || !T || !loss_steps || !(lr > 0.f) || !(lr_min >= 0.f) || !(lr_min <= lr))
        return NMODL_ERR_ARG;
    nmodl_ctx* c = s->ctx;
    DeviceGuard dg(c->device);
    cudaStream_t st = c->stream;
    const int64_t spe = n / batch, total = spe * (int64_t)epochs;
    // the run's step index, then the arrival counter of the kernel that
    // advances it
    int64_t* d_step = nullptr;
    cudaError_t e = dalloc(&d_step, 2);
    if (e != cudaSuccess) return nmodl_cuda_status(e);
    e = cudaMemsetAsync(d_step, 0, 2 * sizeof(int64_t), st);
    unsigned int* d_done = reinterpret_cast<unsigned int*>(d_step + 1);
    FitSched fs{d_step, spe, total, lr, lr_min, s->step, 1};
    auto one_step = [&]() { loss_and_grad(s, batch, X, T, 1, lr, fs, loss_steps, d_done); };
    // graphs of kSteps optimiser steps (the step index lives on the device,
    // so one graph serves every group), then one of the remaining steps: a
    // graph launch per 16 steps instead of one per step
    constexpr int64_t kSteps = 16;
    auto make_exec = [&](int64_t steps, cudaGraphExec_t* ex) -> cudaError_t {
        cudaGraph_t graph = nullptr;
        cudaError_t ge = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (ge == cudaSuccess) {
            for (int64_t k = 0; k < steps; ++k) one_step();
            const cudaError_t le = cudaGetLastError();
            ge = cudaStreamEndCapture(st, &graph);
            if (ge == cudaSuccess) ge = le;
        }
        if (ge == cudaSuccess) ge = cudaGraphInstantiate(ex, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        return ge;
    };
    if (e == cudaSuccess && st != nullptr) {
        const int64_t groups = total / kSteps, rest = total % kSteps;
        cudaGraphExec_t exec = nullptr, exec_rest = nullptr;
        if (groups > 0) e = make_exec(kSteps, &exec);
        for (int64_t k = 0; e == cudaSuccess && k < groups; ++k) e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess && rest > 0) e = make_exec(rest, &exec_rest);
        if (e == cudaSuccess && rest > 0) e = cudaGraphLaunch(exec_rest, st);
        if (exec) cudaGraphExecDestroy(exec);
        if (exec_rest) cudaGraphExecDestroy(exec_rest);
    } else if (e == cudaSuccess) {  // legacy stream: no capture, plain launches
        for (int64_t k = 0; k < total; ++k) one_step();
        e = cudaGetLastError();
    }
    cudaStreamSynchronize(st);
    cudaFree(d_step);
    if (e == cudaSuccess) s->step += (int)total;
    return nmodl_cuda_status(e);
}

NMODL_API int nmodl_surrogate_make_pairs(nmodl_surrogate* s, const nmodl_mech* kin, int64_t n,
                                         const double* v, const double* dt, const double* x,
                                         const double* y, int64_t stride, float* X, float* T) {
    if (!s || !kin || kin->type != NMODL_KIN9 || n < 0 || stride < n) return NMODL_ERR_ARG;
    if (n == 0) return NMODL_OK;
    if (!v || !dt || !x || !y || !X || !T) return NMODL_ERR_ARG;
    DeviceGuard dg(s->ctx->device);
    launch_make_pairs(kin->d_kd, n, v, dt, x, y, stride, s->scaled, X, T, s->ctx->stream);
    return nmodl_cuda_status(cudaGetLastError());
}

// One FP64 (or MIXED, per the context options) implicit Euler Newton step of
// n independent samples of the mechanism's kinetic scheme, each with its own
// voltage v[i] and step dt[i]: y := step(x).  x, y: device SoA, row stride.
NMODL_API int nmodl_kin9_solve(nmodl_mech* kin, int64_t n, const double* v, const double* dt,
                               const double* x, double* y, int64_t stride) {
    if (!kin || kin->type != NMODL_KIN9 || n < 0 || stride < n) return NMODL_ERR_ARG;
    if (n == 0) return NMODL_OK;
    if (!v || !dt || !x || !y) return NMODL_ERR_ARG;
    nmodl_ctx* c = kin->ctx;
    DeviceGuard dg(c->device);
    cudaError_t e = cudaMemcpy2DAsync(y, stride * sizeof(double), x, stride * sizeof(double),
                                      n * sizeof(double), kKinStates, cudaMemcpyDeviceToDevice,
                                      c->stream);
    if (e != cudaSuccess) return nmodl_cuda_status(e);
    const nmodl_options& o = c->opt;
    launch_kin9_state(o.precision, kin->d_kd, kin->kd, n, nullptr, v, y, stride, 0.0, dt, o.newton_tol,
                      o.newton_max_iter, o.ir_max, nullptr, 0, nullptr, nullptr, c->d_err,
                      c->stream);
    return nmodl_cuda_status(cudaGetLastError());
}

NMODL_API int nmodl_mech_attach_surrogate(nmodl_mech* m, nmodl_surrogate* s, double tol) {
    if (!m || m->type != NMODL_KIN9) return NMODL_ERR_ARG;
    DeviceGuard dg(m->ctx->device);
    if (!s || !(tol > 0.0)) {
        m->sur = nullptr;
        nmodl_invalidate_plans(m->ctx, m);
        return NMODL_OK;
    }
    if (s->ctx != m->ctx) return NMODL_ERR_ARG;
    if (!m->d_fb_list && m->n > 0) {
        cudaError_t e = dalloc(&m->d_fb_list, (size_t)m->n);
        if (e == cudaSuccess) e = dalloc(&m->d_fb_count, 1);
        if (e != cudaSuccess) return nmodl_cuda_status(e);
    }
    m->sur = s;
    m->sur_tol = tol;
    nmodl_invalidate_plans(m->ctx, m);  // cached step graphs hold the old kernels
    return NMODL_OK;
}

}  // extern "C"

namespace nmodl {
// surrogate state update of a KIN9 mechanism with an attached surrogate:
// fused MLP + projection + residual test, then Newton on the fallback list
// step: null for the state update alone; else the whole network step of a
// list of this one mechanism with instance i on node i (SurArgs::step)
struct SurStep {
    double cm;
    double* v;
    double* rhs;
    double* d;
    int clamp;
};

static cudaError_t enqueue_surrogate(nmodl_mech* m, double dt, const double* v,
                                     const SurStep* step) {
    nmodl_ctx* c = m->ctx;
    nmodl_surrogate* s = m->sur;
    if (m->n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(m->d_fb_count, 0, sizeof(int32_t), c->stream);
    if (e != cudaSuccess) return e;
    SurArgs a{};
    a.wbf = s->wbf;
    a.params = s->params;
    a.kd = m->d_kd;
    a.n = m->n;
    a.ni = m->d_ni;
    a.v = v;
    a.st = m->d_states;
    a.stride = m->stride;
    a.dt = dt;
    a.tol = (float)m->sur_tol;
    a.scaled = s->scaled;
    a.fb_list = m->d_fb_list;
    a.fb_count = m->d_fb_count;
    a.fb_total = &m->d_cnt->fallback;
    a.err = c->d_err;
    if (step) {
        a.step = 1;
        a.clamp = step->clamp;
        a.open = m->kd.open;
        a.gbar = m->kd.gbar;
        a.e = m->kd.e;
        a.cmdt = 1e-3 * step->cm / dt;
        a.v_step = step->v;
        a.rhs = step->rhs;
        a.d = step->d;
    }
    e = launch_surrogate_step(a, c->stream);
    if (e != cudaSuccess) return e;
    // The fallback solve: the FP32-LU Newton with FP64 residual refinement
    // (its result differs from the FP64 step by about 1e-7, from the FP32
    // rates) wherever the gate's tolerance is 1e-5 or more, so that the
    // fallback's own error stays far inside it; the FP64 Newton below that.
    const nmodl_options& o = c->opt;
    const int fb_prec = (o.precision == NMODL_MIXED || m->sur_tol >= 1e-5) ? NMODL_MIXED
                                                                            : NMODL_FP64;
    launch_kin9_state(fb_prec, m->d_kd, m->kd, m->n, m->d_ni, v, m->d_states, m->stride, dt,
                      nullptr, o.newton_tol, o.newton_max_iter, o.ir_max, m->d_fb_list, m->n,
                      m->d_fb_count, m->d_cnt, c->d_err, c->stream);
    return cudaGetLastError();
}

cudaError_t enqueue_surrogate_state(nmodl_mech* m, double dt, const double* v) {
    return enqueue_surrogate(m, dt, v, nullptr);
}

cudaError_t enqueue_surrogate_network_step(nmodl_mech* m, double dt, double cm, double* v,
                                           double* rhs, double* d, int clamp) {
    const SurStep st{cm, v, rhs, d, clamp};
    return enqueue_surrogate(m, dt, v, &st);
}
}  // namespace nmodl
