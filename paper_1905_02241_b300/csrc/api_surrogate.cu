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

constexpr int kSplitRows = 256;  // split-K chunk of the weight-gradient GEMMs

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
}

void free_sur(nmodl_surrogate* s) {
    void* ptrs[] = {s->params, s->wbf, s->grad, s->m, s->v, s->H0, s->H1, s->H2, s->H3,
                    s->D4, s->D3, s->D2, s->D1, s->Z1, s->Z2, s->Z3, s->OUT, s->part,
                    s->loss_part, s->loss};
    for (void* p : ptrs) cudaFree(p);
    delete s;
}

GemmArgs gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
              int N, int K) {
    GemmArgs g{};
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.k_per_split = K;
    return g;
}

// forward of n <= max_batch rows already packed in H0; OUT = [n][16]
void forward(nmodl_surrogate* s, int64_t n) {
    cudaStream_t st = s->ctx->stream;
    const int B = (int)n;
    GemmArgs g = gemm(s->H0, kIn, s->wbf + kBfW1, kIn, B, kHid, kIn);
    g.bias = s->params + kOffB1; g.Cf = s->Z1; g.ldc = kHid; g.Ch = s->H1; g.ldch = kHid;
    launch_gemm(0, 0, kEpiBiasSilu, g, 1, st);
    g = gemm(s->H1, kHid, s->wbf + kBfW2, kHid, B, kHid, kHid);
    g.bias = s->params + kOffB2; g.Cf = s->Z2; g.ldc = kHid; g.Ch = s->H2; g.ldch = kHid;
    launch_gemm(0, 0, kEpiBiasSilu, g, 1, st);
    g = gemm(s->H2, kHid, s->wbf + kBfW3, kHid, B, kHid, kHid);
    g.bias = s->params + kOffB3; g.Cf = s->Z3; g.ldc = kHid; g.Ch = s->H3; g.ldch = kHid;
    launch_gemm(0, 0, kEpiBiasSilu, g, 1, st);
    g = gemm(s->H3, kHid, s->wbf + kBfW4, kHid, B, kOut, kHid);
    g.bias = s->params + kOffB4; g.Cf = s->OUT; g.ldc = kOut;
    launch_gemm(0, 0, kEpiBias, g, 1, st);
}

// weight gradient dW[out][in] = delta^T H (split-K over the batch), bias
// gradient = column sums of delta; written into s->grad at the offsets.
void weight_grad(nmodl_surrogate* s, int64_t n, const __nv_bfloat16* delta, int n_out,
                 const __nv_bfloat16* H, int n_in, int offW, int offB) {
    cudaStream_t st = s->ctx->stream;
    const int B = (int)n;
    const int splits = (B + kSplitRows - 1) / kSplitRows;
    GemmArgs g = gemm(delta, n_out, H, n_in, n_out, n_in, B);
    g.k_per_split = kSplitRows;
    g.Cf = s->part;
    g.ldc = n_in;
    launch_gemm(1, 1, kEpiPartial, g, splits, st);
    launch_reduce_splits(s->part, splits, (int64_t)n_out * n_in, s->grad + offW, st);
    launch_colsum(delta, n, n_out, s->part, s->grad + offB, st);
}

// delta_prev = (delta W) * SiLU'(Z_prev)
void back_delta(nmodl_surrogate* s, int64_t n, const __nv_bfloat16* delta, int n_out,
                const __nv_bfloat16* W, int n_in, const float* Zprev, __nv_bfloat16* out) {
    GemmArgs g = gemm(delta, n_out, W, n_in, (int)n, n_in, n_out);
    g.Zin = Zprev;
    g.ldz = n_in;
    g.Ch = out;
    g.ldch = n_in;
    launch_gemm(0, 1, kEpiDsilu, g, 1, s->ctx->stream);
}

// loss (device scalar s->loss) and all gradients into s->grad
void loss_and_grad(nmodl_surrogate* s, int64_t n, const float* X, const float* T,
                   FitSched fs = FitSched{}) {
    cudaStream_t st = s->ctx->stream;
    launch_pack_input(X, n, s->H0, st, fs);
    forward(s, n);
    const int blocks = launch_loss_delta(s->OUT, T, n, s->D4, s->loss_part, st, fs);
    launch_reduce_splits(s->loss_part, blocks, 1, s->loss, st);
    weight_grad(s, n, s->D4, kOut, s->H3, kHid, kOffW4, kOffB4);
    back_delta(s, n, s->D4, kOut, s->wbf + kBfW4, kHid, s->Z3, s->D3);
    weight_grad(s, n, s->D3, kHid, s->H2, kHid, kOffW3, kOffB3);
    back_delta(s, n, s->D3, kHid, s->wbf + kBfW3, kHid, s->Z2, s->D2);
    weight_grad(s, n, s->D2, kHid, s->H1, kHid, kOffW2, kOffB2);
    back_delta(s, n, s->D2, kHid, s->wbf + kBfW2, kHid, s->Z1, s->D1);
    weight_grad(s, n, s->D1, kHid, s->H0, kIn, kOffW1, kOffB1);
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
    const int64_t splits = (B + kSplitRows - 1) / kSplitRows;
    s->part_count = std::max<int64_t>(splits * kHid * kHid, (B / 256 + 1) * kHid);
    cudaError_t e = cudaSuccess;
    do {
        if ((e = dalloc(&s->params, kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->wbf, kBfCount)) != cudaSuccess) break;
        if ((e = dalloc(&s->grad, kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->m, kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->v, kParamsPadded)) != cudaSuccess) break;
        if ((e = dalloc(&s->H0, B * kIn)) != cudaSuccess) break;
        if ((e = dalloc(&s->H1, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->H2, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->H3, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->D4, B * kOut)) != cudaSuccess) break;
        if ((e = dalloc(&s->D3, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->D2, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->D1, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->Z1, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->Z2, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->Z3, B * kHid)) != cudaSuccess) break;
        if ((e = dalloc(&s->OUT, B * kOut)) != cudaSuccess) break;
        if ((e = dalloc(&s->part, s->part_count)) != cudaSuccess) break;
        if ((e = dalloc(&s->loss_part, 256)) != cudaSuccess) break;
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
    launch_pack_input(X, n, s->H0, s->ctx->stream);
    forward(s, n);
    cudaError_t e = cudaMemcpy2DAsync(Y, kOutRaw * sizeof(float), s->OUT, kOut * sizeof(float),
                                      kOutRaw * sizeof(float), n, cudaMemcpyDeviceToDevice,
                                      s->ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    return nmodl_cuda_status(e);
}

NMODL_API int nmodl_surrogate_loss_grad(nmodl_surrogate* s, int64_t n, const float* X,
                                        const float* T, float* grad_host, float* loss_host) {
    if (!s || n < 16 || n > s->max_batch || !X || !T) return NMODL_ERR_ARG;
    DeviceGuard dg(s->ctx->device);
    loss_and_grad(s, n, X, T);
    cudaError_t e = cudaStreamSynchronize(s->ctx->stream);
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
    loss_and_grad(s, n, X, T);
    s->step += 1;
    launch_adam(s->params, s->grad, s->m, s->v, kParamsPadded, lr, 0.9f, 0.999f, 1e-8f, s->step,
                st);
    refresh_bf16(s);
    if (loss_dev) cudaMemcpyAsync(loss_dev, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return nmodl_cuda_status(cudaGetLastError());
}

// A whole training run: one optimiser step (loss and gradients, Adam with
// the scheduled learning rate, bf16 refresh, loss record) is captured as a
// CUDA graph whose kernels read the step index from device memory, then
// replayed once per step.
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
    int64_t* d_step = nullptr;
    cudaError_t e = dalloc(&d_step, 1);
    if (e != cudaSuccess) return nmodl_cuda_status(e);
    e = cudaMemsetAsync(d_step, 0, sizeof(int64_t), st);
    FitSched fs{d_step, spe, total, lr, lr_min, s->step, 1};
    auto one_step = [&]() {
        loss_and_grad(s, batch, X, T, fs);
        launch_adam_sched(s->params, s->grad, s->m, s->v, kParamsPadded, 0.9f, 0.999f, 1e-8f,
                          fs, st);
        refresh_bf16(s);
        launch_fit_end(loss_steps, s->loss, fs, st);
    };
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && st != nullptr) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            one_step();
            const cudaError_t le = cudaGetLastError();
            e = cudaStreamEndCapture(st, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        for (int64_t k = 0; e == cudaSuccess && k < total; ++k) e = cudaGraphLaunch(exec, st);
        if (exec) cudaGraphExecDestroy(exec);
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
cudaError_t enqueue_surrogate_state(nmodl_mech* m, double dt, const double* v) {
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
    e = launch_surrogate_step(a, c->stream);
    if (e != cudaSuccess) return e;
    const nmodl_options& o = c->opt;
    launch_kin9_state(o.precision, m->d_kd, m->kd, m->n, m->d_ni, v, m->d_states, m->stride, dt,
                      nullptr, o.newton_tol, o.newton_max_iter, o.ir_max, m->d_fb_list, m->n,
                      m->d_fb_count, m->d_cnt, c->d_err, c->stream);
    return cudaGetLastError();
}
}  // namespace nmodl
