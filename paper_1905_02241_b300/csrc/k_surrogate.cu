// k_surrogate.cu -- learned stand-in for the kinetic Newton solve.
//
// One implicit Euler step of the 9-state scheme has the exact increment
// dx* = J^-1 z with z = dt A(v) x and J = I - dt A column-stochastic, so
// ||dx*||_1 <= s = ||z||_1.  In the scaled form the MLP (3 hidden layers of
// 128, SiLU) sees v_n, dt_n and the 9 states as the normalised explicit
// increment z/s, and its 9 outputs y give dx = s * y: the target J^-1 z / s
// is then a smooth (bilinear) function of its inputs.  In the raw form the
// network sees the states x and predicts dx = y directly.
// x_hat = P(x + dx) with P the Euclidean projection onto the probability
// simplex (Held, Wolfe & Crowder 1974).  The implicit Euler
// residual F(x_hat) = x_hat - x - dt A x_hat decides: ||F||_1 <= tol keeps
// x_hat (then ||x_hat - x*||_1 <= ||J^-1||_1 ||F||_1 = ||F||_1), otherwise the
// instance goes on a fallback list for the Newton kernel.
//
// k_surrogate_step: persistent CTAs (one per SM), 16 warps, weights staged once in shared
// memory (bf16, rows padded by 16 bytes so ldmatrix is conflict-free).  A
// warp owns 16 instances; the accumulator fragments of one layer are the A
// fragments of the next (m16n8k16 C and A layouts coincide pairwise), so
// activations never leave registers.
#include "kernels.cuh"
#include "mlp.cuh"

namespace nmodl {

namespace {
constexpr int kWarps = 16;  // 512 threads, 128 registers: one CTA per SM
constexpr int P1 = kIn + 8;    // W1 row pitch (elements)
constexpr int PH = kHid + 8;   // W2, W3, W4 row pitch
constexpr int kSmemW = (kHid * P1 + 2 * kHid * PH + kOut * PH) * 2;
constexpr int kSmemB = (3 * kHid + kOut) * 4;
constexpr int kWarpFloats = 32 * 16 + 32 * 24 + 32 * 9 + 32 + 32 * 9;
constexpr int kSmemY = kWarps * kWarpFloats * 4;
constexpr int kSmemTotal = kSmemW + kSmemB + kSmemY;
}  // namespace

// FP32 rates dt*k of the 24 transitions and (dt A) x for a state x.
__device__ __forceinline__ void kin_rates_f(const Kin9D& K, float vf, float dtf,
                                            float (&dkf)[kKinEdges], float (&dkb)[kKinEdges]) {
#pragma unroll
    for (int e = 0; e < kKinEdges; ++e) {
        dkf[e] = dtf * ((float)K.af[e] * __expf((float)K.bf[e] * vf));
        dkb[e] = dtf * ((float)K.ab[e] * __expf(-(float)K.bb[e] * vf));
    }
}
__device__ __forceinline__ void dtAx_f(const float (&dkf)[kKinEdges],
                                       const float (&dkb)[kKinEdges], const float* x,
                                       float (&z)[9]) {
#pragma unroll
    for (int a = 0; a < 9; ++a) z[a] = 0.f;
#pragma unroll
    for (int e = 0; e < kKinEdges; ++e) {
        const int lo = edge_lo(e), hi = edge_hi(e);
        const float f = dkf[e] * x[lo], b = dkb[e] * x[hi];
        z[hi] += f - b;
        z[lo] += b - f;
    }
}

__device__ __forceinline__ float l1_9(const float (&z)[9]) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) s += fabsf(z[a]);
    return s;
}

// Network inputs (11) and output scale s of one instance: v_n, dt_n, then
// z/s (scaled form; zero when s == 0) or x (raw form).
__device__ __forceinline__ float sur_inputs(int scaled, float vf, float dtf,
                                            const float (&xf)[9], const float (&z)[9],
                                            float* feat) {
    feat[0] = (vf + kVShift) * (1.0f / kVScale);
    feat[1] = (dtf - kDtShift) * (1.0f / kDtScale);
    if (!scaled) {
#pragma unroll
        for (int a = 0; a < 9; ++a) feat[2 + a] = xf[a];
        return 1.0f;
    }
    const float s = l1_9(z);
    const float inv = s > 0.f ? 1.0f / s : 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) feat[2 + a] = z[a] * inv;
    return s;
}

// Euclidean projection of w onto {x >= 0, sum x = 1}: theta is (S_j - 1)/c_j
// for the largest set {i : w_i >= w_j} whose smallest member stays positive.
__device__ __forceinline__ void project_simplex9(float (&w)[9]) {
    float theta = -1e30f;
    int best = 0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        float S = 0.f;
        int c = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            if (w[i] >= w[j]) {
                S += w[i];
                ++c;
            }
        const float th = (S - 1.0f) / (float)c;
        if (w[j] - th > 0.f && c > best) {
            best = c;
            theta = th;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) w[i] = fmaxf(w[i] - theta, 0.f);
}

__global__ void __launch_bounds__(kWarps * 32, 1) k_surrogate_step(SurArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* W1s = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* W2s = W1s + kHid * P1;
    __nv_bfloat16* W3s = W2s + kHid * PH;
    __nv_bfloat16* W4s = W3s + kHid * PH;
    float* b1s = reinterpret_cast<float*>(smem + kSmemW);
    float* b2s = b1s + kHid;
    float* b3s = b2s + kHid;
    float* b4s = b3s + kHid;
    float* warp_all = b4s + kOut;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // ---- stage weights (16-byte row chunks) and biases
    auto stage = [&](const __nv_bfloat16* src, __nv_bfloat16* dst, int rows, int cols, int pitch) {
        const int ch = cols / 8;
        for (int c = tid; c < rows * ch; c += blockDim.x) {
            const int r = c / ch, cc = (c % ch) * 8;
            *reinterpret_cast<uint4*>(dst + r * pitch + cc) =
                *reinterpret_cast<const uint4*>(src + r * cols + cc);
        }
    };
    // Hidden layers are staged as (W/2, b/2): the accumulator is then
    // h = z/2 and SiLU(z) = z sigma(z) = h + h tanh(h), one tanh and one FMA
    // (halving a bf16 is exact, so the products match the training forward).
    auto stage_half = [&](const __nv_bfloat16* src, __nv_bfloat16* dst, int rows, int cols,
                          int pitch) {
        const int ch = cols / 2;
        for (int c = tid; c < rows * ch; c += blockDim.x) {
            const int r = c / ch, cc = (c % ch) * 2;
            __nv_bfloat162 w = *reinterpret_cast<const __nv_bfloat162*>(src + r * cols + cc);
            *reinterpret_cast<__nv_bfloat162*>(dst + r * pitch + cc) =
                __hmul2(w, __floats2bfloat162_rn(0.5f, 0.5f));
        }
    };
    stage_half(a.wbf + kBfW1, W1s, kHid, kIn, P1);
    stage_half(a.wbf + kBfW2, W2s, kHid, kHid, PH);
    stage_half(a.wbf + kBfW3, W3s, kHid, kHid, PH);
    stage(a.wbf + kBfW4, W4s, kOut, kHid, PH);
    for (int i = tid; i < kHid; i += blockDim.x) {
        b1s[i] = 0.5f * a.params[kOffB1 + i];
        b2s[i] = 0.5f * a.params[kOffB2 + i];
        b3s[i] = 0.5f * a.params[kOffB3 + i];
    }
    if (tid < kOut) b4s[tid] = a.params[kOffB4 + tid];
    __syncthreads();

    const Kin9D& K = *a.kd;
    const float dtf = (float)a.dt;
    const int g = lane >> 2, t = lane & 3, q = lane >> 3, r8 = lane & 7;
    // per-warp staging of 32 instances: features [32][16], rates [32][24],
    // x [32][9], scale [32], outputs [32][9]
    float* wsm = warp_all + warp * kWarpFloats;
    float* feat = wsm;
    float* rates = feat + 32 * 16;
    float* xs = rates + 32 * 2 * kKinEdges;
    float* ss = xs + 32 * 9;
    float* ys = ss + 32;
    const int64_t stride_w = (int64_t)gridDim.x * kWarps * 32;

    for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32; base < a.n;
         base += stride_w) {
        // ---- one lane per instance: rates, dt A x, scale, network inputs
        {
            const int64_t i = base + lane;
            float* f = feat + lane * 16;
            if (i < a.n) {
                float xf[9], dkf[kKinEdges], dkb[kKinEdges], z[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) xf[k] = d2f_int(a.st[k * a.stride + i]);
                const float vf = d2f_int(a.v[a.ni[i]]);
                kin_rates_f(K, vf, dtf, dkf, dkb);
                dtAx_f(dkf, dkb, xf, z);
                ss[lane] = sur_inputs(a.scaled, vf, dtf, xf, z, f);
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    rates[lane * 24 + e] = dkf[e];
                    rates[lane * 24 + 12 + e] = dkb[e];
                }
#pragma unroll
                for (int k = 0; k < 9; ++k) xs[lane * 9 + k] = xf[k];
            } else {
#pragma unroll
                for (int k = 0; k < kInRaw; ++k) f[k] = 0.f;
            }
#pragma unroll
            for (int k = kInRaw; k < 16; ++k) f[k] = 0.f;
        }
        __syncwarp();
        // ---- the MLP on rows 0..15, then 16..31
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const float* fh = feat + half * 16 * 16;
            uint32_t afr[4];
            afr[0] = pack_bf16(fh[g * 16 + 2 * t], fh[g * 16 + 2 * t + 1]);
            afr[1] = pack_bf16(fh[(g + 8) * 16 + 2 * t], fh[(g + 8) * 16 + 2 * t + 1]);
            afr[2] = pack_bf16(fh[g * 16 + 2 * t + 8], fh[g * 16 + 2 * t + 9]);
            afr[3] = pack_bf16(fh[(g + 8) * 16 + 2 * t + 8], fh[(g + 8) * 16 + 2 * t + 9]);
            float acc[16][4];
            // accumulators start at the (halved) bias of their column
            auto init_bias = [&](const float* bias) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float2 bb = *reinterpret_cast<const float2*>(bias + 8 * j + 2 * t);
                    acc[j][0] = bb.x;
                    acc[j][1] = bb.y;
                    acc[j][2] = bb.x;
                    acc[j][3] = bb.y;
                }
            };
            init_bias(b1s);
#pragma unroll
            for (int np = 0; np < 8; ++np) {
                uint32_t b[4];
                ldsm_x4(b, W1s + (16 * np + r8 + (q >> 1) * 8) * P1 + (q & 1) * 8);
                mma_bf16_16816(acc[2 * np], afr, b[0], b[1]);
                mma_bf16_16816(acc[2 * np + 1], afr, b[2], b[3]);
            }
            // C fragments of output tiles 2kk and 2kk+1 are, in this order,
            // the A fragment (a0a1, a2a3, a4a5, a6a7) of k-slice kk of the
            // next layer
            uint32_t ah[8][4];
            auto silu_h = [](float h) { return fmaf(h, tanh_hw(h), h); };
            auto to_frags = [&]() {
#pragma unroll
                for (int kk = 0; kk < 8; ++kk)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = 2 * kk + h;
                        ah[kk][2 * h] = pack_bf16(silu_h(acc[j][0]), silu_h(acc[j][1]));
                        ah[kk][2 * h + 1] = pack_bf16(silu_h(acc[j][2]), silu_h(acc[j][3]));
                    }
            };
            auto hidden = [&](const __nv_bfloat16* Ws, const float* bias) {
                init_bias(bias);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk)
#pragma unroll
                    for (int np = 0; np < 8; ++np) {
                        uint32_t b[4];
                        ldsm_x4(b, Ws + (16 * np + r8 + (q >> 1) * 8) * PH + 16 * kk + (q & 1) * 8);
                        mma_bf16_16816(acc[2 * np], ah[kk], b[0], b[1]);
                        mma_bf16_16816(acc[2 * np + 1], ah[kk], b[2], b[3]);
                    }
            };
            to_frags();
            hidden(W2s, b2s);
            to_frags();
            hidden(W3s, b3s);
            to_frags();
            float o[2][4];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) o[j][e] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                uint32_t b[4];
                ldsm_x4(b, W4s + (r8 + (q >> 1) * 8) * PH + 16 * kk + (q & 1) * 8);
                mma_bf16_16816(o[0], ah[kk], b[0], b[1]);
                mma_bf16_16816(o[1], ah[kk], b[2], b[3]);
            }
            float* yh = ys + half * 16 * 9;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int col = 8 * j + 2 * t + e;
                        if (col < kOutRaw) yh[(g + 8 * h) * 9 + col] = o[j][2 * h + e] + b4s[col];
                    }
        }
        __syncwarp();
        // ---- projection, residual, decision (one lane per instance)
        bool fail = false;
        const int64_t i = base + lane;
        if (i < a.n) {
            float xf[9], w[9], dkf[kKinEdges], dkb[kKinEdges], z[9];
#pragma unroll
            for (int e = 0; e < kKinEdges; ++e) {
                dkf[e] = rates[lane * 24 + e];
                dkb[e] = rates[lane * 24 + 12 + e];
            }
            const float s = ss[lane];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                xf[k] = xs[lane * 9 + k];
                w[k] = xf[k] + s * ys[lane * 9 + k];
            }
            project_simplex9(w);
            dtAx_f(dkf, dkb, w, z);
            float rn = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) rn += fabsf(w[k] - xf[k] - z[k]);
            fail = !(rn <= a.tol);
            if (!fail) {
#pragma unroll
                for (int k = 0; k < 9; ++k) a.st[k * a.stride + i] = f2d_int(w[k]);
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, fail);
        if (mask) {
            int pos = 0;
            if (lane == 0) {
                pos = atomicAdd(a.fb_count, __popc(mask));
                atomicAdd(a.fb_total, (unsigned long long)__popc(mask));
            }
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (fail) a.fb_list[pos + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
        }
        __syncwarp();
    }
}

// Called when a surrogate is created (outside any stream capture).
cudaError_t surrogate_prepare() {
    return cudaFuncSetAttribute(k_surrogate_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemTotal);
}

cudaError_t launch_surrogate_step(const SurArgs& a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    int sms = 148;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (a.n + 31) / 32;
    int64_t grid = std::min<int64_t>((int64_t)sms, (groups + kWarps - 1) / kWarps);
    if (grid < 1) grid = 1;
    k_surrogate_step<<<(int)grid, kWarps * 32, kSmemTotal, s>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------- training pairs

__global__ void k_make_pairs(const Kin9D* __restrict__ kd, int64_t n,
                             const double* __restrict__ v, const double* __restrict__ dt,
                             const double* __restrict__ x, const double* __restrict__ y,
                             int64_t stride, int scaled, float* X, float* T) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float xf[9], dkf[kKinEdges], dkb[kKinEdges], z[9], f[kInRaw];
#pragma unroll
    for (int k = 0; k < 9; ++k) xf[k] = (float)x[k * stride + i];
    const float vf = (float)v[i], dtf = (float)dt[i];
    kin_rates_f(*kd, vf, dtf, dkf, dkb);
    dtAx_f(dkf, dkb, xf, z);
    const float s = sur_inputs(scaled, vf, dtf, xf, z, f);
#pragma unroll
    for (int k = 0; k < kInRaw; ++k) X[i * kInRaw + k] = f[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double inc = y[k * stride + i] - x[k * stride + i];
        T[i * kOutRaw + k] = s > 0.f ? (float)(inc / (double)s) : 0.f;
    }
}

void launch_make_pairs(const Kin9D* kd, int64_t n, const double* v, const double* dt,
                       const double* x, const double* y, int64_t stride, int scaled,
                       float* X, float* T, cudaStream_t s) {
    if (n == 0) return;
    k_make_pairs<<<(int)((n + 127) / 128), 128, 0, s>>>(kd, n, v, dt, x, y, stride, scaled, X, T);
}

}  // namespace nmodl
