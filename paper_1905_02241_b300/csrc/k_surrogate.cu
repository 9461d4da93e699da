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
// k_surrogate_step: persistent CTAs (one per SM) of four warpgroups; each
// warpgroup owns a tile of 128 instances, one thread per instance.  The MLP
// runs on the fifth-generation tensor cores: a single thread per warpgroup
// issues tcgen05.mma (M = 128, K = 16 per instruction) on bf16 operands in
// shared memory, the FP32 accumulator lives in tensor memory (128 columns per
// warpgroup), and every thread reads its own row back with tcgen05.ld for
// the bias + SiLU epilogue, which writes the next layer's A operand.  Weights
// (72 KB) are staged once per CTA.  Completion is signalled through one
// mbarrier per warpgroup; every wait is bounded and a timeout is latched as
// NMODL_ERR_TIMEOUT.
#include "kernels.cuh"
#include "mlp.cuh"
#include "tcgen05.cuh"

namespace nmodl {

namespace {
constexpr int kWG = 4;                 // warpgroups per CTA
constexpr int kThreads = 128 * kWG;    // one CTA per SM (shared memory bound)
constexpr int kTile = 128;             // instances per warpgroup tile (MMA M)
// shared-memory images (K-major, no swizzle; see tcgen05.cuh).  The layer
// inputs (K = 16) sit in columns 0..15 of the warpgroup's H image.  Biases
// enter through the MMAs: layer 1 through input columns 11 and 12 (= 1)
// against W1 columns holding the bias as a bf16 pair hi + lo; layers 2-4
// through one extra K = 16 MMA of ONE (columns 0, 1 = 1) against a bias
// image with hi, lo in columns 0, 1 (hi + lo equals the FP32 bias to 2^-17).
constexpr int kW1Bytes = kHid * kIn * 2;
constexpr int kWHBytes = kHid * kHid * 2;
constexpr int kW4Bytes = kOut * kHid * 2;
constexpr int kHBytes = kTile * kHid * 2;
constexpr int kOneBytes = kTile * 16 * 2;
constexpr int kBHBytes = kHid * 16 * 2;
constexpr int kB4Bytes = kOut * 16 * 2;
constexpr int kOffW1s = 0;
constexpr int kOffW2s = kOffW1s + kW1Bytes;
constexpr int kOffW3s = kOffW2s + kWHBytes;
constexpr int kOffW4s = kOffW3s + kWHBytes;
constexpr int kOffH = kOffW4s + kW4Bytes;
constexpr int kOffOne = kOffH + kWG * kHBytes;
constexpr int kOffB2i = kOffOne + kOneBytes;
constexpr int kOffB3i = kOffB2i + kBHBytes;
constexpr int kOffB4i = kOffB3i + kBHBytes;
constexpr int kOffRate = kOffB4i + kB4Bytes;  // 48 FP32 rate parameters
constexpr int kOffBar = kOffRate + 4 * kKinEdges * 4;
constexpr int kSmemTotal = kOffBar + kWG * 8 + 16;
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert(kSmemTotal <= 227 * 1024, "shared memory per block");
constexpr uint32_t kTmemCols = 128 * kWG;  // 512: the whole tensor memory of the SM
constexpr uint32_t kIdescHid = umma_idesc_bf16(128, kHid);
constexpr uint32_t kIdescOut = umma_idesc_bf16(128, kOut);
constexpr uint32_t kWaitPolls = 1u << 22;
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
// The same rates with the launch's constants folded: dt k = 2^(b' v + c')
// with b' = b log2(e) (negated for the backward rates) and c' = log2(dt a),
// so that each rate is one multiply-add and the hardware exp2 (kp: b'f, c'f,
// b'b, c'b, 12 each, staged once per CTA)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void kin_rates_folded(const float* kp, float vf,
                                                 float (&dkf)[kKinEdges], float (&dkb)[kKinEdges]) {
#pragma unroll
    for (int e = 0; e < kKinEdges; ++e) {
        dkf[e] = ex2_approx(fmaf(kp[e], vf, kp[kKinEdges + e]));
        dkb[e] = ex2_approx(fmaf(kp[2 * kKinEdges + e], vf, kp[3 * kKinEdges + e]));
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

// Euclidean projection of w onto {x >= 0, sum x = 1} by the sort-based
// method (Held, Wolfe & Crowder 1974; as described by Duchi et al. 2008):
// u = w sorted in descending order, S_k its prefix sums, rho the largest k
// with u_k k - (S_k - 1) > 0, theta = (S_rho - 1)/rho, x = max(w - theta, 0).
// The sort is Batcher's odd-even merge network for 16 inputs pruned to 9
// (padding would hold -inf and never move): 28 comparators, checked on all
// 2^9 zero-one inputs (the zero-one principle).
__device__ __forceinline__ void project_simplex9(float (&w)[9]) {
    constexpr int kNet[28][2] = {{0, 1}, {2, 3}, {0, 2}, {1, 3}, {1, 2}, {4, 5}, {6, 7},
                                 {4, 6}, {5, 7}, {5, 6}, {0, 4}, {2, 6}, {2, 4}, {1, 5},
                                 {3, 7}, {3, 5}, {1, 2}, {3, 4}, {5, 6}, {0, 8}, {4, 8},
                                 {2, 4}, {6, 8}, {3, 5}, {1, 2}, {3, 4}, {5, 6}, {7, 8}};
    float u[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = w[i];
#pragma unroll
    for (int c = 0; c < 28; ++c) {
        const float hi = fmaxf(u[kNet[c][0]], u[kNet[c][1]]);
        const float lo = fminf(u[kNet[c][0]], u[kNet[c][1]]);
        u[kNet[c][0]] = hi;
        u[kNet[c][1]] = lo;
    }
    float S = 0.f, bestS = 0.f, bestC = 1.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        S += u[k];
        if (fmaf(u[k], (float)(k + 1), 1.0f - S) > 0.f) {
            bestS = S;
            bestC = (float)(k + 1);
        }
    }
    const float theta = (bestS - 1.0f) / bestC;
#pragma unroll
    for (int i = 0; i < 9; ++i) w[i] = fmaxf(w[i] - theta, 0.f);
}

__global__ void __launch_bounds__(kThreads, 1) k_surrogate_step(SurArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + kWG * 8);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid >> 7;        // warpgroup
    const int t = tid & 127;       // row of the warpgroup's tile
    // ---- stage the weights as K-major core-matrix images.  Hidden layers
    // are staged as (W/2, b/2): the accumulator is then h = z/2 and
    // SiLU(z) = z sigma(z) = h + h tanh(h) (halving a bf16 is exact).
    auto stage = [&](const __nv_bfloat16* src, int off, int rows, int K, bool half) {
        const int ch = K / 8;
        for (int c = tid; c < rows * ch; c += kThreads) {
            const int r = c / ch, k = (c % ch) * 8;
            uint4 w = *reinterpret_cast<const uint4*>(src + r * K + k);
            if (half) {
                __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
                for (int e = 0; e < 4; ++e) h2[e] = __hmul2(h2[e], __floats2bfloat162_rn(0.5f, 0.5f));
            }
            *reinterpret_cast<uint4*>(smem + off + umma_offset(r, k, K)) = w;
        }
    };
    stage(a.wbf + kBfW1, kOffW1s, kHid, kIn, true);
    stage(a.wbf + kBfW2, kOffW2s, kHid, kHid, true);
    stage(a.wbf + kBfW3, kOffW3s, kHid, kHid, true);
    stage(a.wbf + kBfW4, kOffW4s, kOut, kHid, false);
    // bias pairs: layer 1 into W1 columns 11, 12; layers 2-4 into their
    // bias images (columns 0, 1); ONE has ones in columns 0, 1
    auto put = [&](int off, int r, int k, int K, float x) {
        *reinterpret_cast<__nv_bfloat16*>(smem + off + umma_offset(r, k, K)) = __float2bfloat16_rn(x);
    };
    auto put_pair = [&](int off, int r, int k, int K, float b) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(b);
        put(off, r, k, K, b);
        put(off, r, k + 1, K, b - __bfloat162float(hi));
    };
    for (int i = tid; i < kTile * 16; i += kThreads) put(kOffOne, i / 16, i % 16, 16, (i % 16) < 2 ? 1.f : 0.f);
    for (int i = tid; i < kHid * 16; i += kThreads) {
        put(kOffB2i, i / 16, i % 16, 16, 0.f);
        put(kOffB3i, i / 16, i % 16, 16, 0.f);
    }
    for (int i = tid; i < kOut * 16; i += kThreads) put(kOffB4i, i / 16, i % 16, 16, 0.f);
    __syncthreads();
    for (int i = tid; i < kHid; i += kThreads) {
        put_pair(kOffW1s, i, kInRaw, kIn, 0.5f * a.params[kOffB1 + i]);
        put_pair(kOffB2i, i, 0, 16, 0.5f * a.params[kOffB2 + i]);
        put_pair(kOffB3i, i, 0, 16, 0.5f * a.params[kOffB3 + i]);
    }
    if (tid < kOut) put_pair(kOffB4i, tid, 0, 16, a.params[kOffB4 + tid]);
    float* kps = reinterpret_cast<float*>(smem + kOffRate);
    if (tid < kKinEdges) {
        const double kLog2e = 1.4426950408889634;  // log2(e)
        kps[tid] = (float)(a.kd->bf[tid] * kLog2e);
        kps[kKinEdges + tid] = (float)log2(a.dt * a.kd->af[tid]);
        kps[2 * kKinEdges + tid] = (float)(-a.kd->bb[tid] * kLog2e);
        kps[3 * kKinEdges + tid] = (float)log2(a.dt * a.kd->ab[tid]);
    }
    if (tid == 0) {
        for (int k = 0; k < kWG; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t d_tmem = tmem + 128u * g;                        // this warpgroup's columns
    const uint32_t t_row = d_tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes

    const float dtf = (float)a.dt;
    const uint32_t hb = sbase + kOffH + g * kHBytes;
    unsigned char* hp = smem + kOffH + g * kHBytes;
    const uint64_t one_desc = umma_desc(sbase + kOffOne, 128, 256);
    uint64_t* bar = &bars[g];
    const uint32_t bar_id = 1 + g;
    uint32_t phase = 0;
    bool timed_out = false;

    // operands written and earlier TMEM reads done -> the MMA may be issued
    auto publish = [&]() {
        fence_proxy_async_smem();
        tc_fence_before();
        bar_sync(bar_id, 128);
    };
    // every thread waits for the warpgroup's commit; all agree on timeouts
    auto wait_mma = [&]() -> bool {
        const bool ok = mbar_wait(bar, phase, kWaitPolls);
        phase ^= 1u;
        const bool bad = bar_any(bar_id, 128, !ok);
        tc_fence_after();
        return !bad;
    };
    // bias MMA (accumulator := bias), then the K = 128 product in 8 steps
    auto issue_layer = [&](int w_off, int b_off, uint32_t idesc) {
        if (t == 0) {
            tc_fence_after();
            umma_bf16(d_tmem, one_desc, umma_desc(sbase + b_off, 128, 256), idesc, 0);
#pragma unroll
            for (int j = 0; j < kHid / 16; ++j)
                umma_bf16(d_tmem, umma_desc(hb + 256 * j, 128, 16 * kHid),
                          umma_desc(sbase + w_off + 256 * j, 128, 16 * kHid), idesc, 1);
            umma_commit(bar);
        }
    };
    // accumulator row -> bias + SiLU -> bf16 row of the next A operand; the
    // TMEM load of the next 16 columns is in flight while the current 16 are
    // activated (wait::ld waits for every load issued before it)
    auto epilogue = [&]() {
        unsigned char* hrow = hp + (t >> 3) * (16 * kHid) + (t & 7) * 16;
        uint32_t ra[16], rb[16];
        auto act = [&](const uint32_t (&r)[16], int cb) {
            uint32_t pk[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float h0 = __uint_as_float(r[2 * e]), h1 = __uint_as_float(r[2 * e + 1]);
                pk[e] = pack_bf16(fmaf(h0, tanh_hw(h0), h0), fmaf(h1, tanh_hw(h1), h1));
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)
                *reinterpret_cast<uint4*>(hrow + ((cb >> 3) + q) * 128) =
                    make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        };
        tmem_ld16(t_row, ra);
        tmem_ld_wait();
#pragma unroll
        for (int cb = 0; cb < kHid; cb += 32) {
            tmem_ld16(t_row + cb + 16, rb);
            act(ra, cb);
            tmem_ld_wait();
            if (cb + 32 < kHid) tmem_ld16(t_row + cb + 32, ra);
            act(rb, cb + 16);
            tmem_ld_wait();
        }
    };

    const int64_t tile_stride = (int64_t)gridDim.x * kWG;
    for (int64_t tile = (int64_t)blockIdx.x * kWG + g; tile * kTile < a.n && !timed_out;
         tile += tile_stride) {
        const int64_t i = tile * kTile + t;
        const bool valid = i < a.n;
        // ---- inputs of this thread's instance
        float xf[9], dkf[kKinEdges], dkb[kKinEdges], s = 0.f;
        {
            float f[16], z[9];
#pragma unroll
            for (int k = 0; k < 16; ++k) f[k] = 0.f;
            if (valid) {
                double vd = a.v[a.ni[i]];
                if (a.step) {
                    // the node's current, rhs and d, and its diagonal update
                    // (node i holds this one instance), as the current
                    // update, the v update and this state update in turn
                    const double g = a.gbar * a.st[a.open * a.stride + i];
                    const double r = 0.0 - g * (vd - a.e);
                    const double dd = g + a.cmdt;
                    if (!finite_int(r) || !finite_int(dd)) latch_error(a.err, NMODL_ERR_NONFINITE);
                    a.rhs[i] = r;
                    a.d[i] = dd;
                    if (!a.clamp) {
                        vd = vd + ddiv_fast(r, dd);
                        if (!finite_int(vd)) latch_error(a.err, NMODL_ERR_NONFINITE);
                        a.v_step[i] = vd;
                    }
                }
#pragma unroll
                for (int k = 0; k < 9; ++k) xf[k] = d2f_int(a.st[k * a.stride + i]);
                const float vf = d2f_int(vd);
                kin_rates_folded(kps, vf, dkf, dkb);
                dtAx_f(dkf, dkb, xf, z);
                s = sur_inputs(a.scaled, vf, dtf, xf, z, f);
            }
            f[kInRaw] = 1.f;      // bias pair of layer 1
            f[kInRaw + 1] = 1.f;
            unsigned char* arow = hp + (t >> 3) * (16 * kHid) + (t & 7) * 16;
#pragma unroll
            for (int q = 0; q < 2; ++q)
                *reinterpret_cast<uint4*>(arow + q * 128) =
                    make_uint4(pack_bf16(f[8 * q], f[8 * q + 1]), pack_bf16(f[8 * q + 2], f[8 * q + 3]),
                               pack_bf16(f[8 * q + 4], f[8 * q + 5]), pack_bf16(f[8 * q + 6], f[8 * q + 7]));
        }
        publish();
        if (t == 0) {
            tc_fence_after();
            umma_bf16(d_tmem, umma_desc(hb, 128, 16 * kHid), umma_desc(sbase + kOffW1s, 128, 16 * kIn),
                      kIdescHid, 0);
            umma_commit(bar);
        }
        if (!wait_mma()) { timed_out = true; break; }
        epilogue();
        publish();
        issue_layer(kOffW2s, kOffB2i, kIdescHid);
        if (!wait_mma()) { timed_out = true; break; }
        epilogue();
        publish();
        issue_layer(kOffW3s, kOffB3i, kIdescHid);
        if (!wait_mma()) { timed_out = true; break; }
        epilogue();
        publish();
        issue_layer(kOffW4s, kOffB4i, kIdescOut);
        if (!wait_mma()) { timed_out = true; break; }
        uint32_t yo[16];
        tmem_ld16(t_row, yo);
        tmem_ld_wait();
        // ---- projection, residual, decision (one thread per instance)
        bool fail = false;
        if (valid) {
            float w[9], z[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) w[k] = xf[k] + s * __uint_as_float(yo[k]);
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
            const int lane = tid & 31;
            int pos = 0;
            if (lane == 0) {
                pos = atomicAdd(a.fb_count, __popc(mask));
                atomicAdd(a.fb_total, (unsigned long long)__popc(mask));
            }
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (fail) a.fb_list[pos + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
        }
    }
    if (timed_out && t == 0) latch_error(a.err, NMODL_ERR_TIMEOUT);
    // ---- release the tensor memory
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
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
    const int64_t tiles = (a.n + kTile - 1) / kTile;
    int64_t grid = std::min<int64_t>((int64_t)sms, (tiles + kWG - 1) / kWG);
    if (grid < 1) grid = 1;
    k_surrogate_step<<<(int)grid, kThreads, kSmemTotal, s>>>(a);
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
