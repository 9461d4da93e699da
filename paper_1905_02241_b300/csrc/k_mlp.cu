// k_mlp.cu -- BF16 tensor-core training kernels of the kinetic surrogate
// MLP (11 -> 128 -> 128 -> 128 -> 9, SiLU), FP32 accumulation and FP32
// master weights.  Shapes are padded to multiples of 16 (input 11 -> 16,
// output 9 -> 16) with zero weights, which stay exactly zero because their
// gradients are exactly zero.
//
//  k_gemm<TA, TB, EPI>  C = op(A) op(B), op = identity or transpose of the
//                       stored row-major matrix; split-K over gridDim.z;
//                       epilogues: FP32 partial, bias + SiLU (stores the
//                       pre-activation Z and bf16 H), bias only, and
//                       delta * SiLU'(Z) (bf16)
//  k_reduce_splits      deterministic sum of split-K partials
//  k_pack_input         [n][11] FP32 features -> [n][16] bf16
//  k_loss_delta         out - target, 0.5 sum^2 / B, delta (bf16)
//  k_colsum_partial     bias gradients (partial column sums of delta)
//  k_adam               Adam (Kingma & Ba 2015) on the FP32 master weights,
//                       refreshing the bf16 copies used by the GEMMs
#include "kernels.cuh"
#include "mlp.cuh"

namespace nmodl {

namespace {
constexpr int BM = 64, BN = 64, BK = 32;
constexpr int kPad = 8;
}  // namespace

template <int TA, int TB, int EPI>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
    // A tile: TA == 0 -> [BM][BK + pad] (rows m); TA == 1 -> [BK][BM + pad] (rows k)
    constexpr int A_ROWS = TA ? BK : BM, A_COLS = TA ? BM : BK, PA = A_COLS + kPad;
    constexpr int B_ROWS = TB ? BK : BN, B_COLS = TB ? BN : BK, PB = B_COLS + kPad;
    __shared__ __align__(16) __nv_bfloat16 As[2][A_ROWS * PA];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][B_ROWS * PB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * g.k_per_split;
    const int kb1 = min(g.K, kb0 + g.k_per_split);

    auto load_tile = [&](int buf, int k0) {
        // A
        constexpr int A_CH = A_ROWS * (A_COLS / 8);
        for (int c = tid; c < A_CH; c += 128) {
            const int r = c / (A_COLS / 8), cc = (c % (A_COLS / 8)) * 8;
            int gr, gc, rmax, cmax;
            if (TA == 0) { gr = m0 + r; gc = k0 + cc; rmax = g.M; cmax = kb1; }
            else { gr = k0 + r; gc = m0 + cc; rmax = kb1; cmax = g.M; }
            const bool ok = gr < rmax && gc < cmax;
            const __nv_bfloat16* src = g.A + (ok ? ((int64_t)gr * g.lda + gc) : 0);
            cp_async16(&As[buf][r * PA + cc], src, ok ? 16 : 0);
        }
        constexpr int B_CH = B_ROWS * (B_COLS / 8);
        for (int c = tid; c < B_CH; c += 128) {
            const int r = c / (B_COLS / 8), cc = (c % (B_COLS / 8)) * 8;
            int gr, gc, rmax, cmax;
            if (TB == 0) { gr = n0 + r; gc = k0 + cc; rmax = g.N; cmax = kb1; }
            else { gr = k0 + r; gc = n0 + cc; rmax = kb1; cmax = g.N; }
            const bool ok = gr < rmax && gc < cmax;
            const __nv_bfloat16* src = g.B + (ok ? ((int64_t)gr * g.ldb + gc) : 0);
            cp_async16(&Bs[buf][r * PB + cc], src, ok ? 16 : 0);
        }
        cp_async_commit();
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    const int nk = (kb1 - kb0 + BK - 1) / BK;
    if (nk > 0) load_tile(0, kb0);
    for (int it = 0; it < nk; ++it) {
        const int buf = it & 1;
        if (it + 1 < nk) {
            load_tile(buf ^ 1, kb0 + (it + 1) * BK);
            cp_async_wait_1();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const __nv_bfloat16* as = As[buf];
        const __nv_bfloat16* bs = Bs[buf];
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bf[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int mt = wm * 32 + i * 16;
                const int q = lane >> 3, r = lane & 7;
                if (TA == 0)
                    ldsm_x4(af[i], as + (mt + r + (q & 1) * 8) * PA + ks + (q >> 1) * 8);
                else
                    ldsm_x4_t(af[i], as + (ks + r + (q >> 1) * 8) * PA + mt + (q & 1) * 8);
            }
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                const int nt = wn * 32 + jp * 16;
                const int q = lane >> 3, r = lane & 7;
                if (TB == 0)
                    ldsm_x4(bf[jp], bs + (nt + r + (q >> 1) * 8) * PB + ks + (q & 1) * 8);
                else
                    ldsm_x4_t(bf[jp], bs + (ks + r + (q & 1) * 8) * PB + nt + (q >> 1) * 8);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16_16816(acc[i][j], af[i], bf[j >> 1][(j & 1) * 2],
                                   bf[j >> 1][(j & 1) * 2 + 1]);
        }
        __syncthreads();
    }

    // ---- epilogue
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm * 32 + i * 16 + gq + h * 8;
                const int col = n0 + wn * 32 + j * 8 + tq * 2;
                if (row >= g.M || col >= g.N) continue;
                float v0 = acc[i][j][h * 2], v1 = acc[i][j][h * 2 + 1];
                if (EPI == kEpiPartial) {
                    float* o = g.Cf + (int64_t)blockIdx.z * g.M * g.ldc + (int64_t)row * g.ldc + col;
                    o[0] = v0;
                    o[1] = v1;
                } else if (EPI == kEpiBiasSilu) {
                    v0 += g.bias[col];
                    v1 += g.bias[col + 1];
                    float* z = g.Cf + (int64_t)row * g.ldc + col;
                    z[0] = v0;
                    z[1] = v1;
                    *reinterpret_cast<uint32_t*>(g.Ch + (int64_t)row * g.ldch + col) =
                        pack_bf16(silu_f(v0), silu_f(v1));
                } else if (EPI == kEpiBias) {
                    float* o = g.Cf + (int64_t)row * g.ldc + col;
                    o[0] = v0 + g.bias[col];
                    o[1] = v1 + g.bias[col + 1];
                } else {  // kEpiDsilu
                    const float* z = g.Zin + (int64_t)row * g.ldz + col;
                    *reinterpret_cast<uint32_t*>(g.Ch + (int64_t)row * g.ldch + col) =
                        pack_bf16(v0 * dsilu_f(z[0]), v1 * dsilu_f(z[1]));
                }
            }
}

// out[i] = sum_z part[z][i] in order z = 0, 1, ...
__global__ void k_reduce_splits(const float* __restrict__ part, int splits, int64_t count,
                                float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(int64_t)z * count + i];
        out[i] = s;
    }
}

__global__ void k_pack_input(const float* __restrict__ X, int64_t n, __nv_bfloat16* H0,
                             FitSched fs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (fs.active) X += (*fs.step % fs.steps_per_epoch) * n * kInRaw;
#pragma unroll
    for (int f = 0; f < kIn; f += 2) {
        const float a = f < kInRaw ? X[i * kInRaw + f] : 0.f;
        const float b = f + 1 < kInRaw ? X[i * kInRaw + f + 1] : 0.f;
        *reinterpret_cast<uint32_t*>(H0 + i * kIn + f) = pack_bf16(a, b);
    }
}

// delta[b][c] = (out - t)/B for c < 9, 0 otherwise; per-block partial loss.
__global__ void k_loss_delta(const float* __restrict__ out, const float* __restrict__ T,
                             int64_t B, __nv_bfloat16* delta, float* block_loss,
                             FitSched fs) {
    __shared__ float red[256];
    if (fs.active) T += (*fs.step % fs.steps_per_epoch) * B * kOutRaw;
    float l = 0.f;
    const float invB = 1.0f / (float)B;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < kOut; c += 2) {
            float d0 = 0.f, d1 = 0.f;
            if (c < kOutRaw) {
                const float e = out[b * kOut + c] - T[b * kOutRaw + c];
                l += e * e;
                d0 = e * invB;
            }
            if (c + 1 < kOutRaw) {
                const float e = out[b * kOut + c + 1] - T[b * kOutRaw + c + 1];
                l += e * e;
                d1 = e * invB;
            }
            *reinterpret_cast<uint32_t*>(delta + b * kOut + c) = pack_bf16(d0, d1);
        }
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_loss[blockIdx.x] = 0.5f * red[0] * invB;
}

// part[blk][c] = sum of delta[b][c] over rows b of block blk (rows_per_block)
__global__ void k_colsum_partial(const __nv_bfloat16* __restrict__ delta, int64_t B, int N,
                                 int rows_per_block, float* part) {
    const int c = threadIdx.x;
    if (c >= N) return;
    const int64_t b0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t b1 = min(B, b0 + rows_per_block);
    float s = 0.f;
    for (int64_t b = b0; b < b1; ++b) s += __bfloat162float(delta[b * N + c]);
    part[(int64_t)blockIdx.x * N + c] = s;
}

__global__ void k_adam(float* p, const float* __restrict__ grad, float* m, float* v,
                       int64_t count, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * gr;
        const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// Adam with the learning rate and bias corrections of the run's current
// step: lr = lr_min + (lr0 - lr_min)(1 + cos(pi k / total))/2, t = t0 + k + 1.
__global__ void k_adam_sched(float* p, const float* __restrict__ grad, float* m, float* v,
                             int64_t count, float b1, float b2, float eps, FitSched fs) {
    const int64_t k = *fs.step;
    const float lr = fs.lr_min + 0.5f * (fs.lr0 - fs.lr_min) *
                                     (1.0f + cosf(3.14159265358979f * (float)k / (float)fs.total));
    const float t = (float)(fs.t0 + k + 1);
    const float bc1 = 1.f - powf(b1, t), bc2 = 1.f - powf(b2, t);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * gr;
        const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void k_fit_end(float* loss_steps, const float* loss, FitSched fs) {
    loss_steps[*fs.step] = *loss;
    *fs.step += 1;
}

__global__ void k_to_bf16(const float* __restrict__ src, int64_t count, __nv_bfloat16* dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// ------------------------------------------------------------ launchers

template <int TA, int TB, int EPI>
static void gemm_launch(const GemmArgs& g, int splits, cudaStream_t s) {
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, splits);
    k_gemm<TA, TB, EPI><<<grid, 128, 0, s>>>(g);
}

void launch_gemm(int ta, int tb, int epi, const GemmArgs& g, int splits, cudaStream_t s) {
    const int code = ta * 100 + tb * 10 + epi;
    switch (code) {
    case 0 * 100 + 0 * 10 + kEpiBiasSilu: gemm_launch<0, 0, kEpiBiasSilu>(g, splits, s); break;
    case 0 * 100 + 0 * 10 + kEpiBias: gemm_launch<0, 0, kEpiBias>(g, splits, s); break;
    case 0 * 100 + 1 * 10 + kEpiDsilu: gemm_launch<0, 1, kEpiDsilu>(g, splits, s); break;
    case 1 * 100 + 1 * 10 + kEpiPartial: gemm_launch<1, 1, kEpiPartial>(g, splits, s); break;
    case 0 * 100 + 0 * 10 + kEpiPartial: gemm_launch<0, 0, kEpiPartial>(g, splits, s); break;
    case 0 * 100 + 1 * 10 + kEpiPartial: gemm_launch<0, 1, kEpiPartial>(g, splits, s); break;
    case 1 * 100 + 0 * 10 + kEpiPartial: gemm_launch<1, 0, kEpiPartial>(g, splits, s); break;
    default: break;
    }
}

void launch_reduce_splits(const float* part, int splits, int64_t count, float* out,
                          cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((count + 255) / 256, 148 * 8);
    k_reduce_splits<<<grid, 256, 0, s>>>(part, splits, count, out);
}

void launch_pack_input(const float* X, int64_t n, __nv_bfloat16* H0, cudaStream_t s,
                       FitSched fs) {
    if (n == 0) return;
    k_pack_input<<<(int)((n + 255) / 256), 256, 0, s>>>(X, n, H0, fs);
}

int launch_loss_delta(const float* out, const float* T, int64_t B, __nv_bfloat16* delta,
                      float* block_loss, cudaStream_t s, FitSched fs) {
    const int grid = (int)std::min<int64_t>((B + 255) / 256, 256);
    k_loss_delta<<<grid, 256, 0, s>>>(out, T, B, delta, block_loss, fs);
    return grid;
}

void launch_adam_sched(float* p, const float* grad, float* m, float* v, int64_t count,
                       float b1, float b2, float eps, FitSched fs, cudaStream_t s) {
    k_adam_sched<<<148, 256, 0, s>>>(p, grad, m, v, count, b1, b2, eps, fs);
}

void launch_fit_end(float* loss_steps, const float* loss, FitSched fs, cudaStream_t s) {
    k_fit_end<<<1, 1, 0, s>>>(loss_steps, loss, fs);
}

void launch_colsum(const __nv_bfloat16* delta, int64_t B, int N, float* part, float* out,
                   cudaStream_t s) {
    const int rpb = 256;
    const int blocks = (int)((B + rpb - 1) / rpb);
    k_colsum_partial<<<blocks, 128, 0, s>>>(delta, B, N, rpb, part);
    launch_reduce_splits(part, blocks, N, out, s);
}

void launch_adam(float* p, const float* grad, float* m, float* v, int64_t count, float lr,
                 float b1, float b2, float eps, int step, cudaStream_t s) {
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    k_adam<<<148, 256, 0, s>>>(p, grad, m, v, count, lr, b1, b2, eps, bc1, bc2);
}

void launch_to_bf16(const float* src, int64_t count, __nv_bfloat16* dst, cudaStream_t s) {
    k_to_bf16<<<148, 256, 0, s>>>(src, count, dst);
}

}  // namespace nmodl
