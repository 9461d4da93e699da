// k_train.cu -- training and batch forward of the kinetic surrogate MLP
// (11 -> 128 -> 128 -> 128 -> 9, SiLU) on the fifth-generation tensor cores.
//
// k_train_tiles: one CTA per SM, two warpgroups; each CTA takes a run of
// 128-row tiles of the minibatch.  Per tile, one thread issues every
// tcgen05.mma (bf16 operands in shared memory, FP32 accumulators in tensor
// memory) and the 256 threads run the epilogues (thread = row of the tile,
// warpgroup = half of the columns), reading the accumulators with
// tcgen05.ld:
//   forward   Z1 = H0 W1^T, H1 = SiLU(Z1), ... OUT = H3 W4^T (+ biases, fed
//             through the MMAs as bf16 hi/lo pairs against columns of ones)
//   loss      e = OUT - T, loss += e^2, D4 = e / n                 (bf16)
//   backward  D3 = (D4 W4) * SiLU'(Z3), D2 = (D3 W3) * SiLU'(Z2),
//             D1 = (D2 W2) * SiLU'(Z1)                            (bf16;
//             SiLU'(Z) kept by the forward pass in a global scratch in
//             FP16, 2^-11 relative, below the bf16 rounding of D)
//   gradients dW4^T += H3^T D4, dW3^T += H2^T D3, dW2^T += H1^T D2,
//             dW1 += D1^T H0, db2, db3 += D^T 1 (db1 comes with dW1 through
//             H0's column of ones; db4 as column sums on the CUDA cores)
// The weights, the bias pairs and the column of ones arrive as one image
// (kept in global memory in the shared-memory layout by the optimiser step)
// in four bulk copies on the copy engine, waited for only before the first
// MMA.  The same shared-memory image serves both orientations: an activation
// tile stored K-major for the forward product (K = features) is read
// MN-major by the gradient products, whose contraction runs over the 128
// rows of the tile; a weight image stored K-major for the forward (K = in)
// is read MN-major by the backward product (K = out).  The gradient
// accumulators stay in tensor memory over all tiles of the CTA and are
// written once per CTA; k_grad_adam sums the CTA partials in a fixed order
// (deterministic), then either stores the gradient or takes the Adam step
// (Kingma & Ba 2015) and refreshes the bf16 weight copies and the image.
// Every mbarrier wait is bounded; a timeout is latched as
// NMODL_ERR_TIMEOUT and the CTA stops.
#include "kernels.cuh"
#include "mlp.cuh"
#include "tcgen05.cuh"

namespace nmodl {

namespace {
constexpr int kTrGroups = 2;                  // warpgroups
constexpr int kTrThreads = 128 * kTrGroups;
constexpr int kTrRows = 128;                  // rows per tile (MMA M)
constexpr int kTrCols = 128 / kTrGroups;      // hidden columns per warpgroup
static_assert(kTrCols % 16 == 0, "epilogue chunks of 16 columns");
// shared-memory images (K-major core matrices, umma_offset), bytes
constexpr int kImW1 = kHid * kIn * 2, kImWH = kHid * kHid * 2, kImW4 = kOut * kHid * 2;
constexpr int kImH0 = kTrRows * kIn * 2, kImH = kTrRows * kHid * 2, kImD4 = kTrRows * kOut * 2;
constexpr int kImOne = kTrRows * 16 * 2, kImBH = kHid * 16 * 2, kImB4 = kOut * 16 * 2;
// the weight image (the first kImg bytes, as kept in global memory), then
// the activation images; every MMA operand starts on a 1024-byte boundary
constexpr int sW1 = 0, sW2 = sW1 + kImW1, sW3 = sW2 + kImWH, sW4 = sW3 + kImWH;
constexpr int sOne = sW4 + kImW4, sB2 = sOne + kImOne, sB3 = sB2 + kImBH, sB4 = sB3 + kImBH;
constexpr int kImg = sB4 + kImB4;
constexpr int kImgChunk = kImg / 4;  // four bulk copies
static_assert(kImg == kTrImgBytes && kImgChunk % 16 == 0, "weight image");
constexpr int sH0 = (kImg + 1023) / 1024 * 1024, sH1 = sH0 + kImH0, sH2 = sH1 + kImH;
constexpr int sH3 = sH2 + kImH, sD4 = sH3 + kImH;
static_assert(sB4 % 1024 == 0 && sH1 % 1024 == 0 && sD4 % 1024 == 0, "operand alignment");
constexpr int sRed = sD4 + kImD4;        // float [4 warps][16]: per-warp column sums
constexpr int sAcc = sRed + 4 * 16 * 4;  // float [16]: db4 (0..8) and sum e^2 (9) of the CTA
constexpr int sBar = sAcc + 16 * 4;      // two mbarriers, the tensor-memory address
constexpr int kTrSmem = sBar + 32;
static_assert(sBar % 8 == 0, "mbarrier alignment");
static_assert(kTrSmem <= 227 * 1024, "shared memory per block");
// tensor-memory columns: the working accumulator, then the gradient
// accumulators that live across the CTA's tiles (dW2, dW3 transposed: lane
// = input unit, column = output unit)
constexpr uint32_t cAcc = 0, cDW2 = 128, cDW3 = 256, cDW1 = 384, cDW4T = 400, cDB2 = 416,
                   cDB3 = 432;
constexpr uint32_t kTrTmemCols = 512;
constexpr uint32_t kTrPolls = 1u << 22;

// kind::f16 instruction descriptor, M = 128; bit 15 / 16: A / B MN-major
__host__ __device__ constexpr uint32_t tr_idesc(uint32_t N, bool a_mn, bool b_mn) {
    return umma_idesc_bf16(128, N) | (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u);
}
}  // namespace

// Descriptor of an image stored K-major with row width F (elements):
// read K-major (K = its columns; LBO 128 B between core matrices along K,
// SBO 16 F B between 8-row groups) or MN-major (K = its rows: core matrices
// 16 F B apart along K, 128 B apart along MN).
// The weight image entries of master parameter i (value x): a weight's bf16
// value at its place in its K-major image (W1's padding columns 11..15 are
// skipped: 11, 12 hold b1); a bias as the bf16 pair hi + lo, hi = bf16(x),
// lo = bf16(x - hi), in the two columns that meet the ones (W1's columns
// 11, 12 for b1; columns 0, 1 of the B2, B3, B4 images).
__device__ __forceinline__ void img_put(unsigned char* img, int i, float x) {
    auto put = [&](int off, int r, int k, int K, float y) {
        *reinterpret_cast<__nv_bfloat16*>(img + off + umma_offset(r, k, K)) = __float2bfloat16_rn(y);
    };
    auto pair = [&](int off, int r, int k, int K) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        put(off, r, k, K, x);
        put(off, r, k + 1, K, x - __bfloat162float(hi));
    };
    if (i < kOffB1) {
        const int o = (i - kOffW1) / kIn, k = (i - kOffW1) % kIn;
        if (k < kInRaw) put(sW1, o, k, kIn, x);
    } else if (i < kOffW2) {
        pair(sW1, i - kOffB1, kInRaw, kIn);
    } else if (i < kOffB2) {
        put(sW2, (i - kOffW2) / kHid, (i - kOffW2) % kHid, kHid, x);
    } else if (i < kOffW3) {
        pair(sB2, i - kOffB2, 0, 16);
    } else if (i < kOffB3) {
        put(sW3, (i - kOffW3) / kHid, (i - kOffW3) % kHid, kHid, x);
    } else if (i < kOffW4) {
        pair(sB3, i - kOffB3, 0, 16);
    } else if (i < kOffB4) {
        put(sW4, (i - kOffW4) / kHid, (i - kOffW4) % kHid, kHid, x);
    } else if (i < kParamsPadded) {
        pair(sB4, i - kOffB4, 0, 16);
    }
}

// The whole image from the master parameters (img zeroed beforehand): every
// parameter's entries, and the ones of the ONE image's columns 0, 1.
__global__ void k_train_image(const float* __restrict__ p, unsigned char* img) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParamsPadded + 2 * kTrRows;
         i += gridDim.x * blockDim.x) {
        if (i < kParamsPadded) {
            img_put(img, i, p[i]);
        } else {
            const int j = i - kParamsPadded;
            *reinterpret_cast<__nv_bfloat16*>(img + sOne + umma_offset(j / 2, j % 2, 16)) =
                __float2bfloat16_rn(1.f);
        }
    }
}

__device__ __forceinline__ uint64_t desc_k(uint32_t a, int F) { return umma_desc(a, 128, 16 * F); }
__device__ __forceinline__ uint64_t desc_mn(uint32_t a, int F) { return umma_desc(a, 16 * F, 128); }

// D (+)= A B^T over K = 16 ksteps: A, B images at a0, b0 with row widths
// aF, bF, each read K-major or MN-major; the start address moves 32 B x 8
// (two core matrices) per step along K in the K-major view, two 8-row
// groups (32 F B) in the MN-major view.
__device__ __forceinline__ void mma_run(uint32_t d, uint32_t a0, int aF, bool a_mn, uint32_t b0,
                                        int bF, bool b_mn, int ksteps, uint32_t id, bool acc) {
    for (int j = 0; j < ksteps; ++j) {
        const uint32_t aa = a0 + (uint32_t)j * (a_mn ? 32u * aF : 256u);
        const uint32_t bb = b0 + (uint32_t)j * (b_mn ? 32u * bF : 256u);
        umma_bf16(d, a_mn ? desc_mn(aa, aF) : desc_k(aa, aF), b_mn ? desc_mn(bb, bF) : desc_k(bb, bF),
                  id, (acc || j > 0) ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(kTrThreads, 1) k_train_tiles(TrainArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sb = smem_u32(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sBar);
    uint64_t* bar_w = bar + 1;  // the weight image's bulk copies
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + sBar + 16);
    float* red = reinterpret_cast<float*>(smem + sRed);
    float* accs = reinterpret_cast<float*>(smem + sAcc);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = tid & 127;  // row of the tile (tensor-memory lane)
    const int h = tid >> 7;   // warpgroup: hidden columns [kTrCols h, kTrCols (h + 1))
    const int n = (int)a.n;
    const float inv_n = 1.0f / (float)n;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar_w, 1);
        mbar_init_fence();
    }
    if (tid < 16) accs[tid] = 0.f;
    if (warp == 0) {
        tmem_alloc(tmem_slot, kTrTmemCols);
        tmem_relinquish();
    }
    const float* X = a.X;
    const float* T = a.T;
    if (a.fs.active) {
        const int64_t o = (*a.fs.step % a.fs.steps_per_epoch) * a.n;
        X += o * kInRaw;
        T += o * kOutRaw;
    }
    // ---- the weight image: four bulk copies, in flight during the setup
    // and the first tile's input stage
    if (tid == 0) {
        mbar_expect_tx(bar_w, kImg);
#pragma unroll
        for (int c = 0; c < 4; ++c) bulk_g2s(sb + c * kImgChunk, a.img + c * kImgChunk, kImgChunk, bar_w);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
    uint32_t phase = 0;
    bool timed_out = false, w_ready = false;

    // operands in shared memory written, earlier tensor-memory reads done
    auto publish = [&]() {
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
    };
    auto commit_wait = [&]() -> bool {
        if (tid == 0) umma_commit(bar);
        const bool ok = mbar_wait(bar, phase, kTrPolls);
        phase ^= 1u;
        const bool bad = __syncthreads_or(!ok);
        tc_fence_after();
        return !bad;
    };
    auto row_of = [&](int tile) { return (int64_t)tile * kTrRows + t; };

    const int tiles = (n + kTrRows - 1) / kTrRows;
    const int tile0 = blockIdx.x * a.tiles_per_cta;
    const int tile1 = min(tiles, tile0 + a.tiles_per_cta);
    // the CTA's gradient partials (mode 1), every entry of the padded layout
    float* P = a.part + (int64_t)blockIdx.x * kParamsPadded;
    // dW2, dW3 from their transposed accumulators: thread t holds input
    // unit t's gradients for this warpgroup's output units o, stored at
    // o * kHid + t -- for each o a warp's store is 128 contiguous bytes
    auto dump = [&](uint32_t col, float* dst) {  // dst: the matrix's entry (0, 0)
        uint32_t rb[2][16];
        tmem_ld16(lane_base + col + kTrCols * h, rb[0]);
#pragma unroll
        for (int cb = 0; cb < kTrCols; cb += 16) {
            const int o = kTrCols * h + cb;
            tmem_ld_wait(rb[(cb >> 4) & 1]);
            if (cb + 16 < kTrCols) tmem_ld16(lane_base + col + o + 16, rb[((cb >> 4) + 1) & 1]);
            const uint32_t* r = rb[(cb >> 4) & 1];
#pragma unroll
            for (int e = 0; e < 16; ++e) dst[(int64_t)(o + e) * kHid + t] = __uint_as_float(r[e]);
        }
    };
    bool dumped23 = false;
    for (int tile = tile0; tile < tile1 && !timed_out; ++tile) {
        const bool first = tile == tile0;
        const int64_t row = row_of(tile);
        const bool valid = row < n;
        // ---- inputs: row t of H0 (features, then the bias pair's ones)
        if (h == 0) {
            float f[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) f[k] = 0.f;
            if (valid) {
#pragma unroll
                for (int k = 0; k < kInRaw; ++k) f[k] = X[row * kInRaw + k];
                f[kInRaw] = 1.f;
                f[kInRaw + 1] = 1.f;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)
                *reinterpret_cast<uint4*>(smem + sH0 + umma_offset(t, 8 * q, kIn)) =
                    make_uint4(pack_bf16(f[8 * q], f[8 * q + 1]), pack_bf16(f[8 * q + 2], f[8 * q + 3]),
                               pack_bf16(f[8 * q + 4], f[8 * q + 5]), pack_bf16(f[8 * q + 6], f[8 * q + 7]));
        }
        publish();
        if (!w_ready) {  // the weight image landed (the MMA issuer waits)
            const bool bad = tid == 0 && !mbar_wait(bar_w, 0, kTrPolls);
            w_ready = true;
            if (__syncthreads_or(bad)) { timed_out = true; break; }
        }
        // ---- forward: hidden layers
        for (int l = 1; l <= 3 && !timed_out; ++l) {
            const int hin = l == 1 ? sH0 : l == 2 ? sH1 : sH2;
            const int hout = l == 1 ? sH1 : l == 2 ? sH2 : sH3;
            if (tid == 0) {
                tc_fence_after();
                if (l == 1) {
                    mma_run(tmem + cAcc, sb + sH0, kIn, false, sb + sW1, kIn, false, 1,
                            tr_idesc(kHid, false, false), false);
                } else {
                    const int wi = l == 2 ? sW2 : sW3, bi = l == 2 ? sB2 : sB3;
                    mma_run(tmem + cAcc, sb + sOne, 16, false, sb + bi, 16, false, 1,
                            tr_idesc(kHid, false, false), false);
                    mma_run(tmem + cAcc, sb + hin, kHid, false, sb + wi, kHid, false, kHid / 16,
                            tr_idesc(kHid, false, false), true);
                }
            }
            if (!commit_wait()) { timed_out = true; break; }
            __half2* ds = l == 1 ? a.ds1 : l == 2 ? a.ds2 : a.ds3;
            // this warpgroup's columns in chunks of 16, each chunk's
            // tensor-memory read issued before the previous chunk's arithmetic
            uint32_t rb[2][16];
            tmem_ld16(lane_base + cAcc + kTrCols * h, rb[0]);
#pragma unroll
            for (int cb = 0; cb < kTrCols; cb += 16) {
                const int c = kTrCols * h + cb;
                tmem_ld_wait(rb[(cb >> 4) & 1]);
                if (cb + 16 < kTrCols) tmem_ld16(lane_base + cAcc + c + 16, rb[((cb >> 4) + 1) & 1]);
                const uint32_t* r = rb[(cb >> 4) & 1];
                float sv[16], dv[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const float z = __uint_as_float(r[e]);
                    const float s = fmaf(0.5f, tanh_hw(0.5f * z), 0.5f);
                    sv[e] = z * s;
                    dv[e] = s * fmaf(z, 1.0f - s, 1.0f);
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    *reinterpret_cast<uint4*>(smem + hout + umma_offset(t, c + 8 * q, kHid)) =
                        make_uint4(pack_bf16(sv[8 * q], sv[8 * q + 1]), pack_bf16(sv[8 * q + 2], sv[8 * q + 3]),
                                   pack_bf16(sv[8 * q + 4], sv[8 * q + 5]),
                                   pack_bf16(sv[8 * q + 6], sv[8 * q + 7]));
                if (a.mode == 1 && valid) {
                    // the tile's SiLU' block as FP16 column pairs (pair (c,
                    // c + 1) of the tile's 128 rows contiguous): a warp's
                    // store of one pair is 128 contiguous bytes.  FP16 keeps
                    // SiLU' to 2^-11 relative, finer than the bf16 rounding
                    // of the delta it scales.
                    __half2* o = ds + (row - t) * (kHid / 2) + t;
#pragma unroll
                    for (int e = 0; e < 16; e += 2)
                        o[((c + e) / 2) * kTrRows] = __floats2half2_rn(dv[e], dv[e + 1]);
                }
            }
            publish();
        }
        if (timed_out) break;
        // ---- output layer
        if (tid == 0) {
            tc_fence_after();
            mma_run(tmem + cAcc, sb + sOne, 16, false, sb + sB4, 16, false, 1,
                    tr_idesc(kOut, false, false), false);
            mma_run(tmem + cAcc, sb + sH3, kHid, false, sb + sW4, kHid, false, kHid / 16,
                    tr_idesc(kOut, false, false), true);
        }
        if (!commit_wait()) { timed_out = true; break; }
        if (h == 0) {
            uint32_t r[16];
            tmem_ld16(lane_base + cAcc, r);
            tmem_ld_wait();
            if (a.mode == 0) {
                if (valid)
#pragma unroll
                    for (int k = 0; k < kOutRaw; ++k) a.Y[row * kOutRaw + k] = __uint_as_float(r[k]);
            } else {
                // loss and D4 = (OUT - T)/n, rounded to bf16; the column sums
                // of the rounded D4 (db4) and the sum of e^2 per warp
                float dv[16], e2 = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) dv[k] = 0.f;
                if (valid) {
#pragma unroll
                    for (int k = 0; k < kOutRaw; ++k) {
                        const float e = __uint_as_float(r[k]) - T[row * kOutRaw + k];
                        e2 = fmaf(e, e, e2);
                        dv[k] = __bfloat162float(__float2bfloat16_rn(e * inv_n));
                    }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    *reinterpret_cast<uint4*>(smem + sD4 + umma_offset(t, 8 * q, kOut)) =
                        make_uint4(pack_bf16(dv[8 * q], dv[8 * q + 1]), pack_bf16(dv[8 * q + 2], dv[8 * q + 3]),
                                   pack_bf16(dv[8 * q + 4], dv[8 * q + 5]),
                                   pack_bf16(dv[8 * q + 6], dv[8 * q + 7]));
                dv[kOutRaw] = e2;
#pragma unroll
                for (int k = 0; k <= kOutRaw; ++k) {
                    float x = dv[k];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    if (lane == 0) red[warp * 16 + k] = x;
                }
            }
        }
        if (a.mode == 0) {
            publish();  // the next tile's H0 overwrites nothing the MMAs still read
            continue;
        }
        publish();
        if (tid <= kOutRaw) accs[tid] += ((red[tid] + red[16 + tid]) + red[32 + tid]) + red[48 + tid];
        // this thread's columns of SiLU'(Z_l) (stored by the forward pass),
        // loaded as one batch before the tensor-core wait that precedes
        // layer l's backward step, so that their latency hides under it
        __half2 dsv[kTrCols / 2];
        auto load_ds = [&](int l) {
            const __half2* ds = l == 1 ? a.ds1 : l == 2 ? a.ds2 : a.ds3;
            const __half2* ip = ds + (row - t) * (kHid / 2) + t + (int64_t)(kTrCols * h / 2) * kTrRows;
#pragma unroll
            for (int q = 0; q < kTrCols / 2; ++q)
                dsv[q] = valid ? ip[q * kTrRows] : __floats2half2_rn(0.f, 0.f);
        };
        // ---- backward through the output layer: dW4^T += H3^T D4, G3 = D4 W4
        if (tid == 0) {
            tc_fence_after();
            mma_run(tmem + cDW4T, sb + sH3, kHid, true, sb + sD4, kOut, true, kTrRows / 16,
                    tr_idesc(kOut, true, true), !first);
            mma_run(tmem + cAcc, sb + sD4, kOut, false, sb + sW4, kHid, true, 1,
                    tr_idesc(kHid, false, true), false);
        }
        load_ds(3);
        if (!commit_wait()) { timed_out = true; break; }
        // ---- hidden layers, top down: D_l = G_l * SiLU'(Z_l) into H_l's image
        for (int l = 3; l >= 1 && !timed_out; --l) {
            const int dimg = l == 3 ? sH3 : l == 2 ? sH2 : sH1;
            uint32_t rb[2][16];
            tmem_ld16(lane_base + cAcc + kTrCols * h, rb[0]);
#pragma unroll
            for (int cb = 0; cb < kTrCols; cb += 16) {
                const int c = kTrCols * h + cb;
                tmem_ld_wait(rb[(cb >> 4) & 1]);
                if (cb + 16 < kTrCols) tmem_ld16(lane_base + cAcc + c + 16, rb[((cb >> 4) + 1) & 1]);
                const uint32_t* r = rb[(cb >> 4) & 1];
                float dv[16];
                if (valid) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float2 w = __half22float2(dsv[cb / 2 + q]);
                        dv[2 * q] = __uint_as_float(r[2 * q]) * w.x;
                        dv[2 * q + 1] = __uint_as_float(r[2 * q + 1]) * w.y;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) dv[e] = 0.f;
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    *reinterpret_cast<uint4*>(smem + dimg + umma_offset(t, c + 8 * q, kHid)) =
                        make_uint4(pack_bf16(dv[8 * q], dv[8 * q + 1]), pack_bf16(dv[8 * q + 2], dv[8 * q + 3]),
                                   pack_bf16(dv[8 * q + 4], dv[8 * q + 5]),
                                   pack_bf16(dv[8 * q + 6], dv[8 * q + 7]));
            }
            publish();
            if (tid == 0) {
                tc_fence_after();
                if (l > 1) {
                    const int hprev = l == 3 ? sH2 : sH1;
                    const int wl = l == 3 ? sW3 : sW2;
                    const uint32_t cdw = l == 3 ? cDW3 : cDW2, cdb = l == 3 ? cDB3 : cDB2;
                    mma_run(tmem + cdw, sb + hprev, kHid, true, sb + dimg, kHid, true, kTrRows / 16,
                            tr_idesc(kHid, true, true), !first);
                    mma_run(tmem + cdb, sb + dimg, kHid, true, sb + sOne, 16, true, kTrRows / 16,
                            tr_idesc(16, true, true), !first);
                    mma_run(tmem + cAcc, sb + dimg, kHid, false, sb + wl, kHid, true, kHid / 16,
                            tr_idesc(kHid, false, true), false);
                } else {
                    // dW1 (its column 11 is db1: H0 holds ones there)
                    mma_run(tmem + cDW1, sb + dimg, kHid, true, sb + sH0, kIn, true, kTrRows / 16,
                            tr_idesc(kIn, true, true), !first);
                }
            }
            if (l > 1) load_ds(l - 1);
            // the CTA's last tile: an accumulator that an earlier wait
            // completed goes out while this step's MMAs run (dW3 at l = 2,
            // dW2 at l = 1; their columns are not written here)
            if (a.mode == 1 && tile + 1 == tile1 && l < 3) {
                if (l == 2) {
                    dump(cDW3, P + kOffW3);
                } else {
                    dump(cDW2, P + kOffW2);
                    dumped23 = true;
                }
            }
            if (!commit_wait()) { timed_out = true; break; }
        }
    }

    // ---- the rest of the CTA's gradient partials
    if (a.mode == 1 && !timed_out) {
        if (!dumped23) {  // (a CTA without a tile)
            dump(cDW2, P + kOffW2);
            dump(cDW3, P + kOffW3);
        }
        uint32_t r[16];
        if (h == 0) {
            tmem_ld16(lane_base + cDW1, r);
            tmem_ld_wait();
#pragma unroll
            for (int k = 0; k < kIn; ++k) P[kOffW1 + t * kIn + k] = k < kInRaw ? __uint_as_float(r[k]) : 0.f;
            P[kOffB1 + t] = __uint_as_float(r[kInRaw]);
            tmem_ld16(lane_base + cDB2, r);
            tmem_ld_wait();
            P[kOffB2 + t] = __uint_as_float(r[0]);
        } else if (h == 1) {
            tmem_ld16(lane_base + cDW4T, r);  // row t = input feature, columns = outputs
            tmem_ld_wait();
#pragma unroll
            for (int k = 0; k < kOut; ++k) P[kOffW4 + k * kHid + t] = k < kOutRaw ? __uint_as_float(r[k]) : 0.f;
            tmem_ld16(lane_base + cDB3, r);
            tmem_ld_wait();
            P[kOffB3 + t] = __uint_as_float(r[0]);
        }
        if (tid < kOut) P[kOffB4 + tid] = tid < kOutRaw ? accs[tid] : 0.f;
        if (tid == 0) a.loss_part[blockIdx.x] = 0.5f * accs[kOutRaw] * inv_n;
    }
    if (timed_out && tid == 0) latch_error(a.err, NMODL_ERR_TIMEOUT);
    // no bulk copy may still be writing this CTA's shared memory at exit
    // (a CTA without tiles, or one whose wait gave up): wait again, bounded
    if (tid == 0 && (!w_ready || timed_out)) mbar_wait(bar_w, 0, kTrPolls);
    // ---- release the tensor memory
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTrTmemCols);
    }
}

// grad[i] = sum over the CTA partials in a fixed order (below).  adam: then the
// Adam step on the FP32 master parameter (learning rate and bias corrections
// from the arguments, or from the run's step index when fs.active), the bf16
// copy of the weight matrices and the weight image.  The first warp of block
// 0 also sums the loss partials (each lane a fixed strided subset, then a
// fixed butterfly) and, in a replayed run, records the loss; the last block
// to finish advances the run's step index.
__global__ void __launch_bounds__(128) k_grad_adam(const float* __restrict__ part, int n_part,
                            const float* __restrict__ loss_part, float* loss, float* grad,
                            int adam, float* p, float* m, float* v, __nv_bfloat16* wbf,
                            unsigned char* img, float lr, float b1, float b2, float eps,
                            float bc1, float bc2, FitSched fs, float* loss_steps,
                            unsigned int* done) {
    // Sums over the CTA partials in launch order within each quarter of the
    // partials, loads in batches of 16 ahead of their additions; the four
    // warps of a block take the four quarters of the same 32 parameters
    // (coalesced rows), and the quarter sums are added in a fixed order
    // (deterministic)
    __shared__ float qs[4][32];
    auto sum_parts = [](const float* base, int64_t stride, int c, int c1) {
        float acc = 0.f;
        for (; c + 16 <= c1; c += 16) {
            float x[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) x[u] = base[(int64_t)(c + u) * stride];
#pragma unroll
            for (int u = 0; u < 16; ++u) acc += x[u];
        }
        for (; c < c1; ++c) acc += base[(int64_t)c * stride];
        return acc;
    };
    const int lane = threadIdx.x & 31, q4 = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const bool owner = q4 == 0 && i < kParamsPadded;
    // the step index and this parameter's optimiser state first, so that
    // their loads overlap the partial sums
    const int64_t k_run = fs.active ? *fs.step : 0;
    float p0 = 0.f, m0 = 0.f, v0 = 0.f;
    if (adam && owner) {
        p0 = p[i];
        m0 = m[i];
        v0 = v[i];
    }
    if (blockIdx.x == 0 && q4 == 0) {
        float x = 0.f;
        for (int c = lane; c < n_part; c += 32) x += loss_part[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) {
            *loss = x;
            if (fs.active && loss_steps) loss_steps[k_run] = x;
        }
    }
    if (adam && fs.active) {
        lr = fs.lr_min + 0.5f * (fs.lr0 - fs.lr_min) *
                             (1.0f + cosf(3.14159265358979f * (float)k_run / (float)fs.total));
        const float tt = (float)(fs.t0 + k_run + 1);
        bc1 = 1.f - powf(b1, tt);
        bc2 = 1.f - powf(b2, tt);
    }
    const int per = (n_part + 3) / 4;
    const int c0 = min(n_part, q4 * per), c1 = min(n_part, c0 + per);
    qs[q4][lane] = i < kParamsPadded ? sum_parts(part + i, kParamsPadded, c0, c1) : 0.f;
    __syncthreads();
    if (owner) {
        const float g = ((qs[0][lane] + qs[1][lane]) + qs[2][lane]) + qs[3][lane];
        if (!adam) {
            grad[i] = g;
        } else {
            const float mi = b1 * m0 + (1.f - b1) * g;
            const float vi = b2 * v0 + (1.f - b2) * g * g;
            m[i] = mi;
            v[i] = vi;
            const float pi = p0 - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
            p[i] = pi;
            int bi = -1;
            if (i >= kOffW1 && i < kOffB1) bi = kBfW1 + (i - kOffW1);
            else if (i >= kOffW2 && i < kOffB2) bi = kBfW2 + (i - kOffW2);
            else if (i >= kOffW3 && i < kOffB3) bi = kBfW3 + (i - kOffW3);
            else if (i >= kOffW4 && i < kOffB4) bi = kBfW4 + (i - kOffW4);
            if (bi >= 0) wbf[bi] = __float2bfloat16_rn(pi);
            img_put(img, i, pi);
        }
    }
    // every thread of the block read the step index before the barrier
    // above; the last block to arrive advances it for the next step
    if (fs.active && done && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            *done = 0u;
            *fs.step = k_run + 1;
        }
    }
}

// ------------------------------------------------------------ launchers

cudaError_t train_prepare() {
    return cudaFuncSetAttribute(k_train_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kTrSmem);
}

static int device_sms() {
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int train_grid(int64_t n, int* tiles_per_cta) {
    const int sms = device_sms();
    const int64_t tiles = (n + kTrRows - 1) / kTrRows;
    const int64_t g0 = std::min<int64_t>(std::max(1, sms), std::max<int64_t>(1, tiles));
    const int64_t tpc = (tiles + g0 - 1) / g0;
    *tiles_per_cta = (int)std::max<int64_t>(1, tpc);
    return (int)std::max<int64_t>(1, (tiles + *tiles_per_cta - 1) / *tiles_per_cta);
}

int train_max_grid(int64_t max_batch) {
    const int64_t tiles = (max_batch + kTrRows - 1) / kTrRows;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, std::max(1, device_sms())));
}

cudaError_t launch_train_tiles(const TrainArgs& a, int grid, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_train_tiles<<<grid, kTrThreads, kTrSmem, s>>>(a);
    return cudaGetLastError();
}

void launch_grad_adam(const float* part, int n_part, const float* loss_part, float* loss,
                      float* grad, int adam, float* p, float* m, float* v, __nv_bfloat16* wbf,
                      unsigned char* img, float lr, float b1, float b2, float eps, int step,
                      FitSched fs, float* loss_steps, unsigned int* done, cudaStream_t s) {
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    k_grad_adam<<<(kParamsPadded + 31) / 32, 128, 0, s>>>(part, n_part, loss_part, loss, grad,
                                                            adam, p, m, v, wbf, img, lr, b1, b2,
                                                            eps, bc1, bc2, fs, loss_steps, done);
}

void launch_train_image(const float* params, unsigned char* img, cudaStream_t s) {
    cudaMemsetAsync(img, 0, kImg, s);
    k_train_image<<<(kParamsPadded + 2 * kTrRows + 255) / 256, 256, 0, s>>>(params, img);
}

}  // namespace nmodl
