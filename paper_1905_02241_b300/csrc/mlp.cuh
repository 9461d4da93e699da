// mlp.cuh -- shapes, parameter layout and launch interfaces of the kinetic
// surrogate MLP (11 -> 128 -> 128 -> 128 -> 9, SiLU).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bf16_util.cuh"
#include "nmodl_internal.cuh"

namespace nmodl {

constexpr int kInRaw = 11, kIn = 16;    // v_n, dt_n, x0..x8 (padded to 16)
constexpr int kHid = 128;
constexpr int kOutRaw = 9, kOut = 16;   // increments of the 9 states (padded)

// FP32 master parameters, padded, in this order:
//   W1 [128][16], b1 [128], W2 [128][128], b2 [128], W3 [128][128], b3 [128],
//   W4 [16][128], b4 [16]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kOut * kHid;
constexpr int kParamsPadded = kOffB4 + kOut;
// bf16 copies of the weight matrices only: W1 | W2 | W3 | W4
constexpr int kBfW1 = 0, kBfW2 = kBfW1 + kHid * kIn, kBfW3 = kBfW2 + kHid * kHid,
              kBfW4 = kBfW3 + kHid * kHid, kBfCount = kBfW4 + kOut * kHid;
// The training kernel's weight image: the bf16 weights in the K-major
// core-matrix layout of its shared memory (W1 with the bias pair of b1 in
// columns 11, 12 | W2 | W3 | W4), then the column-of-ones image and the bias
// pair images of b2, b3, b4; copied whole into shared memory at the start
// of each training launch and kept current by the optimiser step.
constexpr int kTrImgBytes = 2 * (kHid * kIn + 2 * kHid * kHid + kOut * kHid) +
                            2 * (128 * 16 + 2 * kHid * 16 + kOut * 16);  // 86528
// unpadded public layout (row-major [out][in] weights, then biases)
constexpr int kParamsPublic = kHid * kInRaw + kHid + 2 * (kHid * kHid + kHid) +
                              kOutRaw * kHid + kOutRaw;  // 35721

// Input normalisation of (v, dt): v_n = (v + 20)/80, dt_n = (dt - 0.03125)/0.01875
constexpr float kVShift = 20.f, kVScale = 80.f, kDtShift = 0.03125f, kDtScale = 0.01875f;

// Schedule of a whole training run replayed from one captured step: the
// kernels read the step index from device memory and derive the minibatch
// (rows (k mod steps_per_epoch) * B of X and T), the cosine learning rate
// and Adam's bias corrections from it.  active == 0: plain single step.
struct FitSched {
    int64_t* step;            // device: index of the current step in the run
    int64_t steps_per_epoch;
    int64_t total;
    float lr0, lr_min;
    int32_t t0;               // Adam steps taken before the run
    int32_t active;
};

// Fused training / batch-forward kernel of the surrogate MLP (k_train.cu)
struct TrainArgs {
    const float* X;            // [n][11] normalised inputs (FP32)
    const float* T;            // [n][9] targets (mode 1)
    float* Y;                  // [n][9] network outputs (mode 0)
    int64_t n;                 // rows of the batch
    int tiles_per_cta;         // 128-row tiles per CTA
    int mode;                  // 0: forward outputs; 1: loss and gradient partials
    const unsigned char* img;  // the weight image (kTrImgBytes, 16-byte aligned)
    __half2 *ds1, *ds2, *ds3;  // SiLU'(Z) of the hidden layers (mode 1) in FP16, per 128-row
                               // tile a block of 64 column pairs x 128 rows (pair
                               // (c, c + 1) of row t at 128 (c / 2) + t)
    float* part;               // [grid][kParamsPadded] gradient partials (mode 1)
    float* loss_part;          // [grid] loss partials (mode 1)
    FitSched fs;
    int32_t* err;
};
cudaError_t train_prepare();
// CTAs for a batch of n rows (at most one per SM) and the tiles each takes
int train_grid(int64_t n, int* tiles_per_cta);
// the most CTAs train_grid returns for batches of up to max_batch rows
int train_max_grid(int64_t max_batch);
cudaError_t launch_train_tiles(const TrainArgs& a, int grid, cudaStream_t s);
// gradient = fixed-order sum of the n_part CTA partials; adam: then the
// Adam step (lr and the bias corrections of step `step`, or from fs when
// active) on the master parameters, the bf16 copies and the weight image;
// *loss = the sum of the loss partials.  With fs active and loss_steps
// given, the loss is also recorded at loss_steps[*fs.step] and the last
// block to finish advances *fs.step (done: a zeroed arrival counter).
void launch_grad_adam(const float* part, int n_part, const float* loss_part, float* loss,
                      float* grad, int adam, float* p, float* m, float* v, __nv_bfloat16* wbf,
                      unsigned char* img, float lr, float b1, float b2, float eps, int step,
                      FitSched fs, float* loss_steps, unsigned int* done, cudaStream_t s);
// the whole weight image from the FP32 master parameters
void launch_train_image(const float* params, unsigned char* img, cudaStream_t s);
void launch_to_bf16(const float* src, int64_t count, __nv_bfloat16* dst, cudaStream_t s);

// surrogate state update (fused MLP + projection + residual + fallback list)
struct SurArgs {
    const __nv_bfloat16* wbf;  // kBfCount
    const float* params;       // FP32 master (biases read from here)
    const Kin9D* kd;
    int64_t n;
    const int32_t* ni;
    const double* v;
    double* st;
    int64_t stride;
    double dt;
    float tol;                 // fallback when ||F(x_hat)||_1 > tol
    int scaled;                // output scaled by ||dt A x||_1
    int32_t* fb_list;
    int32_t* fb_count;
    unsigned long long* fb_total;
    int32_t* err;
    // step != 0: the whole network step of a list of this one mechanism with
    // instance i on node i: before its state update each instance forms its
    // current at v_n (g = gbar x_open, i = g (v - e)), writes rhs = -i and
    // d = g + cmdt, and (unless clamp) v = v_n + rhs/d, at which its state
    // update then runs
    int32_t step, clamp, open;
    double gbar, e, cmdt;
    double* v_step;            // v, written (the same array as v)
    double* rhs;
    double* d;
};
cudaError_t launch_surrogate_step(const SurArgs& a, cudaStream_t s);
cudaError_t surrogate_prepare();

// training data: normalised inputs [n][11] and targets [n][9] from
// (v, dt, x, y = Newton step) in FP64
void launch_make_pairs(const Kin9D* kd, int64_t n, const double* v, const double* dt,
                       const double* x, const double* y, int64_t stride, int scaled,
                       float* X, float* T, cudaStream_t s);

}  // namespace nmodl
