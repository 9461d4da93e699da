// k_mlp.cu -- small kernels around the surrogate MLP's training run: the
// per-step loss record of a replayed run and the bf16 refresh of the weight
// copies after new weights are set.  The training contractions themselves
// run on the tensor cores in k_train.cu.
#include "kernels.cuh"
#include "mlp.cuh"

namespace nmodl {

__global__ void k_fit_end(float* loss_steps, const float* loss, FitSched fs) {
    loss_steps[*fs.step] = *loss;
    *fs.step += 1;
}

__global__ void k_to_bf16(const float* __restrict__ src, int64_t count, __nv_bfloat16* dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

void launch_fit_end(float* loss_steps, const float* loss, FitSched fs, cudaStream_t s) {
    k_fit_end<<<1, 1, 0, s>>>(loss_steps, loss, fs);
}

void launch_to_bf16(const float* src, int64_t count, __nv_bfloat16* dst, cudaStream_t s) {
    k_to_bf16<<<148, 256, 0, s>>>(src, count, dst);
}

}  // namespace nmodl
