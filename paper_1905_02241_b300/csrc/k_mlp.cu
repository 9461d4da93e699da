// k_mlp.cu -- the bf16 refresh of the surrogate MLP's weight copies after
// new weights are set.  The training contractions, the optimiser step and
// the weight image of the training kernel are in k_train.cu.
#include "kernels.cuh"
#include "mlp.cuh"

namespace nmodl {

__global__ void k_to_bf16(const float* __restrict__ src, int64_t count, __nv_bfloat16* dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

void launch_to_bf16(const float* src, int64_t count, __nv_bfloat16* dst, cudaStream_t s) {
    k_to_bf16<<<148, 256, 0, s>>>(src, count, dst);
}

}  // namespace nmodl
