// bf16_util.cuh -- small helpers shared by the tensor-core kernels: shared
// addresses, bf16 packing and the SiLU of the surrogate MLP.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace nmodl {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// SiLU used by the surrogate on both its training and inference paths:
// sigma(z) = (1 + tanh(z/2))/2 with the single-instruction hardware tanh
// (max error ~2^-11, below the bf16 rounding of the activations).
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace nmodl
