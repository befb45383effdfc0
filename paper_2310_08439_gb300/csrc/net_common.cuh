// Device helpers shared by the network kernels (FP32 SIMT, BF16 mma.sync and
// BF16 tcgen05 forms): the activation functions of the per-species network
// and BF16 packing.
#pragma once

#include <cuda_bf16.h>

#include "tmd_internal.cuh"

namespace tmd {
namespace {

__device__ __forceinline__ float act_f(int act, float z, float b) {
    if (act == TMD_ACT_TANH) return tanhf(z);
    return 0.5f * (z + sqrtf(fmaf(z, z, b)));
}
// BF16 form: tanh from the hardware approximation (relative error about
// 2^-11, below the 2^-9 rounding of the BF16 activation it feeds)
__device__ __forceinline__ float act_f_bf16(int act, float z, float b) {
    if (act == TMD_ACT_TANH) {
        float r;
        asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(z));
        return r;
    }
    return 0.5f * (z + sqrtf(fmaf(z, z, b)));
}
// derivative expressed through the activation output a
__device__ __forceinline__ float act_da(int act, float a, float b) {
    if (act == TMD_ACT_TANH) return 1.f - a * a;
    const float a2 = 4.f * a * a;
    return a2 / (a2 + b);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t u) {
    const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&u);
    return __bfloat1622float2(v);
}

}  // namespace
}  // namespace tmd
