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
// BF16 form: the activation a and its derivative d from the hardware
// approximations, whose relative errors (about 2^-11 for tanh.approx, 2^-22
// for rsqrt.approx) lie below the 2^-9 rounding of the BF16 operands they
// feed.  SquarePlus through u = 1/sqrt(z^2 + b): sqrt(z^2 + b) = (z^2 + b) u,
// a = (z + sqrt(z^2 + b)) / 2 and da/dz = (1 + z u) / 2.
__device__ __forceinline__ void act_fd_bf16(int act, float z, float b, float &a, float &d) {
    if (act == TMD_ACT_TANH) {
        asm("tanh.approx.f32 %0, %1;" : "=f"(a) : "f"(z));
        d = fmaf(-a, a, 1.f);
        return;
    }
    const float t = fmaf(z, z, b);
    float u;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(u) : "f"(t));
    a = 0.5f * fmaf(t, u, z);
    d = fmaf(0.5f * z, u, 0.5f);
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
