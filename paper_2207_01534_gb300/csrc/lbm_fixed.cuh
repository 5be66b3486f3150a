// lbm_fixed.cuh -- integer fixed-point density accumulators, shared by the
// schedules whose collide-stream pass also accumulates the next densities.
//
// Accumulators are integer fixed point so that the sums do not depend on the
// order of the atomic adds (results are bitwise reproducible): one 64-bit
// word per voxel holds both components, 32 bits each.  A contribution v is
// encoded as round(v * 2^26) + 2^25, non-negative for v >= -1/2; 19 encoded
// contributions stay below 2^32 for v < 3/2, so the low half never carries
// into the high half.  A density is decoded as (sum - 19 * 2^25) / 2^26 and
// a wall's virtual density (or a plane node's density) is stored as one
// encoded total with the same offset.  Resolution 2^-26 = 1.5e-8, finer than
// FP32 at unit density.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int kFixShift = 26;
constexpr uint32_t kFixBias = 1u << 25;
constexpr uint32_t kFixOffset = 19u * kFixBias;  // the bias of 19 contributions

__device__ __forceinline__ uint32_t fix_enc(float v)
{
    return (uint32_t)__float2int_rn(v * (float)(1 << kFixShift)) + kFixBias;
}

__device__ __forceinline__ unsigned long long fix_enc2(float2 v)
{
    return (unsigned long long)fix_enc(v.x) | ((unsigned long long)fix_enc(v.y) << 32);
}

// the sum v of k contributions, added at once: k biases
__device__ __forceinline__ unsigned long long fix_enc2n(float2 v, uint32_t k)
{
    const float sc = (float)(1 << kFixShift);
    const uint32_t a = (uint32_t)__float2int_rn(v.x * sc) + k * kFixBias;
    const uint32_t b = (uint32_t)__float2int_rn(v.y * sc) + k * kFixBias;
    return (unsigned long long)a | ((unsigned long long)b << 32);
}

// one stored total (plane node density, wall virtual density)
__device__ __forceinline__ unsigned long long fix_total2(float2 v)
{
    const uint32_t a = (uint32_t)__float2int_rn(v.x * (float)(1 << kFixShift)) + kFixOffset;
    const uint32_t b = (uint32_t)__float2int_rn(v.y * (float)(1 << kFixShift)) + kFixOffset;
    return (unsigned long long)a | ((unsigned long long)b << 32);
}

__device__ __forceinline__ float2 fix_dec2(unsigned long long w)
{
    const int a = (int)((uint32_t)w - kFixOffset);
    const int b = (int)((uint32_t)(w >> 32) - kFixOffset);
    const float k = 1.0f / (float)(1 << kFixShift);
    return make_float2((float)a * k, (float)b * k);
}

}  // namespace lbm
