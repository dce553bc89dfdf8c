// GELU of the surrogate's hidden layers, tanh form (Hendrycks & Gimpel):
//   gelu(z)  = z/2 (1 + tanh(u)),  u = sqrt(2/pi) (z + 0.044715 z^3)
//   gelu'(z) = (1 + tanh(u))/2 + z/2 (1 - tanh(u)^2) sqrt(2/pi) (1 + 3 * 0.044715 z^2)
// tanh is the hardware approximation (tanh.approx.f32, about 2^-11 relative
// error), one multi-function-unit operation per element.
#pragma once

#include <stdint.h>

namespace mlp {

constexpr float kGeluK = 0.7978845608028654f;  // sqrt(2 / pi)
constexpr float kGeluC = 0.044715f;

__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// u = z (sqrt(2/pi) + sqrt(2/pi) 0.044715 z^2): three FP32 operations
__device__ __forceinline__ float gelu_u(float z, float z2) { return z * fmaf(kGeluK * kGeluC, z2, kGeluK); }

__device__ __forceinline__ float gelu(float z)
{
    const float t = tanh_hw(gelu_u(z, z * z));
    const float hz = 0.5f * z;
    return fmaf(hz, t, hz);
}

__device__ __forceinline__ float gelu_grad(float z)
{
    const float z2 = z * z;
    const float t = tanh_hw(gelu_u(z, z2));
    const float du = kGeluK * fmaf(3.0f * kGeluC, z2, 1.0f);
    return fmaf(0.5f * z * du, fmaf(-t, t, 1.0f), 0.5f * (1.0f + t));
}

// ---- packed half-precision form (two elements per 32-bit register) ----

// f16x2 {lo, hi} from two floats, rounding to nearest and saturating at +-65504.
__device__ __forceinline__ uint32_t f16x2_sat(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// 2 gelu(z) = z (1 + tanh(u)) on both halves: HMUL2 z^2, HFMA2, HMUL2 u, tanh (one
// multi-function operation for two elements), HFMA2.
__device__ __forceinline__ uint32_t gelu2_f16x2(uint32_t z)
{
    const uint32_t kc = 0x28912891u;  // sqrt(2/pi) * 0.044715 = 0.035677 -> f16 0x2891 (both halves)
    const uint32_t k = 0x3a623a62u;   // sqrt(2/pi) = 0.79788 -> f16 0x3a62
    uint32_t z2, p, u, t, h;
    asm("mul.rn.f16x2 %0, %1, %1;" : "=r"(z2) : "r"(z));
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(p) : "r"(kc), "r"(z2), "r"(k));
    asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(u) : "r"(z), "r"(p));
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(u));
    asm("fma.rn.f16x2 %0, %1, %2, %1;" : "=r"(h) : "r"(z), "r"(t));
    return h;
}

// Two E4M3 codes {lo, hi} of an f16x2 (nearest even, saturating at +-448).
__device__ __forceinline__ uint32_t e4m3x2_f16x2(uint32_t x)
{
    unsigned short q;
    asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(q) : "r"(x));
    return q;
}

}  // namespace mlp
