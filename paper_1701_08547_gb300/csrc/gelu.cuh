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

// gelu'(z) from z, z^2 and t = tanh(u) (shared with gelu(z) where both are formed)
__device__ __forceinline__ float gelu_grad_t(float z, float z2, float t)
{
    const float du = kGeluK * fmaf(3.0f * kGeluC, z2, 1.0f);
    return fmaf(0.5f * z * du, fmaf(-t, t, 1.0f), 0.5f * (1.0f + t));
}

// gelu'(Z) of the training forward passes (FP16, [members][rows][256]) is kept in 128-row
// tiles, within a tile in blocks of 16 columns, each block row-major [128 rows][16 columns]:
// a warp whose lanes are 32 consecutive rows (the TMEM lane layout of the epilogues that write
// and read it) then covers 1 KB of contiguous memory with one 32-byte access per lane.
// Offset of (row, column) within one member's array.
__host__ __device__ __forceinline__ long long gprime_at(long long row, int col)
{
    return ((row >> 7) << 15) + ((long long)(col >> 4) << 11) + ((row & 127) << 4) + (col & 15);
}

__device__ __forceinline__ float gelu_grad(float z)
{
    const float z2 = z * z;
    return gelu_grad_t(z, z2, tanh_hw(gelu_u(z, z2)));
}

}  // namespace mlp
