// ge_f32x2.cuh -- packed FP32 pairs for device code: one .f32x2 instruction
// does two FP32 operations, each rounded exactly as the scalar operation
// (fma.rn.f32x2 is two fused multiply-adds), so a packed loop gives the same
// bits as its scalar form with half the instructions.
//
// One difference from the scalar forms: the assembler may fuse a packed
// multiply into a packed add that uses its result, explicit .rn or not
// (measured: the compensated step's d (x_p - x) then differed in the last
// bit).  Where a product must be rounded on its own, f2_mul_alone computes
// it as an FMA whose addend is -0: x + (-0) == x for every x, including
// both zeros, and an FMA result cannot be fused any further.
#pragma once

#include <cstdint>

namespace ge {

__device__ __forceinline__ uint64_t f2(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_split(uint64_t v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// The pair (-0, -0), built from the sign of a non-negative runtime value s
// so that the compiler cannot fold it into a constant.
__device__ __forceinline__ uint64_t f2_neg_zero(float s)
{
    const float z = __int_as_float((__float_as_int(s) & (int)0x80000000) ^ (int)0x80000000);
    return f2(z, z);
}
// a * b, each product rounded on its own (nz = f2_neg_zero(...)).
__device__ __forceinline__ uint64_t f2_mul_alone(uint64_t a, uint64_t b, uint64_t nz) { return f2_fma(a, b, nz); }

}  // namespace ge
