// f32x2.cuh -- two FP32 values in one 64-bit register, operated on by the
// packed single-precision instructions of sm_100-class GPUs (PTX
// fma/add/sub/mul .rn.f32x2): one issue slot yields two IEEE round-to-nearest
// FP32 results, each exactly what the scalar instruction gives for that half.
// The Metropolis kernels are issue bound, so every per-point FP32 operation
// that comes in pairs of points runs packed.
#pragma once
#include <cstdint>

namespace smc {

struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 mk2(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ f2 splat2(float a) { return mk2(a, a); }

__device__ __forceinline__ float lo2(f2 a) { return __uint_as_float((unsigned)a.v); }

__device__ __forceinline__ float hi2(f2 a) { return __uint_as_float((unsigned)(a.v >> 32)); }

// a * b + c, each half rounded once
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

}  // namespace smc
