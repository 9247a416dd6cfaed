// occ_f32x2.cuh -- paired FP32 arithmetic (Blackwell's add/sub/mul/fma .rn.f32x2): one
// instruction applies the same operation to two independent FP32 lanes held in a 64-bit
// register pair.  Each lane rounds exactly like the scalar instruction (round to nearest
// even, no contraction across lanes), so paired and scalar code give bit-identical results
// for the same operation order; the gain is half the issue slots for the arithmetic.
#pragma once

#include <cstdint>

namespace occ {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ f32x2 bc2(float a) { return pk2(a, a); }

__device__ __forceinline__ float2 up2(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// a * b + c per lane with one rounding (fmaf)
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// dot3 of occ_device.cuh (fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z))) for two lanes
__device__ __forceinline__ f32x2 dot3x2(f32x2 ax, f32x2 ay, f32x2 az, f32x2 bx, f32x2 by,
                                        f32x2 bz) {
    return fma2(ax, bx, fma2(ay, by, mul2(az, bz)));
}

}  // namespace occ
