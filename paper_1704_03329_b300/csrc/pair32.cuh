// Single-precision pair arithmetic shared by the FP32 kernels of the
// integrator (atom-index lists in md_kernels.cu, stage-slot lists in
// slots.cu): packed pairs (two neighbours per f32x2 instruction) and
// compensated sums.
#pragma once
#include "common.cuh"
#include "lj.cuh"

namespace ppmd {

typedef unsigned long long f2;  // two FP32 lanes
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Signed minimum-image difference of two fixed-point words, as a float.
__device__ __forceinline__ float fdiff(int32_t a, int32_t b) { return __int2float_rn((int32_t)((uint32_t)a - (uint32_t)b)); }

// Compensated sum of two interleaved streams: value = s - c, kept as cn = -c.
struct Kahan2 {
    f2 s, cn;
    __device__ __forceinline__ void init() { s = cn = 0ull; }
    // adds a * b to each stream
    __device__ __forceinline__ void add_prod(f2 a, f2 b) {
        const f2 yv = fma2(a, b, cn);
        const f2 t = add2(s, yv);
        cn = sub2(yv, sub2(t, s));
        s = t;
    }
    // adds v to each stream
    __device__ __forceinline__ void add(f2 v) {
        const f2 yv = add2(v, cn);
        const f2 t = add2(s, yv);
        cn = sub2(yv, sub2(t, s));
        s = t;
    }
    // the two streams merged: (hi, lo) with hi + lo the sum
    __device__ __forceinline__ void merged(float &hi, float &lo) const {
        float s0, s1, c0, c1;
        upk(s, s0, s1);
        upk(cn, c0, c1);
        hi = s0;
        lo = c0;
        two_sum_merge(hi, lo, s1, c1);
    }
};

}  // namespace ppmd
