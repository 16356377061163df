// nb_pair2.cuh -- paired float32 arithmetic for the pair kernels.
//
// sm_100 and later issue FADD2, FMUL2 and FFMA2: one instruction applies the
// operation to both halves of a float2, each half rounded exactly as the
// scalar instruction rounds it.  The force and energy kernels are bound by
// instruction issue, so they evaluate two atom pairs per instruction, one
// per half.  The double-float steps below are the scalar ones of
// nb_device.cuh, half by half, with identical results.
#pragma once

#include <cuda_runtime.h>

namespace nbgb {

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 sa, sb, sr;\n\tmov.b64 sa, {%2, %3};\n\tmov.b64 sb, {%4, %5};\n\t"
        "sub.rn.f32x2 sr, sa, sb;\n\tmov.b64 {%0, %1}, sr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// per half: c ? a : b
__device__ __forceinline__ float2 sel2(bool c0, bool c1, float2 a, float2 b) {
    return make_float2(c0 ? a.x : b.x, c1 ? a.y : b.y);
}

// s + e = a + b exactly (two-sum), per half.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// s + e = a - b exactly: the two-sum of a and -b, per half.
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
    s = sub2(a, b);
    const float2 bb = sub2(s, a);
    e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
// s + e = a + b exactly for |a| >= |b| (fast two-sum), per half.
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    e = sub2(b, sub2(s, a));
}
// p + e = a b exactly (fused multiply-add residual), per half.
__device__ __forceinline__ void two_prod2(float2 a, float2 b, float2& p, float2& e) {
    p = mul2(a, b);
    e = fma2(a, b, neg2(p));
}
// (ph + pl) = (ah + al)(bh + bl) to about 2^-46 relative, per half.
__device__ __forceinline__ void dd_mul2(float2 ah, float2 al, float2 bh, float2 bl, float2& ph, float2& pl) {
    const float2 p = mul2(ah, bh);
    float2 e = fma2(ah, bh, neg2(p));
    e = fma2(ah, bl, fma2(al, bh, e));
    ph = add2(p, e);
    pl = sub2(e, sub2(ph, p));
}

}  // namespace nbgb
