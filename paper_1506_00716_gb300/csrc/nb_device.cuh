// nb_device.cuh -- device helpers shared by the force and energy kernels:
// SFU approximations issued as single PTX instructions, error-free float32
// transformations (two-sum, two-product) for the compensated ("double-float")
// energy arithmetic, and the exact cut-off decision.
#pragma once

#include "nb_internal.cuh"

namespace nbgb {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ int find_sys_dev(const int* __restrict__ off, int nsys, int idx) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float rsqrt_sfu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_sfu(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_sfu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly, valid when |a| >= |b| (Dekker's fast two-sum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}
// (ph + pl) = (ah + al) (bh + bl) to about 2^-46 relative (double-float
// product; the al bl term is below that and dropped).
__device__ __forceinline__ void dd_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    ph = p + e;
    pl = e - (ph - p);
}
// p + e = a * b exactly (fused multiply-add residual).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// i-atom position displaced by the item's periodic shift, kept as an
// unevaluated sum hi + lo that equals x_i + S exactly.
struct ShiftedI {
    float xh, yh, zh, xl, yl, zl;
};

// x + sum of the terms t_k carried as hi + lo: each addition error-free, the
// low parts summed (exact when at most one term is nonzero).
__device__ __forceinline__ void sum3(float x, float t0, float t1, float t2, float& h, float& l) {
    float e0, e1, e2;
    two_sum(x, t0, h, e0);
    two_sum(h, t1, h, e1);
    two_sum(h, t2, h, e2);
    l = e0 + (e1 + e2);
}

// x_i + S for the item's periodic shift S = sx a + sy b + sz c (box rows a =
// (Lx,0,0), b = (Tbx,Ly,0), c = (Tcx,Tcy,Lz)); every product is exact, so
// the rectangular case is exact and the triclinic one within a rounding of
// the low part.
__device__ __forceinline__ ShiftedI shift_i(float4 xi, int sh, float Lx, float Ly, float Lz, float Tbx,
                                            float Tcx, float Tcy) {
    const float sx = (float)(sh / 9 - 1), sy = (float)((sh / 3) % 3 - 1), sz = (float)(sh % 3 - 1);
    ShiftedI s;
    sum3(xi.x, sx * Lx, sy * Tbx, sz * Tcx, s.xh, s.xl);
    sum3(xi.y, sy * Ly, sz * Tcy, 0.f, s.yh, s.yl);
    two_sum(xi.z, sz * Lz, s.zh, s.zl);
    return s;
}

// Exact cut-off decision for a pair near rc: the float64 squared distance of
// the float32 inputs, summed in the oracle's operation order (no fused
// multiply-add), so that both sides decide every borderline pair alike.
__device__ __forceinline__ bool exact_inside(const ShiftedI& xs, float4 xj, double rc2) {
    const double dx = __dadd_rn(__dadd_rn((double)xs.xh, (double)xs.xl), -(double)xj.x);
    const double dy = __dadd_rn(__dadd_rn((double)xs.yh, (double)xs.yl), -(double)xj.y);
    const double dz = __dadd_rn(__dadd_rn((double)xs.zh, (double)xs.zl), -(double)xj.z);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rc2;
}

}  // namespace nbgb
