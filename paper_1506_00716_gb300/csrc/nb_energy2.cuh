// nb_energy2.cuh -- double-float pair energies, shared by the energy kernel
// (k_energy) and the force kernel's fused energy variant: erfc from the
// Ewald energy table, the energy of two queued pairs at a time (the halves
// of the paired float32 instructions), and the drain of a warp's queue of
// pairs inside (or near) the cut-off.  nb_energy.cu describes the arithmetic.
#pragma once

#include "nb_device.cuh"
#include "nb_pair2.cuh"

namespace nbgb {

namespace {

constexpr unsigned EFULL = FULL_MASK;

// The Ewald energy table as the energy code reads it (KParams::etab): per
// interval k, a[k] = (a0 hi, a0 lo, a1 hi, a1 lo) and b[k] = (a2, a3, a4, -)
// of erfc(beta r) ~ a0 + a1 s + a2 s^2 + a3 s^3 + a4 s^4, s = r / h - k.
struct EwaldE {
    const float4* a;
    const float4* b;
    float invh;     // 1 / h (a power of two)
    unsigned last;  // intervals - 1
};

// 1.5 * 2^23: a float in [2^23, 2^24) holds an integer in its mantissa
constexpr float ET_MAGIC = 12582912.f;

// erfc(beta r) in double-float for r = rh + rl >= 0, from the table; two
// arguments (the halves).  Interval k = floor(rh / h) by a round-down fused
// multiply-add onto 1.5 * 2^23 (clamped to the table: far and masked slots
// give finite values that the caller discards), s = sh + sl with sh = rh / h
// - k exact and sl = rl / h; then a0 + a1 s in double-float (the product of
// the high parts error-free, the terms of sl and of the low parts to first
// order) plus s^2 (a2 + s (a3 + s a4)) in float32, whose rounding (the
// quadratic coefficient is at most 1e-4) stays below 1e-11.
__device__ __forceinline__ void erfc_tab2(float2 rh, float2 rl, const EwaldE& et, float2& eh, float2& el) {
    const float2 m = __ffma2_rd(rh, dup2(et.invh), dup2(ET_MAGIC));
    const float2 sh = fma2(rh, dup2(et.invh), sub2(dup2(ET_MAGIC), m));
    const float2 sl = mul2(rl, dup2(et.invh));
    const unsigned k0 = min((unsigned)(__float_as_int(m.x) - __float_as_int(ET_MAGIC)), et.last);
    const unsigned k1 = min((unsigned)(__float_as_int(m.y) - __float_as_int(ET_MAGIC)), et.last);
    const float4 a0 = et.a[k0], a1 = et.a[k1];
    const float4 b0 = et.b[k0], b1 = et.b[k1];
    float2 t = fma2(make_float2(b0.z, b1.z), sh, make_float2(b0.y, b1.y));
    t = fma2(t, sh, make_float2(b0.x, b1.x));
    // s^2 t, to first order in sl: t sh (sh + 2 sl)
    const float2 q = mul2(mul2(t, sh), fma2(dup2(2.f), sl, sh));
    const float2 c1h = make_float2(a0.z, a1.z), c1l = make_float2(a0.w, a1.w);
    float2 p, pe;
    two_prod2(c1h, sh, p, pe);
    const float2 low = fma2(c1h, sl, fma2(c1l, sh, pe));
    float2 p2, e1, vh, e2;
    two_sum2(p, q, p2, e1);
    two_sum2(make_float2(a0.x, a1.x), p2, vh, e2);
    const float2 vl = add2(add2(e1, e2), add2(low, make_float2(a0.y, a1.y)));
    fast_two_sum2(vh, vl, eh, el);
}

// Energy of two queued pairs (the halves).  `valid`: the lane's half holds
// a pair; `maybe`: its float32 r^2 fell in the band around rc^2 and the
// decision is taken here, exactly; otherwise the pair is inside rc.  The
// i-atom data are per half (the two pairs may have different i-slots).
// The shifted LJ terms c12 (r^-12 - rc^-12) and c6 (r^-6 - rc^-6) are in
// double-float: the shift takes away most of E_LJ, so the float32 terms'
// rounding would no longer be small next to what is left.
struct IPair2 {
    float2 xh, yh, zh, xl, yl, zl, qih, qil;
};

template <int COUL, bool LJSH>
__device__ __forceinline__ void pair_energy2(const float4 xj0, const float4 xj1, float2 c6, float2 c12,
                                             const IPair2& ip, const ShiftedI& xs0, const ShiftedI& xs1,
                                             bool valid0, bool valid1, bool maybe0, bool maybe1,
                                             const KParams& kp, const EwaldE& et, float2& ch, float2& cl,
                                             float2& e12,
                                             float2& e12l, float2& e6, float2& e6l, int& npair) {
    float2 dxh, dxe, dyh, dye, dzh, dze;
    two_diff2(ip.xh, make_float2(xj0.x, xj1.x), dxh, dxe);
    two_diff2(ip.yh, make_float2(xj0.y, xj1.y), dyh, dye);
    two_diff2(ip.zh, make_float2(xj0.z, xj1.z), dzh, dze);
    const float2 dxl = add2(dxe, ip.xl), dyl = add2(dye, ip.yl), dzl = add2(dze, ip.zl);
    float2 px, ex, py, ey, pz, ez;
    two_prod2(dxh, dxh, px, ex);
    two_prod2(dyh, dyh, py, ey);
    two_prod2(dzh, dzh, pz, ez);
    ex = fma2(mul2(dup2(2.f), dxh), dxl, ex);
    ey = fma2(mul2(dup2(2.f), dyh), dyl, ey);
    ez = fma2(mul2(dup2(2.f), dzh), dzl, ez);
    float2 s1, e1, r2h, e2;
    two_sum2(px, py, s1, e1);
    two_sum2(s1, pz, r2h, e2);
    const float2 r2l = add2(add2(e1, e2), add2(ex, add2(ey, ez)));

    // a pair in the band around rc (marked by the screening, or found here:
    // the high part of the double-float r^2 is within 2^-24 of r^2, far
    // inside the band) is decided exactly, in the oracle's arithmetic
    maybe0 = maybe0 || !(r2h.x < kp.rc2_lo);
    maybe1 = maybe1 || !(r2h.y < kp.rc2_lo);
    bool in0 = valid0, in1 = valid1;
    if (valid0 && maybe0) in0 = exact_inside(xs0, xj0, kp.rc2_d);
    if (valid1 && maybe1) in1 = exact_inside(xs1, xj1, kp.rc2_d);
    npair += __popc(__ballot_sync(EFULL, in0)) + __popc(__ballot_sync(EFULL, in1));

    // 1/r = y (1 + h/2), h = 1 - r^2 y^2
    const float2 y = make_float2(rsqrt_sfu(r2h.x), rsqrt_sfu(r2h.y));
    float2 y2, y2e;
    two_prod2(y, y, y2, y2e);
    float2 h = fma2(neg2(r2h), y2, dup2(1.f));
    h = fma2(neg2(r2h), y2e, h);
    h = fma2(neg2(r2l), y2, h);
    const float2 ril = mul2(mul2(dup2(0.5f), y), h);
    const float2 rif = add2(y, ril);

    if (LJSH) {
        float2 ah, al;
        fast_two_sum2(y, ril, ah, al);  // 1/r
        float2 p2h, p2l, p4h, p4l, p6h, p6l, p12h, p12l;
        dd_mul2(ah, al, ah, al, p2h, p2l);
        dd_mul2(p2h, p2l, p2h, p2l, p4h, p4l);
        dd_mul2(p4h, p4l, p2h, p2l, p6h, p6l);
        dd_mul2(p6h, p6l, p6h, p6l, p12h, p12l);
        float2 dh, dl, t6, t6l, t12, t12l;
        two_diff2(p6h, dup2(kp.irc6_h), dh, dl);
        dl = add2(dl, sub2(p6l, dup2(kp.irc6_l)));
        two_prod2(c6, dh, t6, t6l);
        t6l = fma2(c6, dl, t6l);
        two_diff2(p12h, dup2(kp.irc12_h), dh, dl);
        dl = add2(dl, sub2(p12l, dup2(kp.irc12_l)));
        two_prod2(c12, dh, t12, t12l);
        t12l = fma2(c12, dl, t12l);
        t12 = sel2(in0, in1, t12, dup2(0.f));
        t12l = sel2(in0, in1, t12l, dup2(0.f));
        t6 = sel2(in0, in1, t6, dup2(0.f));
        t6l = sel2(in0, in1, t6l, dup2(0.f));
        float2 sh, se;
        two_sum2(e12, t12, sh, se);
        e12 = sh;
        e12l = add2(e12l, add2(se, t12l));
        two_sum2(e6, t6, sh, se);
        e6 = sh;
        e6l = add2(e6l, add2(se, t6l));
    } else {
        const float2 ri2 = mul2(rif, rif);
        const float2 ri6 = mul2(mul2(ri2, ri2), ri2);
        const float2 t6 = mul2(c6, ri6);
        const float2 t12 = mul2(mul2(c12, ri6), ri6);
        e12 = add2(e12, sel2(in0, in1, t12, dup2(0.f)));
        e6 = add2(e6, sel2(in0, in1, t6, dup2(0.f)));
    }

    const float2 qj = make_float2(xj0.w, xj1.w);
    float2 qh, qe;
    two_prod2(ip.qih, qj, qh, qe);
    const float2 ql = fma2(ip.qil, qj, qe);
    float2 vh, vl;
    if (COUL == NB_COUL_RF) {
        float2 kh, ke;
        two_prod2(dup2(kp.krf_h), r2h, kh, ke);
        const float2 kl = fma2(dup2(kp.krf_h), r2l, fma2(dup2(kp.krf_l), r2h, ke));
        float2 sh, es, gh, eg;
        two_sum2(y, kh, sh, es);
        two_diff2(sh, dup2(kp.crf_h), gh, eg);
        const float2 gl = sub2(add2(add2(es, eg), add2(ril, kl)), dup2(kp.crf_l));
        float2 ve;
        two_prod2(qh, gh, vh, ve);
        vl = fma2(qh, gl, fma2(ql, gh, ve));
    } else {
        float2 rh, re;
        two_prod2(r2h, y, rh, re);
        const float2 rl = add2(re, fma2(r2h, ril, mul2(r2l, y)));
        float2 eh, el;
        erfc_tab2(rh, rl, et, eh, el);
        float2 wh, we;
        two_prod2(eh, y, wh, we);
        float2 wl = add2(we, fma2(eh, ril, mul2(el, y)));
        if (kp.mods & NB_MOD_EWALD_SHIFT) {
            float2 dh, de;
            two_diff2(wh, dup2(kp.ewc_h), dh, de);
            wl = add2(de, sub2(wl, dup2(kp.ewc_l)));
            wh = dh;
        }
        float2 ve;
        two_prod2(qh, wh, vh, ve);
        vl = add2(ve, fma2(qh, wl, mul2(ql, wh)));
    }
    vh = sel2(in0, in1, vh, dup2(0.f));
    vl = sel2(in0, in1, vl, dup2(0.f));
    float2 th, te;
    two_sum2(ch, vh, th, te);
    ch = th;
    cl = add2(cl, add2(te, vl));
}

__device__ __forceinline__ void flush_energy(const SysDev* __restrict__ sys, int s, double& dec,
                                             double& d12, double& d6, long long& np, int lane) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dec += __shfl_xor_sync(EFULL, dec, off);
        d12 += __shfl_xor_sync(EFULL, d12, off);
        d6 += __shfl_xor_sync(EFULL, d6, off);
    }
    if (lane == 0) {
        atomicAdd(sys[s].acc + ACC_EC, dec);
        atomicAdd(sys[s].acc + ACC_E12, d12);
        atomicAdd(sys[s].acc + ACC_E6, d6);
        atomicAdd(sys[s].acc + ACC_NPAIR, (double)np);
    }
    dec = d12 = d6 = 0.0;
    np = 0;
}

constexpr int QCAP = 512;  // per-warp ring queue of candidate pairs (>= 63 + 8 * 32)

// i-atom data of the current item, one record per i-slot (shared by the
// lanes that evaluate queued pairs).
struct IRec {
    ShiftedI xs;
    float qih, qil;
    int tirow;
};

// Queue entry: j slot index << 4 | i-slot << 1 | band flag.  A lane takes
// the entries at ring positions k and k + 32 as the two halves of the paired
// evaluation.
template <int COUL, bool LJSH>
__device__ __forceinline__ void drain2(int k, const int* __restrict__ qm, const IRec* __restrict__ irec,
                                       const float4* __restrict__ xq_s, const int* __restrict__ type_s,
                                       const float2* __restrict__ s_lj, const KParams& kp, const EwaldE& et,
                                       float2& ch,
                                       float2& cl, float2& e12, float2& e12l, float2& e6, float2& e6l,
                                       int& npair, bool valid0, bool valid1) {
    const int m0 = valid0 ? qm[k & (QCAP - 1)] : 0;
    const int m1 = valid1 ? qm[(k + 32) & (QCAP - 1)] : 0;
    const int js0 = m0 >> 4, js1 = m1 >> 4;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 xj0 = valid0 ? xq_s[js0] : z4;
    const float4 xj1 = valid1 ? xq_s[js1] : z4;
    const int tj0 = valid0 ? type_s[js0] : 0;
    const int tj1 = valid1 ? type_s[js1] : 0;
    const IRec& r0 = irec[(m0 >> 1) & 7];
    const IRec& r1 = irec[(m1 >> 1) & 7];
    IPair2 ip;
    ip.xh = make_float2(r0.xs.xh, r1.xs.xh);
    ip.yh = make_float2(r0.xs.yh, r1.xs.yh);
    ip.zh = make_float2(r0.xs.zh, r1.xs.zh);
    ip.xl = make_float2(r0.xs.xl, r1.xs.xl);
    ip.yl = make_float2(r0.xs.yl, r1.xs.yl);
    ip.zl = make_float2(r0.xs.zl, r1.xs.zl);
    ip.qih = make_float2(r0.qih, r1.qih);
    ip.qil = make_float2(r0.qil, r1.qil);
    const float2 l0 = s_lj[r0.tirow + tj0], l1 = s_lj[r1.tirow + tj1];
    pair_energy2<COUL, LJSH>(xj0, xj1, make_float2(l0.x, l1.x), make_float2(l0.y, l1.y), ip, r0.xs, r1.xs, valid0,
                             valid1, m0 & 1, m1 & 1, kp, et, ch, cl, e12, e12l, e6, e6l, npair);
}

}  // namespace

}  // namespace nbgb
