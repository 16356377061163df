// nb_energy2.cuh -- double-float pair energies, shared by the energy kernel
// (k_energy) and the force kernel's fused energy variant: the compensated
// erfc and 2^a, the energy of two queued pairs at a time (the halves of the
// paired float32 instructions), and the drain of a warp's queue of pairs
// inside (or near) the cut-off.  nb_energy.cu describes the arithmetic.
#pragma once

#include "erfc_fit.cuh"
#include "nb_device.cuh"
#include "nb_pair2.cuh"

namespace nbgb {

namespace {

constexpr unsigned EFULL = FULL_MASK;

// Number of head coefficients evaluated in double-float; the tail terms are
// small enough (|a_k u^k| <= 5e-4) for plain float32.
constexpr int EF_HEAD = 5;   // erfc fit: k = 0..4
constexpr int EX2_HEAD = 4;  // 2^f fit: k = 0..3

// Horner steps over coefficients hi[k] + lo[k], k = k1 .. 0, in compensated
// (double-float) arithmetic, p = p * u + c with p, u, c all hi + lo; for two
// arguments (the halves).
template <int K1>
__device__ __forceinline__ void horner_dd2(const float* hi, const float* lo, float2 uh, float2 ul, float2& ph,
                                           float2& pl) {
#pragma unroll
    for (int k = K1; k >= 0; --k) {
        float2 m, me, sum, se;
        two_prod2(ph, uh, m, me);
        const float2 cross = fma2(ph, ul, mul2(pl, uh));
        two_sum2(m, dup2(hi[k]), sum, se);
        ph = sum;
        pl = add2(add2(add2(me, se), cross), dup2(lo[k]));
    }
}

// erfc(x) in double-float for x = xh + xl >= 0, from the degree-12 fit and
// the double-float exponential 2^a, a = ah + al = -x^2 log2(e) (given); for
// two arguments (the halves).  Steps: d = 1 + P x; t = 1/d by a refined SFU
// reciprocal; u = UA t + UB; R(u) with a float32 tail and a double-float
// head; 2^a = 2^n 2^f with f = (ah - n) + al in [-0.5, 0.5] (ah - n exact);
// erfc = R 2^a.
__device__ __forceinline__ void erfc_dd2(float2 xh, float2 xl, float2 ah, float2 al, float2& eh, float2& el) {
    const bool c0 = xh.x > EF_XMAX, c1 = xh.y > EF_XMAX;
    xh = sel2(c0, c1, dup2(EF_XMAX), xh);
    xl = sel2(c0, c1, dup2(0.f), xl);
    float2 m, me, dh, de;
    two_prod2(dup2(EF_P), xh, m, me);
    two_sum2(dup2(1.f), m, dh, de);
    const float2 dl = add2(de, fma2(dup2(EF_P), xl, me));
    float2 th = make_float2(rcp_sfu(dh.x), rcp_sfu(dh.y));
    th = mul2(th, fma2(neg2(dh), th, dup2(2.f)));
    float2 r = fma2(neg2(dh), th, dup2(1.f));
    r = fma2(neg2(dl), th, r);
    const float2 tl = mul2(th, r);
    float2 uh, ue, sh, se;
    two_prod2(dup2(EF_UA), th, uh, ue);
    two_sum2(uh, dup2(EF_UB), sh, se);
    const float2 ul = add2(se, fma2(dup2(EF_UA), tl, ue));
    uh = sh;
    float2 ph = dup2(EF_EN_HI[EF_NE - 1]), pl = dup2(0.f);
#pragma unroll
    for (int k = EF_NE - 2; k >= EF_HEAD; --k) ph = fma2(ph, uh, dup2(EF_EN_HI[k]));
    horner_dd2<EF_HEAD - 1>(EF_EN_HI, EF_EN_LO, uh, ul, ph, pl);
    ah = make_float2(fmaxf(ah.x, -120.f), fmaxf(ah.y, -120.f));
    const float2 n = make_float2(rintf(ah.x), rintf(ah.y));
    const float2 fh = sub2(ah, n);
    float2 qh = dup2(EX2_HI[EX2_N - 1]), ql = dup2(0.f);
#pragma unroll
    for (int k = EX2_N - 2; k >= EX2_HEAD; --k) qh = fma2(qh, fh, dup2(EX2_HI[k]));
    horner_dd2<EX2_HEAD - 1>(EX2_HI, EX2_LO, fh, al, qh, ql);
    const float2 scale = make_float2(__int_as_float(((int)n.x + 127) << 23), __int_as_float(((int)n.y + 127) << 23));
    float2 ch, ce;
    two_prod2(ph, qh, ch, ce);
    const float2 cl = add2(ce, fma2(ph, ql, mul2(pl, qh)));
    eh = mul2(ch, scale);
    el = mul2(cl, scale);
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
                                             const KParams& kp, float2& ch, float2& cl, float2& e12,
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
        float2 xh, xe;
        two_prod2(dup2(kp.beta_h), rh, xh, xe);
        const float2 xl = add2(xe, fma2(dup2(kp.beta_h), rl, mul2(dup2(kp.beta_l), rh)));
        float2 ah, ae;
        two_prod2(dup2(kp.mb2l2e_h), r2h, ah, ae);
        const float2 al = fma2(dup2(kp.mb2l2e_h), r2l, fma2(dup2(kp.mb2l2e_l), r2h, ae));
        float2 eh, el;
        erfc_dd2(xh, xl, ah, al, eh, el);
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
                                       const float2* __restrict__ s_lj, const KParams& kp, float2& ch,
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
                             valid1, m0 & 1, m1 & 1, kp, ch, cl, e12, e12l, e6, e6l, npair);
}

}  // namespace

}  // namespace nbgb
