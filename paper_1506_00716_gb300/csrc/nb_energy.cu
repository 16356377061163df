// nb_energy.cu -- the energy kernel: Lennard-Jones and Coulomb energies of
// the cluster-pair list, and the count of interacting pairs.
//
// The system energy of a box of neutral molecules is a sum of pair terms that
// cancel to a few parts in 10^3 - 10^4 (Coulomb), so float32 pair terms
// (relative error ~1e-7 each) cannot give the energy to 1e-6.  This kernel
// therefore evaluates each pair in double-float arithmetic on the float32
// pipes (values carried as unevaluated sums hi + lo of two floats, built
// from error-free two-sum / two-product steps):
//   d = x_i + S - x_j and r^2 in double-float, 1/r = y (1 + h/2) with
//   y = rsqrt(r^2_hi) and the residual h = 1 - r^2 y^2 computed with fused
//   multiply-adds, and then
//   RF:    V = f qi qj (1/r + k_rf r^2 - c_rf) fully in double-float;
//   Ewald: V = f qi qj erfc(b r)/r with erfc(x) = exp(-x^2) R(u) from the
//          degree-12 fit and exp(-x^2) = 2^a by exact range reduction and
//          the degree-10 fit of 2^f (no SFU approximation); x = b r, t, u
//          and the large head terms of both polynomials in double-float
//          (compensated Horner), their small tails in float32;
//   LJ:    c12 r^-12, c6 r^-6 in float32 from the accurate 1/r and the
//          unscaled c6, c12 (pre-scaled 6 c6, 12 c12 would round).
// With the potential-shift modifiers the LJ terms become c12 (r^-12 -
// rc^-12) and c6 (r^-6 - rc^-6), and erfc(beta r)/r becomes erfc(beta r)/r -
// erfc(beta rc)/rc (the constant as hi + lo).
// Coulomb energies accumulate in double-float per lane and work item, and in
// float64 across items and warps.  Cut-off decisions are exact (the float64
// distance of the float32 inputs decides pairs near rc), so the counted pair
// set is the oracle's.  The work distribution is the force kernel's: a
// persistent grid over the (i-cluster, shift) items, four entries in flight
// per warp, j-clusters staged in shared memory.  Only about a third of the
// 8 x 8 pair slots lie inside rc, so each warp first screens its slots in
// float32 and pushes the pairs inside rc (or within the band around it,
// decided exactly later) into a ring queue in shared memory as (j slot,
// i-slot) records; the double-float evaluation then takes 32 queued pairs
// at a time, one per lane, with no idle lanes.
#include "erfc_fit.cuh"
#include "nb_device.cuh"

namespace nbgb {

namespace {

constexpr unsigned FULL = FULL_MASK;
constexpr int EW = 8;  // warps per block

// Horner steps over coefficients hi[k] + lo[k], k = k1 .. 0, in compensated
// (double-float) arithmetic: p = p * u + c with p, u, c all hi + lo.
template <int K1>
__device__ __forceinline__ void horner_dd(const float* hi, const float* lo, float uh, float ul, float& ph,
                                          float& pl) {
#pragma unroll
    for (int k = K1; k >= 0; --k) {
        float m, me, sum, se;
        two_prod(ph, uh, m, me);
        const float cross = fmaf(ph, ul, pl * uh);
        two_sum(m, hi[k], sum, se);
        ph = sum;
        pl = ((me + se) + cross) + lo[k];
    }
}

// Number of head coefficients evaluated in double-float; the tail terms are
// small enough (|a_k u^k| <= 5e-4) for plain float32.
constexpr int EF_HEAD = 5;   // erfc fit: k = 0..4
constexpr int EX2_HEAD = 4;  // 2^f fit: k = 0..3

// erfc(x) in double-float for x = xh + xl >= 0, from the degree-12 fit and
// the double-float exponential 2^a, a = ah + al = -x^2 log2(e) (given).
__device__ __forceinline__ void erfc_dd(float xh, float xl, float ah, float al, float& eh, float& el) {
    if (xh > EF_XMAX) {
        xh = EF_XMAX;
        xl = 0.f;
    }
    // d = 1 + P x
    float m, me, dh, de;
    two_prod(EF_P, xh, m, me);
    two_sum(1.f, m, dh, de);
    const float dl = de + fmaf(EF_P, xl, me);
    // t = 1 / d
    float th = rcp_sfu(dh);
    th = th * fmaf(-dh, th, 2.f);
    float r = fmaf(-dh, th, 1.f);
    r = fmaf(-dl, th, r);
    const float tl = th * r;
    // u = UA t + UB
    float uh, ue, sh, se;
    two_prod(EF_UA, th, uh, ue);
    two_sum(uh, EF_UB, sh, se);
    const float ul = se + fmaf(EF_UA, tl, ue);
    uh = sh;
    // R(u): float32 tail, double-float head
    float ph = EF_EN_HI[EF_NE - 1], pl = 0.f;
#pragma unroll
    for (int k = EF_NE - 2; k >= EF_HEAD; --k) ph = fmaf(ph, uh, EF_EN_HI[k]);
    horner_dd<EF_HEAD - 1>(EF_EN_HI, EF_EN_LO, uh, ul, ph, pl);
    // 2^a = 2^n 2^f, f = (ah - n) + al in [-0.5, 0.5], ah - n exact
    ah = fmaxf(ah, -120.f);
    const float n = rintf(ah);
    const float fh = ah - n;
    float qh = EX2_HI[EX2_N - 1], ql = 0.f;
#pragma unroll
    for (int k = EX2_N - 2; k >= EX2_HEAD; --k) qh = fmaf(qh, fh, EX2_HI[k]);
    horner_dd<EX2_HEAD - 1>(EX2_HI, EX2_LO, fh, al, qh, ql);
    const float scale = __int_as_float(((int)n + 127) << 23);
    // erfc = R 2^a
    float ch, ce;
    two_prod(ph, qh, ch, ce);
    const float cl = ce + fmaf(ph, ql, pl * qh);
    eh = ch * scale;
    el = cl * scale;
}

// Energy of one queued pair.  `valid`: the lane holds a pair; `maybe`: its
// float32 r^2 fell in the band around rc^2 and the decision is taken here,
// exactly; otherwise the pair is inside rc.
template <int COUL, bool LJSH>
__device__ __forceinline__ void pair_energy(const float4 xj, int tj, const ShiftedI& xs, float qih,
                                            float qil, int tirow, const float2* __restrict__ s_lj,
                                            bool valid, bool maybe, const KParams& kp, float& ch,
                                            float& cl, float& e12, float& e12l, float& e6, float& e6l,
                                            int& npair) {
    float dxh, dxe, dyh, dye, dzh, dze;
    two_sum(xs.xh, -xj.x, dxh, dxe);
    two_sum(xs.yh, -xj.y, dyh, dye);
    two_sum(xs.zh, -xj.z, dzh, dze);
    const float dxl = dxe + xs.xl, dyl = dye + xs.yl, dzl = dze + xs.zl;
    float px, ex, py, ey, pz, ez;
    two_prod(dxh, dxh, px, ex);
    two_prod(dyh, dyh, py, ey);
    two_prod(dzh, dzh, pz, ez);
    ex = fmaf(2.f * dxh, dxl, ex);
    ey = fmaf(2.f * dyh, dyl, ey);
    ez = fmaf(2.f * dzh, dzl, ez);
    float s1, e1, r2h, e2;
    two_sum(px, py, s1, e1);
    two_sum(s1, pz, r2h, e2);
    const float r2l = (e1 + e2) + (ex + (ey + ez));

    bool in = valid;
    if (valid && maybe) in = exact_inside(xs, xj, kp.rc2_d);
    npair += __popc(__ballot_sync(FULL, in));

    // 1/r = y (1 + h/2), h = 1 - r^2 y^2
    const float y = rsqrt_sfu(r2h);
    float y2, y2e;
    two_prod(y, y, y2, y2e);
    float h = fmaf(-r2h, y2, 1.f);
    h = fmaf(-r2h, y2e, h);
    h = fmaf(-r2l, y2, h);
    const float ril = 0.5f * y * h;
    const float rif = y + ril;

    const float2 c = s_lj[tirow + tj];
    if (LJSH) {
        // Shifted LJ energies, c12 (r^-12 - rc^-12) and c6 (r^-6 - rc^-6),
        // in double-float: the shift takes away most of E_LJ, so the float32
        // terms' rounding would no longer be small next to what is left.
        float ah, al;
        fast_two_sum(y, ril, ah, al);  // 1/r
        float p2h, p2l, p4h, p4l, p6h, p6l, p12h, p12l;
        dd_mul(ah, al, ah, al, p2h, p2l);
        dd_mul(p2h, p2l, p2h, p2l, p4h, p4l);
        dd_mul(p4h, p4l, p2h, p2l, p6h, p6l);
        dd_mul(p6h, p6l, p6h, p6l, p12h, p12l);
        float dh, dl, t6, t6l, t12, t12l;
        two_sum(p6h, -kp.irc6_h, dh, dl);
        dl += p6l - kp.irc6_l;
        two_prod(c.x, dh, t6, t6l);
        t6l = fmaf(c.x, dl, t6l);
        two_sum(p12h, -kp.irc12_h, dh, dl);
        dl += p12l - kp.irc12_l;
        two_prod(c.y, dh, t12, t12l);
        t12l = fmaf(c.y, dl, t12l);
        if (in) {
            float sh, se;
            two_sum(e12, t12, sh, se);
            e12 = sh;
            e12l += se + t12l;
            two_sum(e6, t6, sh, se);
            e6 = sh;
            e6l += se + t6l;
        }
    } else {
        const float ri2 = rif * rif;
        const float ri6 = ri2 * ri2 * ri2;
        const float t6 = c.x * ri6;
        const float t12 = c.y * ri6 * ri6;
        e12 += in ? t12 : 0.f;
        e6 += in ? t6 : 0.f;
    }

    float qh, qe;
    two_prod(qih, xj.w, qh, qe);
    const float ql = fmaf(qil, xj.w, qe);
    float vh, vl;
    if (COUL == NB_COUL_RF) {
        float kh, ke;
        two_prod(kp.krf_h, r2h, kh, ke);
        const float kl = fmaf(kp.krf_h, r2l, fmaf(kp.krf_l, r2h, ke));
        float sh, es, gh, eg;
        two_sum(y, kh, sh, es);
        two_sum(sh, -kp.crf_h, gh, eg);
        const float gl = ((es + eg) + (ril + kl)) - kp.crf_l;
        float ve;
        two_prod(qh, gh, vh, ve);
        vl = fmaf(qh, gl, fmaf(ql, gh, ve));
    } else {
        // r = r^2 (1/r), x = beta r, all double-float
        float rh, re;
        two_prod(r2h, y, rh, re);
        const float rl = re + fmaf(r2h, ril, r2l * y);
        float xh, xe;
        two_prod(kp.beta_h, rh, xh, xe);
        const float xl = xe + fmaf(kp.beta_h, rl, kp.beta_l * rh);
        float ah, ae;
        two_prod(kp.mb2l2e_h, r2h, ah, ae);
        const float al = fmaf(kp.mb2l2e_h, r2l, fmaf(kp.mb2l2e_l, r2h, ae));
        float eh, el;
        erfc_dd(xh, xl, ah, al, eh, el);
        // w = erfc / r, V = q q w
        float wh, we;
        two_prod(eh, y, wh, we);
        float wl = we + fmaf(eh, ril, el * y);
        if (kp.mods & NB_MOD_EWALD_SHIFT) {
            // w - erfc(beta rc)/rc, in double-float
            float dh, de;
            two_sum(wh, -kp.ewc_h, dh, de);
            wl = de + (wl - kp.ewc_l);
            wh = dh;
        }
        float ve;
        two_prod(qh, wh, vh, ve);
        vl = ve + fmaf(qh, wl, ql * wh);
    }
    if (!in) {
        vh = 0.f;
        vl = 0.f;
    }
    float th, te;
    two_sum(ch, vh, th, te);
    ch = th;
    cl += te + vl;
}

__device__ __forceinline__ void flush_energy(const SysDev* __restrict__ sys, int s, double& dec,
                                             double& d12, double& d6, long long& np, int lane) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dec += __shfl_xor_sync(FULL, dec, off);
        d12 += __shfl_xor_sync(FULL, d12, off);
        d6 += __shfl_xor_sync(FULL, d6, off);
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

constexpr int QCAP = 512;  // per-warp ring queue of candidate pairs (>= 31 + 8 * 32)

// i-atom data of the current item, one record per i-slot (shared by the
// lanes that evaluate queued pairs).
struct IRec {
    ShiftedI xs;
    float qih, qil;
    int tirow;
};

// Queue entry: j slot index << 4 | i-slot << 1 | band flag.
template <int COUL, bool LJSH>
__device__ __forceinline__ void drain(int k, const int* __restrict__ qm, const IRec* __restrict__ irec,
                                      const float4* __restrict__ xq_s, const int* __restrict__ type_s,
                                      const float2* __restrict__ s_lj, const KParams& kp, float& ch,
                                      float& cl, float& e12, float& e12l, float& e6, float& e6l, int& npair,
                                      bool valid) {
    const int m = valid ? qm[k & (QCAP - 1)] : 0;
    const int js = m >> 4;
    const float4 xj = valid ? xq_s[js] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int tj = valid ? type_s[js] : 0;
    const IRec& ir = irec[(m >> 1) & 7];
    pair_energy<COUL, LJSH>(xj, tj, ir.xs, ir.qih, ir.qil, ir.tirow, s_lj, valid, m & 1, kp, ch, cl, e12, e12l, e6,
                      e6l, npair);
}

template <int COUL, bool LJSH>
__global__ void __launch_bounds__(EW * 32)
k_energy(const SysDev* __restrict__ sys, ListDev list, KParams kp) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float2 s_lj[];
    __shared__ __align__(16) float4 s_j[EW][4][2 * CL];
    __shared__ int s_qm[EW][QCAP];
    __shared__ IRec s_irec[EW][CL];

    const int lane = threadIdx.x & 31;
    const int i = lane & 7;
    const int g = lane >> 3;
    const int w = threadIdx.x >> 5;
    const int nt = kp.ntypes;
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) s_lj[k] = kp.lje[k];
    __syncthreads();

    float4* sjg = &s_j[w][g][0];
    int* qm = s_qm[w];
    IRec* irec = s_irec[w];
    // longest-first order for short lists, where the last items decide the
    // launch's length; cluster order otherwise (neighbouring items share
    // j-clusters in L1 and L2)
    const int n_raw = min(list.counters[CNT_ITEMS], list.item_cap);
    const bool ordered = n_raw <= kp.lpt_max_items;
    const int n_long = ordered ? list.counters[CNT_ORD_LONG] : 0;
    const int nitems = ordered ? n_long + list.counters[CNT_ORD_SHORT] : n_raw;
    int cur_sys = -1;
    const float4* xq_s = nullptr;
    const int* type_s = nullptr;
    float Lx = 0.f, Ly = 0.f, Lz = 0.f, Tbx = 0.f, Tcx = 0.f, Tcy = 0.f;
    double dec = 0.0, d12 = 0.0, d6 = 0.0;
    long long np = 0;

    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(list.counters + CNT_EWORK, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= nitems) break;
        const int4 item = list.items[ordered ? ordered_item(list, it, n_long) : it];
        const int sid = item.w >> 5;
        const int sh = item.w & 31;
        if (sid != cur_sys) {
            if (cur_sys >= 0) flush_energy(sys, cur_sys, dec, d12, d6, np, lane);
            cur_sys = sid;
            xq_s = sys[sid].xq_s;
            type_s = sys[sid].type_s;
            Lx = sys[sid].L[0];
            Ly = sys[sid].L[1];
            Lz = sys[sid].L[2];
            Tbx = sys[sid].T[0];
            Tcx = sys[sid].T[1];
            Tcy = sys[sid].T[2];
        }
        const int ci = item.x, jb = item.y, je = item.z;
        if (jb >= je) continue;
        const float4 xi4 = xq_s[ci * CL + i];
        const ShiftedI xs = shift_i(xi4, sh, Lx, Ly, Lz, Tbx, Tcx, Tcy);
        __syncwarp();
        if (g == 0) {
            IRec r;
            r.xs = xs;
            two_prod(kp.fq_h, xi4.w, r.qih, r.qil);
            r.qil = fmaf(kp.fq_l, xi4.w, r.qil);
            r.tirow = type_s[ci * CL + i] * nt;
            irec[i] = r;
        }

        float ch = 0.f, cl = 0.f, e12 = 0.f, e12l = 0.f, e6 = 0.f, e6l = 0.f;
        int npair = 0;
        int head = 0, tail = 0;  // ring positions, identical in every lane

        int e = jb + g;
        bool act = e < je;
        unsigned long long pm = 0ull;
        int pj = 0;
        float4 pxq = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
            pj = list.cj[e] * CL;
            pm = list.mask[e];
            pxq = xq_s[pj + i];
        }
        for (int base = jb; base < je; base += 4) {
            __syncwarp();
            sjg[i] = pxq;
            const int cj0 = pj;
            const unsigned long long cm = pm;
            e = base + 4 + g;
            act = e < je;
            pm = 0ull;
            if (act) {
                pj = list.cj[e] * CL;
                pm = list.mask[e];
                pxq = xq_s[pj + i];
            }
            __syncwarp();
            const unsigned row = (unsigned)(cm >> (8 * i)) & 0xffu;
#pragma unroll
            for (int t = 0; t < CL; ++t) {
                const int js = t ^ i;
                const float4 xj = sjg[js];
                const float dx = xs.xh - xj.x, dy = xs.yh - xj.y, dz = xs.zh - xj.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const bool bit = (row >> t) & 1u;
                const bool in = bit && r2 < kp.rc2_lo;
                const bool maybe = bit && !in && r2 < kp.rc2_hi;
                const bool q = in || maybe;
                const unsigned bal = __ballot_sync(FULL, q);
                if (q) {
                    const int pos = (tail + __popc(bal & ((1u << lane) - 1u))) & (QCAP - 1);
                    qm[pos] = ((cj0 + js) << 4) | (i << 1) | (int)maybe;
                }
                tail += __popc(bal);
            }
            __syncwarp();
            while (tail - head >= 32) {
                drain<COUL, LJSH>(head + lane, qm, irec, xq_s, type_s, s_lj, kp, ch, cl, e12, e12l, e6, e6l, npair,
                            true);
                head += 32;
            }
        }
        if (tail > head)
            drain<COUL, LJSH>(head + lane, qm, irec, xq_s, type_s, s_lj, kp, ch, cl, e12, e12l, e6, e6l, npair,
                        lane < tail - head);
        dec += (double)ch + (double)cl;
        d12 += (double)e12 + (double)e12l;
        d6 += (double)e6 + (double)e6l;
        if (lane == 0) np += npair;
    }
    if (cur_sys >= 0) flush_energy(sys, cur_sys, dec, d12, d6, np, lane);
}

template <int COUL, bool LJSH>
cudaError_t launch_energy_t(const PlanLaunch& p, cudaStream_t st) {
    size_t smem = (size_t)p.kp.ntypes * p.kp.ntypes * sizeof(float2);
    auto kern = k_energy<COUL, LJSH>;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, EW * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    return launch_pdl(kern, (unsigned)(p.num_sms * per_sm), EW * 32, smem, st, p.d_sys, p.list, p.kp);
}

}  // namespace

cudaError_t launch_energy(const PlanLaunch& p, cudaStream_t st) {
    // the shifted LJ terms are a separate instantiation (double-float LJ),
    // so the default kernel keeps its register budget
    const bool ljsh = p.kp.mods & NB_MOD_LJ_SHIFT;
    if (p.kp.coul == NB_COUL_RF)
        return ljsh ? launch_energy_t<NB_COUL_RF, true>(p, st) : launch_energy_t<NB_COUL_RF, false>(p, st);
    return ljsh ? launch_energy_t<NB_COUL_EWALD, true>(p, st) : launch_energy_t<NB_COUL_EWALD, false>(p, st);
}

}  // namespace nbgb
