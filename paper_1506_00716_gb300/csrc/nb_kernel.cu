// nb_kernel.cu -- the cluster-pair force kernel and the per-evaluation
// stages around it (k_prepare: clear + coordinate update; k_finish: unsort +
// finalisation).
//
// Cluster-pair kernel (Section 3.2): the M = 8 atoms of the i-cluster stay
// in registers while the list entries stream past; every entry's j-cluster
// (N = 8 atoms) is staged in shared memory and its M x N pairs are computed
// without further global loads.  Warp mapping on sm_103a: lane = 8 g + i,
// i = i-slot, g = one of four entries in flight.  The pair arithmetic runs
// on the paired float32 instructions (FADD2, FMUL2, FFMA2): a lane takes two
// j-slots per step, 2m and 2m+1 with m = p XOR (i >> 1) at step p, as the
// halves of float2 values, from a staging layout that keeps both halves of
// every operand in one aligned register pair.  The visiting order makes the
// lane's j-force partial sums line up for a three-step transposed butterfly
// that leaves the full force of j-slot i in lane i (21 shuffles per 64
// pairs).  j-forces then go to memory with one float4 atomic per atom and
// entry; i-forces are reduced over the four groups at the end of the item.
// A persistent grid pulls (i-cluster, shift) work items from a global
// counter, so one launch covers every system of a batch.
//
// Per pair (float32): d = x_i + S - x_j with x_i + S carried error-free as
// hi + lo, r^2, interaction iff mask bit and r^2 < rc^2, 1/r by the SFU
// reciprocal square root,
//   LJ:    F/r = (12 c12 r^-12 - 6 c6 r^-6) / r^2
//   RF:    F/r = f qi qj (r^-3 - 2 k_rf)
//   Ewald: F/r = f qi qj (erfc(b r)/r + 2b/sqrt(pi) exp(-b^2 r^2)) / r^2
//              = f qi qj G(r) / r^3, G(r) = erfc(b r) + 2 b r / sqrt(pi)
//                exp(-b^2 r^2), from a cubic Hermite table of G in shared
//                memory (ewald_force_table: error at most 1e-7, absolute,
//                with G between 0 and 1).  Optional virial
// Xi = -1/2 sum_pairs (F/r) d (x) d, summed per pair in float32 and across
// items in float64.
//
// Cut-off decisions are exact: with reaction field (whose force steps at
// rc), pairs whose float32 r^2 lies within a relative 2e-5 of rc^2 are left
// out of the main pass and decided on a rare path from the float64 distance
// of the float32 inputs, the same decision the float64 oracle takes.
#include "nb_energy2.cuh"

namespace nbgb {

namespace {

constexpr unsigned FULL = FULL_MASK;
constexpr int FW = 8;  // warps per block of the force kernel (the default shape)
// The shape of the 96-register budget (force_min_blocks = 4): two blocks of 10
// warps per SM.  The register file is split between the four SM
// sub-partitions, so 20 warps (5 per sub-partition) is the most that fits at
// 96 registers a thread: 16384 / (5 * 32) = 102.

// The Ewald force table in shared memory (KParams::gtab), in R copies:
// entry k of copy c at k R + c, lane l reading copy l mod R.  A 16-byte
// load is served a quarter warp (eight lanes) at a time, so with R = 8 the
// eight lanes read eight different bank quads wherever their entries lie
// (one copy took 199 M bank conflicts per 3M-atom launch).  R is the
// largest power of two up to 8 that keeps the copies within 40 KB.
__host__ __device__ __forceinline__ int gt_log_rep(int n) {
    int lr = 3;
    while (lr > 0 && (long long)n * (16 << lr) > 40 * 1024) --lr;
    return lr;
}
struct EwaldC {
    const float4* tab;  // this lane's copy
    float invh;
    unsigned last;  // gt_n - 1
    int lr;         // log2 R
};

// 1.5 * 2^23: a float in [2^23, 2^24) holds an integer in its mantissa
constexpr float GT_MAGIC = 12582912.f;

// G(r) from the table: interval k = floor(r / h) by the magic constant and
// a round-down fused multiply-add (no conversion instructions), clamped to
// the table (far and masked slots give finite or NaN values that the cut-off
// select discards), and its cubic in s = r / h - k, formed exactly (h is a
// power of two, so r / h is exact, and so is its fractional part).
__device__ __forceinline__ float ewald_g(float r, const EwaldC& ew) {
    const float m = __fmaf_rd(r, ew.invh, GT_MAGIC);
    const float s = fmaf(r, ew.invh, GT_MAGIC - m);
    const unsigned k = min((unsigned)(__float_as_int(m) - __float_as_int(GT_MAGIC)), ew.last);
    const float4 c = ew.tab[k << ew.lr];
    return fmaf(fmaf(fmaf(c.w, s, c.z), s, c.y), s, c.x);
}
__device__ __forceinline__ float2 ewald_g2(float2 r, const EwaldC& ew) {
    const float2 m = __ffma2_rd(r, dup2(ew.invh), dup2(GT_MAGIC));
    const float2 s = fma2(r, dup2(ew.invh), sub2(dup2(GT_MAGIC), m));
    const unsigned k0 = min((unsigned)(__float_as_int(m.x) - __float_as_int(GT_MAGIC)), ew.last);
    const unsigned k1 = min((unsigned)(__float_as_int(m.y) - __float_as_int(GT_MAGIC)), ew.last);
    const float4 c0 = ew.tab[k0 << ew.lr], c1 = ew.tab[k1 << ew.lr];
    float2 g = fma2(make_float2(c0.w, c1.w), s, make_float2(c0.z, c1.z));
    g = fma2(g, s, make_float2(c0.y, c1.y));
    return fma2(g, s, make_float2(c0.x, c1.x));
}

// Force of one pair slot: d, r^2 and the decision `in` are given.
template <int COUL, bool VIR>
__device__ __forceinline__ void pair_force(float dx, float dy, float dz, float r2, bool in, float qi,
                                           float qj, float2 c, const KParams& kp, const EwaldC& ew,
                                           float& fix, float& fiy, float& fiz, float& fjx,
                                           float& fjy, float& fjz, float (&v)[6]) {
    float rinv = rsqrt_sfu(r2);
    rinv = in ? rinv : 0.f;
    const float qq = in ? qi * qj : 0.f;
    const float rinv2 = rinv * rinv;
    const float rinv6 = rinv2 * rinv2 * rinv2;
    const float t6 = c.x * rinv6;
    const float t12 = c.y * rinv6 * rinv6;
    float fr;  // F/r
    if (COUL == NB_COUL_RF) {
        const float fc = qq * fmaf(rinv, rinv2, -kp.two_krf);
        fr = fmaf(t12 - t6, rinv2, fc);
    } else {
        const float g = ewald_g(r2 * rinv, ew);
        fr = (qq * g * rinv + t12 - t6) * rinv2;
    }
    const float fx = fr * dx, fy = fr * dy, fz = fr * dz;
    fix += fx; fiy += fy; fiz += fz;
    fjx -= fx; fjy -= fy; fjz -= fz;
    if (VIR) {
        v[0] = fmaf(fx, dx, v[0]);
        v[1] = fmaf(fy, dy, v[1]);
        v[2] = fmaf(fz, dz, v[2]);
        v[3] = fmaf(fx, dy, v[3]);
        v[4] = fmaf(fx, dz, v[4]);
        v[5] = fmaf(fy, dz, v[5]);
    }
}

// The i-atom of a lane, shifted, with every component duplicated into both
// halves of a float2.
struct IPair {
    float2 xh, yh, zh, xl, yl, zl;
};

// Force of two pair slots (the halves): as pair_force, with the decisions
// in0, in1 applied to F/r at the end (a slot that is out contributes
// nothing, whatever its arithmetic gave).  With LJW the Lennard-Jones
// parameters are the table's single pair (6 C6, 12 C12) and its term is
// multiplied by the pair weight ww = w_i w_j (0 or 1), which reproduces the
// table's values exactly.
template <int COUL, bool VIR, bool LJW = false>
__device__ __forceinline__ void pair_force2(float2 dx, float2 dy, float2 dz, float2 r2, bool in0, bool in1,
                                            float2 qi, float2 qj, float2 c6, float2 c12, const KParams& kp,
                                            const EwaldC& ew, float2 (&fi)[3], float2 (&fj)[3],
                                            float2 (&v)[6], float2 ww = make_float2(1.f, 1.f)) {
    const float2 rinv = make_float2(rsqrt_sfu(r2.x), rsqrt_sfu(r2.y));
    const float2 qq = mul2(qi, qj);
    const float2 rinv2 = mul2(rinv, rinv);
    const float2 rinv6 = mul2(mul2(rinv2, rinv2), rinv2);
    const float2 t6 = mul2(c6, rinv6);
    const float2 t12 = mul2(mul2(c12, rinv6), rinv6);
    float2 fr;  // F/r
    if (COUL == NB_COUL_RF) {
        const float2 fc = mul2(qq, fma2(rinv, rinv2, dup2(-kp.two_krf)));
        fr = fma2(LJW ? mul2(sub2(t12, t6), ww) : sub2(t12, t6), rinv2, fc);
    } else {
        // f qi qj G(r) / r^3 = (qq G / r) / r^2
        const float2 g = ewald_g2(mul2(r2, rinv), ew);
        const float2 coul = mul2(mul2(qq, g), rinv);
        if (LJW)
            fr = mul2(fma2(sub2(t12, t6), ww, coul), rinv2);
        else
            fr = mul2(sub2(add2(coul, t12), t6), rinv2);
    }
    fr.x = in0 ? fr.x : 0.f;
    fr.y = in1 ? fr.y : 0.f;
    const float2 fx = mul2(fr, dx), fy = mul2(fr, dy), fz = mul2(fr, dz);
    fi[0] = add2(fi[0], fx);
    fi[1] = add2(fi[1], fy);
    fi[2] = add2(fi[2], fz);
    fj[0] = sub2(fj[0], fx);
    fj[1] = sub2(fj[1], fy);
    fj[2] = sub2(fj[2], fz);
    if (VIR) {
        v[0] = fma2(fx, dx, v[0]);
        v[1] = fma2(fy, dy, v[1]);
        v[2] = fma2(fz, dz, v[2]);
        v[3] = fma2(fx, dy, v[3]);
        v[4] = fma2(fx, dz, v[4]);
        v[5] = fma2(fy, dz, v[5]);
    }
}

// Shared-memory block of one staged j-cluster (floats): a 12-float record
// per slot pair (2m, 2m+1) at 12m, holding (x_2m, x_2m+1, y_2m, y_2m+1),
// then (z_2m, z_2m+1, q_2m, q_2m+1), then the types as int2.  Every operand
// of the paired arithmetic arrives as one aligned register pair, and a step
// reads its record from one address.  The 48-byte stride keeps the four
// records a group reads at once in distinct banks.
constexpr int JB_REC = 12, JB_Z = 4, JB_T = 8, JB_SIZE = 4 * JB_REC;
// The (12 c12) table starts this many floats after the (6 c6) table, a
// constant, so that both entries of a type pair are addressed from one
// register; the energies' (c6, c12) table follows it (lj_e_offset).
constexpr int LJ_C12 = MAX_TYPES * MAX_TYPES;
__host__ __device__ __forceinline__ int lj_e_offset(int nt) { return (LJ_C12 + nt * nt + 1) & ~1; }
// the Ewald force table (float4, 16-byte aligned) after both
__host__ __device__ __forceinline__ int gt_offset(int nt) { return (lj_e_offset(nt) + 2 * nt * nt + 3) & ~3; }

// The M x N = 8 x 8 pairs of one entry for one lane (i-slot i), two at a
// time: step p takes the j-slots 2m and 2m+1, m = p XOR (i >> 1), as the
// two halves.  `row` holds the lane's mask bits in that order (bit 2p + c
// for half c of step p).  With EXACT, pairs within the band around rc^2 are
// left out and `band` is set; the caller decides them one by one.
//
// With ENER, the slots whose pair lies inside rc (or within the band around
// it, decided exactly later) are also marked for the energies: bit 2p + c of
// ebits for half c of step p, the same bit of mbits if it lies in the band.
//
// With LJW the staged type slots hold the j-atoms' Lennard-Jones weights
// (0.f or 1.f) and wi2 holds the i-atom's, in both halves.
template <int COUL, bool VIR, bool MASKED, bool SHIFTED, bool EXACT, bool ENER, bool LJW>
__device__ __forceinline__ void pair_block2(const float* __restrict__ sj, int h, const IPair& xs, float2 qi,
                                            const float* __restrict__ ljrow, unsigned row, const KParams& kp, const EwaldC& ew,
                                            float2 (&fi)[3], float2 (&fj)[4][3], float2 (&v)[6], bool& band,
                                            unsigned& ebits, unsigned& mbits, float2 wi2) {
#pragma unroll
    for (int p = 0; p < CL / 2; ++p) {
        const float* rec = sj + JB_REC * (p ^ h);
        const float4 a = *reinterpret_cast<const float4*>(rec);
        const float4 b = *reinterpret_cast<const float4*>(rec + JB_Z);
        const int2 tj = *reinterpret_cast<const int2*>(rec + JB_T);
        float2 dx = sub2(xs.xh, make_float2(a.x, a.y));
        float2 dy = sub2(xs.yh, make_float2(a.z, a.w));
        float2 dz = sub2(xs.zh, make_float2(b.x, b.y));
        if (SHIFTED) {
            dx = add2(dx, xs.xl);
            dy = add2(dy, xs.yl);
            dz = add2(dz, xs.zl);
        }
        const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
        const float lim = EXACT ? kp.rc2_lo : kp.rc2;
        bool in0 = r2.x < lim, in1 = r2.y < lim;
        bool b0 = true, b1 = true;
        if (MASKED) {
            b0 = (row >> (2 * p)) & 1u;
            b1 = (row >> (2 * p + 1)) & 1u;
            in0 = in0 && b0;
            in1 = in1 && b1;
        }
        if (EXACT) band = band || (b0 && !in0 && r2.x < kp.rc2_hi) || (b1 && !in1 && r2.y < kp.rc2_hi);
        if (ENER) {
            const bool q0 = b0 && r2.x < kp.rc2_hi, q1 = b1 && r2.y < kp.rc2_hi;
            ebits |= ((q0 ? 1u : 0u) | (q1 ? 2u : 0u)) << (2 * p);
            mbits |= ((q0 && !(r2.x < kp.rc2_lo) ? 1u : 0u) | (q1 && !(r2.y < kp.rc2_lo) ? 2u : 0u)) << (2 * p);
        }
        if (LJW) {
            const float2 ww = mul2(wi2, make_float2(__int_as_float(tj.x), __int_as_float(tj.y)));
            pair_force2<COUL, VIR, true>(dx, dy, dz, r2, in0, in1, qi, make_float2(b.z, b.w), dup2(kp.c6w),
                                         dup2(kp.c12w), kp, ew, fi, fj[p], v, ww);
        } else {
            const float* l0 = ljrow + tj.x;
            const float* l1 = ljrow + tj.y;
            const float2 c6 = make_float2(l0[0], l1[0]);
            const float2 c12 = make_float2(l0[LJ_C12], l1[LJ_C12]);
            pair_force2<COUL, VIR>(dx, dy, dz, r2, in0, in1, qi, make_float2(b.z, b.w), c6, c12, kp, ew, fi, fj[p],
                                   v);
        }
    }
}

// With ENER (an evaluation with NB_F_ENERGY), the kernel also computes the
// energies: the pairs that the force pass finds inside rc (or in the band
// around it) go to a per-warp ring queue in shared memory as (j slot, i-slot,
// band) records, and whenever 64 are queued the warp evaluates them in
// double-float (nb_energy2.cuh, the energy kernel's arithmetic), two per lane;
// the queue is emptied at the end of every work item.  The energy kernel's
// second pass over the list (staging, screening) is saved.
//
// With LJW (KParams::lj_weights) the Lennard-Jones parameters come from the
// atoms' weights instead of the type-pair table.
//
// With MARK (an evaluation with energies on the separate energy kernel) the
// kernel writes, per entry and i-row, the slots inside rc or in the band
// around it (ListDev::marks), from the distances it has just computed, so
// that the energy kernel needs no second distance pass (it finds the band
// pairs among them from its own double-float distances).
template <int COUL, bool VIR, int MINB, bool ENER, bool LJSH, bool LJW = false, bool MARK = false, int FWT = FW>
__global__ void __launch_bounds__(FWT * 32, MINB)
k_forces(const SysDev* __restrict__ sys, ListDev list, KParams kp) {
    pdl_wait();
    pdl_trigger();
    constexpr bool EXACT = COUL == NB_COUL_RF;
    // (6 c6) table [ntypes^2] at 0, (12 c12) table at LJ_C12; with ENER the
    // (c6, c12) table of the energies (float2) at lj_e_offset(ntypes)
    extern __shared__ float s_ljt[];
    __shared__ __align__(16) float s_j[FWT][4][JB_SIZE];
    __shared__ double s_acc[FWT][6];
    __shared__ float s_fix[FWT][4][CL][3];
    __shared__ int s_qm[ENER ? FWT : 1][ENER ? QCAP : 1];
    __shared__ IRec s_irec[ENER ? FWT : 1][CL];

    const int lane = threadIdx.x & 31;
    const int i = lane & 7;
    const int g = lane >> 3;
    const int w = threadIdx.x >> 5;
    const int h = i >> 1, odd = i & 1;
    const int nt = kp.ntypes;
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
        const float2 c = kp.lj[k];
        s_ljt[k] = c.x;
        s_ljt[LJ_C12 + k] = c.y;
    }
    float2* const s_lje = reinterpret_cast<float2*>(s_ljt + lj_e_offset(nt));
    if (ENER)
        for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) s_lje[k] = kp.lje[k];
    const int gt_lr = gt_log_rep(kp.gt_n);
    if (COUL == NB_COUL_EWALD)
        for (int k = threadIdx.x; k < (kp.gt_n << gt_lr); k += blockDim.x)
            reinterpret_cast<float4*>(s_ljt + gt_offset(nt))[k] = kp.gtab[k >> gt_lr];
    if (lane < 6) s_acc[w][lane] = 0.0;
    __syncthreads();
    int* const qm = s_qm[ENER ? w : 0];
    IRec* const irec = s_irec[ENER ? w : 0];
    double dec = 0.0, d12 = 0.0, d6 = 0.0;
    long long np = 0;

    // the energies' Ewald table (ENER), read through L1
    EwaldE et;
    et.a = kp.etab;
    et.b = kp.etab + ET_MAX;
    et.invh = kp.et_invh;
    et.last = (unsigned)max(kp.et_n - 1, 0);
    EwaldC ew;
    ew.tab = reinterpret_cast<const float4*>(s_ljt + gt_offset(nt)) + (lane & ((1 << gt_lr) - 1));
    ew.invh = kp.gt_invh;
    ew.last = (unsigned)max(kp.gt_n - 1, 0);
    ew.lr = gt_lr;

    float* const sjg = &s_j[w][g][0];
    // the list's j-atoms of this lane's j-slot i: slot cjl[e] * jmul + i
    // (ListDev: 8 x 8 entries name the j-cluster, 8 x 4 entries the first
    // slot of each half, j-slots 4-7 offset by -4)
    const int* const cjl = list.jgeo && i >= 4 ? list.cjb : list.cj;
    const int jmul = list.jgeo ? 1 : CL;
    // where lane i stages j-slot i: x and y at 12 (i >> 1) + (i & 1) (+ 2),
    // z and q 4 floats further, the type 8 floats further
    const int st = JB_REC * h + odd;
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
    float4* f_s = nullptr;
    float Lx = 0.f, Ly = 0.f, Lz = 0.f, Tbx = 0.f, Tcx = 0.f, Tcy = 0.f;

    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(list.counters + CNT_WORK, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= nitems) break;
        const int4 item = list.items[ordered ? ordered_item(list, it, n_long) : it];
        const int sid = item.w >> 5;
        const int sh = item.w & 31;
        if (sid != cur_sys) {
            if (ENER && cur_sys >= 0) flush_energy(sys, cur_sys, dec, d12, d6, np, lane);
            if (VIR && cur_sys >= 0) {
                __syncwarp();
                if (lane < 6 && s_acc[w][lane] != 0.0) atomicAdd(sys[cur_sys].acc + ACC_VXX + lane, s_acc[w][lane]);
                __syncwarp();
                if (lane < 6) s_acc[w][lane] = 0.0;
                __syncwarp();
            }
            cur_sys = sid;
            xq_s = sys[sid].xq_s;
            type_s = sys[sid].type_s;
            f_s = sys[sid].f_s;
            Lx = sys[sid].L[0];
            Ly = sys[sid].L[1];
            Lz = sys[sid].L[2];
            Tbx = sys[sid].T[0];
            Tcx = sys[sid].T[1];
            Tcy = sys[sid].T[2];
        }
        const int ci = item.x, jb = item.y, je = item.z;
        if (jb >= je) continue;
        const bool shifted = sh != SHIFT_ZERO;
        const float4 xi4 = xq_s[ci * CL + i];
        const ShiftedI xs = shift_i(xi4, sh, Lx, Ly, Lz, Tbx, Tcx, Tcy);
        const IPair xp = {dup2(xs.xh), dup2(xs.yh), dup2(xs.zh), dup2(xs.xl), dup2(xs.yl), dup2(xs.zl)};
        const float qi = xi4.w * kp.fq;
        const int ti = type_s[ci * CL + i];
        const int tirow = ti * nt;
        const float* const ljrow = s_ljt + tirow;
        // the weights by selects: converting the 64-bit mask bit to float ran on
        // the FP64 pipe (12.7% busy on the 3M-atom box)
        const float wi = LJW && ((kp.ljw_mask >> ti) & 1ull) ? 1.f : 0.f;
        float2 ch = dup2(0.f), cl = dup2(0.f), e12 = dup2(0.f), e12l = dup2(0.f), e6 = dup2(0.f),
               e6l = dup2(0.f);
        int npair = 0;
        int head = 0, tail = 0;  // energy ring positions, identical in every lane
        if (ENER) {
            __syncwarp();
            if (g == 0) {
                IRec r;
                r.xs = xs;
                two_prod(kp.fq_h, xi4.w, r.qih, r.qil);
                r.qil = fmaf(kp.fq_l, xi4.w, r.qil);
                r.tirow = tirow;
                irec[i] = r;
            }
        }

        float2 fi[3] = {dup2(0.f), dup2(0.f), dup2(0.f)};
        float2 v[6] = {dup2(0.f), dup2(0.f), dup2(0.f), dup2(0.f), dup2(0.f), dup2(0.f)};

        int e = jb + g;
        bool act = e < je;
        int cjn = 0;
        unsigned long long pm = 0ull;
        float4 pxq = make_float4(0.f, 0.f, 0.f, 0.f);
        int pty = 0;
        if (act) {
            cjn = cjl[e];
            pm = list.mask[e];
            pxq = xq_s[cjn * jmul + i];
            pty = type_s[cjn * jmul + i];
        }
        // the list entries one step further ahead, so that the coordinate
        // loads of the next step never wait on them
        int e2 = jb + 4 + g;
        bool act2 = e2 < je;
        int cjn2 = act2 ? cjl[e2] : 0;
        unsigned long long pm2 = act2 ? list.mask[e2] : 0ull;
        for (int base = jb; base < je; base += 4) {
            __syncwarp();
            sjg[st] = pxq.x;
            sjg[st + 2] = pxq.y;
            sjg[JB_Z + st] = pxq.z;
            sjg[JB_Z + st + 2] = pxq.w;
            reinterpret_cast<int*>(sjg)[JB_T + st] = LJW ? (((kp.ljw_mask >> pty) & 1ull) ? __float_as_int(1.f) : 0) : pty;
            const int ccj = cjn;
            const bool cact = act;
            const unsigned long long cm = pm;
            act = act2;
            cjn = cjn2;
            pm = pm2;
            if (act) {
                pxq = xq_s[cjn * jmul + i];
                pty = type_s[cjn * jmul + i];
            }
            e2 = base + 8 + g;
            act2 = e2 < je;
            cjn2 = 0;
            pm2 = 0ull;
            if (act2) {
                cjn2 = cjl[e2];
                pm2 = list.mask[e2];
            }
            __syncwarp();
            // the lane's mask row (bit t: j-slot t XOR i) in the order of the
            // paired steps (bit 2p + c: j-slot 2 (p XOR (i >> 1)) + c), i.e.
            // adjacent bits swapped on odd lanes
            const unsigned row = (unsigned)(cm >> (8 * i)) & 0xffu;
            const unsigned rowp = odd ? (((row & 0x55u) << 1) | ((row >> 1) & 0x55u)) : row;
            float2 fj[CL / 2][3];
#pragma unroll
            for (int p = 0; p < CL / 2; ++p) fj[p][0] = fj[p][1] = fj[p][2] = dup2(0.f);
            bool band = false;
            unsigned ebits = 0u, mbits = 0u;
            const bool full = __all_sync(FULL, row == 0xffu);
            if (full && !shifted)
                pair_block2<COUL, VIR, false, false, EXACT, ENER || MARK, LJW>(sjg, h, xp, dup2(qi), ljrow, rowp, kp, ew,
                                                                      fi, fj, v, band, ebits, mbits, dup2(wi));
            else if (full)
                pair_block2<COUL, VIR, false, true, EXACT, ENER || MARK, LJW>(sjg, h, xp, dup2(qi), ljrow, rowp, kp, ew,
                                                                     fi, fj, v, band, ebits, mbits, dup2(wi));
            else
                pair_block2<COUL, VIR, true, true, EXACT, ENER || MARK, LJW>(sjg, h, xp, dup2(qi), ljrow, rowp, kp, ew,
                                                                    fi, fj, v, band, ebits, mbits, dup2(wi));
            // transposed butterfly over the 8 lanes of the group: half c of
            // fj[p] holds j-slot 2 (p XOR (i >> 1)) + c, so the partners at
            // XOR 4 and 2 hold the same slots in fj[p ^ 2] and fj[p ^ 1]; at
            // XOR 1 each lane keeps its own slot's half and sends the other
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    fj[p][c] = add2(fj[p][c], make_float2(__shfl_xor_sync(FULL, fj[p + 2][c].x, 4),
                                                          __shfl_xor_sync(FULL, fj[p + 2][c].y, 4)));
#pragma unroll
            for (int c = 0; c < 3; ++c)
                fj[0][c] = add2(fj[0][c], make_float2(__shfl_xor_sync(FULL, fj[1][c].x, 2),
                                                      __shfl_xor_sync(FULL, fj[1][c].y, 2)));
            float fjt[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float keep = odd ? fj[0][c].y : fj[0][c].x;
                const float send = odd ? fj[0][c].x : fj[0][c].y;
                fjt[c] = keep + __shfl_xor_sync(FULL, send, 1);
            }
            if (EXACT && __any_sync(FULL, band)) {
                // rare path: pairs within the band around rc, found again with
                // the main pass's arithmetic and decided exactly
                s_fix[w][g][i][0] = s_fix[w][g][i][1] = s_fix[w][g][i][2] = 0.f;
                __syncwarp();
                if (band) {
                    float fsx = 0.f, fsy = 0.f, fsz = 0.f;
                    for (int t = 0; t < CL; ++t) {
                        if (!((row >> t) & 1u)) continue;
                        const int js = t ^ i;
                        const int o = JB_REC * (js >> 1) + (js & 1);
                        const float4 xj = make_float4(sjg[o], sjg[o + 2], sjg[o + JB_Z], sjg[o + JB_Z + 2]);
                        const float dx = (xs.xh - xj.x) + xs.xl;
                        const float dy = (xs.yh - xj.y) + xs.yl;
                        const float dz = (xs.zh - xj.z) + xs.zl;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (r2 < kp.rc2_lo || !(r2 < kp.rc2_hi)) continue;
                        if (!exact_inside(xs, xj, kp.rc2_d)) continue;
                        const int tj = reinterpret_cast<const int*>(sjg)[o + JB_T];
                        const float wij = LJW ? wi * __int_as_float(tj) : 0.f;
                        const float2 c = LJW ? make_float2(kp.c6w * wij, kp.c12w * wij)
                                             : make_float2(ljrow[tj], ljrow[LJ_C12 + tj]);
                        float gx = 0.f, gy = 0.f, gz = 0.f;
                        float vs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        pair_force<COUL, VIR>(dx, dy, dz, r2, true, qi, xj.w, c, kp, ew, fsx, fsy, fsz, gx, gy,
                                              gz, vs);
                        if (VIR) {
#pragma unroll
                            for (int k = 0; k < 6; ++k) v[k].x += vs[k];
                        }
                        atomicAdd(&s_fix[w][g][js][0], gx);
                        atomicAdd(&s_fix[w][g][js][1], gy);
                        atomicAdd(&s_fix[w][g][js][2], gz);
                    }
                    fi[0].x += fsx;
                    fi[1].x += fsy;
                    fi[2].x += fsz;
                }
                __syncwarp();
                fjt[0] += s_fix[w][g][i][0];
                fjt[1] += s_fix[w][g][i][1];
                fjt[2] += s_fix[w][g][i][2];
            }
            if (cact) atomicAdd(f_s + ccj * jmul + i, make_float4(fjt[0], fjt[1], fjt[2], 0.f));
            if (MARK && cact) list.marks[(size_t)(base + g) * CL + i] = (unsigned char)ebits;
            if (ENER) {
                // queue this entry's candidate pairs (bit 2p + c: j-slot
                // 2 (p XOR (i >> 1)) + c), then evaluate them 64 at a time
                const int cnt = __popc(ebits);
                int incl = cnt;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int t = __shfl_up_sync(FULL, incl, off);
                    if (lane >= off) incl += t;
                }
                const int tot = __shfl_sync(FULL, incl, 31);
                int pos = tail + incl - cnt;
                // the slots of the entry's j-slots 0-3 and 4-7 (minus 4), from
                // the group's lanes 0 and 4
                const int jlo = __shfl_sync(FULL, ccj, 8 * g) * jmul, jhi = __shfl_sync(FULL, ccj, 8 * g + 4) * jmul;
                for (unsigned bits = ebits; bits != 0u; bits &= bits - 1u, ++pos) {
                    const int t = __ffs(bits) - 1;
                    const int jt = 2 * ((t >> 1) ^ h) + (t & 1);
                    const int js = jt + (jt < 4 ? jlo : jhi);
                    qm[pos & (QCAP - 1)] = (js << 4) | (i << 1) | (int)((mbits >> t) & 1u);
                }
                tail += tot;
                __syncwarp();
                while (tail - head >= 64) {
                    drain2<COUL, LJSH>(head + lane, qm, irec, xq_s, type_s, s_lje, kp, et, ch, cl, e12, e12l, e6, e6l,
                                       npair, true, true);
                    head += 64;
                }
            }
        }
        if (ENER) {
            if (tail > head)
                drain2<COUL, LJSH>(head + lane, qm, irec, xq_s, type_s, s_lje, kp, et, ch, cl, e12, e12l, e6, e6l, npair,
                                   lane < tail - head, lane + 32 < tail - head);
            dec += ((double)ch.x + (double)cl.x) + ((double)ch.y + (double)cl.y);
            d12 += ((double)e12.x + (double)e12l.x) + ((double)e12.y + (double)e12l.y);
            d6 += ((double)e6.x + (double)e6l.x) + ((double)e6.y + (double)e6l.y);
            if (lane == 0) np += npair;
        }
        float fix = fi[0].x + fi[0].y, fiy = fi[1].x + fi[1].y, fiz = fi[2].x + fi[2].y;
        fix += __shfl_xor_sync(FULL, fix, 8);
        fiy += __shfl_xor_sync(FULL, fiy, 8);
        fiz += __shfl_xor_sync(FULL, fiz, 8);
        fix += __shfl_xor_sync(FULL, fix, 16);
        fiy += __shfl_xor_sync(FULL, fiy, 16);
        fiz += __shfl_xor_sync(FULL, fiz, 16);
        if (g == 0) atomicAdd(f_s + ci * CL + i, make_float4(fix, fiy, fiz, 0.f));
        if (VIR) {
            float vt[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                vt[k] = v[k].x + v[k].y;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) vt[k] += __shfl_xor_sync(FULL, vt[k], off);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) s_acc[w][k] += (double)vt[k];
            }
        }
    }
    if (VIR && cur_sys >= 0) {
        __syncwarp();
        if (lane < 6 && s_acc[w][lane] != 0.0) atomicAdd(sys[cur_sys].acc + ACC_VXX + lane, s_acc[w][lane]);
    }
    if (ENER && cur_sys >= 0) flush_energy(sys, cur_sys, dec, d12, d6, np, lane);
}

// Start of an evaluation: zero the sorted force buffers, the accumulators of
// every system and the work counters; with COORD, also copy new coordinates
// into the sorted slots without re-sorting, applying the box multiples
// recorded by the last grid put (stale-list evaluations).
template <bool COORD>
__global__ void k_prepare(const SysDev* __restrict__ sys, const int* __restrict__ cl_off, int nsys,
                          int tot_slots, int* __restrict__ counters, const float* __restrict__ x_ext) {
    pdl_wait();
    pdl_trigger();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        counters[CNT_WORK] = 0;
        counters[CNT_EWORK] = 0;
    }
    if (t >= tot_slots) return;
    int s = find_sys_dev(cl_off, nsys, t / CL);
    const SysDev& d = sys[s];
    int slot = t - cl_off[s] * CL;
    d.f_s[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (slot < NACC) d.acc[slot] = 0.0;
    if (!COORD) return;
    if (slot >= d.col_cl0[d.ncol] * CL) return;
    int a = d.perm[slot];
    if (a < 0) return;
    int wk = d.wrapk[slot];
    int kx = (int)(signed char)(wk & 0xff);
    int ky = (int)(signed char)((wk >> 8) & 0xff);
    int kz = (int)(signed char)((wk >> 16) & 0xff);
    const float* xn = x_ext ? x_ext : d.x_new;
    // minus the lattice vector the last grid put removed: kx a + ky b + kz c
    float4 v = d.xq_s[slot];
    v.x = xn[3 * a + 0] - (float)kx * d.L[0] - (float)ky * d.T[0] - (float)kz * d.T[1];
    v.y = xn[3 * a + 1] - (float)ky * d.L[1] - (float)kz * d.T[2];
    v.z = xn[3 * a + 2] - (float)kz * d.L[2];
    d.xq_s[slot] = v;
}

// End of an evaluation: forces back to the caller's atom order and, with
// ENER_VIR, the final FP64 combination of each system's accumulators.
template <bool ENER_VIR>
__global__ void k_finish(const SysDev* __restrict__ sys, const int* __restrict__ atom_off, int nsys,
                         int tot_atoms, float* __restrict__ f_ext, double* __restrict__ e_ext,
                         double* __restrict__ v_ext) {
    pdl_wait();
    pdl_trigger();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (ENER_VIR && t < nsys) {
        const SysDev& d = sys[t];
        const double* a = d.acc;
        double* r = d.res;
        r[0] = a[ACC_E12] - a[ACC_E6];
        r[1] = a[ACC_EC] + a[ACC_ECLO] + (a[ACC_EREC] + a[ACC_ESELF] + a[ACC_EEXCL]);
        r[2] = -0.5 * a[ACC_VXX];
        r[3] = -0.5 * a[ACC_VXY];
        r[4] = -0.5 * a[ACC_VXZ];
        r[5] = -0.5 * a[ACC_VXY];
        r[6] = -0.5 * a[ACC_VYY];
        r[7] = -0.5 * a[ACC_VYZ];
        r[8] = -0.5 * a[ACC_VXZ];
        r[9] = -0.5 * a[ACC_VYZ];
        r[10] = -0.5 * a[ACC_VZZ];
        r[11] = a[ACC_NPAIR];
        r[12] = a[ACC_EREC];
        r[13] = a[ACC_ESELF];
        r[14] = a[ACC_EEXCL];
        if (e_ext) {
            e_ext[0] = r[0];
            e_ext[1] = r[1];
        }
        if (v_ext)
            for (int k = 0; k < 9; ++k) v_ext[k] = r[2 + k];
    }
    if (t >= tot_atoms) return;
    int s = find_sys_dev(atom_off, nsys, t);
    const SysDev& d = sys[s];
    int a = t - atom_off[s];
    float4 f = d.f_s[d.iperm[a]];
    d.f_out[3 * a + 0] = f.x;
    d.f_out[3 * a + 1] = f.y;
    d.f_out[3 * a + 2] = f.z;
    if (f_ext) {
        f_ext[3 * a + 0] = f.x;
        f_ext[3 * a + 1] = f.y;
        f_ext[3 * a + 2] = f.z;
    }
}

template <int COUL, bool VIR, int MINB, bool ENER = false, bool LJSH = false, bool LJW = false, bool MARK = false,
          int FWT = FW>
cudaError_t launch_forces_t(const PlanLaunch& p, cudaStream_t st) {
    const size_t nt2 = (size_t)p.kp.ntypes * p.kp.ntypes;
    // LJ tables (the energies' too with ENER), then the Ewald force table
    const size_t smem = COUL == NB_COUL_EWALD ? (gt_offset(p.kp.ntypes) + ((4 * (size_t)p.kp.gt_n) << gt_log_rep(p.kp.gt_n))) * sizeof(float)
                        : ENER ? (lj_e_offset(p.kp.ntypes) + 2 * nt2) * sizeof(float)
                               : (LJ_C12 + nt2) * sizeof(float);
    auto kern = k_forces<COUL, VIR, MINB, ENER, LJSH, LJW, MARK, FWT>;
    if (ENER || smem > 48 * 1024) {
        // the energy queue (or a large Ewald table) makes static + dynamic
        // shared memory pass 48 KB: allow the dynamic part explicitly
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FWT * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    return launch_pdl(kern, (unsigned)(p.num_sms * per_sm), FWT * 32, smem, st, p.d_sys, p.list, p.kp);
}

}  // namespace

cudaError_t launch_prepare(const PlanLaunch& p, bool coords, cudaStream_t st) {
    int tot = p.tot_clcap * CL;
    int bs = 256;
    unsigned blocks = (unsigned)((tot + bs - 1) / bs + 1);
    const float* x_ext = p.nsys == 1 ? p.x_ext : nullptr;
    if (coords)
        return launch_pdl(k_prepare<true>, blocks, bs, 0, st, p.d_sys, p.d_cl_off, p.nsys, tot, p.list.counters, x_ext);
    return launch_pdl(k_prepare<false>, blocks, bs, 0, st, p.d_sys, p.d_cl_off, p.nsys, tot, p.list.counters,
                      (const float*)nullptr);
}

// The force kernel writing the energy kernel's marks (register budgets 2, 3
// and 4: two or three blocks of 8 warps, two of 10).
template <int COUL, bool VIR>
cudaError_t launch_forces_m(const PlanLaunch& p, cudaStream_t st) {
    const bool w = p.kp.lj_weights != 0;
    if (p.kp.force_min_blocks == 4)
        return w ? launch_forces_t<COUL, VIR, 2, false, false, true, true, 10>(p, st)
                 : launch_forces_t<COUL, VIR, 2, false, false, false, true, 10>(p, st);
    if (p.kp.force_min_blocks == 2)
        return w ? launch_forces_t<COUL, VIR, 2, false, false, true, true>(p, st)
                 : launch_forces_t<COUL, VIR, 2, false, false, false, true>(p, st);
    return w ? launch_forces_t<COUL, VIR, 3, false, false, true, true>(p, st)
             : launch_forces_t<COUL, VIR, 3, false, false, false, true>(p, st);
}

template <int COUL, bool VIR>
cudaError_t launch_forces_v(const PlanLaunch& p, cudaStream_t st) {
    // Lennard-Jones by weights for the register budgets of 2 and 3 blocks per
    // SM (the others take the table)
    const bool w = p.kp.lj_weights != 0;
    switch (p.kp.force_min_blocks) {
        case 1: return launch_forces_t<COUL, VIR, 1>(p, st);
        case 2: return w ? launch_forces_t<COUL, VIR, 2, false, false, true>(p, st) : launch_forces_t<COUL, VIR, 2>(p, st);
        case 4:
            return w ? launch_forces_t<COUL, VIR, 2, false, false, true, false, 10>(p, st)
                     : launch_forces_t<COUL, VIR, 2, false, false, false, false, 10>(p, st);
        default: return w ? launch_forces_t<COUL, VIR, 3, false, false, true>(p, st) : launch_forces_t<COUL, VIR, 3>(p, st);
    }
}

// The force kernel with the energies fused in (NB_F_ENERGY evaluations when
// the tuning's energy_mode is 1): one register budget (2 blocks per SM).
template <int COUL, bool VIR>
cudaError_t launch_forces_e(const PlanLaunch& p, cudaStream_t st) {
    if (p.kp.mods & NB_MOD_LJ_SHIFT) return launch_forces_t<COUL, VIR, 2, true, true>(p, st);
    return launch_forces_t<COUL, VIR, 2, true, false>(p, st);
}

bool energy_fused(const PlanLaunch& p) { return p.kp.energy_mode == 1; }

bool energy_marks(const PlanLaunch& p, unsigned flags) {
    return (flags & NB_F_ENERGY) && !energy_fused(p) && p.list.marks != nullptr && p.kp.force_min_blocks != 1;
}

cudaError_t launch_forces(const PlanLaunch& p, unsigned flags, cudaStream_t st) {
    bool vi = flags & NB_F_VIRIAL;
    if ((flags & NB_F_ENERGY) && energy_fused(p)) {
        if (p.kp.coul == NB_COUL_RF)
            return vi ? launch_forces_e<NB_COUL_RF, true>(p, st) : launch_forces_e<NB_COUL_RF, false>(p, st);
        return vi ? launch_forces_e<NB_COUL_EWALD, true>(p, st) : launch_forces_e<NB_COUL_EWALD, false>(p, st);
    }
    if (energy_marks(p, flags)) {
        if (p.kp.coul == NB_COUL_RF)
            return vi ? launch_forces_m<NB_COUL_RF, true>(p, st) : launch_forces_m<NB_COUL_RF, false>(p, st);
        return vi ? launch_forces_m<NB_COUL_EWALD, true>(p, st) : launch_forces_m<NB_COUL_EWALD, false>(p, st);
    }
    if (p.kp.coul == NB_COUL_RF)
        return vi ? launch_forces_v<NB_COUL_RF, true>(p, st) : launch_forces_v<NB_COUL_RF, false>(p, st);
    return vi ? launch_forces_v<NB_COUL_EWALD, true>(p, st) : launch_forces_v<NB_COUL_EWALD, false>(p, st);
}

cudaError_t launch_finalize(const PlanLaunch& p, unsigned flags, cudaStream_t st) {
    int bs = 256;
    int n = p.tot_atoms > p.nsys ? p.tot_atoms : p.nsys;
    unsigned blocks = (unsigned)((n + bs - 1) / bs);
    const bool one = p.nsys == 1;
    float* f_ext = one ? p.f_ext : nullptr;
    double* e_ext = one && (flags & NB_F_ENERGY) ? p.e_ext : nullptr;
    double* v_ext = one && (flags & NB_F_VIRIAL) ? p.v_ext : nullptr;
    if (flags & (NB_F_ENERGY | NB_F_VIRIAL))
        return launch_pdl(k_finish<true>, blocks, bs, 0, st, p.d_sys, p.d_atom_off, p.nsys, p.tot_atoms, f_ext, e_ext,
                          v_ext);
    return launch_pdl(k_finish<false>, blocks, bs, 0, st, p.d_sys, p.d_atom_off, p.nsys, p.tot_atoms, f_ext,
                      (double*)nullptr, (double*)nullptr);
}

}  // namespace nbgb
