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
//   Ewald: V = f qi qj erfc(b r)/r, r = r^2 (1/r) in double-float and
//          erfc(b r) from a table of quartics in s = r / h - k (interval
//          width h = 2^-n, built on the host by ewald_energy_table): the
//          constant and linear terms in double-float, the small rest in
//          float32 (error at most about 1.3e-11, no SFU approximation);
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
// i-slot) records; the double-float evaluation then takes 64 queued pairs
// at a time, two per lane as the halves of the paired float32 instructions
// (FADD2, FMUL2, FFMA2), with no idle lanes.
#include "nb_energy2.cuh"

namespace nbgb {

namespace {

constexpr unsigned FULL = FULL_MASK;
constexpr int EW = 8;  // warps per block

// With MK the force kernel of the same evaluation has marked, per entry and
// i-row, the slots inside rc or in the band (ListDev::marks): the warp queues
// them from those bits, without staging the j-clusters or computing any
// distance (the screening is 41% of this kernel's time otherwise).
template <int COUL, bool LJSH, bool MK>
__global__ void __launch_bounds__(EW * 32, 3)
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
    // the Ewald energy table after the Lennard-Jones pairs (16-byte aligned)
    float4* const s_et = reinterpret_cast<float4*>(s_lj + ((nt * nt + 1) & ~1));
    const int etn = COUL == NB_COUL_EWALD ? kp.et_n : 0;
    for (int k = threadIdx.x; k < etn; k += blockDim.x) {
        s_et[k] = kp.etab[k];
        s_et[etn + k] = kp.etab[ET_MAX + k];
    }
    EwaldE et;
    et.a = s_et;
    et.b = s_et + etn;
    et.invh = kp.et_invh;
    et.last = (unsigned)max(etn - 1, 0);
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

        float2 ch = dup2(0.f), cl = dup2(0.f), e12 = dup2(0.f), e12l = dup2(0.f), e6 = dup2(0.f),
               e6l = dup2(0.f);
        int npair = 0;
        int head = 0, tail = 0;  // ring positions, identical in every lane

        if (MK) {
            const int h = i >> 1;
            int e = jb + g;
            unsigned pmk = 0u;
            int pjl = 0, pjh = 0;
            if (e < je) {
                pmk = list.marks[(size_t)e * CL + i];
                entry_slots(list, e, pjl, pjh);
            }
            for (int base = jb; base < je; base += 4) {
                const unsigned mk = pmk;
                const int cjl0 = pjl, cjh0 = pjh;
                e = base + 4 + g;
                pmk = 0u;
                if (e < je) {
                    pmk = list.marks[(size_t)e * CL + i];
                    entry_slots(list, e, pjl, pjh);
                }
                // bit b: j-slot 2 ((b >> 1) XOR h) + (b & 1) is queued (the
                // drain finds the band pairs from its own distances)
#pragma unroll
                for (int b = 0; b < CL; ++b) {
                    const bool q = (mk >> b) & 1u;
                    const unsigned bal = __ballot_sync(FULL, q);
                    if (q) {
                        const int js = 2 * ((b >> 1) ^ h) + (b & 1);
                        const int pos = (tail + __popc(bal & ((1u << lane) - 1u))) & (QCAP - 1);
                        qm[pos] = ((js + (js < 4 ? cjl0 : cjh0)) << 4) | (i << 1);
                    }
                    tail += __popc(bal);
                }
                __syncwarp();
                while (tail - head >= 64) {
                    drain2<COUL, LJSH>(head + lane, qm, irec, xq_s, type_s, s_lj, kp, et, ch, cl, e12, e12l, e6, e6l,
                                       npair, true, true);
                    head += 64;
                }
            }
        } else {
        int e = jb + g;
        bool act = e < je;
        unsigned long long pm = 0ull;
        int pjl = 0, pjh = 0;
        float4 pxq = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
            entry_slots(list, e, pjl, pjh);
            pm = list.mask[e];
            pxq = xq_s[i + (i < 4 ? pjl : pjh)];
        }
        for (int base = jb; base < je; base += 4) {
            __syncwarp();
            sjg[i] = pxq;
            const int cjl0 = pjl, cjh0 = pjh;
            const unsigned long long cm = pm;
            e = base + 4 + g;
            act = e < je;
            pm = 0ull;
            if (act) {
                entry_slots(list, e, pjl, pjh);
                pm = list.mask[e];
                pxq = xq_s[i + (i < 4 ? pjl : pjh)];
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
                    qm[pos] = ((js + (js < 4 ? cjl0 : cjh0)) << 4) | (i << 1) | (int)maybe;
                }
                tail += __popc(bal);
            }
            __syncwarp();
            while (tail - head >= 64) {
                drain2<COUL, LJSH>(head + lane, qm, irec, xq_s, type_s, s_lj, kp, et, ch, cl, e12, e12l, e6, e6l,
                                   npair, true, true);
                head += 64;
            }
        }
        }
        if (tail > head)
            drain2<COUL, LJSH>(head + lane, qm, irec, xq_s, type_s, s_lj, kp, et, ch, cl, e12, e12l, e6, e6l, npair,
                               lane < tail - head, lane + 32 < tail - head);
        dec += ((double)ch.x + (double)cl.x) + ((double)ch.y + (double)cl.y);
        d12 += ((double)e12.x + (double)e12l.x) + ((double)e12.y + (double)e12l.y);
        d6 += ((double)e6.x + (double)e6l.x) + ((double)e6.y + (double)e6l.y);
        if (lane == 0) np += npair;
    }
    if (cur_sys >= 0) flush_energy(sys, cur_sys, dec, d12, d6, np, lane);
}

template <int COUL, bool LJSH>
cudaError_t launch_energy_t(const PlanLaunch& p, cudaStream_t st) {
    // Lennard-Jones pairs, then (Ewald) the energy table's two halves
    const size_t nt2 = (size_t)p.kp.ntypes * p.kp.ntypes;
    size_t smem = ((nt2 + 1) & ~(size_t)1) * sizeof(float2) + (COUL == NB_COUL_EWALD ? 32 * (size_t)p.kp.et_n : 0);
    auto kern = energy_marks(p, NB_F_ENERGY) ? k_energy<COUL, LJSH, true> : k_energy<COUL, LJSH, false>;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, EW * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    return launch_pdl(kern, (unsigned)(p.num_sms * per_sm), EW * 32, smem, st, p.d_sys, p.list, p.kp);
}

}  // namespace

cudaError_t launch_energy(const PlanLaunch& p, cudaStream_t st) {
    if (energy_fused(p)) return cudaSuccess;  // computed by the force kernel
    // the shifted LJ terms are a separate instantiation (double-float LJ),
    // so the default kernel keeps its register budget
    const bool ljsh = p.kp.mods & NB_MOD_LJ_SHIFT;
    if (p.kp.coul == NB_COUL_RF)
        return ljsh ? launch_energy_t<NB_COUL_RF, true>(p, st) : launch_energy_t<NB_COUL_RF, false>(p, st);
    return ljsh ? launch_energy_t<NB_COUL_EWALD, true>(p, st) : launch_energy_t<NB_COUL_EWALD, false>(p, st);
}

}  // namespace nbgb
