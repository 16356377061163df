// nb_excl.cu -- reaction-field correction of excluded pairs (NB_MOD_RF_EXCL).
//
// With the modifier, every excluded atom pair (i, j) whose minimum-image
// distance is inside rc contributes V = f qi qj / eps_r (k_rf r^2 - c_rf) to
// the Coulomb energy, the force of that potential, F_i = -2 f qi qj / eps_r
// k_rf (x_i - x_j) = -F_j, and its virial.  The pairs are few (about one per
// atom in water) and are taken straight from the symmetric exclusion list,
// each unordered pair once (j > i), in float64: the cut-off decision is then
// the float64 one and the energy needs no compensation.  One thread per atom
// of every system of the plan; the coordinates are the sorted slots' current
// ones (the same the force kernel used), reached through the atom's slot.
#include "nb_device.cuh"

namespace nbgb {

namespace {

constexpr unsigned FULL = FULL_MASK;

__device__ __forceinline__ double min_image_d(double d, double L) { return d - L * rint(d / L); }

template <bool ENER, bool VIR>
__global__ void k_excl_rf(const SysDev* __restrict__ sys, const int* __restrict__ atom_off, int nsys,
                          int tot_atoms, KParams kp) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    double e = 0.0;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int s = -1;
    if (t < tot_atoms) {
        s = find_sys_dev(atom_off, nsys, t);
        const SysDev& d = sys[s];
        const int a = t - atom_off[s];
        if (d.excl_index) {
            const int sa = d.iperm[a];
            const float4 xa = d.xq_s[sa];
            const double Lx = d.L[0], Ly = d.L[1], Lz = d.L[2];
            float fx = 0.f, fy = 0.f, fz = 0.f;
            for (int k = d.excl_index[a]; k < d.excl_index[a + 1]; ++k) {
                const int b = d.excl_atoms[k];
                if (b <= a) continue;
                const int sb = d.iperm[b];
                const float4 xb = d.xq_s[sb];
                const double dx = min_image_d((double)xa.x - (double)xb.x, Lx);
                const double dy = min_image_d((double)xa.y - (double)xb.y, Ly);
                const double dz = min_image_d((double)xa.z - (double)xb.z, Lz);
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < kp.rc2_d)) continue;
                const double fqq = kp.fq_d * (double)xa.w * (double)xb.w;
                const double fr = -2.0 * fqq * kp.krf_d;  // F/r
                if (ENER) e += fqq * (kp.krf_d * r2 - kp.crf_d);
                if (VIR) {
                    v[0] += fr * dx * dx;
                    v[1] += fr * dy * dy;
                    v[2] += fr * dz * dz;
                    v[3] += fr * dx * dy;
                    v[4] += fr * dx * dz;
                    v[5] += fr * dy * dz;
                }
                const float gx = (float)(fr * dx), gy = (float)(fr * dy), gz = (float)(fr * dz);
                fx += gx;
                fy += gy;
                fz += gz;
                atomicAdd(d.f_s + sb, make_float4(-gx, -gy, -gz, 0.f));
            }
            if (fx != 0.f || fy != 0.f || fz != 0.f) atomicAdd(d.f_s + sa, make_float4(fx, fy, fz, 0.f));
        }
    }
    if (!ENER && !VIR) return;
    // sums per system: over the warp when all its atoms are of one system
    const int s0 = __shfl_sync(FULL, s, 0);
    if (__all_sync(FULL, s == s0 || s < 0)) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            if (ENER) e += __shfl_xor_sync(FULL, e, off);
            if (VIR) {
#pragma unroll
                for (int c = 0; c < 6; ++c) v[c] += __shfl_xor_sync(FULL, v[c], off);
            }
        }
        if (lane != 0 || s0 < 0) return;
        s = s0;
    } else if (s < 0) {
        return;
    }
    double* acc = sys[s].acc;
    if (ENER && e != 0.0) atomicAdd(acc + ACC_EC, e);
    if (VIR) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (v[c] != 0.0) atomicAdd(acc + ACC_VXX + c, v[c]);
    }
}

}  // namespace

cudaError_t launch_excl_corr(const PlanLaunch& p, unsigned flags, cudaStream_t st) {
    if (!(p.kp.mods & NB_MOD_RF_EXCL) || p.tot_atoms <= 0) return cudaSuccess;
    const unsigned bs = 256;
    const unsigned blocks = (unsigned)((p.tot_atoms + bs - 1) / bs);
    const bool en = flags & NB_F_ENERGY, vi = flags & NB_F_VIRIAL;
    if (en && vi) return launch_pdl(k_excl_rf<true, true>, blocks, bs, 0, st, p.d_sys, p.d_atom_off, p.nsys,
                                    p.tot_atoms, p.kp);
    if (en) return launch_pdl(k_excl_rf<true, false>, blocks, bs, 0, st, p.d_sys, p.d_atom_off, p.nsys,
                              p.tot_atoms, p.kp);
    if (vi) return launch_pdl(k_excl_rf<false, true>, blocks, bs, 0, st, p.d_sys, p.d_atom_off, p.nsys,
                              p.tot_atoms, p.kp);
    return launch_pdl(k_excl_rf<false, false>, blocks, bs, 0, st, p.d_sys, p.d_atom_off, p.nsys, p.tot_atoms,
                      p.kp);
}

}  // namespace nbgb
