// nb_internal.cuh -- device data layout and kernel launch interfaces shared by
// the library's translation units.  Not part of the public ABI (include/nb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nb.h"

namespace nbgb {

// Cluster size: every i- and j-cluster holds exactly CL atom slots (Section
// 3.2 groups the atoms into clusters of a fixed size M); here M = N = 8 so
// that one 8-lane group of a warp covers one cluster, and the 8 x 4 geometry
// (ListDev::jgeo) takes the two 4-slot halves of a cluster as j-clusters.
constexpr int CL = 8;
constexpr int MAX_TYPES = 64;
constexpr int COL_MAX = 4096;      // atoms per column sorted in shared memory
constexpr int NSHIFT = 27;         // periodic images (sx, sy, sz) in {-1,0,1}^3
constexpr int SHIFT_ZERO = 13;     // index of the zero shift
constexpr int SEARCH_BUF = 384;    // entries a search warp buffers before flushing
constexpr int EXCL_BUF = 128;      // exclusion partners a search warp caches
constexpr int GT_MAX = 2048;       // intervals of the Ewald force table, at most
constexpr int ET_MAX = 2048;       // intervals of the Ewald energy table, at most

// Counter slots of a list (ListDev::counters).
enum {
    CNT_ITEMS = 0,      // work items written (may exceed capacity: then overflow)
    CNT_ENTRIES = 1,    // raw entries written by the search
    CNT_OVERFLOW = 2,   // bit 0: items, bit 1: entries
    CNT_WORK = 3,       // persistent-kernel work counter
    CNT_PRUNED = 4,     // entries kept by the prune
    CNT_EWORK = 5,      // energy-kernel work counter
    CNT_ORD_LONG = 6,   // non-empty items the prune ordered first (long ones)
    CNT_ORD_SHORT = 7,  // non-empty items the prune ordered last (short ones)
    CNT_NEED = 8,       // thread-per-cluster search: most entries of one cluster
    CNT_N = 9
};

// Entries per cluster slab of the thread-per-cluster search: the list's
// entry capacity spread over the clusters, a multiple of 8.
__host__ __device__ inline int slab_stride(long long entry_cap, long long tot_clcap) {
    if (tot_clcap <= 0) return 0;
    long long s = entry_cap / tot_clcap;
    if (s > (1 << 24)) s = 1 << 24;
    return (int)(s & ~7ll);
}

// The entry capacity a search's counters ask for: the entries written, and
// (thread-per-cluster search) a slab as large as the largest cluster's
// count for every cluster.
inline long long entries_needed(const int* counters, long long tot_clcap) {
    const long long slab = ((long long)counters[CNT_NEED] + 7) & ~7ll;
    const long long a = counters[CNT_ENTRIES], b = slab * tot_clcap;
    return a > b ? a : b;
}

// Per-system device descriptor.  Every pointer is a device pointer owned by
// the system (nb_sys).  "slot" arrays have clcap * CL elements in the sorted
// (grid) order; "atom" arrays have natoms elements in the caller's order.
struct SysDev {
    float L[3];          // box: ax, by, cz (the edges of a rectangular box)
    float T[3];          // off-diagonal components bx, cx, cy of a triclinic box
                         // (rows a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz)); 0 otherwise
    float cw[2];         // column widths in x, y
    float icw[2];        // 1 / column width
    int ncx, ncy, ncol;  // grid columns
    int natoms;
    int clcap;           // cluster capacity = ceil(natoms / CL) + ncol
    // inputs, caller's order
    float4* xq_in;       // [natoms] x y z q
    int* type_in;        // [natoms]
    float* x_new;        // [natoms * 3] staged coordinates for nb_forces(x_new)
    // grid
    int* col_count;      // [ncol] atoms per column
    int* col_cl0;        // [ncol + 1] first cluster of each column; [ncol] = #clusters
    int* atom_col;       // [natoms]
    int* atom_slot;      // [natoms] arrival slot inside the column (pre-sort)
    unsigned long long* keys;  // [slots] (z key << 32 | atom) in column order
    float4* xq_s;        // [slots] sorted x y z q (fillers: far away, q = 0)
    int* type_s;         // [slots]
    int* perm;           // [slots] original atom of each slot, -1 = filler
    int* iperm;          // [natoms] slot of each atom
    int* wrapk;          // [slots] box multiples added by wrapping (3 x int8 packed)
    float4* bb;          // [clcap * 2] cluster bounding boxes: lo (w = #real), hi
    // exclusions: symmetric CSR in the caller's order (may be empty)
    const int* excl_index;  // [natoms + 1] or nullptr
    const int* excl_atoms;
    // outputs
    float4* f_s;         // [slots] forces in sorted order (w unused)
    float* f_out;        // [natoms * 3] forces in the caller's order
    double* acc;         // [NACC] FP64 energy/virial accumulators
    double* res;         // [NRES] E_LJ, E_C, virial row-major, pair count
    // list radius of this system, padded for the float32 rounding of
    // coordinates of this box's magnitude; per system, so that a system's
    // list does not depend on the other systems of a batch
    float rl_search;     // used by the bounding-box test
    float rl2_prune;     // its square, used by the prune
};

// Accumulator layout of SysDev::acc.  The virial slots hold sum (F/r) d (x) d,
// i.e. -2 Xi; the last three are the long-range (PME) energy parts.
enum { ACC_E12 = 0, ACC_E6 = 1, ACC_EC = 2, ACC_VXX = 3, ACC_VYY = 4, ACC_VZZ = 5,
       ACC_VXY = 6, ACC_VXZ = 7, ACC_VYZ = 8, ACC_NPAIR = 9, ACC_ECLO = 10,
       ACC_EREC = 11, ACC_ESELF = 12, ACC_EEXCL = 13, NACC = 14 };
// SysDev::res: E_LJ, E_C (every Coulomb part), virial[9], interacting pairs,
// then the long-range parts E_rec, E_self, E_excl
constexpr int NRES = 15;

// Per-plan (one system, or one batch of systems) cluster-pair list.
struct ListDev {
    int4* items;         // (ci, first entry, end entry, sys << 5 | shift)
    // j-atoms of an entry, by geometry (jgeo):
    //   0 (M x N = 8 x 8): cj = the j-cluster; j-slot t is sorted slot 8 cj + t.
    //   1 (8 x 4, two 4-atom j-clusters per entry): the j-clusters are the
    //     halves (z-halves after the column sort) of the 8-atom clusters;
    //     j-slots 0-3 are slots cj + t, j-slots 4-7 are slots cjb + t, i.e.
    //     cj is the first slot of the first half and cjb + 4 that of the
    //     second.  The prune writes this form, pairing the halves that keep
    //     a pair within the list radius two by two in each item; an item's
    //     odd last half is paired with itself under a zero mask.
    // Search output (before the prune) is always of the first form.
    int* cj;
    int* cjb;            // [entry_cap] with jgeo = 1, else unused
    int jgeo;
    unsigned long long* mask;  // 8x8 interaction bits per entry (rotated layout)
    // per entry and i-row (entry * 8 + i-slot), written by the force kernel of
    // an evaluation with energies: the slots inside rc or in the band around
    // it, bit 2p + c standing for j-slot 2 (p XOR (i >> 1)) + c; the energy
    // kernel queues from them instead of computing every slot's distance
    // again.  NULL: the energy kernel screens the slots itself.
    unsigned char* marks;
    int* counters;       // [CNT_N]
    // evaluation order of the non-empty items, written by the prune: the
    // long items (more than max_entries / 2 entries) from the front, the
    // short ones from the back, so that the persistent kernels take the
    // longest work first and end on short items
    int* order;          // [item_cap]
    int item_cap;
    int entry_cap;
};

// The prune writes that order, and the persistent kernels follow it, when the
// list has at most this many items per warp the force kernel can keep
// resident (KParams::lpt_max_items); longer lists are taken in cluster order.
constexpr int LPT_ITEMS_PER_WARP = 4;
constexpr int LPT_WARPS_PER_SM = 24;

// Bits of j-slots 0-3 in the rotated mask layout (bit 8 i + (j XOR i) for
// the pair of i-slot i and j-slot j): the low nibble of bytes 0-3 and the
// high nibble of bytes 4-7.  j-slots 4-7 hold the complement.
constexpr unsigned long long MASK_JLO = 0xF0F0F0F00F0F0F0Full;

// First sorted slot of j-slots 0-3 (lo) and j-slots 4-7 minus 4 (hi) of
// entry e: j-slot t lies at slot t + (t < 4 ? lo : hi).
__device__ __forceinline__ void entry_slots(const ListDev& list, int e, int& lo, int& hi) {
    if (list.jgeo) {
        lo = list.cj[e];
        hi = list.cjb[e];
    } else {
        lo = hi = list.cj[e] * 8;
    }
}

// Item index of the k-th item in evaluation order (k < n_long + n_short).
__device__ __forceinline__ int ordered_item(const ListDev& list, int k, int n_long) {
    return k < n_long ? list.order[k] : list.order[list.item_cap - 1 - (k - n_long)];
}

// Interaction constants (identical for all systems of a plan).
struct KParams {
    double rc2_d;        // cut-off^2 in float64 (exact decisions near rc)
    float rc2;           // cut-off^2
    float rc2_lo, rc2_hi;  // band around rc^2 decided exactly
    float fq;            // fcoul / eps_r
    float krf, two_krf, crf;
    float beta;          // Ewald splitting parameter
    // double-float (hi + lo) constants of the energy kernel
    float krf_h, krf_l, crf_h, crf_l, fq_h, fq_l;
    int coul;
    int ntypes;
    unsigned mods;       // NB_MOD_* potential modifiers
    float irc6_h, irc6_l, irc12_h, irc12_l;  // rc^-6, rc^-12 as hi + lo (NB_MOD_LJ_SHIFT)
    float ewc_h, ewc_l;  // erfc(beta rc) / rc as hi + lo (NB_MOD_EWALD_SHIFT)
    double fq_d, krf_d, crf_d;  // f / eps_r, k_rf, c_rf in float64 (NB_MOD_RF_EXCL)
    int max_entries;     // list entries per work item (items are split beyond)
    int search_mode;     // 0: by size, 1: a warp per i-cluster, 2: a thread per i-cluster
    int energy_mode;     // 0: a separate energy kernel, 1: energies fused into the force kernel
    int lpt_max_items;   // item count up to which items run longest first
    int force_min_blocks;  // force-kernel launch-bounds variant: 1, 2, 3 or 4 (nb_tuning)
    // Lennard-Jones as weights: when the table has one nonzero parameter
    // pair, c6_ij = C6 w_i w_j and c12_ij = C12 w_i w_j with w = 1 for the
    // types in ljw_mask and 0 otherwise, exactly; the force kernel then takes
    // w from the type instead of looking the pair up
    int lj_weights;                 // 1: the table is of that form
    unsigned long long ljw_mask;    // bit t: type t has w = 1
    float c6w, c12w;                // 6 C6, 12 C12 (the force table's values)
    // Ewald force table (force kernel): cubic Hermite pieces of G(r) =
    // erfc(beta r) + 2 beta r / sqrt(pi) exp(-beta^2 r^2) on intervals of
    // width h = 1 / gt_invh, coefficients (b0, b1, b2, b3) of s = r / h - k
    const float4* gtab;  // [gt_n]
    int gt_n;            // intervals (0: reaction field)
    float gt_invh;
    // Ewald energy table (energy kernels): erfc(beta r) on intervals of
    // width h = 1 / et_invh as quartics in s = r / h - k, interval k at
    // etab[k] = (a0 hi, a0 lo, a1 hi, a1 lo) and etab[ET_MAX + k] =
    // (a2, a3, a4, 0), the constant and linear coefficients as hi + lo
    const float4* etab;  // [2 * ET_MAX]
    int et_n;            // intervals (0: reaction field)
    float et_invh;
    const float2* lj;    // [ntypes^2] (6 c6, 12 c12), force kernel
    const float2* lje;   // [ntypes^2] (c6, c12), energy kernel
};

// ---------------------------------------------------- long-range part (PME)
// One axis of the mesh FFT: a Stockham transform of length n in `nst`
// stages of radix 16, 4, 2, 3 or 5.
constexpr int FFT_MAX_STAGES = 16;
struct FftAxis {
    int n;
    int nst;
    int rad[FFT_MAX_STAGES];  // radix of each stage
    const float2* tw;  // [n] exp(-2 pi i j / n), rounded from float64
};

// Smooth particle-mesh Ewald state of one rectangular system (device
// pointers owned by the system).  Mesh layout: x slowest, z fastest; the
// spectrum keeps kz = 0..K[2]/2 of the real-to-complex transform.
struct PmeDev {
    int K[3];
    int Kzh;           // K[2] / 2 + 1
    int order;         // B-spline order p (4, 6 or 8)
    double kl[3];      // K_d / L_d: mesh units per nm
    float kl_h[3], kl_l[3];  // the same as an unevaluated float sum hi + lo
    // Triclinic cell (box rows a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz)):
    // the mesh coordinates are u = x M, M = B^-1 diag(K), lower-triangular
    // with diagonal K_d / L_d (kl) and the off-diagonal entries M10, M20, M21
    // here as hi + lo; wave vectors are m = k R^T with R = B^-1 (diagonal
    // 1 / L_d, off-diagonal R10, R20, R21).  All off-diagonals are zero in a
    // rectangular box.
    int tri;
    float mo_h[3], mo_l[3];  // M10, M20, M21
    float rd[3], ro[3];      // R00, R11, R22 and R10, R20, R21
    float* Q;          // [K0 K1 K2] charges spread on the mesh, then the potential
    float2* S;         // [K0 K1 Kzh] half spectrum
    FftAxis ax[3];
    // per mesh index k of axis d, with k' its signed frequency (k' = +K/2 at
    // the index K/2 of an even mesh): rectangular cell, (m_d, |b_d(k)|^2
    // exp(-pi^2 m_d^2 / beta^2)) with m_d = k' / L_d; triclinic cell, (k',
    // |b_d(k)|^2), the exponential then taken per wave vector
    const float2* tab[3];
    float cpre;        // f / (pi V)
    float pi2_b2;      // pi^2 / beta^2
    double self_pre;   // -f beta / sqrt(pi)
    double beta;       // splitting parameter (excluded-pair correction)
    double fq;         // f = fcoul / eps_r
    // excluded-pair constants as hi + lo: f, 2 beta / sqrt(pi), 4 beta^3 / (3 sqrt(pi))
    float fq_h, fq_l, ke_h, ke_l, kf_h, kf_l;
    float beta2;       // beta^2
};

// Host-side view of a plan, used to size launches.
struct PlanLaunch {
    int nsys;
    const SysDev* d_sys;     // [nsys]
    const int* d_atom_off;   // [nsys + 1] prefix of natoms
    const int* d_col_off;    // [nsys + 1] prefix of ncol
    const int* d_cl_off;     // [nsys + 1] prefix of clcap
    int tot_atoms, tot_cols, tot_clcap;
    ListDev list;
    KParams kp;
    int num_sms;
    // single-system evaluations only (nsys == 1), each may be null: the
    // caller's device arrays read or written directly instead of through a
    // staging copy
    const float* x_ext;      // [natoms * 3] new coordinates (k_prepare)
    float* f_ext;            // [natoms * 3] forces (k_finish)
    double* e_ext;           // [2] E_LJ, E_C (k_finish)
    double* v_ext;           // [9] virial (k_finish)
};

// Programmatic dependent launch.  The path's kernels are launched with
// programmatic stream serialization: a kernel may be scheduled onto the SMs
// while the previous kernel of the stream finishes, which hides the launch
// latency between the many short stages.  Every such kernel calls pdl_wait()
// as its first statement, which returns once the previous grid has completed
// and its memory operations are visible, so no kernel reads anything early;
// pdl_trigger() lets the next kernel be scheduled once every block of this
// one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Shift index <-> vector.
__host__ __device__ inline int shift_index(int sx, int sy, int sz) {
    return (sx + 1) * 9 + (sy + 1) * 3 + (sz + 1);
}

// The lattice vector sx a + sy b + sz c of shift index sh (float32; every
// product is exact, the sums round only in a triclinic box).
__device__ __forceinline__ float3 shift_vec(int sh, const float (&L)[3], const float (&T)[3]) {
    const float sx = (float)(sh / 9 - 1), sy = (float)((sh / 3) % 3 - 1), sz = (float)(sh % 3 - 1);
    return make_float3(fmaf(sz, T[1], fmaf(sy, T[0], sx * L[0])), fmaf(sz, T[2], sy * L[1]), sz * L[2]);
}

// Bytes of a system's parameter tables: the Lennard-Jones tables ((6 c6, 12
// c12) then (c6, c12), 16 per type pair) and the Ewald force table after them.
inline size_t param_table_bytes(int ntypes) {
    return 16 * (size_t)ntypes * ntypes + 16 * (size_t)GT_MAX + 32 * (size_t)ET_MAX;
}
// Float2 offset of the Ewald energy table from the start of the parameter
// tables (after both Lennard-Jones tables and the force table).
inline size_t etab_offset2(int ntypes) { return 2 * (size_t)ntypes * ntypes + 2 * (size_t)GT_MAX; }
// The Ewald force table for splitting parameter beta and cut-off rc: writes
// up to GT_MAX float4 coefficients, sets *invh, returns the number of
// intervals (0 if it would need more than GT_MAX; never for beta rc <= 10).
// Each interval k of width h = 2^-n covers [k h, (k + 1) h); its cubic in
// s = r / h - k is the Hermite interpolant of G and dG/dr at both ends, with
// h the largest power of two for which every interval's error bound
// h^4 / 384 max|d^4 G / dr^4| is at most 1e-7 of G at its far end (G
// decreases; G taken as at least 1e-7), and the intervals reach rc (1 + 1e-4).
int ewald_force_table(double beta, double rc, float4* coef, float* invh);
// The Ewald energy table for beta and rc: writes 2 * ET_MAX float4 (the
// KParams::etab layout; entries past the intervals are left as they are),
// sets *invh, returns the number of intervals (0 if more than ET_MAX would
// be needed; never for beta rc <= 10).  Interval k of width h = 2^-n covers
// [k h, (k + 1) h); its quartic in s = r / h - k interpolates erfc(beta r)
// at the five Chebyshev points of the interval, in float64.  h is the
// largest power of two for which the interpolation error bound
// 2 (h / 4)^5 max|d^5 erfc(beta r) / dr^5| / 5! is at most 1e-12 and the
// quadratic coefficient, evaluated in float32, at most 1e-4 (so that its
// float32 rounding is below 1e-11), with the intervals reaching rc (1 + 1e-4).
int ewald_energy_table(double beta, double rc, float4* coef, float* invh);

// Host helpers of nb_api.cu shared with the allocation-free entry point.
nb_status api_fail(nb_status s, const char* msg);
nb_status api_check_system(const nb_params* params, int natoms, const double box[3]);
// Geometry and buffer layout of one system inside `base` (nullptr: size only);
// returns the bytes used, the LJ tables occupying the last 16 * ntypes^2.
size_t api_sys_layout(int natoms, const double box[3], int ntypes, SysDev* h, char* base);
KParams api_kparams(const nb_params& p, const double box[3], float2* lj);
// Padded list radius of a system (SysDev::rl_search, rl2_prune).
void api_list_radii(double rlist, const double box[3], SysDev* h);
void api_list_estimate(const nb_params& p, int natoms, const double box[3], int clcap, long long* items,
                       long long* entries);

// Kernel launchers (each returns the launch status).
cudaError_t launch_grid_put(const PlanLaunch& p, cudaStream_t st);
cudaError_t launch_search(const PlanLaunch& p, cudaStream_t st);
cudaError_t launch_prune(const PlanLaunch& p, cudaStream_t st);
// Prune src out of place into dst (same capacities) at radius^2 rl2_inner;
// dst's counters must be zero.
cudaError_t launch_prune_into(const PlanLaunch& p, const ListDev& src, const ListDev& dst, float rl2_inner,
                              cudaStream_t st);
// Start of an evaluation: clear forces, accumulators and work counters; with
// coords, also move the staged x_new into the sorted slots.
cudaError_t launch_prepare(const PlanLaunch& p, bool coords, cudaStream_t st);
// Forces (and, per flags, virial; with NB_F_ENERGY and energy_fused(p) also
// the energies, in the same kernel).
cudaError_t launch_forces(const PlanLaunch& p, unsigned flags, cudaStream_t st);
bool energy_fused(const PlanLaunch& p);
// Whether the force kernel of an evaluation with these flags writes the
// list's marks and the energy kernel queues from them (separate energies,
// a list with marks, a force register budget of 2 or 3 blocks per SM).
bool energy_marks(const PlanLaunch& p, unsigned flags);
// The separate energy kernel (nothing when the energies are fused).
cudaError_t launch_energy(const PlanLaunch& p, cudaStream_t st);
cudaError_t launch_finalize(const PlanLaunch& p, unsigned flags, cudaStream_t st);
// Reaction-field correction of excluded pairs (NB_MOD_RF_EXCL; nothing
// otherwise): after the force and energy kernels, before the finalisation.
cudaError_t launch_excl_corr(const PlanLaunch& p, unsigned flags, cudaStream_t st);
// Long-range part of a single-system plan (spread, mesh FFT and solve, gather,
// excluded-pair correction): adds its forces to the sorted force buffer and
// its energies and virial to the accumulators.  After the force kernels,
// before the finalisation.
// acc: the system's accumulators (SysDev::acc).  Three launch groups, in
// this order: mesh clear and spreading; FFT, solve and inverse FFT; gathering
// and the excluded-pair correction.
cudaError_t launch_pme_spread(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags,
                              cudaStream_t st);
cudaError_t launch_pme_fft(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags, cudaStream_t st);
cudaError_t launch_pme_gather(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags,
                              cudaStream_t st);
// Raise the dynamic shared-memory limit of the mesh-FFT kernels to what the
// mesh of pm needs; pme_smem_need gives that amount for a mesh K.
cudaError_t pme_prepare_kernels(const PmeDev& pm);
size_t pme_smem_need(const int K[3]);

}  // namespace nbgb
