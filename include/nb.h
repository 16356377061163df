/*
 * nb.h -- C ABI of the GB300 short-range non-bonded library.
 *
 * The library evaluates the short-range non-bonded forces, energies and
 * virial of periodic particle systems with the cluster-pair scheme of
 * Pall et al. (arXiv:1506.00716, Section 3.2 "SIMD parallelism"):
 *   - particles are put on a grid of x-y columns and sorted along z inside
 *     each column, and every column is cut into clusters of exactly M = 8
 *     particles (nb_grid_put);
 *   - a buffered list of cluster pairs (bounding-box distance < rlist, with
 *     rlist > rc) is built once and reused over many force evaluations, with
 *     per-pair interaction masks, then pruned to the pairs that have at least
 *     one particle pair inside rlist (nb_pairlist_build; Section 3.2 and the
 *     "Heterogeneous parallelization" part of Section 3.2.1, where the list
 *     is pruned on the GPU and reused for many steps);
 *   - a cluster-pair kernel computes M x N interactions per list entry
 *     (nb_forces; Section 3.2).
 * With Ewald electrostatics the long-range part (smooth particle-mesh Ewald,
 * which the paper runs next to the pair kernel) is available too
 * (nb_pme_init, nb_pme_forces, NB_F_PME).  Batches of systems and a serving
 * engine evaluate many systems per launch (nb_batch_*, nb_server_*).
 * All work runs on one CUDA device; there is no CPU fallback.
 *
 * Units: nm, kJ/mol, elementary charge.  Boxes are rectangular (periodic in
 * x, y and z) or triclinic (nb_sys_create_box); every edge must be at least
 * 2 * rlist.
 *
 * Conventions shared by every call:
 *   - Every call returns an nb_status; none aborts.  NB_OK is 0.  A failing
 *     call leaves a message for nb_last_error() in thread-local storage.
 *   - Buffers are owned by the caller.  A pointer argument described as
 *     "host or device" is read or written through cudaMemcpyAsync on the
 *     context's stream, so both kinds work; calls that return results into
 *     host memory synchronise the stream before returning.  Device pointers
 *     must stay valid until the stream has passed the call.
 *   - All device work of a context is ordered on the CUDA stream given to
 *     nb_ctx_create (NULL = the legacy default stream).
 *   - Handles are not thread-safe: one host thread at a time per context.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx;
typedef struct nb_sys nb_sys;
typedef struct nb_batch nb_batch;

typedef enum {
    NB_OK = 0,
    NB_ERR_ARG = 1,      /* invalid argument (NULL handle, bad size or flag) */
    NB_ERR_BOX = 2,      /* a box edge is shorter than 2 * rlist */
    NB_ERR_OOM = 3,      /* a device allocation failed */
    NB_ERR_BUDGET = 4,   /* the context's HBM budget would be exceeded */
    NB_ERR_CUDA = 5,     /* a CUDA runtime call or kernel launch failed */
    NB_ERR_NOT_READY = 6,/* the batch ticket has not completed yet */
    NB_ERR_TIMEOUT = 7,  /* a bounded wait ran out */
    NB_ERR_STATE = 8,    /* call out of order, e.g. nb_forces before a list exists */
    NB_ERR_CAPACITY = 9  /* a fixed device capacity was exceeded (reported, no overrun) */
} nb_status;

enum { NB_COUL_RF = 0, NB_COUL_EWALD = 1 };

/* Flags of nb_forces, nb_batch_submit. */
enum {
    NB_F_ENERGY = 1u,  /* compute E_LJ and E_Coulomb */
    NB_F_VIRIAL = 2u,  /* compute the 3x3 virial */
    NB_F_PME = 4u      /* nb_forces only: add the long-range part (nb_pme_init) */
};

/*
 * Interaction parameters (Section 3.2: van der Waals and electrostatics
 * inside a spherical cut-off, with a list buffer rlist > rc).
 *   rc          interaction cut-off (nm); a pair interacts iff r^2 < rc^2
 *   rlist       list radius (nm), rlist >= rc
 *   coul        NB_COUL_RF: reaction field, V = f qi qj / eps_r
 *                 (1/r + k_rf r^2 - c_rf), k_rf = (eps_rf - eps_r) /
 *                 ((2 eps_rf + eps_r) rc^3), c_rf = 1/rc + k_rf rc^2
 *                 (eps_rf = 0 means infinity: k_rf = 1/(2 rc^3));
 *               NB_COUL_EWALD: Ewald real space, V = f qi qj / eps_r
 *                 erfc(beta r) / r (ewald_beta > 0, ewald_beta rc <= 10)
 *   fcoul       electric conversion factor f = 1/(4 pi eps_0), 138.935458
 *   ntypes      number of Lennard-Jones types, 1..64
 *   c6, c12     host arrays of ntypes*ntypes floats, row-major [ti*ntypes+tj],
 *               V_LJ = c12/r^12 - c6/r^6; copied during nb_sys_create
 *   modifiers   bits of NB_MOD_* (0: none).  Without modifiers, excluded
 *               pairs contribute nothing and the potentials are cut plainly
 *               at rc (the reaction-field one is zero there by its c_rf).
 *               The paper states no cut-off treatment; these are the
 *               common alternatives:
 *     NB_MOD_LJ_SHIFT     every interacting pair's Lennard-Jones energy is
 *                         taken relative to its value at rc (forces unchanged)
 *     NB_MOD_EWALD_SHIFT  likewise for the Ewald real-space energy,
 *                         f qi qj / eps_r (erfc(beta r)/r - erfc(beta rc)/rc);
 *                         NB_COUL_EWALD only
 *     NB_MOD_RF_EXCL      every excluded pair with r^2 < rc^2 contributes
 *                         f qi qj / eps_r (k_rf r^2 - c_rf) to E_Coulomb, with
 *                         its force and virial (no self term); NB_COUL_RF only.
 *                         Evaluated in float64 over the exclusion list.
 *               Other bits, or a modifier with the other electrostatics,
 *               fail with NB_ERR_ARG.
 */
enum { NB_MOD_LJ_SHIFT = 1u, NB_MOD_EWALD_SHIFT = 2u, NB_MOD_RF_EXCL = 4u };

typedef struct {
    double rc, rlist;
    int coul;
    double eps_r, eps_rf, ewald_beta, fcoul;
    int ntypes;
    const float *c6, *c12;
    unsigned modifiers;
} nb_params;

/* Counts of the current pair list (nb_pairlist_info). */
typedef struct {
    long long n_clusters;    /* clusters of M = 8 slots, fillers included */
    long long n_items;       /* (i-cluster, periodic shift) work items */
    long long n_entries;     /* cluster-pair entries after pruning */
    long long n_entries_raw; /* entries that passed the bounding-box test */
    long long n_slots;       /* M*N atom-pair slots the kernel evaluates */
    long long n_entries_inner; /* entries of the inner list (nb_pairlist_prune),
                                  n_entries when there is none */
} nb_list_info;

/* Result counts of the last evaluation (nb_eval_info). */
typedef struct {
    long long n_pairs;  /* atom pairs inside rc, not excluded, counted by the kernel
                           (float32 distance test); set by evaluations with NB_F_ENERGY */
} nb_eval_stats;

/* Stages timed by nb_ctx_timing. */
enum {
    NB_STAGE_GRID = 0,    /* nb_grid_put kernels */
    NB_STAGE_SEARCH = 1,  /* cluster-pair search */
    NB_STAGE_PRUNE = 2,   /* list prune */
    NB_STAGE_COORD = 3,   /* staging copy of nb_forces(x_new) */
    NB_STAGE_ZERO = 4,    /* force-buffer clear + coordinate update */
    NB_STAGE_FORCES = 5,  /* the cluster-pair force kernel (all evaluations; with
                             nb_tuning.energy_mode = 1 those without energies) */
    NB_STAGE_FINAL = 6,   /* unsort + FP64 energy/virial finalisation */
    NB_STAGE_ENERGY = 7,  /* NB_F_ENERGY evaluations: the double-float energy kernel, or
                             (energy_mode = 1) the force kernel with the energies fused in */
    NB_STAGE_PME_SPREAD = 8,  /* long-range part: mesh clear + charge spreading */
    NB_STAGE_PME_FFT = 9,     /* long-range part: forward FFT, solve, inverse FFT */
    NB_STAGE_PME_GATHER = 10, /* long-range part: force gathering + excluded pairs */
    NB_NSTAGE = 11
};

/*
 * Launch tuning of a context (chosen per system size by the project's
 * autotuner, paper_1506_00716_gb300/autotune.py).  Takes effect at the next
 * list build or batch submission.
 *   max_entries       list entries per work item: (i-cluster, shift) runs
 *                     longer than this are split into several items, which
 *                     balances the persistent force kernel on small systems;
 *                     4..4096 (default 32)
 *   force_min_blocks  register budget of the force kernel, as the number of
 *                     256-thread blocks guaranteed resident per SM: 1 (up to
 *                     255 registers per thread), 2 (128) or 3 (80, default);
 *                     or 4: two 320-thread blocks per SM (96 registers, 20
 *                     warps per SM).  Evaluations with energies fused into the
 *                     force kernel (energy_mode 1) take budget 2.
 *   search_mode       cluster-pair search: 1 = one warp per i-cluster (lanes
 *                     share its candidates), 2 = one thread per i-cluster
 *                     (count, scan and write passes, no atomics), 0 = by
 *                     size (default: a thread per cluster from about eight
 *                     warps' worth of clusters per SM).  The list is the same.
 *   energy_mode       evaluations with NB_F_ENERGY: 0 = a separate energy
 *                     kernel after the force kernel (default), 1 = the force
 *                     kernel also evaluates the energies of the pairs it
 *                     finds inside rc.  The results are the same.
 *   jcluster          j-cluster size N of the list (Section 3.2's cluster
 *                     geometry; the i-cluster size M is 8): 8 (or 0, the
 *                     default) = 8 x 8 entries; 4 = the z-halves of the
 *                     8-atom clusters as 4-atom j-clusters, those without a
 *                     pair within the list radius dropped by the prune and
 *                     the rest paired two per entry (fewer pair slots per
 *                     interacting pair, more list entries per slot).  The
 *                     interacting pairs and the results are the same.
 */
typedef struct {
    int max_entries;
    int force_min_blocks;
    int search_mode;
    int energy_mode;
    int jcluster;
} nb_tuning;

/* Message of the calling thread's last failure ("" if none). */
const char *nb_last_error(void);

/*
 * Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream).  `hbm_budget_bytes` caps the device memory
 * the context's systems and batches may hold (0 = no cap); requests over the
 * cap fail with NB_ERR_BUDGET and allocate nothing.
 */
nb_status nb_ctx_create(int device, void *cuda_stream, size_t hbm_budget_bytes, nb_ctx **out);
nb_status nb_ctx_destroy(nb_ctx *ctx);
/*
 * Per-stage device timing: when enabled, every stage launched by the context
 * is bracketed by CUDA events on the context's stream.  nb_ctx_timing
 * synchronises the stream and returns, per NB_STAGE_*, the summed elapsed
 * milliseconds and the number of timed launches since the last reset
 * (ms and launches: NB_NSTAGE entries, either may be NULL); reset != 0
 * clears the totals.  nb_ctx_set_timing(ctx, enable) times every stage
 * (enable != 0) or none; nb_ctx_set_timing_stages times only the stages whose
 * bit (1 << NB_STAGE_*) is set in stage_mask.  Each timed stage adds two
 * event records to the stream, which separate the stage's kernels from
 * their neighbours on the device: time only what is needed.
 */
nb_status nb_ctx_set_tuning(nb_ctx *ctx, const nb_tuning *tuning);
nb_status nb_ctx_get_tuning(nb_ctx *ctx, nb_tuning *tuning);
nb_status nb_ctx_set_timing(nb_ctx *ctx, int enable);
nb_status nb_ctx_set_timing_stages(nb_ctx *ctx, unsigned stage_mask);
nb_status nb_ctx_timing(nb_ctx *ctx, double *ms, long long *launches, int reset);
/* Device bytes currently held by the context's systems and batches. */
nb_status nb_ctx_memory(nb_ctx *ctx, size_t *bytes_in_use, size_t *budget);
/*
 * Test hook (fault injection on the host): the next `count` device
 * allocations of this context fail as an out-of-memory would, with
 * NB_ERR_OOM and nothing allocated, so that callers can test their recovery
 * without exhausting the GPU.  count = 0 clears it.  Every call that
 * allocates leaves the context and its systems usable after such a failure.
 */
nb_status nb_ctx_inject_alloc_failures(nb_ctx *ctx, int count);
/* Device bytes nb_sys_create would reserve for a system of natoms atoms. */
nb_status nb_sys_footprint(const nb_params *params, int natoms, const double box[3], size_t *bytes);

/*
 * Create a system of `natoms` atoms in a rectangular box box[0..2] (nm).
 * The device uses float(box[k]); pass float-representable values to make
 * host and device see the same box.  Fails with NB_ERR_BOX if any edge is
 * below 2 * rlist, NB_ERR_BUDGET / NB_ERR_OOM if the memory is not there.
 */
nb_status nb_sys_create(nb_ctx *ctx, const nb_params *params, int natoms, const double box[3],
                        nb_sys **out);
/*
 * The same for a triclinic box.  box[9] holds the rows a = (ax, 0, 0),
 * b = (bx, by, 0), c = (cx, cy, cz) of the periodic lattice.  Restrictions
 * (NB_ERR_BOX otherwise): |bx| + |cx| <= ax/2, |cy| <= by/2; rlist <= ax/2,
 * by/2 and < cz; every lattice vector at least 2 rlist long.  These admit
 * the rectangular boxes and, among others, the rhombic dodecahedron in its
 * xy-square form (a = (d,0,0), b = (0,d,0), c = (d/2, d/2, d sqrt(2)/2)).
 * Coordinates are wrapped into the cell [0, ax) x [0, by) x [0, cz) (z by
 * c, then y by b, then x by a); pairs interact through their minimum image.
 */
nb_status nb_sys_create_box(nb_ctx *ctx, const nb_params *params, int natoms, const double box[9],
                            nb_sys **out);
nb_status nb_sys_destroy(nb_sys *sys);

/*
 * Exclusions as a CSR over atoms in the caller's order: the partners of
 * atom a are excl_atoms[excl_index[a] .. excl_index[a+1]-1].  A pair is
 * excluded if either atom lists the other (the list is symmetrised here).
 * Host pointers.  Excluded pairs do not interact.  Takes effect at the next
 * nb_pairlist_build.
 */
nb_status nb_set_exclusions(nb_sys *sys, const int *excl_index, const int *excl_atoms);

/*
 * Grid put (Section 3.2): take coordinates and charges xq (natoms * 4 floats,
 * x y z q, caller's order; host or device) and Lennard-Jones types (natoms
 * ints in [0, ntypes); host or device), wrap the coordinates into the box,
 * bin atoms into x-y columns, sort each column along z (ties by atom index)
 * and cut it into clusters of 8, padding with non-interacting fillers, and
 * compute each cluster's bounding box.  Invalidates the pair list.
 */
nb_status nb_grid_put(nb_sys *sys, const float *xq, const int *type);

/*
 * Build the buffered cluster-pair list (Section 3.2): every pair of
 * clusters whose bounding boxes come closer than rlist under some periodic
 * image, kept once per unordered pair (half list), with an 8x8 interaction
 * mask that removes excluded pairs, fillers and the lower triangle of
 * self-pairs; then prune entries with no atom pair inside rlist.  Needs a
 * preceding nb_grid_put.  Synchronises the stream to check the list
 * capacity, and grows it and rebuilds if needed.
 */
nb_status nb_pairlist_build(nb_sys *sys);
nb_status nb_pairlist_info(nb_sys *sys, nb_list_info *info);
/*
 * Dynamic pruning (Section 3.2.1: the list is built with a buffer, pruned on
 * the GPU and reused): prune the list of the last nb_pairlist_build, out of
 * place, to the radius r_inner (rc <= r_inner <= rlist) using the current
 * coordinates (those of the last nb_grid_put or nb_forces).  Until the next
 * nb_pairlist_build, evaluations use this inner list; the outer one is kept,
 * so the call can be repeated as the atoms move.  The caller keeps every
 * displacement since the call small enough for r_inner - rc to cover it, as
 * rlist - rc must cover those since the build.  NB_ERR_STATE without a list,
 * NB_ERR_ARG for r_inner outside [rc, rlist].
 */
nb_status nb_pairlist_prune(nb_sys *sys, double r_inner);

/*
 * Evaluate forces (and, per flags, energies and virial) with the current
 * list (Section 3.2 cluster-pair kernel).
 *   x_new   NULL: use the coordinates of the last nb_grid_put; otherwise
 *           natoms * 3 floats (host or device), the new positions in the
 *           caller's order.  They must be continuous with those of the last
 *           nb_grid_put (no re-wrapping into the box between list builds),
 *           and the list stays valid while every atom has moved less than
 *           (rlist - rc) / 2.
 *   f       natoms * 3 floats (host or device), the force on each atom in the
 *           caller's order (overwritten); NULL skips the copy-out.
 *   energy  2 doubles (host or device): E_LJ, E_Coulomb; NULL allowed.
 *   virial  9 doubles (host or device): Xi = -1/2 sum_pairs d (x) F,
 *           row-major; NULL allowed.
 *   flags   NB_F_ENERGY | NB_F_VIRIAL; energy / virial must be non-NULL when
 *           their flag is set.
 * Buffers: device memory and pinned host memory (cudaHostAlloc, registered
 * or pinned tensors) are read and written by the kernels themselves, pinned
 * host memory through its mapped device address (no separate copy; over
 * NVLink-C2C on a Grace-Blackwell node); pageable host memory goes through
 * the system's staging buffers.  With any host buffer the call returns after
 * the stream has finished with it.
 * Forces and virial: float32 pair arithmetic and per-atom accumulation, the
 * virial summed over the system in float64.  Energies (NB_F_ENERGY, an extra
 * kernel): double-float pair arithmetic on the float32 pipes, summed in
 * float64.  Cut-off decisions are exact for the float32 inputs.
 */
nb_status nb_forces(nb_sys *sys, const float *x_new, float *f, double *energy, double *virial,
                    unsigned flags);

/* Counts of the last evaluation of this system (synchronises the stream). */
nb_status nb_eval_info(nb_sys *sys, nb_eval_stats *stats);

/*
 * Test hook: copy the current list to host memory.  Any output pointer may
 * be NULL.  Sizes come from nb_pairlist_info, except that of the entry
 * arrays: a call with cj = mask = NULL returns it in n_entries_total.
 *   perm        n_clusters * 8 ints: original atom index of each sorted slot,
 *               -1 for fillers
 *   items       n_items * 4 ints: (i-cluster, first entry, end entry, shift)
 *               where shift = (sx+1)*9 + (sy+1)*3 + (sz+1), the i-cluster
 *               being displaced by (sx Lx, sy Ly, sz Lz)
 *   cj          n_entries_total ints, j-cluster of each entry (indices up to
 *               the largest item end; entries outside every item's range
 *               are gaps and hold no list data)
 *   mask        n_entries_total unsigned long long: bit 8*i + t set means the
 *               pair (i-slot i, j-slot t XOR i) may interact
 *   n_entries_total  receives the size of the entry arrays
 */
nb_status nb_pairlist_export(nb_sys *sys, int *perm, int *items, int *cj,
                             unsigned long long *mask, long long *n_entries_total);
/*
 * Test hook: as nb_pairlist_export, for either j-cluster geometry
 * (nb_tuning.jcluster), with the j-atoms of each entry given by sorted slot
 * instead of by j-cluster.  Section 3.2 sets the cluster sizes by the SIMD
 * width of the hardware; with 4-atom j-clusters one entry holds two of them.
 *   jslot   2 * n_entries_total ints: entry e's j-slots 0-3 are the sorted
 *           slots jslot[2e] + 0..3 and its j-slots 4-7 the slots
 *           jslot[2e + 1] + 0..3 (8 x 8 lists: 8 cj and 8 cj + 4)
 * nb_pairlist_export itself refuses (NB_ERR_STATE) to write cj for a list of
 * 4-atom j-clusters, which have no single j-cluster per entry.
 */
nb_status nb_pairlist_export_slots(nb_sys *sys, int *perm, int *items, int *jslot,
                                   unsigned long long *mask, long long *n_entries_total);

/*
 * Test hook (host only, no device work): the Ewald force table of the
 * force kernel for splitting parameter beta (nm^-1) and cut-off rc (nm).
 * With NB_COUL_EWALD the force kernel takes the real-space force factor as
 * F/r = f qi qj G(r) / r^3, with G(r) = erfc(beta r) + 2 beta r / sqrt(pi)
 * exp(-beta^2 r^2) (the derivative of the energy term of Section 3.2's
 * pair interaction, see nb_params), from a cubic Hermite table of G on
 * intervals of width h = 2^-n: interval k covers [k h, (k + 1) h) and holds
 * (b0, b1, b2, b3), G(r) ~ b0 + b1 s + b2 s^2 + b3 s^3 with s = r / h - k.
 * h is the largest power of two for which every interval's interpolation
 * error bound (h^4 / 384 times the maximum of |d^4 G / dr^4| on it) is at
 * most 1e-7 of G at the interval's far end (G decreases; G taken as at least
 * 1e-7 there), and the intervals reach rc (1 + 1e-4).
 *   coef          4 * max_intervals floats (host), or NULL for the size only
 *   n_intervals   receives the number of intervals (at most 2048)
 *   h             receives the interval width (nm); may be NULL
 * NB_ERR_ARG unless beta > 0, rc > 0 and beta rc <= 10 (the limit of
 * nb_sys_create for NB_COUL_EWALD), or if coef holds fewer intervals.
 */
nb_status nb_ewald_force_table(double beta, double rc, float *coef, int max_intervals, int *n_intervals,
                               double *h);

/*
 * Test hook (host only, no device work): the Ewald energy table of the
 * energy kernels for splitting parameter beta (nm^-1) and cut-off rc (nm).
 * With NB_COUL_EWALD the energy kernels take erfc(beta r) of the pair energy
 * f qi qj erfc(beta r) / r (Section 3.2's pair interaction, see nb_params)
 * from a table of quartics on intervals of width h = 2^-n: interval k covers
 * [k h, (k + 1) h) and gives erfc(beta r) ~ a0 + a1 s + a2 s^2 + a3 s^3 +
 * a4 s^4, s = r / h - k, the polynomial interpolating erfc(beta r) (float64)
 * at the five Chebyshev points (1 - cos((2 j + 1) pi / 10)) / 2 of s.  h is
 * the largest power of two for which the interpolation error bound
 * 2 (h / 4)^5 max|d^5 erfc(beta r) / dr^5| / 5! is at most 1e-12 and
 * max|a2| at most 1e-4, and the intervals reach rc (1 + 1e-4).  The kernels
 * evaluate a0 + a1 s in double-float and the rest in float32.
 *   coef          8 * max_intervals floats (host), or NULL for the size only:
 *                 per interval (a0 hi, a0 lo, a1 hi, a1 lo, a2, a3, a4, 0),
 *                 a0 = a0 hi + a0 lo and a1 = a1 hi + a1 lo as float sums
 *   n_intervals   receives the number of intervals (at most 2048)
 *   h             receives the interval width (nm); may be NULL
 * NB_ERR_ARG unless beta > 0, rc > 0 and beta rc <= 10 (the limit of
 * nb_sys_create for NB_COUL_EWALD), or if coef holds fewer intervals.
 */
nb_status nb_ewald_energy_table(double beta, double rc, float *coef, int max_intervals, int *n_intervals,
                                double *h);

/*
 * Batched evaluation of many independent systems (the paper's ensemble
 * simulations, Section 3.3): one launch per stage covers every system, the
 * force stage is one persistent kernel over a flattened worklist of all
 * systems' cluster pairs, and the whole sequence is captured once in a CUDA
 * graph and replayed.
 *
 * nb_batch_create: the systems must share one context and equal parameters;
 * each needs a preceding nb_sys_set_coords (or nb_grid_put).  The batch
 * holds its own list buffers (counted against the budget).
 */
nb_status nb_batch_create(nb_ctx *ctx, nb_sys *const *systems, int n, nb_batch **out);
nb_status nb_batch_destroy(nb_batch *batch);
/*
 * Stage new coordinates for one system without running anything: xq is
 * natoms * 4 floats and type natoms ints (host or device).  The next batch
 * submission grids, lists and evaluates from them.
 */
nb_status nb_sys_set_coords(nb_sys *sys, const float *xq, const int *type);
/*
 * Launch grid put, list build, prune and force evaluation for every system
 * of the batch (flags as nb_forces).  Returns at once; *ticket identifies
 * the submission.
 */
nb_status nb_batch_submit(nb_batch *batch, unsigned flags, unsigned long long *ticket);
/*
 * Wait up to timeout_us microseconds (0 = just test) for a submission.
 * *done = 1 once it has finished.  Returns NB_ERR_TIMEOUT if it has not
 * finished in time, NB_ERR_CAPACITY if a list outgrew its buffer (the batch
 * then grows its buffers; submit again).
 */
nb_status nb_batch_poll(nb_batch *batch, unsigned long long ticket, long long timeout_us, int *done);
/*
 * Copy one system's results of the last completed submission: f (natoms*3
 * floats), energy (2 doubles), virial (9 doubles); host or device; NULL
 * skips.
 */
nb_status nb_sys_results(nb_sys *sys, float *f, double *energy, double *virial);

/*
 * Serving (continuous batching of independent single-point evaluations, the
 * serving form of the paper's ensemble workloads, Section 3.3).  A server
 * owns a scheduler thread and two CUDA streams.  Requests are queued by
 * nb_server_submit; whenever a stream is free, the scheduler admits the
 * oldest pending requests that fit the server's HBM budget (at most max_wave
 * of them) as one wave: their grid put, list build, prune, forces and
 * energies run as one launch per stage over all of them.  Two waves are in
 * flight at a time, so the upload, grid and search of one wave overlap the
 * force kernel of the other, and requests that arrive meanwhile join the
 * next wave as memory frees up.  Device state of a request exists only while
 * its wave runs.
 */
typedef struct nb_server nb_server;

/* Timings of one request (seconds, steady clock). */
typedef struct {
    double latency_s;  /* submission to results available */
    double queue_s;    /* submission to admission into a wave */
    long long n_pairs; /* interacting pairs (requests with NB_F_ENERGY) */
    int wave_size;     /* requests in the wave that served it */
} nb_request_stats;

/*
 * Create a server on ctx's device with the given parameters (copied).
 * hbm_budget_bytes caps the device memory of the waves in flight (0 = no
 * cap); max_wave caps the requests per wave (1..4096).
 */
nb_status nb_server_create(nb_ctx *ctx, const nb_params *params, size_t hbm_budget_bytes, int max_wave,
                           nb_server **out);
/* Stop accepting requests, finish all pending and in-flight work, free. */
nb_status nb_server_destroy(nb_server *srv);
/*
 * Queue one evaluation.  natoms, box as nb_sys_create; xq, type as
 * nb_grid_put but host memory only (copied before returning); exclusions
 * as nb_set_exclusions (host, may be NULL); flags as nb_forces.  Returns a
 * ticket.  A request larger than the whole budget fails at nb_server_wait
 * with NB_ERR_BUDGET.
 */
nb_status nb_server_submit(nb_server *srv, int natoms, const double box[3], const float *xq,
                           const int *type, const int *excl_index, const int *excl_atoms, unsigned flags,
                           unsigned long long *ticket);
/*
 * Wait up to timeout_us (< 0: no limit) for a ticket and copy its results
 * to host memory: f (natoms*3 floats), energy (2), virial (9), stats; any
 * may be NULL.  NB_ERR_TIMEOUT if not finished in time (the ticket stays
 * valid); each ticket's results can be collected once.  One thread at a
 * time may wait on a ticket: a second concurrent wait on the same ticket
 * fails at once with NB_ERR_ARG.
 */
nb_status nb_server_wait(nb_server *srv, unsigned long long ticket, long long timeout_us, float *f,
                         double *energy, double *virial, nb_request_stats *stats);

/*
 * Allocation-free evaluation, for callers that cannot allocate device
 * memory: code that runs where cudaMalloc is unavailable or not allowed
 * (inside another framework's memory manager, a latency-critical loop that
 * must not hit the allocator, a plug-in that only receives a stream).  The
 * paper has no counterpart; this is an interface of this library.
 *
 * One call runs grid put, pair search, prune, forces and (per flags)
 * energies and virial for one system of at most NB_NOALLOC_MAX_ATOMS atoms,
 * using as scratch a fixed device array of NB_NOALLOC_SCRATCH_BYTES that is
 * part of the library (every GPU that loads it holds it until the process
 * exits; see below for when it is loaded).  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   params, natoms, box  as nb_sys_create
 *   excl_index,          host CSR of exclusions (may both be NULL); unlike
 *   excl_atoms           nb_set_exclusions, every excluded pair must be
 *                        listed under both of its atoms
 *   xq, type             as nb_grid_put (host or device)
 *   f, energy, virial,   as nb_forces (host or device; f may be NULL)
 *   flags
 *   cuda_stream          the stream to run on (NULL = legacy default stream);
 *                        the calling thread's current CUDA device is used
 * Returns NB_ERR_CAPACITY if natoms exceeds the maximum or the pair list
 * does not fit the scratch array; the outputs are then left untouched (the
 * overflow is detected after the search, before any force is evaluated).
 * After any other error the contents of f, energy and virial are undefined.
 * Synchronises the stream after the search and before returning.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress), so make the first call before any stream capture.
 * Under lazy module loading (CUDA_MODULE_LOADING=LAZY, the default of recent
 * CUDA releases) that lookup also loads the library's module holding the
 * array, so the first call on each device is the one that reserves its
 * NB_NOALLOC_SCRATCH_BYTES, and it fails with NB_ERR_CUDA (out of memory)
 * if the device has no room left for it.
 * All calls share the scratch array: calls whose GPU work overlaps (other
 * streams or host threads on the same device) race and must be serialised
 * by the caller.
 */
#define NB_NOALLOC_MAX_ATOMS 32768
#define NB_NOALLOC_SCRATCH_BYTES (32u << 20)
nb_status nb_eval_noalloc(const nb_params *params, int natoms, const double box[3],
                          const int *excl_index, const int *excl_atoms, const float *xq,
                          const int *type, float *f, double *energy, double *virial,
                          unsigned flags, void *cuda_stream);

/*
 * Long-range electrostatics by smooth particle-mesh Ewald (the paper runs
 * PME next to the short-range kernel for the part of the Ewald sum beyond
 * rc: Sections 1 and 2).  With NB_COUL_EWALD, the short-range kernel
 * computes the real-space term f qi qj erfc(beta r) / r of non-excluded
 * pairs inside rc; the long-range part adds
 *   E_rec   the reciprocal sum, f / (2 pi V) sum_{m != 0} exp(-pi^2 m^2 /
 *           beta^2) / m^2 |S(m)|^2 with S(m) = sum_j q_j exp(2 pi i m.x_j),
 *           evaluated by spreading the charges with cardinal B-splines of
 *           order p onto a K_x x K_y x K_z mesh, a 3D FFT, multiplication by
 *           the influence function (with the B-spline moduli) and the
 *           inverse FFT; forces by interpolating the potential mesh with the
 *           splines' derivatives (they are the exact gradient of this E_rec)
 *   E_self  -f beta / sqrt(pi) sum_j q_j^2
 *   E_excl  -f sum over excluded pairs (each once, minimum image, any
 *           distance) of q_i q_j erf(beta r) / r, with its forces
 * and the virial of E_rec (Xi_rec = -1/2 sum_m E_m (delta - 2 (1 + pi^2 m^2
 * / beta^2) m m / m^2)) and of E_excl, all with f = fcoul / eps_r.  The
 * total electrostatic energy is then the Ewald sum with conducting
 * boundary conditions.
 *
 * nb_pme_init: enable the long-range part for an NB_COUL_EWALD system, in a
 * rectangular (nb_sys_create) or triclinic (nb_sys_create_box) cell, or
 * change its mesh; allocates the mesh (4 K_x K_y K_z + 8 K_x K_y (K_z / 2 +
 * 1) bytes, counted against the budget).  In a triclinic cell with rows a,
 * b, c the mesh coordinates are u = x B^-1 diag(K) and the wave vectors m =
 * k B^-T (smooth PME in a general periodic cell), V = ax by cz; the
 * excluded pairs take the image reached by reducing z by c, then y by b,
 * then x by a, which is the minimum image for pairs closer than half the
 * shortest cell height (the molecules' own exclusions).
 *   grid[3]  mesh points along x, y, z: each 8..1024, a product of the
 *            primes 2, 3 and 5 only, with K_d >= 2 p
 *   order    B-spline order p: 4 (cubic, the usual choice), 6 or 8.  Odd
 *            orders are not offered: their B-spline modulus has a pole at
 *            k = K/2 for even K.
 * NB_ERR_ARG for a bad mesh or order or a non-Ewald system.
 */
typedef struct {
    int grid[3];
    int order;
} nb_pme_params;
nb_status nb_pme_init(nb_sys *sys, const nb_pme_params *pme);

/*
 * The long-range part alone, for the coordinates of the last nb_grid_put,
 * or for x_new (as nb_forces: continuous with the last nb_grid_put).
 *   f       natoms * 3 floats (host or device), the long-range force on
 *           each atom in the caller's order (overwritten); NULL allowed
 *   energy  3 doubles (host or device): E_rec, E_self, E_excl; NULL allowed
 *   virial  9 doubles (host or device): Xi_rec + Xi_excl; NULL allowed
 *   flags   NB_F_ENERGY | NB_F_VIRIAL
 * Needs nb_pme_init and a pair list (nb_pairlist_build: the atoms are taken
 * in the grid's sorted order).  Mesh, transforms and forces are float32;
 * the mesh coordinates and the excluded-pair terms are formed as unevaluated
 * float sums (hi + lo, about 48 bits), energies and virial accumulated in
 * float64.
 *
 * nb_forces with NB_F_PME adds the long-range part to the short-range
 * result: the forces are the sum, E_Coulomb = real space + E_rec + E_self +
 * E_excl, the virial the sum.
 */
nb_status nb_pme_forces(nb_sys *sys, const float *x_new, float *f, double *energy, double *virial,
                        unsigned flags);

#ifdef __cplusplus
}
#endif

#endif /* NB_H */
