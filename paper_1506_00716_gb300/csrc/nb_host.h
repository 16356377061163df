// nb_host.h -- host-side state of the library (contexts, systems, plans)
// and the helpers of nb_api.cu that other translation units use (the
// serving engine).  Not part of the public ABI.
#pragma once

#include <string>
#include <vector>

#include "nb_internal.cuh"

namespace nbgb {

struct Geometry {
    int ncx, ncy, ncol, clcap;
    float cw[2], icw[2];
};

}  // namespace nbgb

struct Plan;
using nbgb::Geometry;

struct TimedLaunch {
    int stage;
    cudaEvent_t a, b;
};

struct nb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    size_t in_use = 0;
    int fail_allocs = 0;  // nb_ctx_inject_alloc_failures
    int num_sms = 0;
    unsigned timing = 0;  // mask of timed stages (1 << NB_STAGE_*)
    bool capturing = false;
    nb_tuning tuning{32, 3, 0, 0};
    unsigned tuning_gen = 0;
    std::vector<TimedLaunch> pending;
    std::vector<cudaEvent_t> pool;
    // pinned counter read-back blocks of plans, carved from slabs so that
    // creating and destroying a plan allocates and frees no pinned memory
    std::vector<int*> cnt_free;
    std::vector<void*> cnt_slabs;
    double tot_ms[NB_NSTAGE] = {0};
    long long launches[NB_NSTAGE] = {0};
};

// Long-range (PME) state of a system: the device view and the one
// allocation holding its mesh, spectrum and tables.
struct PmeHost {
    nbgb::PmeDev dev{};
    void* block = nullptr;
    size_t bytes = 0;
};

struct nb_sys {
    nb_ctx* ctx = nullptr;
    nb_params p{};
    std::vector<float> c6, c12;
    int natoms = 0;
    double box[3] = {0, 0, 0};
    nbgb::Geometry geo{};
    nbgb::SysDev h{};              // descriptor (device pointers)
    void* block = nullptr;   // one allocation holding all per-system buffers
    size_t bytes = 0;
    int* d_excl = nullptr;   // exclusion CSR (index then atoms)
    size_t excl_bytes = 0;
    float2* d_lj = nullptr;
    Plan* plan = nullptr;    // standalone plan (lazy)
    PmeHost* pme = nullptr;  // nb_pme_init
    bool has_coords = false;
    bool gridded = false;
    bool listed = false;
};

struct Plan {
    nb_ctx* ctx = nullptr;
    std::vector<nb_sys*> systems;
    nbgb::SysDev* d_sys = nullptr;
    int* d_off = nullptr;     // atom, col, cl prefix arrays (3 * (nsys + 1))
    nbgb::ListDev list{};
    void* list_block = nullptr;
    size_t list_bytes = 0;
    // inner list (nb_pairlist_prune): the outer list pruned, out of place, to
    // a smaller radius; the evaluations use it while use_inner is set
    nbgb::ListDev inner{};
    void* inner_block = nullptr;
    size_t inner_bytes = 0;
    bool use_inner = false;
    size_t fixed_bytes = 0;
    int tot_atoms = 0, tot_cols = 0, tot_clcap = 0;
    long long item_cap = 0, entry_cap = 0;
    int* h_counters = nullptr;  // pinned readback
    nbgb::KParams kp{};
    // graph state (batches)
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned graph_tuning_gen = 0;
    cudaEvent_t done_ev = nullptr;
    unsigned long long ticket = 0;
    unsigned long long done_ticket = 0;
};

struct nb_batch {
    nb_ctx* ctx = nullptr;
    Plan* plan = nullptr;
};

namespace nbgb {

nb_status fail(nb_status s, const std::string& msg);
nb_status cuda_fail(cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
bool is_pinned_ptr(const void* p);
Geometry make_geometry(int natoms, const double box[3]);
void list_estimate(const nb_params& p, int natoms, const double box[3], int clcap, int max_entries,
                   long long* items, long long* entries);
nb_status dev_alloc(nb_ctx* ctx, void** ptr, size_t bytes);
void dev_free(nb_ctx* ctx, void* ptr, size_t bytes);
// boost scales the estimated list capacity (retries after an overflow)
nb_status plan_create(nb_ctx* ctx, nb_sys* const* systems, int n, Plan** out, double boost = 1.0);
void plan_destroy(Plan* pl);
// Set the geometry of the list the next search and prune write (from the
// context's tuning); call before launch_of of a build.
void plan_set_geometry(Plan* pl);
PlanLaunch launch_of(const Plan* pl);
nb_status stage_coords(nb_sys* s, const float* xq, const int* type);
// Symmetric, sorted, duplicate-free exclusion CSR from the caller's CSR
// (validated).  *out_idx / *out_at point at the caller's arrays when they
// already have that form, else at idx / at, which receive the symmetrised CSR.
nb_status excl_symmetrise(int n, const int* excl_index, const int* excl_atoms, std::vector<int>& idx,
                          std::vector<int>& at, const int** out_idx, const int** out_at);
// Upload a CSR made by excl_symmetrise (idx: natoms + 1 entries, at: idx[natoms])
// to the system's device buffers.  Pageable sources are consumed when the call
// returns; pinned sources must stay valid until the stream has passed the copies.
nb_status sys_upload_exclusions(nb_sys* sys, const int* idx, const int* at);

}  // namespace nbgb
