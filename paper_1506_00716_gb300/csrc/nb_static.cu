// nb_static.cu -- nb_eval_noalloc: a whole evaluation (grid put, pair search,
// prune, forces, energies) whose scratch memory is a fixed file-scope device
// array instead of allocations, for callers that cannot allocate device
// memory (code running where cudaMalloc is unavailable or forbidden, such as
// inside another library's allocator-managed region, a real-time loop, or a
// host process that only owns a stream).
//
// The scratch array below is part of this library's device image: every GPU
// that loads the library's device code reserves NB_NOALLOC_SCRATCH_BYTES for
// it until the process exits.  Under lazy module loading (CUDA_MODULE_LOADING
// = LAZY, the default of recent CUDA releases) that happens at the first
// nb_eval_noalloc call on a device, whose cudaGetSymbolAddress loads this
// file's module; that call can therefore fail with out-of-memory on a device
// that is already full.  Host code cannot use the array's name as a device address
// (in host code it names a host-side shadow), so its device address is
// looked up once per device with cudaGetSymbolAddress and passed to the
// kernels as a plain pointer.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears what must start at zero (counters, column
// counts, force and energy accumulators).  Two calls whose GPU work overlaps
// (different streams, or different host threads on one device) race on the
// array.
#include <algorithm>
#include <mutex>

#include "nb_internal.cuh"

namespace nbgb {

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NB_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
nb_status scratch_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return api_fail(NB_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return api_fail(NB_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return api_fail(NB_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return NB_OK;
}

__global__ void k_lj_tables(const float* __restrict__ c6, const float* __restrict__ c12, int n2,
                            float2* __restrict__ lj, float2* __restrict__ lje) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n2) return;
    lj[k] = make_float2(6.0f * c6[k], 12.0f * c12[k]);
    lje[k] = make_float2(c6[k], c12[k]);
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

}  // namespace nbgb

using namespace nbgb;

extern "C" nb_status nb_eval_noalloc(const nb_params* params, int natoms, const double box[3],
                                     const int* excl_index, const int* excl_atoms, const float* xq,
                                     const int* type, float* f, double* energy, double* virial,
                                     unsigned flags, void* cuda_stream) {
    nb_status s = api_check_system(params, natoms, box);
    if (s != NB_OK) return s;
    if (natoms > NB_NOALLOC_MAX_ATOMS)
        return api_fail(NB_ERR_CAPACITY, "nb_eval_noalloc: natoms exceeds NB_NOALLOC_MAX_ATOMS (32768)");
    if (!xq || !type) return api_fail(NB_ERR_ARG, "xq and type must be non-NULL");
    if (flags & ~(unsigned)(NB_F_ENERGY | NB_F_VIRIAL)) return api_fail(NB_ERR_ARG, "unknown flag bits");
    if ((flags & NB_F_ENERGY) && !energy) return api_fail(NB_ERR_ARG, "NB_F_ENERGY needs energy");
    if ((flags & NB_F_VIRIAL) && !virial) return api_fail(NB_ERR_ARG, "NB_F_VIRIAL needs virial");
    int nnz = 0;
    if (excl_index) {
        // the index array first (non-decreasing from 0), so that no partner
        // range read below lies outside excl_atoms[0 .. nnz)
        if (excl_index[0] != 0) return api_fail(NB_ERR_ARG, "excl_index[0] must be 0");
        for (int a = 0; a < natoms; ++a)
            if (excl_index[a + 1] < excl_index[a]) return api_fail(NB_ERR_ARG, "excl_index must be non-decreasing");
        nnz = excl_index[natoms];
        if (nnz > 0 && !excl_atoms) return api_fail(NB_ERR_ARG, "excl_atoms is NULL but excl_index lists partners");
        // then every partner, before any partner's own range is read
        for (int k = 0; k < nnz; ++k)
            if (excl_atoms[k] < 0 || excl_atoms[k] >= natoms) return api_fail(NB_ERR_ARG, "bad exclusion partner");
        for (int a = 0; a < natoms; ++a) {
            for (int k = excl_index[a]; k < excl_index[a + 1]; ++k) {
                int b = excl_atoms[k];
                if (b == a) return api_fail(NB_ERR_ARG, "bad exclusion partner");
                bool mirrored = false;
                for (int m = excl_index[b]; m < excl_index[b + 1]; ++m) mirrored = mirrored || excl_atoms[m] == a;
                if (!mirrored) return api_fail(NB_ERR_ARG, "exclusions must list every pair under both atoms");
            }
        }
    }
    const int nt = params->ntypes;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void* basev = nullptr;
    s = scratch_base(&basev);
    if (s != NB_OK) return s;
    char* base = (char*)basev;

    // carve the scratch array: descriptor, prefix offsets, system buffers,
    // raw LJ parameters, exclusions, list
    size_t off = 0;
    SysDev* d_sys = (SysDev*)(base + off);
    off += up256(sizeof(SysDev));
    int* d_off = (int*)(base + off);
    off += up256(6 * sizeof(int));
    SysDev h{};
    size_t sys_bytes = api_sys_layout(natoms, box, nt, &h, nullptr);
    if (h.ncol > NB_NOALLOC_MAX_ATOMS / 2)
        return api_fail(NB_ERR_CAPACITY, "nb_eval_noalloc: the box needs too many grid columns");
    char* sys_base = base + off;
    api_sys_layout(natoms, box, nt, &h, sys_base);
    api_list_radii(params->rlist, box, &h);
    off += up256(sys_bytes);
    float2* d_lj = (float2*)(sys_base + sys_bytes - up256(param_table_bytes(nt)));
    float2* d_lje = d_lj + (size_t)nt * nt;
    float* d_c6 = (float*)(base + off);
    off += up256(4 * (size_t)nt * nt);
    float* d_c12 = (float*)(base + off);
    off += up256(4 * (size_t)nt * nt);
    int* d_excl = (int*)(base + off);
    off += up256(4 * ((size_t)natoms + 1 + (size_t)nnz));
    int* d_counters = (int*)(base + off);
    off += up256(4 * CNT_N);
    long long est_items, est_entries;
    api_list_estimate(*params, natoms, box, h.clcap, &est_items, &est_entries);
    if (off >= NB_NOALLOC_SCRATCH_BYTES)
        return api_fail(NB_ERR_CAPACITY, "nb_eval_noalloc: system does not fit the scratch array");
    size_t rest = NB_NOALLOC_SCRATCH_BYTES - off;
    long long items = std::min<long long>(est_items + est_entries / 8, (long long)(rest / 8 / 20));
    int4* d_items = (int4*)(base + off);
    off += up256(16 * (size_t)items);
    int* d_order = (int*)(base + off);
    off += up256(4 * (size_t)items);
    rest = NB_NOALLOC_SCRATCH_BYTES > off ? NB_NOALLOC_SCRATCH_BYTES - off : 0;
    long long entries = (long long)(rest / 12) - 64;
    if (entries < est_entries / 2)
        return api_fail(NB_ERR_CAPACITY, "nb_eval_noalloc: the pair list does not fit the scratch array");
    int* d_cj = (int*)(base + off);
    off += up256(4 * (size_t)entries);
    unsigned long long* d_mask = (unsigned long long*)(base + off);
    off += up256(8 * (size_t)entries);
    if (off > NB_NOALLOC_SCRATCH_BYTES)
        return api_fail(NB_ERR_CAPACITY, "nb_eval_noalloc: scratch layout overflow");

    if (excl_index) {
        h.excl_index = d_excl;
        h.excl_atoms = d_excl + natoms + 1;
    }
    int offs[6] = {0, natoms, 0, h.ncol, 0, h.clcap};

    PlanLaunch p{};
    p.nsys = 1;
    p.d_sys = d_sys;
    p.d_atom_off = d_off;
    p.d_col_off = d_off + 2;
    p.d_cl_off = d_off + 4;
    p.tot_atoms = natoms;
    p.tot_cols = h.ncol;
    p.tot_clcap = h.clcap;
    p.list.items = d_items;
    p.list.cj = d_cj;
    p.list.mask = d_mask;
    p.list.counters = d_counters;
    p.list.order = d_order;
    p.list.item_cap = (int)items;
    p.list.entry_cap = (int)entries;
    p.kp = api_kparams(*params, box, d_lj);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
    p.kp.lpt_max_items = LPT_ITEMS_PER_WARP * LPT_WARPS_PER_SM * p.num_sms;

#define NA_CK(call)                                                  \
    do {                                                             \
        if (e == cudaSuccess) e = (call);                            \
    } while (0)
    NA_CK(cudaMemcpyAsync(d_sys, &h, sizeof(SysDev), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_off, offs, sizeof(offs), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_c6, params->c6, 4 * (size_t)nt * nt, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_c12, params->c12, 4 * (size_t)nt * nt, cudaMemcpyHostToDevice, st));
    if (excl_index) {
        NA_CK(cudaMemcpyAsync(d_excl, excl_index, 4 * ((size_t)natoms + 1), cudaMemcpyHostToDevice, st));
        if (nnz > 0)
            NA_CK(cudaMemcpyAsync(d_excl + natoms + 1, excl_atoms, 4 * (size_t)nnz, cudaMemcpyHostToDevice, st));
    }
    NA_CK(cudaMemcpyAsync(h.xq_in, xq, 16 * (size_t)natoms, cudaMemcpyDefault, st));
    NA_CK(cudaMemcpyAsync(h.type_in, type, 4 * (size_t)natoms, cudaMemcpyDefault, st));
    NA_CK(cudaMemsetAsync(d_counters, 0, 4 * CNT_N, st));
    NA_CK(cudaMemsetAsync(h.acc, 0, 8 * NACC, st));
    if (e == cudaSuccess) {
        k_lj_tables<<<(nt * nt + 255) / 256, 256, 0, st>>>(d_c6, d_c12, nt * nt, d_lj, d_lje);
        e = cudaGetLastError();
    }
    // the Ewald force table, after the Lennard-Jones tables (built on the host,
    // in a buffer on this call's stack)
    float4 gtab[GT_MAX];
    float4 etab[2 * ET_MAX];
    if (params->coul == NB_COUL_EWALD) {
        float invh = 0.f;
        const int gt_n = ewald_force_table(params->ewald_beta, params->rc, gtab, &invh);
        if (gt_n > 0)
            NA_CK(cudaMemcpyAsync((float4*)(d_lj + 2 * (size_t)nt * nt), gtab, 16 * (size_t)gt_n,
                                  cudaMemcpyHostToDevice, st));
        // the energy table after it (the KParams::etab layout)
        const int et_n = ewald_energy_table(params->ewald_beta, params->rc, etab, &invh);
        if (et_n > 0) {
            float4* d_et = (float4*)(d_lj + etab_offset2(nt));
            NA_CK(cudaMemcpyAsync(d_et, etab, 16 * (size_t)et_n, cudaMemcpyHostToDevice, st));
            NA_CK(cudaMemcpyAsync(d_et + ET_MAX, etab + ET_MAX, 16 * (size_t)et_n, cudaMemcpyHostToDevice, st));
        }
        // the copy reads the stack buffer: let it finish before the buffer goes
        NA_CK(cudaStreamSynchronize(st));
    }
    NA_CK(launch_grid_put(p, st));
    NA_CK(launch_search(p, st));
    // the search reports a list that outgrew the scratch array; stop there,
    // before anything is evaluated or written to the caller's outputs
    int counters[CNT_N] = {0};
    NA_CK(cudaMemcpyAsync(counters, d_counters, sizeof(counters), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (e != cudaSuccess) return api_fail(NB_ERR_CUDA, cudaGetErrorString(e));
    if (counters[CNT_OVERFLOW] & 3)
        return api_fail(NB_ERR_CAPACITY, "nb_eval_noalloc: the pair list outgrew the scratch array");
    NA_CK(launch_prune(p, st));
    NA_CK(launch_prepare(p, false, st));
    NA_CK(launch_forces(p, flags, st));
    if (flags & NB_F_ENERGY) NA_CK(launch_energy(p, st));
    NA_CK(launch_excl_corr(p, flags, st));
    NA_CK(launch_finalize(p, flags, st));
    if (f) NA_CK(cudaMemcpyAsync(f, h.f_out, 12 * (size_t)natoms, cudaMemcpyDefault, st));
    if (flags & NB_F_ENERGY) NA_CK(cudaMemcpyAsync(energy, h.res, 16, cudaMemcpyDefault, st));
    if (flags & NB_F_VIRIAL) NA_CK(cudaMemcpyAsync(virial, h.res + 2, 72, cudaMemcpyDefault, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    if (e != cudaSuccess) return api_fail(NB_ERR_CUDA, cudaGetErrorString(e));
    return NB_OK;
}
