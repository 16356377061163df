// nb_api.cu -- the C ABI (include/nb.h): contexts, systems, plans, the
// batch engine and the long-range (PME) set-up.  Host code only; every
// arithmetic step of the method runs in the kernels of nb_grid.cu,
// nb_search.cu, nb_kernel.cu, nb_energy.cu, nb_excl.cu and nb_pme.cu, with
// the paired float32 helpers of nb_pair2.cuh (the host computes only
// per-mesh constant tables: twiddle factors, B-spline moduli, the influence
// function's per-axis factors).
//
// A "plan" is a set of systems evaluated by one sequence of launches: a
// standalone system owns a plan of one, a batch owns a plan over all of its
// systems.  Each system owns its per-atom, per-slot and per-cluster device
// buffers; a plan owns the cluster-pair list (work items, entries, masks)
// and the device descriptor array the kernels index by system.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "nb_host.h"

using namespace nbgb;

namespace nbgb {

thread_local std::string g_err;

nb_status fail(nb_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

nb_status cuda_fail(cudaError_t e, const char* what) {
    return fail(NB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NB_CK(call)                                        \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool is_pinned_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The address at which kernels may read or write a caller's buffer directly:
// device or managed memory as it is, pinned host memory through its mapped
// device address (on a Grace-Blackwell node the kernels then reach host
// memory over the coherent NVLink-C2C link, with no separate copy); nullptr
// for pageable host memory, which goes through the staging buffers.  *host
// is set when the address is host memory.
void* direct_ptr(const void* p, bool* host) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return const_cast<void*>(p);
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *host = true;
        return a.devicePointer;
    }
    return nullptr;
}



Geometry make_geometry(int natoms, const double box[3]) {
    Geometry g;
    double vol = box[0] * box[1] * box[2];
    double rho = natoms / vol;
    double side = std::cbrt((double)CL / rho);
    g.ncx = std::max(1, (int)std::floor(box[0] / side));
    g.ncy = std::max(1, (int)std::floor(box[1] / side));
    g.ncol = g.ncx * g.ncy;
    g.clcap = (natoms + CL - 1) / CL + g.ncol;
    g.cw[0] = (float)(box[0] / g.ncx);
    g.cw[1] = (float)(box[1] / g.ncy);
    g.icw[0] = (float)(g.ncx / box[0]);
    g.icw[1] = (float)(g.ncy / box[1]);
    return g;
}

// Expected list sizes (half list, before pruning) for capacity planning.
void list_estimate(const nb_params& p, int natoms, const double box[3], int clcap, int max_entries,
                   long long* items, long long* entries) {
    double vol = box[0] * box[1] * box[2];
    double rho = natoms / vol;
    double ext = std::cbrt((double)CL / rho);
    double s = 2.0 * ext, r = p.rlist;
    double steiner = s * s * s + 6.0 * s * s * r + 3.0 * M_PI * s * r * r + 4.0 / 3.0 * M_PI * r * r * r;
    double per_cl = steiner * rho / CL / 2.0;
    double shift = 1.0;
    for (int d = 0; d < 3; ++d) shift *= 1.0 + 2.0 * std::min(1.0, (r + ext) / box[d]);
    // the thread-per-cluster search gives every cluster a slab as large as
    // the largest cluster's count: up to the whole neighbourhood (twice the
    // half-list average) for the clusters whose periodic neighbours all
    // have higher indices
    *entries = (long long)(clcap * (per_cl * 2.6 + 16.0) * std::max(1.0, shift / 4.0)) + 4096;
    // one item per (cluster, shift) run, plus the splits of runs longer than
    // max_entries
    *items = (long long)(clcap * std::min(27.0, shift * 1.25)) + *entries / std::max(1, max_entries) + 256;
}

}  // namespace nbgb

namespace nbgb {

nb_status excl_symmetrise(int n, const int* excl_index, const int* excl_atoms, std::vector<int>& idx,
                          std::vector<int>& at, const int** out_idx, const int** out_at) {
    if (!excl_index) return fail(NB_ERR_ARG, "excl_index is NULL");
    if (excl_index[0] != 0) return fail(NB_ERR_ARG, "excl_index[0] must be 0");
    // one pass: validate, and see whether the list is already symmetric,
    // strictly ascending per atom and free of self pairs (then it is used
    // as it is)
    bool canon = true;
    for (int a = 0; a < n; ++a) {
        const int k0 = excl_index[a], k1 = excl_index[a + 1];
        if (k1 < k0) return fail(NB_ERR_ARG, "excl_index must be non-decreasing");
        if (k1 > k0 && !excl_atoms) return fail(NB_ERR_ARG, "excl_atoms is NULL");
        int prev = -1;
        for (int k = k0; k < k1; ++k) {
            const int b = excl_atoms[k];
            if ((unsigned)b >= (unsigned)n) return fail(NB_ERR_ARG, "exclusion partner out of range");
            if (!canon) continue;
            if (b == a || b <= prev) {
                canon = false;
                continue;
            }
            prev = b;
            // b must list a (rows are short: a linear scan; a malformed row
            // of b is reported when b is visited)
            bool found = false;
            for (int q = excl_index[b]; q < excl_index[b + 1]; ++q) found = found || excl_atoms[q] == a;
            canon = found;
        }
    }
    if (canon) {
        *out_idx = excl_index;
        *out_at = excl_atoms;
        return NB_OK;
    }
    // symmetrise with flat arrays: degree count, prefix, fill, then sort and
    // de-duplicate each atom's (short) partner list
    std::vector<int> deg(n + 1, 0);
    for (int a = 0; a < n; ++a)
        for (int k = excl_index[a]; k < excl_index[a + 1]; ++k) {
            const int b = excl_atoms[k];
            if (b == a) continue;
            ++deg[a + 1];
            ++deg[b + 1];
        }
    for (int a = 0; a < n; ++a) deg[a + 1] += deg[a];
    std::vector<int> fillp(deg.begin(), deg.end() - 1), flat(deg[n]);
    for (int a = 0; a < n; ++a)
        for (int k = excl_index[a]; k < excl_index[a + 1]; ++k) {
            const int b = excl_atoms[k];
            if (b == a) continue;
            flat[fillp[a]++] = b;
            flat[fillp[b]++] = a;
        }
    idx.assign(n + 1, 0);
    at.clear();
    at.reserve(flat.size());
    for (int a = 0; a < n; ++a) {
        int* first = flat.data() + deg[a];
        int* last = flat.data() + deg[a + 1];
        std::sort(first, last);
        int* end_u = std::unique(first, last);
        at.insert(at.end(), first, end_u);
        idx[a + 1] = (int)at.size();
    }
    *out_idx = idx.data();
    *out_at = at.data();
    return NB_OK;
}

nb_status sys_upload_exclusions(nb_sys* sys, const int* idx, const int* at) {
    const size_t nidx = (size_t)sys->natoms + 1;
    const size_t nat = (size_t)idx[sys->natoms];
    size_t bytes = 4 * (nidx + std::max<size_t>(1, nat));
    // the new buffer first: if it cannot be had, the old exclusions stay
    void* p = nullptr;
    nb_status s = dev_alloc(sys->ctx, &p, bytes);
    if (s != NB_OK) return s;
    if (sys->d_excl) dev_free(sys->ctx, sys->d_excl, sys->excl_bytes);
    sys->d_excl = (int*)p;
    sys->excl_bytes = bytes;
    NB_CK(cudaMemcpyAsync(sys->d_excl, idx, 4 * nidx, cudaMemcpyHostToDevice, sys->ctx->stream));
    if (nat > 0)
        NB_CK(cudaMemcpyAsync(sys->d_excl + nidx, at, 4 * nat, cudaMemcpyHostToDevice, sys->ctx->stream));
    sys->h.excl_index = sys->d_excl;
    sys->h.excl_atoms = sys->d_excl + nidx;
    // descriptors held by plans are stale now
    if (sys->plan) { plan_destroy(sys->plan); sys->plan = nullptr; }
    sys->listed = false;
    return NB_OK;
}

cudaEvent_t pool_event(nb_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one stage with CUDA events on the context's stream when timing is on.
struct StageScope {
    nb_ctx* c;
    int stage;
    cudaEvent_t a = nullptr;
    StageScope(nb_ctx* ctx, int st) : c(ctx), stage(st) {
        if (((c->timing >> st) & 1u) && !c->capturing) {
            a = pool_event(c);
            if (a) cudaEventRecord(a, c->stream);
        }
    }
    ~StageScope() {
        if (!a) return;
        cudaEvent_t b = pool_event(c);
        if (!b) return;
        cudaEventRecord(b, c->stream);
        c->pending.push_back({stage, a, b});
    }
};

nb_status ctx_reserve(nb_ctx* ctx, size_t bytes) {
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return fail(NB_ERR_BUDGET, "HBM budget exceeded: " + std::to_string(ctx->in_use) + " + " +
                                       std::to_string(bytes) + " > " + std::to_string(ctx->budget));
    return NB_OK;
}

nb_status dev_alloc(nb_ctx* ctx, void** ptr, size_t bytes) {
    if (ctx->fail_allocs > 0) {
        --ctx->fail_allocs;
        *ptr = nullptr;
        return fail(NB_ERR_OOM, "device allocation failed (injected)");
    }
    nb_status s = ctx_reserve(ctx, bytes);
    if (s != NB_OK) return s;
    cudaError_t e = cudaMallocAsync(ptr, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NB_ERR_OOM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    ctx->in_use += bytes;
    return NB_OK;
}

void dev_free(nb_ctx* ctx, void* ptr, size_t bytes) {
    if (!ptr) return;
    cudaFreeAsync(ptr, ctx->stream);
    ctx->in_use -= std::min(ctx->in_use, bytes);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Per-system buffer layout inside one allocation.
size_t sys_layout(int natoms, const Geometry& g, int ntypes, SysDev* h, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    size_t n = (size_t)natoms, S = (size_t)g.clcap * CL;
    char* xq_in = take(16 * n);
    char* type_in = take(4 * n);
    char* x_new = take(12 * n);
    char* atom_col = take(4 * n);
    char* atom_slot = take(4 * n);
    char* iperm = take(4 * n);
    char* f_out = take(12 * n);
    char* keys = take(8 * S);
    char* xq_s = take(16 * S);
    char* type_s = take(4 * S);
    char* perm = take(4 * S);
    char* wrapk = take(4 * S);
    char* f_s = take(16 * S);
    char* bb = take(32 * (size_t)g.clcap);
    char* col_count = take(4 * (size_t)g.ncol);
    char* col_cl0 = take(4 * ((size_t)g.ncol + 1));
    char* acc = take(8 * NACC);
    char* res = take(8 * NRES);
    char* lj = take(param_table_bytes(ntypes));  // (6 c6, 12 c12), (c6, c12), Ewald force table
    (void)lj;
    if (h) {
        h->xq_in = (float4*)xq_in;
        h->type_in = (int*)type_in;
        h->x_new = (float*)x_new;
        h->atom_col = (int*)atom_col;
        h->atom_slot = (int*)atom_slot;
        h->iperm = (int*)iperm;
        h->f_out = (float*)f_out;
        h->keys = (unsigned long long*)keys;
        h->xq_s = (float4*)xq_s;
        h->type_s = (int*)type_s;
        h->perm = (int*)perm;
        h->wrapk = (int*)wrapk;
        h->f_s = (float4*)f_s;
        h->bb = (float4*)bb;
        h->col_count = (int*)col_count;
        h->col_cl0 = (int*)col_cl0;
        h->acc = (double*)acc;
        h->res = (double*)res;
    }
    return off;
}

float2* sys_lj_ptr(nb_sys* s) {
    size_t total = sys_layout(s->natoms, s->geo, s->p.ntypes, nullptr, nullptr);
    size_t lj = align256(param_table_bytes(s->p.ntypes));
    return (float2*)((char*)s->block + total - lj);
}

// The list radius is padded by 1e-5 (1 + the longest box edge): float32
// coordinates of that magnitude carry rounding errors far below the pad, so
// no pair inside rlist can be lost to them.
void list_radii(double rlist, const double box[3], SysDev* h) {
    double maxL = std::max(box[0], std::max(box[1], box[2]));
    double rl = rlist + 1e-5 * (1.0 + maxL);
    h->rl_search = (float)rl;
    h->rl2_prune = (float)(rl * rl);
}

int ewald_force_table(double beta, double rc, float4* coef, float* invh) {
    // the last table built is kept and handed out again while beta and rc
    // stay the same: building one takes a few hundred microseconds
    static std::mutex memo_mu;
    static double memo_beta = -1.0, memo_rc = -1.0;
    static int memo_n = 0;
    static float memo_invh = 0.f;
    static float4 memo[GT_MAX];
    {
        std::lock_guard<std::mutex> lk(memo_mu);
        if (beta == memo_beta && rc == memo_rc) {
            std::memcpy(coef, memo, sizeof(float4) * (size_t)memo_n);
            *invh = memo_invh;
            return memo_n;
        }
    }
    const double isqpi = 0.5641895835477563;
    // G(r) = erfc(x) + 2 x exp(-x^2) / sqrt(pi), x = beta r, decreasing in r;
    // its x-derivatives are -4 x^2 exp(-x^2) / sqrt(pi), then -8 (x - x^3),
    // -8 (1 - 5 x^2 + 2 x^4) and -8 (-12 x + 18 x^3 - 4 x^5), each times
    // exp(-x^2) / sqrt(pi); the r-derivatives carry powers of beta
    auto G = [&](double r) { const double x = beta * r; return std::erfc(x) + 2.0 * isqpi * x * std::exp(-x * x); };
    auto dG = [&](double r) { const double x = beta * r; return -4.0 * isqpi * beta * x * x * std::exp(-x * x); };
    auto d4G = [&](double r) {
        const double x = beta * r;
        const double x2 = x * x, b2 = beta * beta;
        return std::fabs(8.0 * isqpi * x * (-12.0 + x2 * (18.0 - 4.0 * x2)) * std::exp(-x2)) * b2 * b2;
    };
    // relative to G at the interval's far end, G taken as at least 1e-7
    // (where a pair's force factor is below 1e-7 of its value at contact:
    // an absolute error of at most 1e-14 there)
    const double tol = 1e-7;
    const double rmax = rc * (1.0 + 1e-4);
    for (int n = 0; n <= 30; ++n) {
        const double h = std::ldexp(1.0, -n);
        if (h > rmax) continue;
        const int K = (int)std::ceil(rmax / h);
        if (K > GT_MAX) return 0;
        bool ok = true;
        for (int k = 0; k < K && ok; ++k) {
            double m4 = 0.0;
            for (int q = 0; q <= 16; ++q) m4 = std::max(m4, d4G((k + q / 16.0) * h));
            ok = h * h * h * h / 384.0 * m4 <= tol * std::max(G((k + 1) * h), 1e-7);
        }
        if (!ok) continue;
        for (int k = 0; k < K; ++k) {
            const double g0 = G(k * h), g1 = G((k + 1) * h);
            const double d0 = h * dG(k * h), d1 = h * dG((k + 1) * h);
            coef[k] = make_float4((float)g0, (float)d0, (float)(3.0 * (g1 - g0) - 2.0 * d0 - d1),
                                  (float)(2.0 * (g0 - g1) + d0 + d1));
        }
        *invh = (float)(1.0 / h);
        std::lock_guard<std::mutex> lk(memo_mu);
        std::memcpy(memo, coef, sizeof(float4) * (size_t)K);
        memo_n = K;
        memo_invh = *invh;
        memo_beta = beta;
        memo_rc = rc;
        return K;
    }
    return 0;
}

int ewald_energy_table(double beta, double rc, float4* coef, float* invh) {
    static std::mutex memo_mu;
    static double memo_beta = -1.0, memo_rc = -1.0;
    static int memo_n = 0;
    static float memo_invh = 0.f;
    static float4 memo[2 * ET_MAX];
    {
        std::lock_guard<std::mutex> lk(memo_mu);
        if (beta == memo_beta && rc == memo_rc) {
            std::memcpy(coef, memo, sizeof(float4) * (size_t)memo_n);
            std::memcpy(coef + ET_MAX, memo + ET_MAX, sizeof(float4) * (size_t)memo_n);
            *invh = memo_invh;
            return memo_n;
        }
    }
    // the largest |d^2 erfc / dx^2| = (4 / sqrt(pi)) max x exp(-x^2) =
    // 2 sqrt(2 / (e pi)), and |d^5 erfc / dx^5| = (2 / sqrt(pi)) |H4(x)|
    // exp(-x^2) <= 24 / sqrt(pi) (H4 the Hermite polynomial, largest at 0)
    const double pi = 3.14159265358979323846;
    const double m2 = 2.0 * std::sqrt(2.0 / (std::exp(1.0) * pi)), m5 = 24.0 / std::sqrt(pi);
    const double rmax = rc * (1.0 + 1e-4);
    for (int n = 0; n <= 30; ++n) {
        const double h = std::ldexp(1.0, -n);
        if (h > rmax) continue;
        const double bh = beta * h;
        if (0.5 * bh * bh * m2 > 1e-4) continue;
        if (2.0 * std::pow(bh / 4.0, 5) * m5 / 120.0 > 1e-12) continue;
        const int K = (int)std::ceil(rmax / h);
        if (K > ET_MAX) return 0;
        for (int k = 0; k < K; ++k) {
            // interpolation at s_j = (1 - cos((2 j + 1) pi / 10)) / 2: the
            // Vandermonde system in s, solved by Gaussian elimination with
            // partial pivoting
            double A[5][6];
            for (int j = 0; j < 5; ++j) {
                const double sj = 0.5 * (1.0 - std::cos((2 * j + 1) * pi / 10.0));
                double pw = 1.0;
                for (int c = 0; c < 5; ++c, pw *= sj) A[j][c] = pw;
                A[j][5] = std::erfc(beta * h * (k + sj));
            }
            for (int c = 0; c < 5; ++c) {
                int piv = c;
                for (int r = c + 1; r < 5; ++r)
                    if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
                for (int q = 0; q < 6; ++q) std::swap(A[c][q], A[piv][q]);
                for (int r = c + 1; r < 5; ++r) {
                    const double f = A[r][c] / A[c][c];
                    for (int q = c; q < 6; ++q) A[r][q] -= f * A[c][q];
                }
            }
            double a[5];
            for (int c = 4; c >= 0; --c) {
                double t = A[c][5];
                for (int q = c + 1; q < 5; ++q) t -= A[c][q] * a[q];
                a[c] = t / A[c][c];
            }
            const float a0h = (float)a[0], a1h = (float)a[1];
            coef[k] = make_float4(a0h, (float)(a[0] - (double)a0h), a1h, (float)(a[1] - (double)a1h));
            coef[ET_MAX + k] = make_float4((float)a[2], (float)a[3], (float)a[4], 0.f);
        }
        *invh = (float)(1.0 / h);
        std::lock_guard<std::mutex> lk(memo_mu);
        std::memcpy(memo, coef, sizeof(float4) * (size_t)K);
        std::memcpy(memo + ET_MAX, coef + ET_MAX, sizeof(float4) * (size_t)K);
        memo_n = K;
        memo_invh = *invh;
        memo_beta = beta;
        memo_rc = rc;
        return K;
    }
    return 0;
}

KParams make_kparams(const nb_sys* s) {
    KParams k{};
    const nb_params& p = s->p;
    k.rc2_d = p.rc * p.rc;
    k.rc2 = (float)(p.rc * p.rc);
    k.rc2_lo = (float)(p.rc * p.rc * (1.0 - 2e-5));
    k.rc2_hi = (float)(p.rc * p.rc * (1.0 + 2e-5));
    k.fq = (float)(p.fcoul / p.eps_r);
    double krf = p.eps_rf == 0.0 ? 1.0 / (2.0 * p.rc * p.rc * p.rc)
                                 : (p.eps_rf - p.eps_r) / ((2.0 * p.eps_rf + p.eps_r) * p.rc * p.rc * p.rc);
    k.krf = (float)krf;
    k.two_krf = (float)(2.0 * krf);
    k.crf = (float)(1.0 / p.rc + krf * p.rc * p.rc);
    k.beta = (float)p.ewald_beta;
    double crf = 1.0 / p.rc + krf * p.rc * p.rc;
    double fq = p.fcoul / p.eps_r;
    k.krf_h = (float)krf;
    k.krf_l = (float)(krf - (double)k.krf_h);
    k.crf_h = (float)crf;
    k.crf_l = (float)(crf - (double)k.crf_h);
    k.fq_h = (float)fq;
    k.fq_l = (float)(fq - (double)k.fq_h);
    k.mods = p.modifiers;
    const double irc6 = 1.0 / (p.rc * p.rc * p.rc * p.rc * p.rc * p.rc);
    k.irc6_h = (float)irc6;
    k.irc6_l = (float)(irc6 - (double)k.irc6_h);
    k.irc12_h = (float)(irc6 * irc6);
    k.irc12_l = (float)(irc6 * irc6 - (double)k.irc12_h);
    const double ewc = p.coul == NB_COUL_EWALD ? std::erfc(p.ewald_beta * p.rc) / p.rc : 0.0;
    k.ewc_h = (float)ewc;
    k.ewc_l = (float)(ewc - (double)k.ewc_h);
    k.fq_d = fq;
    k.krf_d = krf;
    k.crf_d = crf;
    k.max_entries = 32;
    k.force_min_blocks = 3;
    k.coul = p.coul;
    k.ntypes = p.ntypes;
    {
        // Lennard-Jones as weights (KParams::lj_weights): every nonzero entry
        // is the same (c6, c12) and the nonzero entries are exactly the pairs
        // of types in one set
        const int nt = p.ntypes;
        const float* c6 = s->c6.empty() ? p.c6 : s->c6.data();
        const float* c12 = s->c12.empty() ? p.c12 : s->c12.data();
        unsigned long long m = 0;
        float C6 = 0.f, C12 = 0.f;
        for (int t = 0; t < nt; ++t)
            if (c6[t * nt + t] != 0.f || c12[t * nt + t] != 0.f) {
                m |= 1ull << t;
                C6 = c6[t * nt + t];
                C12 = c12[t * nt + t];
            }
        bool ok = nt <= 64;
        for (int i = 0; i < nt && ok; ++i)
            for (int j = 0; j < nt && ok; ++j) {
                const bool in = ((m >> i) & 1ull) && ((m >> j) & 1ull);
                ok = in ? (c6[i * nt + j] == C6 && c12[i * nt + j] == C12) : (c6[i * nt + j] == 0.f && c12[i * nt + j] == 0.f);
            }
        k.lj_weights = ok ? 1 : 0;
        k.ljw_mask = m;
        k.c6w = 6.0f * C6;
        k.c12w = 12.0f * C12;
    }
    k.lj = s->d_lj;
    k.lje = s->d_lj + (size_t)p.ntypes * p.ntypes;
    k.gtab = reinterpret_cast<const float4*>(s->d_lj + 2 * (size_t)p.ntypes * p.ntypes);
    k.gt_n = 0;
    k.gt_invh = 0.f;
    k.etab = reinterpret_cast<const float4*>(s->d_lj + etab_offset2(p.ntypes));
    k.et_n = 0;
    k.et_invh = 0.f;
    if (p.coul == NB_COUL_EWALD) {
        std::vector<float4> tab(2 * (size_t)std::max(GT_MAX, ET_MAX));
        k.gt_n = ewald_force_table(p.ewald_beta, p.rc, tab.data(), &k.gt_invh);
        k.et_n = ewald_energy_table(p.ewald_beta, p.rc, tab.data(), &k.et_invh);
    }
    return k;
}

bool same_params(const nb_sys* a, const nb_sys* b) {
    const nb_params &p = a->p, &q = b->p;
    return p.rc == q.rc && p.rlist == q.rlist && p.coul == q.coul && p.eps_r == q.eps_r &&
           p.eps_rf == q.eps_rf && p.ewald_beta == q.ewald_beta && p.fcoul == q.fcoul &&
           p.ntypes == q.ntypes && p.modifiers == q.modifiers && a->c6 == b->c6 && a->c12 == b->c12;
}

void plan_free_inner(Plan* pl) {
    if (pl->inner_block) dev_free(pl->ctx, pl->inner_block, pl->inner_bytes);
    pl->inner_block = nullptr;
    pl->inner_bytes = 0;
    pl->inner = ListDev{};
    pl->use_inner = false;
}

void plan_free_list(Plan* pl) {
    plan_free_inner(pl);
    if (pl->list_block) dev_free(pl->ctx, pl->list_block, pl->list_bytes);
    pl->list_block = nullptr;
    pl->list_bytes = 0;
}

// Buffers of the inner list, with the outer list's capacities.
nb_status plan_alloc_inner(Plan* pl) {
    if (pl->inner_block && pl->inner.item_cap == pl->list.item_cap && pl->inner.entry_cap == pl->list.entry_cap)
        return NB_OK;
    plan_free_inner(pl);
    const size_t items = (size_t)pl->list.item_cap, entries = (size_t)pl->list.entry_cap;
    size_t bytes = align256(16 * items) + align256(4 * items) + 2 * align256(4 * entries) + align256(8 * entries) +
                   align256(8 * entries) + align256(4 * CNT_N);
    void* blk = nullptr;
    nb_status s = dev_alloc(pl->ctx, &blk, bytes);
    if (s != NB_OK) return s;
    char* b = (char*)blk;
    pl->inner.items = (int4*)b;
    b += align256(16 * items);
    pl->inner.order = (int*)b;
    b += align256(4 * items);
    pl->inner.cj = (int*)b;
    b += align256(4 * entries);
    pl->inner.cjb = (int*)b;
    b += align256(4 * entries);
    pl->inner.mask = (unsigned long long*)b;
    b += align256(8 * entries);
    pl->inner.marks = (unsigned char*)b;
    b += align256(8 * entries);
    pl->inner.counters = (int*)b;
    pl->inner.item_cap = pl->list.item_cap;
    pl->inner.entry_cap = pl->list.entry_cap;
    pl->inner_block = blk;
    pl->inner_bytes = bytes;
    return NB_OK;
}

void plan_drop_graphs(Plan* pl) {
    for (auto& g : pl->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// The list buffers of the plan, at the given capacities.  The new block is
// allocated before the old one is freed, so that a failure (budget or device
// memory) leaves the plan with its old, still valid list.
nb_status plan_alloc_list(Plan* pl, long long items, long long entries) {
    items = std::min<long long>(items, (1ll << 31) - 1);
    entries = std::min<long long>(entries, (1ll << 31) - 1);
    size_t bytes = align256(16 * (size_t)items) + align256(4 * (size_t)items) + 2 * align256(4 * (size_t)entries) +
                   align256(8 * (size_t)entries) + align256(8 * (size_t)entries) + align256(4 * CNT_N);
    void* blk = nullptr;
    nb_status s = dev_alloc(pl->ctx, &blk, bytes);
    if (s != NB_OK) return s;
    plan_free_list(pl);
    char* b = (char*)blk;
    pl->list.items = (int4*)b;
    b += align256(16 * (size_t)items);
    pl->list.order = (int*)b;
    b += align256(4 * (size_t)items);
    pl->list.cj = (int*)b;
    b += align256(4 * (size_t)entries);
    pl->list.cjb = (int*)b;
    b += align256(4 * (size_t)entries);
    pl->list.mask = (unsigned long long*)b;
    b += align256(8 * (size_t)entries);
    pl->list.marks = (unsigned char*)b;
    b += align256(8 * (size_t)entries);
    pl->list.counters = (int*)b;
    pl->list.item_cap = (int)items;
    pl->list.entry_cap = (int)entries;
    pl->item_cap = items;
    pl->entry_cap = entries;
    pl->list_block = blk;
    pl->list_bytes = bytes;
    NB_CK(cudaMemsetAsync(pl->list.counters, 0, 4 * CNT_N, pl->ctx->stream));
    plan_drop_graphs(pl);
    return NB_OK;
}

constexpr int CNT_BLOCK_INTS = 16;  // >= CNT_N, 64 bytes
static_assert(CNT_BLOCK_INTS >= CNT_N, "counter block too small");

int* ctx_counters_get(nb_ctx* c) {
    if (c->cnt_free.empty()) {
        const int per_slab = 256;
        void* slab = nullptr;
        if (cudaMallocHost(&slab, sizeof(int) * CNT_BLOCK_INTS * per_slab) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c->cnt_slabs.push_back(slab);
        for (int k = per_slab - 1; k >= 0; --k) c->cnt_free.push_back((int*)slab + CNT_BLOCK_INTS * k);
    }
    int* p = c->cnt_free.back();
    c->cnt_free.pop_back();
    return p;
}

void plan_destroy(Plan* pl) {
    if (!pl) return;
    plan_drop_graphs(pl);
    plan_free_list(pl);
    if (pl->d_sys) dev_free(pl->ctx, pl->d_sys, pl->fixed_bytes);
    if (pl->h_counters) pl->ctx->cnt_free.push_back(pl->h_counters);
    if (pl->done_ev) cudaEventDestroy(pl->done_ev);
    delete pl;
}

nb_status plan_create(nb_ctx* ctx, nb_sys* const* systems, int n, Plan** out, double boost) {
    Plan* pl = new Plan();
    pl->ctx = ctx;
    pl->systems.assign(systems, systems + n);
    std::vector<SysDev> hs(n);
    std::vector<int> off(3 * (n + 1), 0);
    long long items = 0, entries = 0;
    for (int k = 0; k < n; ++k) {
        nb_sys* s = systems[k];
        hs[k] = s->h;
        off[k + 1] = off[k] + s->natoms;
        off[(n + 1) + k + 1] = off[(n + 1) + k] + s->geo.ncol;
        off[2 * (n + 1) + k + 1] = off[2 * (n + 1) + k] + s->geo.clcap;
        long long it, en;
        list_estimate(s->p, s->natoms, s->box, s->geo.clcap, ctx->tuning.max_entries, &it, &en);
        items += (long long)(it * boost);
        entries += (long long)(en * boost);
    }
    pl->tot_atoms = off[n];
    pl->tot_cols = off[(n + 1) + n];
    pl->tot_clcap = off[2 * (n + 1) + n];
    size_t fixed = align256(sizeof(SysDev) * n) + align256(4 * off.size());
    void* blk = nullptr;
    nb_status st = dev_alloc(ctx, &blk, fixed);
    if (st != NB_OK) { delete pl; return st; }
    pl->fixed_bytes = fixed;
    pl->d_sys = (SysDev*)blk;
    pl->d_off = (int*)((char*)blk + align256(sizeof(SysDev) * n));
    cudaError_t e = cudaMemcpyAsync(pl->d_sys, hs.data(), sizeof(SysDev) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->d_off, off.data(), 4 * off.size(), cudaMemcpyHostToDevice, ctx->stream);
    // (copies from pageable host memory return once the source is consumed,
    // so the host vectors may go out of scope)
    if (e == cudaSuccess) {
        pl->h_counters = ctx_counters_get(ctx);
        if (!pl->h_counters) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        plan_destroy(pl);
        return cuda_fail(e, "plan_create");
    }
    st = plan_alloc_list(pl, items, entries);
    if (st != NB_OK) { plan_destroy(pl); return st; }
    pl->kp = make_kparams(systems[0]);
    *out = pl;
    return NB_OK;
}

PlanLaunch launch_of(const Plan* pl) {
    PlanLaunch p{};
    const_cast<Plan*>(pl)->kp.max_entries = pl->ctx->tuning.max_entries;
    const_cast<Plan*>(pl)->kp.force_min_blocks = pl->ctx->tuning.force_min_blocks;
    const_cast<Plan*>(pl)->kp.search_mode = pl->ctx->tuning.search_mode;
    const_cast<Plan*>(pl)->kp.energy_mode = pl->ctx->tuning.energy_mode;
    const_cast<Plan*>(pl)->kp.lpt_max_items = LPT_ITEMS_PER_WARP * LPT_WARPS_PER_SM * pl->ctx->num_sms;
    int n = (int)pl->systems.size();
    p.nsys = n;
    p.d_sys = pl->d_sys;
    p.d_atom_off = pl->d_off;
    p.d_col_off = pl->d_off + (n + 1);
    p.d_cl_off = pl->d_off + 2 * (n + 1);
    p.tot_atoms = pl->tot_atoms;
    p.tot_cols = pl->tot_cols;
    p.tot_clcap = pl->tot_clcap;
    p.list = pl->use_inner ? pl->inner : pl->list;
    p.kp = pl->kp;
    p.num_sms = pl->ctx->num_sms;
    return p;
}

// Copy one system's inputs into its device buffers.
nb_status stage_coords(nb_sys* s, const float* xq, const int* type) {
    if (!xq || !type) return fail(NB_ERR_ARG, "xq and type must be non-NULL");
    cudaStream_t st = s->ctx->stream;
    NB_CK(cudaMemcpyAsync(s->h.xq_in, xq, 16 * (size_t)s->natoms, cudaMemcpyDefault, st));
    NB_CK(cudaMemcpyAsync(s->h.type_in, type, 4 * (size_t)s->natoms, cudaMemcpyDefault, st));
    s->has_coords = true;
    return NB_OK;
}

// The j-cluster geometry of the list the next build writes (the context's
// nb_tuning.jcluster); the evaluations of that list read it from the list.
void plan_set_geometry(Plan* pl) { pl->list.jgeo = pl->ctx->tuning.jcluster == 4 ? 1 : 0; }

// Search + prune with capacity growth.  Synchronises the stream.
nb_status plan_build_list(Plan* pl) {
    cudaStream_t st = pl->ctx->stream;
    pl->use_inner = false;  // a new outer list supersedes any inner one
    plan_set_geometry(pl);
    for (int attempt = 0; attempt < 4; ++attempt) {
        NB_CK(cudaMemsetAsync(pl->list.counters + CNT_ITEMS, 0, 4 * 2, st));
        NB_CK(cudaMemsetAsync(pl->list.counters + CNT_PRUNED, 0, 4 * (CNT_N - CNT_PRUNED), st));
        PlanLaunch p = launch_of(pl);
        {
            StageScope sc(pl->ctx, NB_STAGE_SEARCH);
            NB_CK(launch_search(p, st));
        }
        NB_CK(cudaMemcpyAsync(pl->h_counters, pl->list.counters, 4 * CNT_N, cudaMemcpyDeviceToHost, st));
        NB_CK(cudaStreamSynchronize(st));
        int ov = pl->h_counters[CNT_OVERFLOW];
        if (ov & 3) {
            long long ni = std::max<long long>(pl->h_counters[CNT_ITEMS], pl->item_cap);
            long long ne = std::max<long long>(entries_needed(pl->h_counters, pl->tot_clcap), pl->entry_cap);
            NB_CK(cudaMemsetAsync(pl->list.counters + CNT_OVERFLOW, 0, 4, st));
            nb_status s = plan_alloc_list(pl, ni + ni / 4 + 256, ne + ne / 4 + 4096);
            if (s != NB_OK) return s;
            continue;
        }
        {
            StageScope sc(pl->ctx, NB_STAGE_PRUNE);
            NB_CK(launch_prune(p, st));
        }
        return NB_OK;
    }
    return fail(NB_ERR_CAPACITY, "pair list did not fit after growing its buffers");
}

// The long-range launches of one evaluation, each group a timing stage.
nb_status pme_record(nb_ctx* ctx, const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags,
                     cudaStream_t st) {
    {
        StageScope sc(ctx, NB_STAGE_PME_SPREAD);
        NB_CK(launch_pme_spread(p, pm, acc, flags, st));
    }
    {
        StageScope sc(ctx, NB_STAGE_PME_FFT);
        NB_CK(launch_pme_fft(p, pm, acc, flags, st));
    }
    {
        StageScope sc(ctx, NB_STAGE_PME_GATHER);
        NB_CK(launch_pme_gather(p, pm, acc, flags, st));
    }
    return NB_OK;
}

// One evaluation of a plan.  With pme (single-system plans), the long-range
// part runs after the short-range kernels (flags may carry NB_F_PME).
nb_status plan_eval(Plan* pl, unsigned flags, bool coords, const PlanLaunch* ext, const PmeHost* pme = nullptr) {
    cudaStream_t st = pl->ctx->stream;
    PlanLaunch p = launch_of(pl);
    if (ext) {
        p.x_ext = ext->x_ext;
        p.f_ext = ext->f_ext;
        p.e_ext = ext->e_ext;
        p.v_ext = ext->v_ext;
    }
    {
        StageScope sc(pl->ctx, NB_STAGE_ZERO);
        NB_CK(launch_prepare(p, coords, st));
    }
    if ((flags & NB_F_ENERGY) && energy_fused(p)) {
        // one kernel: forces and energies, timed as the energy stage
        StageScope sc(pl->ctx, NB_STAGE_ENERGY);
        NB_CK(launch_forces(p, flags, st));
    } else {
        {
            StageScope sc(pl->ctx, NB_STAGE_FORCES);
            NB_CK(launch_forces(p, flags, st));
        }
        if (flags & NB_F_ENERGY) {
            StageScope sc(pl->ctx, NB_STAGE_ENERGY);
            NB_CK(launch_energy(p, st));
        }
    }
    if (pme && (flags & NB_F_PME)) {
        nb_status s = pme_record(pl->ctx, p, pme->dev, pl->systems[0]->h.acc, flags, st);
        if (s != NB_OK) return s;
    }
    {
        StageScope sc(pl->ctx, NB_STAGE_FINAL);
        NB_CK(launch_excl_corr(p, flags, st));
        NB_CK(launch_finalize(p, flags, st));
    }
    return NB_OK;
}

nb_status copy_out(nb_sys* s, float* f, double* energy, double* virial, unsigned flags, bool* need_sync) {
    cudaStream_t st = s->ctx->stream;
    bool host = false;
    if (f) {
        NB_CK(cudaMemcpyAsync(f, s->h.f_out, 12 * (size_t)s->natoms, cudaMemcpyDefault, st));
        host = host || !is_device_ptr(f);
    }
    if (energy && (flags & NB_F_ENERGY)) {
        NB_CK(cudaMemcpyAsync(energy, s->h.res, 16, cudaMemcpyDefault, st));
        host = host || !is_device_ptr(energy);
    }
    if (virial && (flags & NB_F_VIRIAL)) {
        NB_CK(cudaMemcpyAsync(virial, s->h.res + 2, 72, cudaMemcpyDefault, st));
        host = host || !is_device_ptr(virial);
    }
    *need_sync = host;
    return NB_OK;
}

nb_status check_params(const nb_params* p) {
    if (!p) return fail(NB_ERR_ARG, "params is NULL");
    if (!(p->rc > 0) || !(p->rlist >= p->rc)) return fail(NB_ERR_ARG, "need 0 < rc <= rlist");
    if (p->coul != NB_COUL_RF && p->coul != NB_COUL_EWALD) return fail(NB_ERR_ARG, "unknown coul");
    if (!(p->eps_r > 0)) return fail(NB_ERR_ARG, "eps_r must be > 0");
    if (p->coul == NB_COUL_EWALD && !(p->ewald_beta > 0)) return fail(NB_ERR_ARG, "ewald_beta must be > 0");
    if (p->coul == NB_COUL_EWALD && !(p->ewald_beta * p->rc <= 10.0))
        return fail(NB_ERR_ARG, "ewald_beta * rc must be at most 10 (Ewald force table)");
    if (p->ntypes < 1 || p->ntypes > MAX_TYPES) return fail(NB_ERR_ARG, "ntypes must be in 1..64");
    if (!p->c6 || !p->c12) return fail(NB_ERR_ARG, "c6 / c12 are NULL");
    if (p->modifiers & ~(unsigned)(NB_MOD_LJ_SHIFT | NB_MOD_EWALD_SHIFT | NB_MOD_RF_EXCL))
        return fail(NB_ERR_ARG, "unknown modifier bits");
    if ((p->modifiers & NB_MOD_EWALD_SHIFT) && p->coul != NB_COUL_EWALD)
        return fail(NB_ERR_ARG, "NB_MOD_EWALD_SHIFT needs NB_COUL_EWALD");
    if ((p->modifiers & NB_MOD_RF_EXCL) && p->coul != NB_COUL_RF)
        return fail(NB_ERR_ARG, "NB_MOD_RF_EXCL needs NB_COUL_RF");
    return NB_OK;
}

nb_status check_box(const nb_params* p, const double box[3]) {
    if (!box) return fail(NB_ERR_ARG, "box is NULL");
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0) || !std::isfinite(box[d])) return fail(NB_ERR_ARG, "box edges must be positive");
        if ((float)box[d] < (float)(2.0 * p->rlist))
            return fail(NB_ERR_BOX, "box edge shorter than 2 * rlist");
    }
    return NB_OK;
}

size_t plan_bytes_estimate(const nb_params* p, int natoms, const double box[3], const Geometry& g) {
    long long it, en;
    list_estimate(*p, natoms, box, g.clcap, 8, &it, &en);
    return align256(20 * (size_t)it) + align256(20 * (size_t)en) + 4096;
}

}  // namespace nbgb

// Helpers shared with the allocation-free entry point (nb_static.cu).
namespace nbgb {

nb_status api_fail(nb_status s, const char* msg) { return fail(s, msg); }

nb_status api_check_system(const nb_params* params, int natoms, const double box[3]) {
    nb_status s = check_params(params);
    if (s != NB_OK) return s;
    if (natoms <= 0) return fail(NB_ERR_ARG, "natoms must be > 0");
    return check_box(params, box);
}

size_t api_sys_layout(int natoms, const double box[3], int ntypes, SysDev* h, char* base) {
    Geometry g = make_geometry(natoms, box);
    if (h) {
        for (int d = 0; d < 3; ++d) h->L[d] = (float)box[d];
        h->cw[0] = g.cw[0];
        h->cw[1] = g.cw[1];
        h->icw[0] = g.icw[0];
        h->icw[1] = g.icw[1];
        h->ncx = g.ncx;
        h->ncy = g.ncy;
        h->ncol = g.ncol;
        h->natoms = natoms;
        h->clcap = g.clcap;
        h->excl_index = nullptr;
        h->excl_atoms = nullptr;
    }
    return sys_layout(natoms, g, ntypes, h, base);
}

void api_list_radii(double rlist, const double box[3], SysDev* h) { list_radii(rlist, box, h); }

KParams api_kparams(const nb_params& p, const double box[3], float2* lj) {
    nb_sys tmp;
    tmp.p = p;
    for (int d = 0; d < 3; ++d) tmp.box[d] = box[d];
    tmp.d_lj = lj;
    return make_kparams(&tmp);
}

void api_list_estimate(const nb_params& p, int natoms, const double box[3], int clcap, long long* items,
                       long long* entries) {
    list_estimate(p, natoms, box, clcap, 32, items, entries);
}

// ------------------------------------------------------------- PME (host)

// Stockham stages of a length-n transform: radix 16 while possible, then 4,
// 2, 3 and 5.  False if n has another prime factor or needs too many stages.
bool fft_radices(int n, FftAxis* ax) {
    ax->n = n;
    ax->nst = 0;
    const int order[5] = {16, 4, 2, 3, 5};
    for (int r : order) {
        while (n % r == 0) {
            if (ax->nst == FFT_MAX_STAGES) return false;
            ax->rad[ax->nst++] = r;
            n /= r;
        }
    }
    return n == 1;
}

// Cardinal B-spline M_p at the integers 0..p-1 (float64), by the recursion
// M_k(x) = (x M_{k-1}(x) + (k - x) M_{k-1}(x - 1)) / (k - 1) from M_2.
std::vector<double> bspline_at_integers(int p) {
    std::vector<double> m(p, 0.0);
    m[1] = 1.0;  // M_2(1) = 1, M_2(0) = 0
    for (int k = 3; k <= p; ++k)
        for (int j = k - 1; j >= 1; --j) m[j] = (j * m[j] + (k - j) * m[j - 1]) / (k - 1);
    return m;
}

// |b(k)|^2 = 1 / |sum_{j=0}^{p-2} M_p(j + 1) exp(2 pi i k j / K)|^2, k = 0..K-1.
std::vector<double> bspline_moduli(int K, int p) {
    const std::vector<double> m = bspline_at_integers(p);
    std::vector<double> out(K);
    for (int k = 0; k < K; ++k) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j <= p - 2; ++j) {
            const double a = 2.0 * M_PI * (double)k * j / K;
            re += m[j + 1] * std::cos(a);
            im += m[j + 1] * std::sin(a);
        }
        out[k] = 1.0 / (re * re + im * im);
    }
    return out;
}

}  // namespace nbgb

extern "C" {

const char* nb_last_error(void) { return g_err.c_str(); }

nb_status nb_ctx_create(int device, void* cuda_stream, size_t hbm_budget_bytes, nb_ctx** out) {
    if (!out) return fail(NB_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(NB_ERR_ARG, "no such CUDA device");
    NB_CK(cudaSetDevice(device));
    nb_ctx* c = new nb_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->budget = hbm_budget_bytes;
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaDeviceGetAttribute"); }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return NB_OK;
}

nb_status nb_ctx_destroy(nb_ctx* ctx) {
    if (!ctx) return fail(NB_ERR_ARG, "ctx is NULL");
    cudaStreamSynchronize(ctx->stream);
    for (auto& t : ctx->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    for (void* slab : ctx->cnt_slabs) cudaFreeHost(slab);
    delete ctx;
    return NB_OK;
}

nb_status nb_ctx_set_tuning(nb_ctx* ctx, const nb_tuning* t) {
    if (!ctx || !t) return fail(NB_ERR_ARG, "ctx / tuning is NULL");
    if (t->max_entries < 4 || t->max_entries > 4096) return fail(NB_ERR_ARG, "max_entries must be in 4..4096");
    if (t->force_min_blocks < 1 || t->force_min_blocks > 4)
        return fail(NB_ERR_ARG, "force_min_blocks must be 1, 2, 3 or 4");
    if (t->search_mode < 0 || t->search_mode > 2) return fail(NB_ERR_ARG, "search_mode must be 0, 1 or 2");
    if (t->energy_mode < 0 || t->energy_mode > 1) return fail(NB_ERR_ARG, "energy_mode must be 0 or 1");
    if (t->jcluster != 0 && t->jcluster != 8 && t->jcluster != 4)
        return fail(NB_ERR_ARG, "jcluster must be 0, 8 or 4");
    ctx->tuning = *t;
    ctx->tuning_gen += 1;
    return NB_OK;
}

nb_status nb_ctx_get_tuning(nb_ctx* ctx, nb_tuning* t) {
    if (!ctx || !t) return fail(NB_ERR_ARG, "ctx / tuning is NULL");
    *t = ctx->tuning;
    return NB_OK;
}

nb_status nb_ctx_set_timing(nb_ctx* ctx, int enable) {
    if (!ctx) return fail(NB_ERR_ARG, "ctx is NULL");
    ctx->timing = enable != 0 ? (1u << NB_NSTAGE) - 1u : 0u;
    return NB_OK;
}

nb_status nb_ctx_set_timing_stages(nb_ctx* ctx, unsigned stage_mask) {
    if (!ctx) return fail(NB_ERR_ARG, "ctx is NULL");
    if (stage_mask >> NB_NSTAGE) return fail(NB_ERR_ARG, "stage_mask has bits beyond NB_NSTAGE");
    ctx->timing = stage_mask;
    return NB_OK;
}

nb_status nb_ctx_timing(nb_ctx* ctx, double* ms, long long* launches, int reset) {
    if (!ctx) return fail(NB_ERR_ARG, "ctx is NULL");
    NB_CK(cudaStreamSynchronize(ctx->stream));
    for (auto& t : ctx->pending) {
        float el = 0.f;
        NB_CK(cudaEventElapsedTime(&el, t.a, t.b));
        ctx->tot_ms[t.stage] += el;
        ctx->launches[t.stage] += 1;
        ctx->pool.push_back(t.a);
        ctx->pool.push_back(t.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < NB_NSTAGE; ++k) {
        if (ms) ms[k] = ctx->tot_ms[k];
        if (launches) launches[k] = ctx->launches[k];
        if (reset) {
            ctx->tot_ms[k] = 0;
            ctx->launches[k] = 0;
        }
    }
    return NB_OK;
}

nb_status nb_ctx_memory(nb_ctx* ctx, size_t* bytes_in_use, size_t* budget) {
    if (!ctx) return fail(NB_ERR_ARG, "ctx is NULL");
    if (bytes_in_use) *bytes_in_use = ctx->in_use;
    if (budget) *budget = ctx->budget;
    return NB_OK;
}

nb_status nb_ctx_inject_alloc_failures(nb_ctx* ctx, int count) {
    if (!ctx || count < 0) return fail(NB_ERR_ARG, "ctx is NULL or count < 0");
    ctx->fail_allocs = count;
    return NB_OK;
}

nb_status nb_sys_footprint(const nb_params* params, int natoms, const double box[3], size_t* bytes) {
    nb_status s = check_params(params);
    if (s != NB_OK) return s;
    if (natoms <= 0) return fail(NB_ERR_ARG, "natoms must be > 0");
    s = check_box(params, box);
    if (s != NB_OK) return s;
    if (!bytes) return fail(NB_ERR_ARG, "bytes is NULL");
    Geometry g = make_geometry(natoms, box);
    *bytes = sys_layout(natoms, g, params->ntypes, nullptr, nullptr) + plan_bytes_estimate(params, natoms, box, g);
    return NB_OK;
}

static nb_status sys_create(nb_ctx* ctx, const nb_params* params, int natoms, const double box[3],
                            const double skew[3], nb_sys** out) {
    nb_status s;
    nb_sys* y = new nb_sys();
    y->ctx = ctx;
    y->p = *params;
    int nt = params->ntypes;
    y->c6.assign(params->c6, params->c6 + nt * nt);
    y->c12.assign(params->c12, params->c12 + nt * nt);
    y->p.c6 = y->c6.data();
    y->p.c12 = y->c12.data();
    y->natoms = natoms;
    for (int d = 0; d < 3; ++d) y->box[d] = box[d];
    y->geo = make_geometry(natoms, box);
    size_t bytes = sys_layout(natoms, y->geo, nt, nullptr, nullptr);
    s = dev_alloc(ctx, &y->block, bytes);
    if (s != NB_OK) { delete y; return s; }
    y->bytes = bytes;
    sys_layout(natoms, y->geo, nt, &y->h, (char*)y->block);
    y->d_lj = sys_lj_ptr(y);
    SysDev& h = y->h;
    for (int d = 0; d < 3; ++d) {
        h.L[d] = (float)box[d];
        h.T[d] = (float)skew[d];
    }
    list_radii(params->rlist, box, &h);
    h.cw[0] = y->geo.cw[0];
    h.cw[1] = y->geo.cw[1];
    h.icw[0] = y->geo.icw[0];
    h.icw[1] = y->geo.icw[1];
    h.ncx = y->geo.ncx;
    h.ncy = y->geo.ncy;
    h.ncol = y->geo.ncol;
    h.natoms = natoms;
    h.clcap = y->geo.clcap;
    h.excl_index = nullptr;
    h.excl_atoms = nullptr;
    // parameter tables: the Lennard-Jones pairs, then (Ewald) the force table
    std::vector<float2> lj(etab_offset2(nt) + 4 * (size_t)ET_MAX, make_float2(0.f, 0.f));
    for (int k = 0; k < nt * nt; ++k) {
        lj[k] = make_float2(6.0f * y->c6[k], 12.0f * y->c12[k]);
        lj[nt * nt + k] = make_float2(y->c6[k], y->c12[k]);
    }
    int gt_n = 0, et_n = 0;
    if (y->p.coul == NB_COUL_EWALD) {
        float invh = 0.f;
        gt_n = ewald_force_table(y->p.ewald_beta, y->p.rc, reinterpret_cast<float4*>(lj.data() + 2 * nt * nt), &invh);
        float einvh = 0.f;
        et_n = ewald_energy_table(y->p.ewald_beta, y->p.rc, reinterpret_cast<float4*>(lj.data() + etab_offset2(nt)),
                                  &einvh);
    }
    // the filled parts only: the Lennard-Jones pairs with the force table
    // after them, then the energy table's two halves
    cudaError_t e = cudaMemcpyAsync(y->d_lj, lj.data(), 8 * (2 * (size_t)nt * nt + 2 * (size_t)gt_n),
                                    cudaMemcpyHostToDevice, ctx->stream);
    for (int half = 0; half < 2 && et_n > 0 && e == cudaSuccess; ++half) {
        const size_t off = etab_offset2(nt) + 2 * (size_t)ET_MAX * half;
        e = cudaMemcpyAsync(y->d_lj + off, lj.data() + off, 16 * (size_t)et_n, cudaMemcpyHostToDevice, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h.acc, 0, 8 * NACC, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h.res, 0, 8 * NRES, ctx->stream);
    if (e != cudaSuccess) {
        dev_free(ctx, y->block, y->bytes);
        delete y;
        return cuda_fail(e, "nb_sys_create");
    }
    *out = y;
    return NB_OK;
}

nb_status nb_sys_create(nb_ctx* ctx, const nb_params* params, int natoms, const double box[3], nb_sys** out) {
    if (!ctx || !out) return fail(NB_ERR_ARG, "ctx / out is NULL");
    *out = nullptr;
    nb_status s = check_params(params);
    if (s != NB_OK) return s;
    if (natoms <= 0) return fail(NB_ERR_ARG, "natoms must be > 0");
    s = check_box(params, box);
    if (s != NB_OK) return s;
    const double zero[3] = {0.0, 0.0, 0.0};
    return sys_create(ctx, params, natoms, box, zero, out);
}

nb_status nb_sys_create_box(nb_ctx* ctx, const nb_params* params, int natoms, const double m[9], nb_sys** out) {
    if (!ctx || !out || !m) return fail(NB_ERR_ARG, "ctx / box / out is NULL");
    *out = nullptr;
    nb_status s = check_params(params);
    if (s != NB_OK) return s;
    if (natoms <= 0) return fail(NB_ERR_ARG, "natoms must be > 0");
    // the float32 box the device uses
    const double ax = (float)m[0], bx = (float)m[3], by = (float)m[4], cx = (float)m[6], cy = (float)m[7],
                 cz = (float)m[8];
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(m[k])) return fail(NB_ERR_ARG, "box components must be finite");
    if (m[1] != 0.0 || m[2] != 0.0 || m[5] != 0.0)
        return fail(NB_ERR_BOX, "box rows must be a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz)");
    if (!(ax > 0 && by > 0 && cz > 0)) return fail(NB_ERR_BOX, "ax, by and cz must be positive");
    if (std::fabs(bx) + std::fabs(cx) > 0.5 * ax * (1.0 + 1e-6) || std::fabs(cy) > 0.5 * by * (1.0 + 1e-6))
        return fail(NB_ERR_BOX, "box too skewed: need |bx| + |cx| <= ax/2 and |cy| <= by/2");
    const double rl = params->rlist;
    if (rl > 0.5 * ax || rl > 0.5 * by || !(rl < cz))
        return fail(NB_ERR_BOX, "box too small for rlist: need rlist <= ax/2, by/2 and < cz");
    // a pair inside rlist must have one image only: every lattice vector at
    // least 2 rlist long
    double shortest = 1e300;
    for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j)
            for (int k = -1; k <= 1; ++k) {
                if (!i && !j && !k) continue;
                const double vx = i * ax + j * bx + k * cx, vy = j * by + k * cy, vz = k * cz;
                shortest = std::min(shortest, std::sqrt(vx * vx + vy * vy + vz * vz));
            }
    if (shortest < 2.0 * rl) return fail(NB_ERR_BOX, "a lattice vector is shorter than 2 * rlist");
    const double box[3] = {m[0], m[4], m[8]}, skew[3] = {m[3], m[6], m[7]};
    return sys_create(ctx, params, natoms, box, skew, out);
}

nb_status nb_sys_destroy(nb_sys* sys) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    nb_ctx* ctx = sys->ctx;
    plan_destroy(sys->plan);
    if (sys->pme) {
        dev_free(ctx, sys->pme->block, sys->pme->bytes);
        delete sys->pme;
    }
    if (sys->d_excl) dev_free(ctx, sys->d_excl, sys->excl_bytes);
    dev_free(ctx, sys->block, sys->bytes);
    delete sys;
    return NB_OK;
}

nb_status nb_set_exclusions(nb_sys* sys, const int* excl_index, const int* excl_atoms) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    std::vector<int> idx, at;
    const int *pi = nullptr, *pa = nullptr;
    nb_status s = excl_symmetrise(sys->natoms, excl_index, excl_atoms, idx, at, &pi, &pa);
    if (s != NB_OK) return s;
    // copies from pageable memory have consumed their source when they
    // return; a pinned caller array would be read later, so it is copied
    // to pageable memory first (the call copies its inputs)
    if (pi == excl_index && (is_pinned_ptr(excl_index) || is_pinned_ptr(excl_atoms))) {
        idx.assign(excl_index, excl_index + sys->natoms + 1);
        at.assign(excl_atoms, excl_atoms + excl_index[sys->natoms]);
        pi = idx.data();
        pa = at.data();
    }
    return sys_upload_exclusions(sys, pi, pa);
}

static nb_status ensure_plan(nb_sys* sys) {
    if (sys->plan) return NB_OK;
    nb_sys* one[1] = {sys};
    return plan_create(sys->ctx, one, 1, &sys->plan);
}

nb_status nb_grid_put(nb_sys* sys, const float* xq, const int* type) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    nb_status s = stage_coords(sys, xq, type);
    if (s != NB_OK) return s;
    s = ensure_plan(sys);
    if (s != NB_OK) return s;
    cudaStream_t st = sys->ctx->stream;
    NB_CK(cudaMemsetAsync(sys->plan->list.counters + CNT_OVERFLOW, 0, 4, st));
    {
        StageScope sc(sys->ctx, NB_STAGE_GRID);
        NB_CK(launch_grid_put(launch_of(sys->plan), st));
    }
    sys->gridded = true;
    sys->listed = false;
    return NB_OK;
}

nb_status nb_pairlist_build(nb_sys* sys) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    if (!sys->gridded) return fail(NB_ERR_STATE, "nb_pairlist_build needs a preceding nb_grid_put");
    nb_status s = plan_build_list(sys->plan);
    if (s != NB_OK) return s;
    sys->listed = true;
    return NB_OK;
}

nb_status nb_pairlist_prune(nb_sys* sys, double r_inner) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    if (!sys->listed) return fail(NB_ERR_STATE, "nb_pairlist_prune needs a pair list (nb_pairlist_build)");
    if (!(r_inner >= sys->p.rc) || !(r_inner <= sys->p.rlist))
        return fail(NB_ERR_ARG, "r_inner must lie in [rc, rlist]");
    Plan* pl = sys->plan;
    cudaStream_t st = sys->ctx->stream;
    nb_status s = plan_alloc_inner(pl);
    if (s != NB_OK) return s;
    NB_CK(cudaMemsetAsync(pl->inner.counters, 0, 4 * CNT_N, st));
    // padded like the outer radius, for the float32 rounding of coordinates
    double maxL = std::max(sys->box[0], std::max(sys->box[1], sys->box[2]));
    double r = r_inner + 1e-5 * (1.0 + maxL);
    pl->use_inner = false;
    pl->inner.jgeo = pl->list.jgeo;
    PlanLaunch p = launch_of(pl);
    {
        StageScope sc(sys->ctx, NB_STAGE_PRUNE);
        NB_CK(launch_prune_into(p, pl->list, pl->inner, (float)(r * r), st));
    }
    pl->use_inner = true;
    return NB_OK;
}

nb_status nb_pairlist_info(nb_sys* sys, nb_list_info* info) {
    if (!sys || !info) return fail(NB_ERR_ARG, "sys / info is NULL");
    if (!sys->listed) return fail(NB_ERR_STATE, "no pair list");
    Plan* pl = sys->plan;
    cudaStream_t st = sys->ctx->stream;
    int ncl = 0;
    NB_CK(cudaMemcpyAsync(pl->h_counters, pl->list.counters, 4 * CNT_N, cudaMemcpyDeviceToHost, st));
    NB_CK(cudaMemcpyAsync(&ncl, sys->h.col_cl0 + sys->geo.ncol, 4, cudaMemcpyDeviceToHost, st));
    NB_CK(cudaStreamSynchronize(st));
    info->n_clusters = ncl;
    info->n_items = pl->h_counters[CNT_ITEMS];
    info->n_entries_raw = pl->h_counters[CNT_ENTRIES];
    info->n_entries = pl->h_counters[CNT_PRUNED];
    info->n_entries_inner = info->n_entries;
    if (pl->use_inner) {
        NB_CK(cudaMemcpyAsync(pl->h_counters, pl->inner.counters, 4 * CNT_N, cudaMemcpyDeviceToHost, st));
        NB_CK(cudaStreamSynchronize(st));
        info->n_entries_inner = pl->h_counters[CNT_PRUNED];
    }
    info->n_slots = info->n_entries_inner * CL * CL;
    return NB_OK;
}

nb_status nb_eval_info(nb_sys* sys, nb_eval_stats* stats) {
    if (!sys || !stats) return fail(NB_ERR_ARG, "sys / stats is NULL");
    double np = 0;
    NB_CK(cudaMemcpyAsync(&np, sys->h.res + 11, 8, cudaMemcpyDeviceToHost, sys->ctx->stream));
    NB_CK(cudaStreamSynchronize(sys->ctx->stream));
    stats->n_pairs = (long long)np;
    return NB_OK;
}

nb_status nb_ewald_energy_table(double beta, double rc, float* coef, int max_intervals, int* n_intervals,
                                double* h) {
    if (!(beta > 0) || !(rc > 0) || !(beta * rc <= 10.0)) return fail(NB_ERR_ARG, "need beta > 0, rc > 0, beta rc <= 10");
    if (!n_intervals) return fail(NB_ERR_ARG, "n_intervals is NULL");
    std::vector<float4> tab(2 * (size_t)ET_MAX);
    float invh = 0.f;
    const int K = ewald_energy_table(beta, rc, tab.data(), &invh);
    if (K <= 0) return fail(NB_ERR_ARG, "the table needs more intervals than it may hold");
    *n_intervals = K;
    if (h) *h = 1.0 / (double)invh;
    if (coef) {
        if (max_intervals < K) return fail(NB_ERR_ARG, "coef holds fewer intervals than the table");
        for (int k = 0; k < K; ++k) {
            const float4 a = tab[(size_t)k], b = tab[(size_t)ET_MAX + k];
            const float row[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            std::memcpy(coef + 8 * (size_t)k, row, sizeof(row));
        }
    }
    return NB_OK;
}

nb_status nb_ewald_force_table(double beta, double rc, float* coef, int max_intervals, int* n_intervals,
                               double* h) {
    if (!(beta > 0) || !(rc > 0) || !(beta * rc <= 10.0)) return fail(NB_ERR_ARG, "need beta > 0, rc > 0, beta rc <= 10");
    if (!n_intervals) return fail(NB_ERR_ARG, "n_intervals is NULL");
    float4 tab[GT_MAX];
    float invh = 0.f;
    const int K = ewald_force_table(beta, rc, tab, &invh);
    if (K <= 0) return fail(NB_ERR_ARG, "the table needs more intervals than it may hold");
    *n_intervals = K;
    if (h) *h = 1.0 / (double)invh;
    if (coef) {
        if (max_intervals < K) return fail(NB_ERR_ARG, "coef holds fewer intervals than the table");
        std::memcpy(coef, tab, 16 * (size_t)K);
    }
    return NB_OK;
}

// The list's items and masks (and, for a list of the 8 x 8 geometry, its
// j-clusters) in host or device arrays.
static nb_status nb_pairlist_export_any(nb_sys* sys, int* perm, int* items, int* cj, unsigned long long* mask,
                                        long long* n_entries_total) {
    nb_list_info info;
    nb_status s = nb_pairlist_info(sys, &info);
    if (s != NB_OK) return s;
    Plan* pl = sys->plan;
    cudaStream_t st = sys->ctx->stream;
    // the entry arrays reach the largest item end (the thread-per-cluster
    // search leaves gaps between the clusters' slabs)
    const long long n_items = std::min<long long>(info.n_items, pl->item_cap);
    std::vector<int4> it((size_t)std::max<long long>(n_items, 1));
    if (n_items > 0)
        NB_CK(cudaMemcpyAsync(it.data(), pl->list.items, 16 * (size_t)n_items, cudaMemcpyDeviceToHost, st));
    NB_CK(cudaStreamSynchronize(st));
    long long ne = 0;
    for (long long k = 0; k < n_items; ++k) ne = std::max<long long>(ne, it[k].z);
    ne = std::min<long long>(ne, pl->entry_cap);
    if (n_entries_total) *n_entries_total = ne;
    if (perm) NB_CK(cudaMemcpyAsync(perm, sys->h.perm, 4 * (size_t)info.n_clusters * CL, cudaMemcpyDefault, st));
    if (items && n_items > 0) std::memcpy(items, it.data(), 16 * (size_t)n_items);
    if (cj) NB_CK(cudaMemcpyAsync(cj, pl->list.cj, 4 * (size_t)ne, cudaMemcpyDefault, st));
    if (mask) NB_CK(cudaMemcpyAsync(mask, pl->list.mask, 8 * (size_t)ne, cudaMemcpyDefault, st));
    NB_CK(cudaStreamSynchronize(st));
    return NB_OK;
}

nb_status nb_pairlist_export(nb_sys* sys, int* perm, int* items, int* cj, unsigned long long* mask,
                             long long* n_entries_total) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    if (!sys->listed) return fail(NB_ERR_STATE, "no pair list");
    if (cj && sys->plan->list.jgeo)
        return fail(NB_ERR_STATE, "the list has 4-atom j-clusters: nb_pairlist_export_slots gives its j-atoms");
    return nb_pairlist_export_any(sys, perm, items, cj, mask, n_entries_total);
}

nb_status nb_pairlist_export_slots(nb_sys* sys, int* perm, int* items, int* jslot, unsigned long long* mask,
                                   long long* n_entries_total) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    if (!sys->listed) return fail(NB_ERR_STATE, "no pair list");
    long long ne = 0;
    nb_status s = nb_pairlist_export_any(sys, perm, items, nullptr, mask, &ne);
    if (s != NB_OK) return s;
    if (n_entries_total) *n_entries_total = ne;
    if (!jslot || ne == 0) return NB_OK;
    Plan* pl = sys->plan;
    cudaStream_t st = sys->ctx->stream;
    std::vector<int> a((size_t)ne), b(pl->list.jgeo ? (size_t)ne : 0);
    NB_CK(cudaMemcpyAsync(a.data(), pl->list.cj, 4 * (size_t)ne, cudaMemcpyDeviceToHost, st));
    if (pl->list.jgeo) NB_CK(cudaMemcpyAsync(b.data(), pl->list.cjb, 4 * (size_t)ne, cudaMemcpyDeviceToHost, st));
    NB_CK(cudaStreamSynchronize(st));
    for (long long e = 0; e < ne; ++e) {
        jslot[2 * e] = pl->list.jgeo ? a[(size_t)e] : a[(size_t)e] * CL;
        jslot[2 * e + 1] = pl->list.jgeo ? b[(size_t)e] + 4 : a[(size_t)e] * CL + 4;
    }
    return NB_OK;
}

nb_status nb_forces(nb_sys* sys, const float* x_new, float* f, double* energy, double* virial, unsigned flags) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    if (flags & ~(unsigned)(NB_F_ENERGY | NB_F_VIRIAL | NB_F_PME)) return fail(NB_ERR_ARG, "unknown flag bits");
    if ((flags & NB_F_PME) && !sys->pme) return fail(NB_ERR_STATE, "NB_F_PME needs nb_pme_init");
    if ((flags & NB_F_ENERGY) && !energy) return fail(NB_ERR_ARG, "NB_F_ENERGY needs energy");
    if ((flags & NB_F_VIRIAL) && !virial) return fail(NB_ERR_ARG, "NB_F_VIRIAL needs virial");
    if (!sys->listed) return fail(NB_ERR_STATE, "nb_forces needs a pair list (nb_pairlist_build)");
    Plan* pl = sys->plan;
    cudaStream_t st = sys->ctx->stream;
    // device and pinned host arrays of the caller are read and written by
    // the kernels themselves; pageable host arrays go through the system's
    // staging buffers
    PlanLaunch ext{};
    bool direct_host = false;
    ext.x_ext = static_cast<const float*>(direct_ptr(x_new, &direct_host));
    ext.f_ext = static_cast<float*>(direct_ptr(f, &direct_host));
    ext.e_ext = static_cast<double*>(direct_ptr(energy, &direct_host));
    ext.v_ext = static_cast<double*>(direct_ptr(virial, &direct_host));
    if (x_new && !ext.x_ext) {
        StageScope sc(sys->ctx, NB_STAGE_COORD);
        NB_CK(cudaMemcpyAsync(sys->h.x_new, x_new, 12 * (size_t)sys->natoms, cudaMemcpyHostToDevice, st));
    }
    nb_status s = plan_eval(pl, flags, x_new != nullptr, &ext, sys->pme);
    if (s != NB_OK) return s;
    bool need_sync = false;
    s = copy_out(sys, ext.f_ext ? nullptr : f, ext.e_ext ? nullptr : energy, ext.v_ext ? nullptr : virial,
                 flags, &need_sync);
    if (s != NB_OK) return s;
    // host memory read or written by the kernels is done with when the call
    // returns, as with the staged copies
    if (need_sync || direct_host) NB_CK(cudaStreamSynchronize(st));
    return NB_OK;
}

// ------------------------------------------------------------------ batches

nb_status nb_sys_set_coords(nb_sys* sys, const float* xq, const int* type) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    nb_status s = stage_coords(sys, xq, type);
    if (s != NB_OK) return s;
    sys->gridded = false;
    sys->listed = false;
    return NB_OK;
}

nb_status nb_batch_create(nb_ctx* ctx, nb_sys* const* systems, int n, nb_batch** out) {
    if (!ctx || !systems || !out || n <= 0) return fail(NB_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!systems[k] || systems[k]->ctx != ctx) return fail(NB_ERR_ARG, "system from another context");
        if (!same_params(systems[0], systems[k])) return fail(NB_ERR_ARG, "systems differ in parameters");
    }
    nb_batch* b = new nb_batch();
    b->ctx = ctx;
    nb_status s = plan_create(ctx, systems, n, &b->plan);
    if (s != NB_OK) { delete b; return s; }
    *out = b;
    return NB_OK;
}

nb_status nb_batch_destroy(nb_batch* batch) {
    if (!batch) return fail(NB_ERR_ARG, "batch is NULL");
    cudaStreamSynchronize(batch->ctx->stream);
    plan_destroy(batch->plan);
    delete batch;
    return NB_OK;
}

static nb_status batch_record(Plan* pl, unsigned flags) {
    cudaStream_t st = pl->ctx->stream;
    plan_set_geometry(pl);
    PlanLaunch p = launch_of(pl);
    // per-stage timing applies when the sequence runs directly (not captured)
    NB_CK(cudaMemsetAsync(pl->list.counters, 0, 4 * CNT_N, st));
    {
        StageScope sc(pl->ctx, NB_STAGE_GRID);
        NB_CK(launch_grid_put(p, st));
    }
    {
        StageScope sc(pl->ctx, NB_STAGE_SEARCH);
        NB_CK(launch_search(p, st));
    }
    {
        StageScope sc(pl->ctx, NB_STAGE_PRUNE);
        NB_CK(launch_prune(p, st));
    }
    {
        StageScope sc(pl->ctx, NB_STAGE_ZERO);
        NB_CK(launch_prepare(p, false, st));
    }
    if ((flags & NB_F_ENERGY) && energy_fused(p)) {
        // one kernel: forces and energies, timed as the energy stage
        StageScope sc(pl->ctx, NB_STAGE_ENERGY);
        NB_CK(launch_forces(p, flags, st));
    } else {
        {
            StageScope sc(pl->ctx, NB_STAGE_FORCES);
            NB_CK(launch_forces(p, flags, st));
        }
        if (flags & NB_F_ENERGY) {
            StageScope sc(pl->ctx, NB_STAGE_ENERGY);
            NB_CK(launch_energy(p, st));
        }
    }
    {
        StageScope sc(pl->ctx, NB_STAGE_FINAL);
        NB_CK(launch_excl_corr(p, flags, st));
        NB_CK(launch_finalize(p, flags, st));
    }
    NB_CK(cudaMemcpyAsync(pl->h_counters, pl->list.counters, 4 * CNT_N, cudaMemcpyDeviceToHost, st));
    return NB_OK;
}

nb_status nb_batch_submit(nb_batch* batch, unsigned flags, unsigned long long* ticket) {
    if (!batch || !ticket) return fail(NB_ERR_ARG, "batch / ticket is NULL");
    if (flags & ~(unsigned)(NB_F_ENERGY | NB_F_VIRIAL)) return fail(NB_ERR_ARG, "unknown flag bits");
    Plan* pl = batch->plan;
    for (nb_sys* s : pl->systems)
        if (!s->has_coords) return fail(NB_ERR_STATE, "a batch system has no coordinates");
    cudaStream_t st = batch->ctx->stream;
    if (pl->graph_tuning_gen != batch->ctx->tuning_gen) {
        plan_drop_graphs(pl);
        pl->graph_tuning_gen = batch->ctx->tuning_gen;
    }
    cudaGraphExec_t& ge = pl->graph[flags & 3];
    if (!ge) {
        if (st == nullptr) {
            // the legacy default stream cannot be captured: run the launches directly
            nb_status s = batch_record(pl, flags);
            if (s != NB_OK) return s;
        } else {
            cudaGraph_t g = nullptr;
            NB_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            batch->ctx->capturing = true;
            nb_status s = batch_record(pl, flags);
            batch->ctx->capturing = false;
            cudaError_t e = cudaStreamEndCapture(st, &g);
            if (s != NB_OK) { if (g) cudaGraphDestroy(g); return s; }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { ge = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
        }
    }
    if (ge) NB_CK(cudaGraphLaunch(ge, st));
    NB_CK(cudaEventRecord(pl->done_ev, st));
    *ticket = ++pl->ticket;
    for (nb_sys* s : pl->systems) {
        s->gridded = false;
        s->listed = false;
    }
    return NB_OK;
}

nb_status nb_batch_poll(nb_batch* batch, unsigned long long ticket, long long timeout_us, int* done) {
    if (!batch || !done) return fail(NB_ERR_ARG, "batch / done is NULL");
    Plan* pl = batch->plan;
    *done = 0;
    if (ticket == 0 || ticket > pl->ticket) return fail(NB_ERR_ARG, "unknown ticket");
    if (ticket < pl->ticket || ticket <= pl->done_ticket) {
        *done = 1;
        return NB_OK;
    }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(pl->done_ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
        long long el = std::chrono::duration_cast<std::chrono::microseconds>(
                           std::chrono::steady_clock::now() - t0).count();
        if (el >= timeout_us) return fail(NB_ERR_TIMEOUT, "batch not finished within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    pl->done_ticket = ticket;
    *done = 1;
    int ov = pl->h_counters[CNT_OVERFLOW];
    if (ov & 3) {
        long long ni = std::max<long long>(pl->h_counters[CNT_ITEMS], pl->item_cap);
        long long ne = std::max<long long>(entries_needed(pl->h_counters, pl->tot_clcap), pl->entry_cap);
        nb_status s = plan_alloc_list(pl, ni + ni / 4 + 256, ne + ne / 4 + 4096);
        if (s != NB_OK) return s;
        NB_CK(cudaStreamSynchronize(batch->ctx->stream));
        return fail(NB_ERR_CAPACITY, "batch pair list outgrew its buffer; buffers grown, submit again");
    }
    return NB_OK;
}

// ---------------------------------------------------------------- PME

nb_status nb_pme_init(nb_sys* sys, const nb_pme_params* pp) {
    if (!sys || !pp) return fail(NB_ERR_ARG, "sys / pme is NULL");
    if (sys->p.coul != NB_COUL_EWALD) return fail(NB_ERR_ARG, "the long-range part needs NB_COUL_EWALD");
    const int p = pp->order;
    if (p != 4 && p != 6 && p != 8) return fail(NB_ERR_ARG, "PME order must be 4, 6 or 8");
    FftAxis axis[3];
    for (int d = 0; d < 3; ++d) {
        const int K = pp->grid[d];
        if (K < 8 || K > 1024 || K < 2 * p || !fft_radices(K, &axis[d]))
            return fail(NB_ERR_ARG, "each PME mesh size must be in 8..1024, >= 2 * order, with prime factors 2, 3, 5");
    }
    if ((size_t)pme_smem_need(pp->grid) > 227 * 1024) return fail(NB_ERR_ARG, "PME mesh too large");
    const int K0 = pp->grid[0], K1 = pp->grid[1], K2 = pp->grid[2], Kzh = K2 / 2 + 1;
    // one block: tables, twiddles, spectrum, mesh
    size_t off = 0;
    size_t o_tab[3], o_tw[3];
    for (int d = 0; d < 3; ++d) {
        o_tab[d] = off;
        off = align256(off + 8 * (size_t)pp->grid[d]);
        o_tw[d] = off;
        off = align256(off + 8 * (size_t)pp->grid[d]);
    }
    const size_t o_S = off;
    off = align256(off + 8 * (size_t)K0 * K1 * Kzh);
    const size_t o_Q = off;
    off = align256(off + 4 * (size_t)K0 * K1 * K2);
    PmeHost* ph = new PmeHost();
    nb_status s = dev_alloc(sys->ctx, &ph->block, off);
    if (s != NB_OK) {
        delete ph;
        return s;
    }
    ph->bytes = off;
    char* base = (char*)ph->block;
    PmeDev& pm = ph->dev;
    const double f = sys->p.fcoul / sys->p.eps_r, beta = sys->p.ewald_beta;
    // the cell the device uses (float32 box rows a = (ax,0,0), b = (bx,by,0),
    // c = (cx,cy,cz)) and its inverse R = B^-1, lower-triangular
    const double ax = sys->h.L[0], by = sys->h.L[1], cz = sys->h.L[2];
    const double bx = sys->h.T[0], cx = sys->h.T[1], cy = sys->h.T[2];
    const bool tri = bx != 0.0 || cx != 0.0 || cy != 0.0;
    const double R10 = -bx / (ax * by), R21 = -cy / (by * cz), R20 = (bx * cy - by * cx) / (ax * by * cz);
    const double V = ax * by * cz;
    std::vector<float2> host(off / 8, make_float2(0.f, 0.f));
    const double Ld[3] = {ax, by, cz};
    for (int d = 0; d < 3; ++d) {
        const int K = pp->grid[d];
        pm.K[d] = K;
        pm.kl[d] = K / Ld[d];
        pm.ax[d] = axis[d];
        pm.ax[d].tw = (const float2*)(base + o_tw[d]);
        pm.tab[d] = (const float2*)(base + o_tab[d]);
        const std::vector<double> bm = bspline_moduli(K, p);
        for (int k = 0; k < K; ++k) {
            const double ks = (k <= K / 2 ? k : k - K);
            const double m = ks / Ld[d];
            host[o_tab[d] / 8 + k] =
                tri ? make_float2((float)ks, (float)bm[k])
                    : make_float2((float)m, (float)(bm[k] * std::exp(-M_PI * M_PI * m * m / (beta * beta))));
            const double a = -2.0 * M_PI * (double)k / K;
            host[o_tw[d] / 8 + k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    }
    pm.tri = tri ? 1 : 0;
    const double mo[3] = {R10 * pp->grid[0], R20 * pp->grid[0], R21 * pp->grid[1]};
    const double rdg[3] = {1.0 / ax, 1.0 / by, 1.0 / cz}, ro[3] = {R10, R20, R21};
    pm.Kzh = Kzh;
    pm.order = p;
    pm.S = (float2*)(base + o_S);
    pm.Q = (float*)(base + o_Q);
    pm.cpre = (float)(f / (M_PI * V));
    pm.pi2_b2 = (float)(M_PI * M_PI / (beta * beta));
    pm.self_pre = -f * beta / std::sqrt(M_PI);
    pm.beta = beta;
    pm.fq = f;
    auto split = [](double v, float& h, float& l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    for (int d = 0; d < 3; ++d) {
        split(pm.kl[d], pm.kl_h[d], pm.kl_l[d]);
        split(mo[d], pm.mo_h[d], pm.mo_l[d]);
        pm.rd[d] = (float)rdg[d];
        pm.ro[d] = (float)ro[d];
    }
    split(f, pm.fq_h, pm.fq_l);
    split(2.0 * beta / std::sqrt(M_PI), pm.ke_h, pm.ke_l);
    split(4.0 / 3.0 * beta * beta * beta / std::sqrt(M_PI), pm.kf_h, pm.kf_l);
    pm.beta2 = (float)(beta * beta);
    cudaStream_t st = sys->ctx->stream;
    // tables only (the mesh and spectrum are written by every evaluation)
    cudaError_t e = cudaMemcpyAsync(base, host.data(), o_S, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = pme_prepare_kernels(pm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(sys->ctx, ph->block, ph->bytes);
        delete ph;
        return cuda_fail(e, "nb_pme_init");
    }
    if (sys->pme) {
        dev_free(sys->ctx, sys->pme->block, sys->pme->bytes);
        delete sys->pme;
    }
    sys->pme = ph;
    return NB_OK;
}

nb_status nb_pme_forces(nb_sys* sys, const float* x_new, float* f, double* energy, double* virial,
                        unsigned flags) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    if (flags & ~(unsigned)(NB_F_ENERGY | NB_F_VIRIAL)) return fail(NB_ERR_ARG, "unknown flag bits");
    if ((flags & NB_F_ENERGY) && !energy) return fail(NB_ERR_ARG, "NB_F_ENERGY needs energy");
    if ((flags & NB_F_VIRIAL) && !virial) return fail(NB_ERR_ARG, "NB_F_VIRIAL needs virial");
    if (!sys->pme) return fail(NB_ERR_STATE, "nb_pme_forces needs nb_pme_init");
    if (!sys->listed) return fail(NB_ERR_STATE, "nb_pme_forces needs a pair list (nb_pairlist_build)");
    Plan* pl = sys->plan;
    cudaStream_t st = sys->ctx->stream;
    PlanLaunch p = launch_of(pl);
    if (x_new && is_device_ptr(x_new)) p.x_ext = x_new;
    if (f && is_device_ptr(f)) p.f_ext = f;
    if (virial && is_device_ptr(virial)) p.v_ext = virial;
    if (x_new && !p.x_ext) {
        StageScope sc(sys->ctx, NB_STAGE_COORD);
        NB_CK(cudaMemcpyAsync(sys->h.x_new, x_new, 12 * (size_t)sys->natoms, cudaMemcpyHostToDevice, st));
    }
    {
        StageScope sc(sys->ctx, NB_STAGE_ZERO);
        NB_CK(launch_prepare(p, x_new != nullptr, st));
    }
    nb_status s = pme_record(sys->ctx, p, sys->pme->dev, sys->h.acc, flags, st);
    if (s != NB_OK) return s;
    {
        StageScope sc(sys->ctx, NB_STAGE_FINAL);
        NB_CK(launch_finalize(p, flags, st));
    }
    bool host = false;
    if (f && !p.f_ext) {
        NB_CK(cudaMemcpyAsync(f, sys->h.f_out, 12 * (size_t)sys->natoms, cudaMemcpyDefault, st));
        host = true;
    }
    if (energy && (flags & NB_F_ENERGY)) {
        NB_CK(cudaMemcpyAsync(energy, sys->h.res + 12, 24, cudaMemcpyDefault, st));
        host = host || !is_device_ptr(energy);
    }
    if (virial && (flags & NB_F_VIRIAL) && !p.v_ext) {
        NB_CK(cudaMemcpyAsync(virial, sys->h.res + 2, 72, cudaMemcpyDefault, st));
        host = true;
    }
    if (host) NB_CK(cudaStreamSynchronize(st));
    return NB_OK;
}

nb_status nb_sys_results(nb_sys* sys, float* f, double* energy, double* virial) {
    if (!sys) return fail(NB_ERR_ARG, "sys is NULL");
    bool need_sync = false;
    nb_status s = copy_out(sys, f, energy, virial, (energy ? NB_F_ENERGY : 0) | (virial ? NB_F_VIRIAL : 0),
                           &need_sync);
    if (s != NB_OK) return s;
    if (need_sync) NB_CK(cudaStreamSynchronize(sys->ctx->stream));
    return NB_OK;
}

}  // extern "C"
