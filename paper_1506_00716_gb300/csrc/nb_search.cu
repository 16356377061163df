// nb_search.cu -- cluster-pair search and list pruning.
//
// Search (Section 3.2): for every i-cluster and every periodic image of it
// that can reach the central box, visit the grid columns whose footprint
// lies within rlist of the (shifted) i-cluster bounding box, take the
// z-range of clusters in each column that can be within rlist, and keep the
// j-clusters whose bounding boxes are closer than rlist.  The list is a half
// list: an unordered cluster pair is kept once, by the lower cluster index
// (ci < cj with any shift; ci == cj with the zero shift or a "positive"
// shift, index > 13).  Only the lower index ever makes the keep decision, so
// rounding in the float32 box test can neither drop nor duplicate a pair;
// the test radius is padded to stay conservative.
//
// Each kept entry carries an 8 x 8 interaction mask in a rotated layout:
// bit 8*i + t refers to the pair (i-slot i, j-slot t XOR i).  Bits are
// cleared for filler slots, for the lower triangle and diagonal of a
// cluster's pair with itself (zero shift), and for excluded atom pairs.
//
// Prune (Section 3.2.1, "Heterogeneous parallelization": the list is pruned
// on the GPU and then reused): entries with no unmasked atom pair closer
// than rlist are removed, compacting each work item's entries in place.
#include "nb_internal.cuh"

namespace nbgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SEARCH_WARPS = 4;

__device__ __forceinline__ int find_sys(const int* __restrict__ off, int nsys, int idx) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int rot_bit(int i, int j) { return 8 * i + (i ^ j); }

// bits of pairs (i, j) with j > i
__device__ unsigned long long diag_mask() {
    unsigned long long m = 0;
    for (int i = 0; i < CL; ++i)
        for (int j = i + 1; j < CL; ++j) m |= 1ull << rot_bit(i, j);
    return m;
}

// bits of pairs with i < ni and j < nj
__device__ unsigned long long real_mask(int ni, int nj) {
    unsigned long long m = 0;
    for (int i = 0; i < ni; ++i)
        for (int j = 0; j < nj; ++j) m |= 1ull << rot_bit(i, j);
    return m;
}

struct SearchWarpSmem {
    int cj[SEARCH_BUF];
    unsigned long long mask[SEARCH_BUF];
    unsigned char sh[SEARCH_BUF];
    int ex_slot[EXCL_BUF];
    unsigned char ex_i[EXCL_BUF];
    int n_ex;
};

__device__ __forceinline__ float gap(float alo, float ahi, float blo, float bhi) {
    return fmaxf(0.f, fmaxf(blo - ahi, alo - bhi));
}

// Write the buffered entries as work items: one per run of equal shift,
// split into pieces of at most max_entries entries.
__device__ void flush(SearchWarpSmem& sm, int nbuf, int ci, int sid, const ListDev& list, int lane,
                      int max_entries) {
    if (nbuf == 0) return;
    // items per run start, and their total
    int nitems = 0;
    for (int base = 0; base < nbuf; base += 32) {
        int k = base + lane;
        int nch = 0;
        if (k < nbuf && (k == 0 || sm.sh[k] != sm.sh[k - 1])) {
            int e = k + 1;
            while (e < nbuf && sm.sh[e] == sm.sh[k]) ++e;
            nch = (e - k + max_entries - 1) / max_entries;
        }
        for (int off = 16; off > 0; off >>= 1) nch += __shfl_xor_sync(FULL, nch, off);
        nitems += nch;
    }
    int ibase = 0, ebase = 0;
    if (lane == 0) {
        ibase = atomicAdd(list.counters + CNT_ITEMS, nitems);
        ebase = atomicAdd(list.counters + CNT_ENTRIES, nbuf);
    }
    ibase = __shfl_sync(FULL, ibase, 0);
    ebase = __shfl_sync(FULL, ebase, 0);
    bool ok_e = (long long)ebase + nbuf <= list.entry_cap;
    bool ok_i = (long long)ibase + nitems <= list.item_cap;
    if (lane == 0 && !ok_e) atomicOr(list.counters + CNT_OVERFLOW, 2);
    if (lane == 0 && !ok_i) atomicOr(list.counters + CNT_OVERFLOW, 1);
    if (ok_e) {
        for (int k = lane; k < nbuf; k += 32) {
            list.cj[ebase + k] = sm.cj[k];
            list.mask[ebase + k] = sm.mask[k];
        }
    }
    if (ok_i) {
        // on entry overflow the items are still written, empty, so that the
        // counted item range never holds stale data
        int ord = 0;
        for (int base = 0; base < nbuf; base += 32) {
            int k = base + lane;
            int e = k, nch = 0;
            if (k < nbuf && (k == 0 || sm.sh[k] != sm.sh[k - 1])) {
                e = k + 1;
                while (e < nbuf && sm.sh[e] == sm.sh[k]) ++e;
                nch = (e - k + max_entries - 1) / max_entries;
            }
            int incl = nch;
            for (int off = 1; off < 32; off <<= 1) {
                int v = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += v;
            }
            int idx = ibase + ord + incl - nch;
            for (int q = 0; q < nch; ++q) {
                int a = k + q * max_entries;
                int b = min(e, a + max_entries);
                list.items[idx + q] = ok_e ? make_int4(ci, ebase + a, ebase + b, (sid << 5) | sm.sh[k])
                                           : make_int4(ci, 0, 0, (sid << 5) | sm.sh[k]);
            }
            ord += __shfl_sync(FULL, incl, 31);
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(SEARCH_WARPS * 32)
k_search(const SysDev* __restrict__ sys, const int* __restrict__ cl_off, int nsys, int tot_clcap,
         ListDev list, KParams kp) {
    __shared__ SearchWarpSmem s_w[SEARCH_WARPS];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int gw = blockIdx.x * SEARCH_WARPS + w;
    if (gw >= tot_clcap) return;
    const int sid = find_sys(cl_off, nsys, gw);
    const SysDev& d = sys[sid];
    const int ci = gw - cl_off[sid];
    const int ncl = d.col_cl0[d.ncol];
    if (ci >= ncl) return;
    SearchWarpSmem& sm = s_w[w];

    const float4 lo_i = d.bb[2 * ci];
    const float4 hi_i = d.bb[2 * ci + 1];
    const int nri = (int)lo_i.w;
    const float rl = kp.rl_search;
    const float rl2 = rl * rl;
    const float eps = 1e-5f * fmaxf(1.f, fmaxf(d.L[0], fmaxf(d.L[1], d.L[2])));

    // cache the exclusion partners (as sorted slots) of this cluster's atoms
    if (lane == 0) sm.n_ex = 0;
    __syncwarp();
    bool ex_overflow = false;
    if (d.excl_index != nullptr && lane < nri) {
        int a = d.perm[ci * CL + lane];
        for (int e = d.excl_index[a]; e < d.excl_index[a + 1]; ++e) {
            int p = d.iperm[d.excl_atoms[e]];
            int k = atomicAdd(&sm.n_ex, 1);
            if (k < EXCL_BUF) {
                sm.ex_slot[k] = p;
                sm.ex_i[k] = (unsigned char)lane;
            }
        }
    }
    __syncwarp();
    const int n_ex = min(sm.n_ex, EXCL_BUF);
    ex_overflow = sm.n_ex > EXCL_BUF;
    const unsigned long long dmask = diag_mask();

    int nbuf = 0;
    for (int sx = -1; sx <= 1; ++sx) {
        if (sx == 1 && !(lo_i.x < rl)) continue;
        if (sx == -1 && !(hi_i.x > d.L[0] - rl)) continue;
        for (int sy = -1; sy <= 1; ++sy) {
            if (sy == 1 && !(lo_i.y < rl)) continue;
            if (sy == -1 && !(hi_i.y > d.L[1] - rl)) continue;
            for (int sz = -1; sz <= 1; ++sz) {
                if (sz == 1 && !(lo_i.z < rl)) continue;
                if (sz == -1 && !(hi_i.z > d.L[2] - rl)) continue;
                const int shift = shift_index(sx, sy, sz);
                const float Sx = sx * d.L[0], Sy = sy * d.L[1], Sz = sz * d.L[2];
                const float lx = lo_i.x + Sx, ly = lo_i.y + Sy, lz = lo_i.z + Sz;
                const float hx = hi_i.x + Sx, hy = hi_i.y + Sy, hz = hi_i.z + Sz;
                int cx0 = max(0, (int)floorf((lx - rl) * d.icw[0]) - 1);
                int cx1 = min(d.ncx - 1, (int)floorf((hx + rl) * d.icw[0]) + 1);
                int cy0 = max(0, (int)floorf((ly - rl) * d.icw[1]) - 1);
                int cy1 = min(d.ncy - 1, (int)floorf((hy + rl) * d.icw[1]) + 1);
                if (cx0 > cx1 || cy0 > cy1) continue;
                const int nyc = cy1 - cy0 + 1;
                const int ncand = (cx1 - cx0 + 1) * nyc;
                const float zmin = lz - rl, zmax = hz + rl;
                for (int cbase = 0; cbase < ncand; cbase += 32) {
                    int k = cbase + lane;
                    bool has = k < ncand;
                    int cur = 0, cend = 0;
                    if (has) {
                        int cx = cx0 + k / nyc, cy = cy0 + k % nyc;
                        float fx0 = cx * d.cw[0] - eps, fx1 = (cx + 1) * d.cw[0] + eps;
                        float fy0 = cy * d.cw[1] - eps, fy1 = (cy + 1) * d.cw[1] + eps;
                        float gx = gap(lx, hx, fx0, fx1), gy = gap(ly, hy, fy0, fy1);
                        if (gx * gx + gy * gy >= rl2) has = false;
                        if (has) {
                            int col = cx * d.ncy + cy;
                            int c0 = d.col_cl0[col], c1 = d.col_cl0[col + 1];
                            // first cluster whose top is at or above zmin
                            int a = c0, b = c1;
                            while (a < b) {
                                int m = (a + b) >> 1;
                                if (d.bb[2 * m + 1].z < zmin) a = m + 1; else b = m;
                            }
                            cur = a;
                            cend = c1;
                        }
                    }
                    for (;;) {
                        bool cand = has && cur < cend;
                        float4 lj = make_float4(0.f, 0.f, 0.f, 0.f), hj;
                        if (cand) {
                            lj = d.bb[2 * cur];
                            if (lj.z > zmax) { cand = false; has = false; }
                        }
                        if (!__any_sync(FULL, cand)) break;
                        bool pass = false;
                        if (cand) {
                            hj = d.bb[2 * cur + 1];
                            float gx = gap(lx, hx, lj.x, hj.x);
                            float gy = gap(ly, hy, lj.y, hj.y);
                            float gz = gap(lz, hz, lj.z, hj.z);
                            pass = gx * gx + gy * gy + gz * gz < rl2 &&
                                   (cur > ci || (cur == ci && shift >= SHIFT_ZERO));
                        }
                        unsigned bal = __ballot_sync(FULL, pass);
                        int np = __popc(bal);
                        if (nbuf + np > SEARCH_BUF) {
                            flush(sm, nbuf, ci, sid, list, lane, kp.max_entries);
                            nbuf = 0;
                        }
                        if (pass) {
                            unsigned long long m = ~0ull;
                            if (cur == ci && shift == SHIFT_ZERO) m = dmask;
                            int nrj = (int)lj.w;
                            if (nri < CL || nrj < CL) m &= real_mask(nri, nrj);
                            if (!ex_overflow) {
                                for (int q = 0; q < n_ex; ++q) {
                                    int p = sm.ex_slot[q];
                                    if ((p >> 3) == cur) m &= ~(1ull << rot_bit(sm.ex_i[q], p & 7));
                                }
                            } else {
                                for (int ii = 0; ii < nri; ++ii) {
                                    int a = d.perm[ci * CL + ii];
                                    for (int e = d.excl_index[a]; e < d.excl_index[a + 1]; ++e) {
                                        int p = d.iperm[d.excl_atoms[e]];
                                        if ((p >> 3) == cur) m &= ~(1ull << rot_bit(ii, p & 7));
                                    }
                                }
                            }
                            int idx = nbuf + __popc(bal & ((1u << lane) - 1u));
                            sm.cj[idx] = cur;
                            sm.mask[idx] = m;
                            sm.sh[idx] = (unsigned char)shift;
                        }
                        nbuf += np;
                        __syncwarp();
                        if (cand) ++cur;
                    }
                }
            }
        }
    }
    flush(sm, nbuf, ci, sid, list, lane, kp.max_entries);
}

constexpr int PRUNE_WARPS = 8;

__global__ void __launch_bounds__(PRUNE_WARPS * 32)
k_prune(const SysDev* __restrict__ sys, ListDev list, KParams kp) {
    const int lane = threadIdx.x & 31;
    const int nitems = min(list.counters[CNT_ITEMS], list.item_cap);
    const float rl2 = kp.rl2_prune;
    for (int it = blockIdx.x * PRUNE_WARPS + (threadIdx.x >> 5); it < nitems;
         it += gridDim.x * PRUNE_WARPS) {
        int4 item = list.items[it];
        const SysDev& d = sys[item.w >> 5];
        int sh = item.w & 31;
        float Sx = (sh / 9 - 1) * d.L[0], Sy = ((sh / 3) % 3 - 1) * d.L[1], Sz = (sh % 3 - 1) * d.L[2];
        float3 xi[CL];
#pragma unroll
        for (int k = 0; k < CL; ++k) {
            float4 v = d.xq_s[item.x * CL + k];
            xi[k] = make_float3(v.x + Sx, v.y + Sy, v.z + Sz);
        }
        int write = item.y;
        for (int base = item.y; base < item.z; base += 32) {
            int e = base + lane;
            bool keep = false;
            int cjv = 0;
            unsigned long long m = 0;
            if (e < item.z) {
                cjv = list.cj[e];
                m = list.mask[e];
                for (int jj = 0; jj < CL && !keep; ++jj) {
                    float4 xj = d.xq_s[cjv * CL + jj];
#pragma unroll
                    for (int ii = 0; ii < CL; ++ii) {
                        float dx = xi[ii].x - xj.x, dy = xi[ii].y - xj.y, dz = xi[ii].z - xj.z;
                        float r2 = dx * dx + dy * dy + dz * dz;
                        bool bit = (m >> rot_bit(ii, jj)) & 1ull;
                        keep = keep || (bit && r2 < rl2);
                    }
                }
            }
            unsigned bal = __ballot_sync(FULL, keep);
            if (keep) {
                int idx = write + __popc(bal & ((1u << lane) - 1u));
                list.cj[idx] = cjv;
                list.mask[idx] = m;
            }
            write += __popc(bal);
        }
        if (lane == 0) {
            list.items[it].z = write;
            atomicAdd(list.counters + CNT_PRUNED, write - item.y);
        }
    }
}

}  // namespace

cudaError_t launch_search(const PlanLaunch& p, cudaStream_t st) {
    if (p.tot_clcap <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((p.tot_clcap + SEARCH_WARPS - 1) / SEARCH_WARPS);
    k_search<<<blocks, SEARCH_WARPS * 32, 0, st>>>(p.d_sys, p.d_cl_off, p.nsys, p.tot_clcap, p.list, p.kp);
    return cudaGetLastError();
}

cudaError_t launch_prune(const PlanLaunch& p, cudaStream_t st) {
    unsigned blocks = (unsigned)(p.num_sms * 8);
    k_prune<<<blocks, PRUNE_WARPS * 32, 0, st>>>(p.d_sys, p.list, p.kp);
    return cudaGetLastError();
}

}  // namespace nbgb
