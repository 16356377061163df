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
#include "nb_pair2.cuh"

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

// bits of pairs with j < nj (all i), and with i < ni (all j)
__device__ unsigned long long col_mask(int nj) {
    unsigned long long m = 0;
    for (int i = 0; i < CL; ++i)
        for (int j = 0; j < nj; ++j) m |= 1ull << rot_bit(i, j);
    return m;
}
__device__ __forceinline__ unsigned long long row_mask(int ni) {
    return ni >= CL ? ~0ull : ((1ull << (8 * ni)) - 1ull);
}

constexpr int MAX_RUNS = 32;

// Entries of cluster pairs whose bounding boxes lie closer than the list
// radius minus this margin (nm) are kept without testing their atom pairs:
// with clusters about 0.4 nm across, such a pair practically always has an
// atom pair inside the radius, and an entry kept without one only adds
// masked-out work.  The others carry PRUNE_CHECK in their cluster index
// until the prune has tested them.
constexpr float PRUNE_SURE_MARGIN = 0.3f;
constexpr int PRUNE_CHECK = 1 << 30;

struct SearchWarpSmem {
    int cj[SEARCH_BUF];
    unsigned long long mask[SEARCH_BUF];
    int run_start[MAX_RUNS];
    int run_shift[MAX_RUNS];
    int ex_slot[EXCL_BUF];
    unsigned char ex_i[EXCL_BUF];
    int n_ex;
};

__device__ __forceinline__ float gap(float alo, float ahi, float blo, float bhi) {
    return fmaxf(0.f, fmaxf(blo - ahi, alo - bhi));
}

// Partition point of a column's clusters [lo, hi): with TOP, the first
// cluster whose top z is >= z; otherwise the first whose bottom z is > z.
// The clusters of a column are z-sorted, so both keys ascend.  The guess
// (the column's atoms spread evenly over the box height) is usually within a
// cluster or two of the answer, so the keys of the PROBE clusters around it
// are loaded at once, independent loads in one round trip; an answer outside
// that window is found by bisecting the rest.
constexpr int PROBE = 6;  // clusters guess - 3 .. guess + 2

template <bool TOP>
__device__ __forceinline__ int window_bound(const float4* __restrict__ bb, int lo, int hi, float z, int guess) {
    auto before = [&](int m) {  // cluster m lies before the partition point
        return TOP ? bb[2 * m + 1].z < z : bb[2 * m].z <= z;
    };
    const int p0 = min(max(guess - PROBE / 2, lo), hi);  // first probed cluster
    bool bf[PROBE];
#pragma unroll
    for (int k = 0; k < PROBE; ++k) bf[k] = p0 + k < hi ? before(p0 + k) : false;
    if (p0 > lo && !bf[0]) {
        // the answer lies in [lo, p0]
        hi = p0;
    } else {
        int k = 0;
#pragma unroll
        for (int q = 0; q < PROBE; ++q) k += bf[q] ? 1 : 0;  // the keys ascend: bf is true, then false
        if (k < PROBE || p0 + PROBE >= hi) return min(p0 + k, hi);
        lo = p0 + PROBE;  // the answer lies in [p0 + PROBE, hi]
    }
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (before(m)) lo = m + 1; else hi = m;
    }
    return lo;
}

// Write the buffered entries as work items: one per run of equal shift
// (runs are recorded while appending), split into pieces of at most
// max_entries entries.
__device__ void flush(SearchWarpSmem& sm, int nbuf, int nruns, int ci, int sid, const ListDev& list,
                      int lane, int max_entries) {
    if (nbuf == 0) return;
    int nch = 0, rs = 0, re = 0;
    if (lane < nruns) {
        rs = sm.run_start[lane];
        re = lane + 1 < nruns ? sm.run_start[lane + 1] : nbuf;
        nch = (re - rs + max_entries - 1) / max_entries;
    }
    int incl = nch;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int v = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += v;
    }
    const int nitems = __shfl_sync(FULL, incl, 31);
    int ibase = 0, ebase = 0;
    if (lane == 0) {
        ibase = atomicAdd(list.counters + CNT_ITEMS, nitems);
        ebase = atomicAdd(list.counters + CNT_ENTRIES, nbuf);
    }
    ibase = __shfl_sync(FULL, ibase, 0);
    ebase = __shfl_sync(FULL, ebase, 0);
    const bool ok_e = (long long)ebase + nbuf <= list.entry_cap;
    const bool ok_i = (long long)ibase + nitems <= list.item_cap;  // only reported
    if (lane == 0 && !ok_e) atomicOr(list.counters + CNT_OVERFLOW, 2);
    if (lane == 0 && !ok_i) atomicOr(list.counters + CNT_OVERFLOW, 1);
    if (ok_e) {
        for (int k = lane; k < nbuf; k += 32) {
            list.cj[ebase + k] = sm.cj[k];
            list.mask[ebase + k] = sm.mask[k];
        }
    }
    if (lane < nruns) {
        // Every reserved item slot below the capacity is written, so that the
        // item range the kernels read (up to min(count, capacity)) never holds
        // stale data: a real item if this flush's entries fit, otherwise an
        // empty one.  Slots at or beyond the capacity are not written.
        const int w = (sid << 5) | sm.run_shift[lane];
        int idx = ibase + incl - nch;
        for (int a = rs; a < re; a += max_entries, ++idx) {
            if (idx >= list.item_cap) break;
            const int b = min(re, a + max_entries);
            list.items[idx] = ok_e ? make_int4(ci, ebase + a, ebase + b, w) : make_int4(ci, 0, 0, w);
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(SEARCH_WARPS * 32, 7)
k_search(const SysDev* __restrict__ sys, const int* __restrict__ cl_off, int nsys, int tot_clcap,
         ListDev list, KParams kp) {
    pdl_wait();
    pdl_trigger();
    __shared__ SearchWarpSmem s_w[SEARCH_WARPS];
    __shared__ unsigned long long s_colmask[CL + 1];
    __shared__ unsigned long long s_diag;
    if (threadIdx.x <= CL) s_colmask[threadIdx.x] = col_mask(threadIdx.x);
    if (threadIdx.x == 32) s_diag = diag_mask();
    __syncthreads();
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
    const unsigned long long rmask_i = row_mask(nri);
    const float rl = d.rl_search;
    const float rl2 = rl * rl;
    const float izl = 1.f / d.L[2];
    const float rbb = fmaxf(0.f, rl - PRUNE_SURE_MARGIN);
    const float rbb2 = rbb * rbb;
    const float eps = 1e-5f * fmaxf(1.f, fmaxf(d.L[0], fmaxf(d.L[1], d.L[2])));

    // exclusion partners (sorted slots) of this cluster's atoms, and a
    // 64-bit filter of their clusters for a quick test of each candidate
    if (lane == 0) sm.n_ex = 0;
    __syncwarp();
    unsigned long long xfilter = 0;
    if (d.excl_index != nullptr && lane < nri) {
        int a = d.perm[ci * CL + lane];
        for (int e = d.excl_index[a]; e < d.excl_index[a + 1]; ++e) {
            int p = d.iperm[d.excl_atoms[e]];
            xfilter |= 1ull << ((p >> 3) & 63);
            int k = atomicAdd(&sm.n_ex, 1);
            if (k < EXCL_BUF) {
                sm.ex_slot[k] = p;
                sm.ex_i[k] = (unsigned char)lane;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) xfilter |= __shfl_xor_sync(FULL, xfilter, off);
    __syncwarp();
    const int n_ex = min(sm.n_ex, EXCL_BUF);
    const bool ex_overflow = sm.n_ex > EXCL_BUF;

    int nbuf = 0, nruns = 0;
    // images of the i-cluster: S = sx a + sy b + sz c; an image is visited when
    // its bounding box comes within the list radius of the cell [0, ax) x
    // [0, by) x [0, cz), which holds every atom (the box restrictions keep all
    // such images within |s| <= 1)
    // (z first: the gap of each coordinate is known once its shift terms are)
    const float rle2 = (rl + eps) * (rl + eps);
    for (int sz = -1; sz <= 1; ++sz) {
        const float Sz = sz * d.L[2];
        const float lz = lo_i.z + Sz, hz = hi_i.z + Sz;
        const float gz = gap(lz, hz, 0.f, d.L[2]);
        if (gz * gz >= rle2) continue;
        for (int sy = -1; sy <= 1; ++sy) {
            const float Sy = fmaf((float)sz, d.T[2], sy * d.L[1]);
            const float ly = lo_i.y + Sy, hy = hi_i.y + Sy;
            const float gy = gap(ly, hy, 0.f, d.L[1]);
            if (gy * gy + gz * gz >= rle2) continue;
            for (int sx = -1; sx <= 1; ++sx) {
                const float Sx = fmaf((float)sz, d.T[1], fmaf((float)sy, d.T[0], sx * d.L[0]));
                const float lx = lo_i.x + Sx, hx = hi_i.x + Sx;
                const float gx = gap(lx, hx, 0.f, d.L[0]);
                if (gx * gx + gy * gy + gz * gz >= rle2) continue;
                const int shift = shift_index(sx, sy, sz);
                const int cx0 = max(0, (int)floorf((lx - rl) * d.icw[0]) - 1);
                const int cx1 = min(d.ncx - 1, (int)floorf((hx + rl) * d.icw[0]) + 1);
                const int cy0 = max(0, (int)floorf((ly - rl) * d.icw[1]) - 1);
                const int cy1 = min(d.ncy - 1, (int)floorf((hy + rl) * d.icw[1]) + 1);
                if (cx0 > cx1 || cy0 > cy1) continue;
                const int nyc = cy1 - cy0 + 1;
                const int ncand = (cx1 - cx0 + 1) * nyc;
                const float zmin = lz - rl, zmax = hz + rl;
                bool run_open = false;
                for (int cbase = 0; cbase < ncand; cbase += 32) {
                    // each lane: one candidate column, its z-window of clusters
                    const int k = cbase + lane;
                    int c0 = 0, cnt = 0;
                    if (k < ncand) {
                        const int cx = cx0 + k / nyc, cy = cy0 + k % nyc;
                        const float fx0 = cx * d.cw[0] - eps, fx1 = (cx + 1) * d.cw[0] + eps;
                        const float fy0 = cy * d.cw[1] - eps, fy1 = (cy + 1) * d.cw[1] + eps;
                        const float gx = gap(lx, hx, fx0, fx1), gy = gap(ly, hy, fy0, fy1);
                        const int col = cx * d.ncy + cy;
                        // the half list keeps cur > ci (cur == ci only for the
                        // zero and "positive" shifts): columns numbered wholly
                        // below ci hold no candidate
                        const int lo_c = shift >= SHIFT_ZERO ? ci : ci + 1;
                        const int b0 = d.col_cl0[col + 1];
                        if (gx * gx + gy * gy < rl2 && b0 > lo_c) {
                            const int a0 = d.col_cl0[col];
                            const float cl_per_z = (float)(b0 - a0) * izl;
                            // first cluster with top >= zmin, and first with
                            // bottom > zmax (tops and bottoms ascend along the
                            // column)
                            // (independent of each other: clusters before a
                            // have bottom <= top < zmin <= zmax)
                            const int a = max(lo_c, window_bound<true>(d.bb, a0, b0, zmin, a0 + (int)(zmin * cl_per_z)));
                            const int u = window_bound<false>(d.bb, a0, b0, zmax, a0 + (int)(zmax * cl_per_z));
                            c0 = a;
                            cnt = max(0, u - a);
                        }
                    }
                    int incl = cnt;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int vv = __shfl_up_sync(FULL, incl, off);
                        if (lane >= off) incl += vv;
                    }
                    const int total = __shfl_sync(FULL, incl, 31);
                    // lanes stride over the flattened candidates of the 32 columns
                    for (int t0 = 0; t0 < total; t0 += 32) {
                        const int t = t0 + lane;
                        // owner lane: first lane whose inclusive count exceeds t
                        int lo = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const int probe = __shfl_sync(FULL, incl, lo + step - 1);
                            if (probe <= t) lo += step;
                        }
                        const int own_incl = __shfl_sync(FULL, incl, lo);
                        const int own_cnt = __shfl_sync(FULL, cnt, lo);
                        const int own_c0 = __shfl_sync(FULL, c0, lo);
                        const int cur = own_c0 + t - (own_incl - own_cnt);
                        bool pass = false;
                        float g2 = 0.f;
                        float4 lj = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (t < total) {
                            lj = d.bb[2 * cur];
                            const float4 hj = d.bb[2 * cur + 1];
                            const float gx = gap(lx, hx, lj.x, hj.x);
                            const float gy = gap(ly, hy, lj.y, hj.y);
                            const float gz = gap(lz, hz, lj.z, hj.z);
                            g2 = gx * gx + gy * gy + gz * gz;
                            pass = g2 < rl2 && (cur > ci || (cur == ci && shift >= SHIFT_ZERO));
                        }
                        const unsigned bal = __ballot_sync(FULL, pass);
                        const int np = __popc(bal);
                        if (np == 0) continue;
                        if (nbuf + np > SEARCH_BUF || (!run_open && nruns == MAX_RUNS)) {
                            flush(sm, nbuf, nruns, ci, sid, list, lane, kp.max_entries);
                            nbuf = 0;
                            nruns = 0;
                            run_open = false;
                        }
                        if (!run_open) {
                            if (lane == 0) {
                                sm.run_start[nruns] = nbuf;
                                sm.run_shift[nruns] = shift;
                            }
                            ++nruns;
                            run_open = true;
                        }
                        if (pass) {
                            unsigned long long m = ~0ull;
                            if (cur == ci && shift == SHIFT_ZERO) m = s_diag;
                            const int nrj = (int)lj.w;
                            m &= rmask_i & s_colmask[nrj];
                            if ((xfilter >> (cur & 63)) & 1ull) {
                                if (!ex_overflow) {
                                    for (int q = 0; q < n_ex; ++q) {
                                        const int p = sm.ex_slot[q];
                                        if ((p >> 3) == cur) m &= ~(1ull << rot_bit(sm.ex_i[q], p & 7));
                                    }
                                } else {
                                    for (int ii = 0; ii < nri; ++ii) {
                                        const int a = d.perm[ci * CL + ii];
                                        for (int e = d.excl_index[a]; e < d.excl_index[a + 1]; ++e) {
                                            const int p = d.iperm[d.excl_atoms[e]];
                                            if ((p >> 3) == cur) m &= ~(1ull << rot_bit(ii, p & 7));
                                        }
                                    }
                                }
                            }
                            const int idx = nbuf + __popc(bal & ((1u << lane) - 1u));
                            // entries whose boxes are not clearly inside the
                            // list radius get their atom pairs tested by the prune
                            sm.cj[idx] = g2 < rbb2 ? cur : (cur | PRUNE_CHECK);
                            sm.mask[idx] = m;
                        }
                        nbuf += np;
                        __syncwarp();
                    }
                }
            }
        }
    }
    flush(sm, nbuf, nruns, ci, sid, list, lane, kp.max_entries);
}

// ------------------------------------------- search, one thread per cluster
//
// For systems with many clusters the search takes one thread per i-cluster.
// It tests the same candidates with the same rule as k_search, but a thread
// walks its cluster's images, columns and z-windows on its own, with no
// coordination between lanes, and writes into a range of the list reserved
// for its cluster, with no atomics.  Three launches:
//   k_tsearch<false>  count, per cluster, the entries that pass the box test
//                     and the work items they make (one per run of equal
//                     shift, split into pieces of at most max_entries);
//                     exclusive scan of both over the block
//   k_tsearch_scan    exclusive scan of the block totals (one block), the
//                     list's entry and item counts, capacity check
//   k_tsearch<true>   the same walk again, writing each entry (mask, and
//                     the PRUNE_CHECK mark of entries whose boxes are not
//                     clearly inside the radius) and each item at the
//                     cluster's offsets; the prune follows as for k_search.
// The per-cluster offsets live in the grid put's sort-key buffer, which is
// not used again until the next grid put: cluster c's first key slot holds
// its (entries, items) offsets packed into 64 bits, and the second slot of a
// block's first cluster holds the block's totals, then its offsets.
constexpr int TS_BLOCK = 128;
constexpr int TS_EXK = 16;  // exclusion partners of a cluster kept in registers

__device__ __forceinline__ unsigned long long* ts_slot(const SysDev& d, int c, int k) {
    return d.keys + (size_t)c * CL + k;
}

// Walk one i-cluster's candidates.  Counting: returns the entry and item
// counts.  Writing: writes the entries from base_e and the items from
// base_i.
template <bool WRITE>
__device__ void ts_cluster(const SysDev& d, int sid, int ci, int max_entries, const ListDev& list,
                           const unsigned long long* s_colmask, unsigned long long s_diag, int base_e, int base_i,
                           int& n_e, int& n_i) {
    const float4 lo_i = d.bb[2 * ci];
    const float4 hi_i = d.bb[2 * ci + 1];
    const int nri = (int)lo_i.w;
    const unsigned long long rmask_i = row_mask(nri);
    const float rl = d.rl_search;
    const float rl2 = rl * rl;
    const float izl = 1.f / d.L[2];
    const float rbb = fmaxf(0.f, rl - PRUNE_SURE_MARGIN);
    const float rbb2 = rbb * rbb;
    const float eps = 1e-5f * fmaxf(1.f, fmaxf(d.L[0], fmaxf(d.L[1], d.L[2])));

    // exclusion partners (sorted slot << 3 | i-slot) of the cluster's atoms
    int exs[TS_EXK];
    int n_ex = 0;
    unsigned long long xfilter = 0;
    if (WRITE && d.excl_index != nullptr) {
        for (int ii = 0; ii < nri; ++ii) {
            const int a = d.perm[ci * CL + ii];
            for (int e = d.excl_index[a]; e < d.excl_index[a + 1]; ++e) {
                const int p = d.iperm[d.excl_atoms[e]];
                xfilter |= 1ull << ((p >> 3) & 63);
                if (n_ex < TS_EXK) exs[n_ex] = (p << 3) | ii;
                ++n_ex;
            }
        }
    }

    int w_e = 0, w_i = 0;
    // images of the i-cluster (as in k_search; z first)
    const float rle2 = (rl + eps) * (rl + eps);
    for (int sz = -1; sz <= 1; ++sz) {
        const float Sz = sz * d.L[2];
        const float lz = lo_i.z + Sz, hz = hi_i.z + Sz;
        const float gz = gap(lz, hz, 0.f, d.L[2]);
        if (gz * gz >= rle2) continue;
        for (int sy = -1; sy <= 1; ++sy) {
            const float Sy = fmaf((float)sz, d.T[2], sy * d.L[1]);
            const float ly = lo_i.y + Sy, hy = hi_i.y + Sy;
            const float gy = gap(ly, hy, 0.f, d.L[1]);
            if (gy * gy + gz * gz >= rle2) continue;
            for (int sx = -1; sx <= 1; ++sx) {
                const float Sx = fmaf((float)sz, d.T[1], fmaf((float)sy, d.T[0], sx * d.L[0]));
                const float lx = lo_i.x + Sx, hx = hi_i.x + Sx;
                const float gx = gap(lx, hx, 0.f, d.L[0]);
                if (gx * gx + gy * gy + gz * gz >= rle2) continue;
                const int shift = shift_index(sx, sy, sz);
                const int cx0 = max(0, (int)floorf((lx - rl) * d.icw[0]) - 1);
                const int cx1 = min(d.ncx - 1, (int)floorf((hx + rl) * d.icw[0]) + 1);
                const int cy0 = max(0, (int)floorf((ly - rl) * d.icw[1]) - 1);
                const int cy1 = min(d.ncy - 1, (int)floorf((hy + rl) * d.icw[1]) + 1);
                const float zmin = lz - rl, zmax = hz + rl;
                const int run0 = w_e;
                for (int cx = cx0; cx <= cx1; ++cx) {
                    const float fx0 = cx * d.cw[0] - eps, fx1 = (cx + 1) * d.cw[0] + eps;
                    const float gcx = gap(lx, hx, fx0, fx1);
                    if (gcx * gcx >= rl2) continue;
                    for (int cy = cy0; cy <= cy1; ++cy) {
                        const float fy0 = cy * d.cw[1] - eps, fy1 = (cy + 1) * d.cw[1] + eps;
                        const float gcy = gap(ly, hy, fy0, fy1);
                        if (gcx * gcx + gcy * gcy >= rl2) continue;
                        const int col = cx * d.ncy + cy;
                        const int a0 = d.col_cl0[col], b0 = d.col_cl0[col + 1];
                        // the half list keeps cur > ci (cur == ci only for the zero
                        // and "positive" shifts): columns numbered wholly below ci
                        // hold no candidate
                        const int lo_c = shift >= SHIFT_ZERO ? ci : ci + 1;
                        if (b0 <= lo_c) continue;
                        const float cl_per_z = (float)(b0 - a0) * izl;
                        const int a = max(lo_c, window_bound<true>(d.bb, a0, b0, zmin, a0 + (int)(zmin * cl_per_z)));
                        const int u = window_bound<false>(d.bb, a0, b0, zmax, a0 + (int)(zmax * cl_per_z));
                        // each candidate's box is loaded one step ahead
                        float4 ln = make_float4(0.f, 0.f, 0.f, 0.f), hn = ln;
                        if (a < u) {
                            ln = d.bb[2 * a];
                            hn = d.bb[2 * a + 1];
                        }
                        for (int cur = a; cur < u; ++cur) {
                            const float4 lj = ln;
                            const float4 hj = hn;
                            if (cur + 1 < u) {
                                ln = d.bb[2 * cur + 2];
                                hn = d.bb[2 * cur + 3];
                            }
                            const float gjx = gap(lx, hx, lj.x, hj.x);
                            const float gjy = gap(ly, hy, lj.y, hj.y);
                            const float gjz = gap(lz, hz, lj.z, hj.z);
                            const float g2 = gjx * gjx + gjy * gjy + gjz * gjz;
                            if (!(g2 < rl2)) continue;
                            if (WRITE) {
                                unsigned long long m = (cur == ci && shift == SHIFT_ZERO) ? s_diag : ~0ull;
                                m &= rmask_i & s_colmask[(int)lj.w];
                                if ((xfilter >> (cur & 63)) & 1ull) {
                                    if (n_ex <= TS_EXK) {
                                        for (int q = 0; q < n_ex; ++q) {
                                            const int p = exs[q] >> 3;
                                            if ((p >> 3) == cur) m &= ~(1ull << rot_bit(exs[q] & 7, p & 7));
                                        }
                                    } else {
                                        for (int ii = 0; ii < nri; ++ii) {
                                            const int aa = d.perm[ci * CL + ii];
                                            for (int e = d.excl_index[aa]; e < d.excl_index[aa + 1]; ++e) {
                                                const int p = d.iperm[d.excl_atoms[e]];
                                                if ((p >> 3) == cur) m &= ~(1ull << rot_bit(ii, p & 7));
                                            }
                                        }
                                    }
                                }
                                list.cj[base_e + w_e] = g2 < rbb2 ? cur : (cur | PRUNE_CHECK);
                                list.mask[base_e + w_e] = m;
                            }
                            ++w_e;
                        }
                    }
                }
                // the run of this shift as items of at most max_entries entries
                const int len = w_e - run0;
                if (len > 0) {
                    if (WRITE) {
                        const int w = (sid << 5) | shift;
                        for (int x = 0; x < len; x += max_entries) {
                            const int y = min(len, x + max_entries);
                            list.items[base_i + w_i] = make_int4(ci, base_e + run0 + x, base_e + run0 + y, w);
                            ++w_i;
                        }
                    } else {
                        w_i += (len + max_entries - 1) / max_entries;
                    }
                }
            }
        }
    }
    n_e = w_e;
    n_i = w_i;
}

// Exclusive scan of packed (entries << 32 | items) counts over a block of
// TS_BLOCK threads; returns the thread's offset and sets *total.
__device__ __forceinline__ unsigned long long ts_block_scan(unsigned long long v, unsigned long long* s_warp,
                                                            unsigned long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int k = 0; k < TS_BLOCK / 32; ++k) {
        if (k < w) before += s_warp[k];
        all += s_warp[k];
    }
    *total = all;
    return before + incl - v;
}

template <bool WRITE>
__global__ void __launch_bounds__(TS_BLOCK)
k_tsearch(const SysDev* __restrict__ sys, const int* __restrict__ cl_off, int nsys, int tot_clcap, ListDev list,
          KParams kp) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_colmask[CL + 1];
    __shared__ unsigned long long s_diag;
    __shared__ unsigned long long s_warp[TS_BLOCK / 32];
    if (threadIdx.x <= CL) s_colmask[threadIdx.x] = col_mask(threadIdx.x);
    if (threadIdx.x == 32) s_diag = diag_mask();
    __syncthreads();
    const int gc = blockIdx.x * TS_BLOCK + threadIdx.x;
    int sid = 0, ci = 0;
    bool real = false;
    if (gc < tot_clcap) {
        sid = find_sys(cl_off, nsys, gc);
        ci = gc - cl_off[sid];
        real = ci < sys[sid].col_cl0[sys[sid].ncol];
    }
    const SysDev& d = sys[sid];
    if (!WRITE) {
        int n_e = 0, n_i = 0;
        if (real) ts_cluster<false>(d, sid, ci, kp.max_entries, list, s_colmask, s_diag, 0, 0, n_e, n_i);
        unsigned long long total = 0;
        const unsigned long long off =
            ts_block_scan(((unsigned long long)n_e << 32) | (unsigned)n_i, s_warp, &total);
        if (gc < tot_clcap) *ts_slot(d, ci, 0) = off;
        if (threadIdx.x == 0) *ts_slot(d, ci, 1) = total;  // the block's first cluster
        return;
    }
    if (gc >= tot_clcap) return;
    // offsets: the block's (in its first cluster) plus the cluster's own
    const int g0 = blockIdx.x * TS_BLOCK;
    const int s0 = find_sys(cl_off, nsys, g0);
    const unsigned long long boff = *ts_slot(sys[s0], g0 - cl_off[s0], 1);
    const unsigned long long off = boff + *ts_slot(d, ci, 0);
    const int base_e = (int)(off >> 32), base_i = (int)(off & 0xffffffffull);
    if (list.counters[CNT_OVERFLOW] & 3) {
        // the list does not fit: write empty items into the reserved item
        // slots below the capacity, so that no kernel reads stale items
        if (!real) return;
        int n_e = 0, n_i = 0;
        ts_cluster<false>(d, sid, ci, kp.max_entries, list, s_colmask, s_diag, 0, 0, n_e, n_i);
        for (int k = 0; k < n_i && base_i + k < list.item_cap; ++k)
            list.items[base_i + k] = make_int4(ci, 0, 0, (sid << 5) | SHIFT_ZERO);
        return;
    }
    if (!real) return;
    int n_e = 0, n_i = 0;
    ts_cluster<true>(d, sid, ci, kp.max_entries, list, s_colmask, s_diag, base_e, base_i, n_e, n_i);
}

// One block: exclusive scan of the block totals of k_tsearch<false>, in
// place; the list's entry and item counts; overflow bits if they exceed the
// capacities (the write pass then writes no entries).
__global__ void __launch_bounds__(1024)
k_tsearch_scan(const SysDev* __restrict__ sys, const int* __restrict__ cl_off, int nsys, int tot_clcap,
               ListDev list) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nblk = (tot_clcap + TS_BLOCK - 1) / TS_BLOCK;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        const int b = base + threadIdx.x;
        unsigned long long v = 0;
        unsigned long long* slot = nullptr;
        if (b < nblk) {
            const int g0 = b * TS_BLOCK;
            const int s0 = find_sys(cl_off, nsys, g0);
            slot = ts_slot(sys[s0], g0 - cl_off[s0], 1);
            v = *slot;
        }
        unsigned long long incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long t = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        unsigned long long before = s_carry;
        for (int k = 0; k < w; ++k) before += s_warp[k];
        if (slot) *slot = before + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long tot = s_carry;
        const long long n_e = (long long)(tot >> 32), n_i = (long long)(tot & 0xffffffffull);
        list.counters[CNT_ENTRIES] = (int)min(n_e, (long long)0x7fffffff);
        list.counters[CNT_ITEMS] = (int)min(n_i, (long long)0x7fffffff);
        int ov = 0;
        if (n_i > list.item_cap) ov |= 1;
        if (n_e > list.entry_cap) ov |= 2;
        if (ov) atomicOr(list.counters + CNT_OVERFLOW, ov);
    }
}

constexpr int PRUNE_WARPS = 8;
// checks in flight per lane (16 per round of independent j-atom loads; eight
// per lane, one round per chunk, needs more registers and ran slower)
constexpr int PRUNE_U = 4;

// Prune (Section 3.3): drop the entries of which no atom pair whose mask bit
// is set lies within the list radius.  A warp takes one work item at a time.
// Per chunk of 32 entries, lane k loads entry k's j-cluster index and mask
// (coalesced).  Entries the search marked as certain are kept as they are;
// the others are tested 16 at a time, lane = 8 g + j holding j-atom j of four
// of them (four independent coalesced loads in flight) against the eight
// i-atoms of the item, which every lane keeps in registers.  Kept entries are
// compacted in place, in order, without the mark; a write never passes the
// entries still to be read.
//
// The same kernel prunes out of place (dst != src, the inner list of
// nb_pairlist_prune): it then tests every entry against the radius rl2_inner
// and writes the kept entries to the same positions of dst, with dst's items,
// counters and order.
__global__ void __launch_bounds__(PRUNE_WARPS * 32, 3)
k_prune(const SysDev* __restrict__ sys, ListDev src, ListDev dst, KParams kp, float rl2_inner) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned char s_rank[PRUNE_WARPS][32];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int jj = lane & 7;
    const int g = lane >> 3;
    const bool inner = rl2_inner > 0.f;
    const int nitems = min(src.counters[CNT_ITEMS], src.item_cap);
    const bool ordered = nitems <= kp.lpt_max_items;
    if (inner && blockIdx.x == 0 && threadIdx.x == 0) dst.counters[CNT_ITEMS] = nitems;
    for (int it = blockIdx.x * PRUNE_WARPS + w; it < nitems; it += gridDim.x * PRUNE_WARPS) {
        const int4 item = src.items[it];
        if (item.y >= item.z) {
            if (inner && (threadIdx.x & 31) == 0) dst.items[it] = item;
            continue;
        }
        const SysDev& d = sys[item.w >> 5];
        const float rl2 = inner ? rl2_inner : d.rl2_prune;
        const int sh = item.w & 31;
        const float3 S = shift_vec(sh, d.L, d.T);
        const float Sx = S.x, Sy = S.y, Sz = S.z;
        // the i-atoms in pairs (2k, 2k+1), for the paired float32 arithmetic
        float2 xi[CL / 2], yi[CL / 2], zi[CL / 2];
#pragma unroll
        for (int k = 0; k < CL / 2; ++k) {
            const float4 v0 = d.xq_s[item.x * CL + 2 * k], v1 = d.xq_s[item.x * CL + 2 * k + 1];
            xi[k] = make_float2(v0.x + Sx, v1.x + Sx);
            yi[k] = make_float2(v0.y + Sy, v1.y + Sy);
            zi[k] = make_float2(v0.z + Sz, v1.z + Sz);
        }
        int write = item.y;
        // each chunk's entries are loaded while the previous chunk is tested
        int c_next = 0;
        unsigned long long m_next = 0ull;
        if (lane < item.z - item.y) {
            c_next = src.cj[item.y + lane];
            m_next = src.mask[item.y + lane];
        }
        for (int base = item.y; base < item.z; base += 32) {
            const int n = min(32, item.z - base);
            int cjv = 0;
            unsigned long long m = 0ull;
            bool chk = false;
            if (lane < n) {
                const int c = c_next;
                chk = inner || (c & PRUNE_CHECK) != 0;
                cjv = c & ~PRUNE_CHECK;
                m = m_next;
            }
            if (base + 32 + lane < item.z) {
                c_next = src.cj[base + 32 + lane];
                m_next = src.mask[base + 32 + lane];
            }
            const unsigned chk_bal = __ballot_sync(FULL, chk);
            unsigned keep = __ballot_sync(FULL, lane < n && !chk);  // bit k: entry base + k is kept
            const int nchk = __popc(chk_bal);
            if (chk) s_rank[w][__popc(chk_bal & ((1u << lane) - 1u))] = (unsigned char)lane;
            __syncwarp();
            for (int q0 = 0; q0 < nchk; q0 += 4 * PRUNE_U) {
                float4 xj[PRUNE_U];
                unsigned long long mq[PRUNE_U];
#pragma unroll
                for (int u = 0; u < PRUNE_U; ++u) {
                    const int k = q0 + 4 * u + g;
                    const int src = k < nchk ? s_rank[w][k] : 0;
                    const int cjk = __shfl_sync(FULL, cjv, src);
                    mq[u] = __shfl_sync(FULL, m, src);
                    xj[u] = k < nchk ? d.xq_s[cjk * CL + jj] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < PRUNE_U; ++u) {
                    // bit ii: i-atom ii lies within the list radius of this j-atom
                    // (two i-atoms per paired instruction)
                    unsigned nb8 = 0;
                    const float2 jx = dup2(xj[u].x), jy = dup2(xj[u].y), jz = dup2(xj[u].z);
#pragma unroll
                    for (int k = 0; k < CL / 2; ++k) {
                        const float2 dx = sub2(xi[k], jx), dy = sub2(yi[k], jy), dz = sub2(zi[k], jz);
                        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                        nb8 |= (r2.x < rl2 ? 1u : 0u) << (2 * k);
                        nb8 |= (r2.y < rl2 ? 1u : 0u) << (2 * k + 1);
                    }
                    // the mask column of j-slot jj (bit ii = pair (ii, jj)), only
                    // when one of the four entries has a partial mask
                    if (__any_sync(FULL, mq[u] != ~0ull)) {
                        const unsigned lo = (unsigned)mq[u], hi = (unsigned)(mq[u] >> 32);
                        unsigned col = 0;
#pragma unroll
                        for (int ii = 0; ii < CL; ++ii)
                            col |= (((ii < 4 ? lo : hi) >> (8 * (ii & 3) + (ii ^ jj))) & 1u) << ii;
                        nb8 &= col;
                    }
                    const unsigned bal = __ballot_sync(FULL, nb8 != 0u);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = q0 + 4 * u + q;
                        if (k < nchk && ((bal >> (8 * q)) & 0xffu) != 0u) keep |= 1u << s_rank[w][k];
                    }
                }
            }
            __syncwarp();
            if (lane < n && ((keep >> lane) & 1u)) {
                const int idx = write + __popc(keep & ((1u << lane) - 1u));
                dst.cj[idx] = cjv;
                dst.mask[idx] = m;
            }
            write += __popc(keep);
        }
        if (lane == 0) {
            const int len = write - item.y;
            dst.items[it] = make_int4(item.x, item.y, write, item.w);
            atomicAdd(dst.counters + CNT_PRUNED, len);
            if (ordered && len > kp.max_entries / 2)
                dst.order[atomicAdd(dst.counters + CNT_ORD_LONG, 1)] = it;
            else if (ordered && len > 0)
                dst.order[dst.item_cap - 1 - atomicAdd(dst.counters + CNT_ORD_SHORT, 1)] = it;
        }
    }
}

}  // namespace

// Clusters from which the search takes one thread per cluster (about eight
// warps per SM); smaller systems take one warp per cluster.
static bool thread_search(const PlanLaunch& p) {
    if (p.kp.search_mode == 1) return false;
    if (p.kp.search_mode == 2) return true;
    return (long long)p.tot_clcap >= (long long)p.num_sms * 8 * 32;
}

cudaError_t launch_search(const PlanLaunch& p, cudaStream_t st) {
    if (p.tot_clcap <= 0) return cudaSuccess;
    if (thread_search(p)) {
        const unsigned blocks = (unsigned)((p.tot_clcap + TS_BLOCK - 1) / TS_BLOCK);
        cudaError_t e = launch_pdl(k_tsearch<false>, blocks, TS_BLOCK, 0, st, p.d_sys, p.d_cl_off, p.nsys,
                                   p.tot_clcap, p.list, p.kp);
        if (e == cudaSuccess)
            e = launch_pdl(k_tsearch_scan, 1u, 1024, 0, st, p.d_sys, p.d_cl_off, p.nsys, p.tot_clcap, p.list);
        if (e == cudaSuccess)
            e = launch_pdl(k_tsearch<true>, blocks, TS_BLOCK, 0, st, p.d_sys, p.d_cl_off, p.nsys, p.tot_clcap,
                           p.list, p.kp);
        return e;
    }
    unsigned blocks = (unsigned)((p.tot_clcap + SEARCH_WARPS - 1) / SEARCH_WARPS);
    return launch_pdl(k_search, blocks, SEARCH_WARPS * 32, 0, st, p.d_sys, p.d_cl_off, p.nsys, p.tot_clcap, p.list,
                      p.kp);
}

cudaError_t launch_prune(const PlanLaunch& p, cudaStream_t st) {
    unsigned blocks = (unsigned)(p.num_sms * 8);
    return launch_pdl(k_prune, blocks, PRUNE_WARPS * 32, 0, st, p.d_sys, p.list, p.list, p.kp, -1.f);
}

cudaError_t launch_prune_into(const PlanLaunch& p, const ListDev& src, const ListDev& dst, float rl2_inner,
                              cudaStream_t st) {
    unsigned blocks = (unsigned)(p.num_sms * 8);
    return launch_pdl(k_prune, blocks, PRUNE_WARPS * 32, 0, st, p.d_sys, src, dst, p.kp, rl2_inner);
}

}  // namespace nbgb
