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
// The margin for lists of 4-atom j-clusters (ListDev::jgeo): the prune keeps
// both halves of a certain entry, so only the closest pairs of clusters
// skip the per-half test.
constexpr float PRUNE_SURE_MARGIN4 = 0.6f;
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
    const float rbb = fmaxf(0.f, rl - (list.jgeo ? PRUNE_SURE_MARGIN4 : PRUNE_SURE_MARGIN));
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
// For systems with many clusters the search takes one thread per i-cluster,
// in one pass.  It tests the same candidates with the same rule as
// k_search, but a thread walks its cluster's images, columns and z-windows
// on its own, with no coordination between lanes, and writes the entries
// into a slab of `ce` entries reserved for its cluster (cluster gc's
// entries at gc * ce; ce is a multiple of 8).  The work items reference
// ranges of those slabs, so the slabs need no compaction: the gaps between
// clusters are never read.  Entries are collected four at a time and
// written as one 16-byte (cluster indices) and one 32-byte (masks) store.
// The threads of a warp walk the 27 images in step; after each image the
// warp reserves the items of its runs with one atomic add and writes them.
// A cluster with more than ce entries sets the entries' overflow bit and
// reports its count (CNT_NEED, the maximum over clusters); its items are
// clipped to its slab.
constexpr int TS_BLOCK = 128;
constexpr int TS_XS = 16;  // exclusion partner clusters of an i-cluster kept in shared memory

__device__ __forceinline__ void ts_store4(const ListDev& list, long long at, const int (&c)[4],
                                          const unsigned long long (&m)[4]) {
    *reinterpret_cast<int4*>(list.cj + at) = make_int4(c[0], c[1], c[2], c[3]);
    ulonglong4_32a v;
    v.x = m[0];
    v.y = m[1];
    v.z = m[2];
    v.w = m[3];
    *reinterpret_cast<ulonglong4_32a*>(list.mask + at) = v;
}

__global__ void __launch_bounds__(TS_BLOCK)
k_tsearch(const SysDev* __restrict__ sys, const int* __restrict__ cl_off, int nsys, int tot_clcap, int ce,
          ListDev list, KParams kp) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_colmask[CL + 1];
    __shared__ unsigned long long s_diag;
    __shared__ unsigned long long s_xm[TS_XS][TS_BLOCK];
    __shared__ int s_xc[TS_XS][TS_BLOCK];
    if (threadIdx.x <= CL) s_colmask[threadIdx.x] = col_mask(threadIdx.x);
    if (threadIdx.x == 32) s_diag = diag_mask();
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // a warp whose clusters all lie past the end leaves as a whole (the warp
    // collectives below need every lane)
    if (blockIdx.x * TS_BLOCK + (threadIdx.x & ~31) >= tot_clcap) return;
    const int gc = blockIdx.x * TS_BLOCK + threadIdx.x;
    int sid = 0, ci = 0;
    bool real = false;
    if (gc < tot_clcap) {
        sid = find_sys(cl_off, nsys, gc);
        ci = gc - cl_off[sid];
        real = ci < sys[sid].col_cl0[sys[sid].ncol];
    }
    const SysDev& d = sys[sid];
    const int max_entries = kp.max_entries;
    float4 lo_i = make_float4(0.f, 0.f, 0.f, 0.f), hi_i = lo_i;
    if (real) {
        lo_i = d.bb[2 * ci];
        hi_i = d.bb[2 * ci + 1];
    }
    const int nri = (int)lo_i.w;
    const unsigned long long rmask_i = row_mask(nri);
    const float rl = d.rl_search;
    const float rl2 = rl * rl;
    const float izl = 1.f / d.L[2];
    const float rbb = fmaxf(0.f, rl - (list.jgeo ? PRUNE_SURE_MARGIN4 : PRUNE_SURE_MARGIN));
    const float rbb2 = rbb * rbb;
    const float eps = 1e-5f * fmaxf(1.f, fmaxf(d.L[0], fmaxf(d.L[1], d.L[2])));

    // the clusters holding exclusion partners of the cluster's atoms, each
    // with the mask bits of its excluded pairs, in shared memory (TS_XS per
    // thread); a 64-bit filter (bit c mod 64 of every partner cluster c)
    // sends only the candidates that may be partners to the table.  More
    // partner clusters than the table holds take the slow path through the
    // exclusion lists for the candidates that hit the filter.
    int n_xc = 0;
    unsigned long long x_filter = 0ull;
    bool x_slow = false;
    if (real && d.excl_index != nullptr) {
        for (int ii = 0; ii < nri; ++ii) {
            const int a = d.perm[ci * CL + ii];
            for (int e = d.excl_index[a]; e < d.excl_index[a + 1]; ++e) {
                const int p = d.iperm[d.excl_atoms[e]];
                const int c = p >> 3;
                const unsigned long long bit = 1ull << rot_bit(ii, p & 7);
                x_filter |= 1ull << (c & 63);
                int k = 0;
                while (k < n_xc && s_xc[k][threadIdx.x] != c) ++k;
                if (k < n_xc) {
                    s_xm[k][threadIdx.x] |= bit;
                } else if (n_xc < TS_XS) {
                    s_xc[n_xc][threadIdx.x] = c;
                    s_xm[n_xc][threadIdx.x] = bit;
                    ++n_xc;
                } else {
                    x_slow = true;
                }
            }
        }
    }

    const long long ebase = (long long)gc * ce;
    int bc[4] = {0, 0, 0, 0};
    unsigned long long bm[4] = {0ull, 0ull, 0ull, 0ull};
    int w_e = 0;
    const float rle2 = (rl + eps) * (rl + eps);
    // images of the i-cluster (as in k_search; z first); every lane takes
    // all 27 steps (one loop, not unrolled: its body is large)
#pragma unroll 1
    for (int img = 0; img < NSHIFT; ++img) {
        const int sz = img / 9 - 1, sy = (img / 3) % 3 - 1, sx = img % 3 - 1;
        const int run0 = w_e;
        const int shift = shift_index(sx, sy, sz);
        const float Sz = sz * d.L[2];
        const float lz = lo_i.z + Sz, hz = hi_i.z + Sz;
        const float gz = gap(lz, hz, 0.f, d.L[2]);
        const float Sy = fmaf((float)sz, d.T[2], sy * d.L[1]);
        const float ly = lo_i.y + Sy, hy = hi_i.y + Sy;
        const float gy = gap(ly, hy, 0.f, d.L[1]);
        const float Sx = fmaf((float)sz, d.T[1], fmaf((float)sy, d.T[0], sx * d.L[0]));
        const float lx = lo_i.x + Sx, hx = hi_i.x + Sx;
        const float gx = gap(lx, hx, 0.f, d.L[0]);
        if (real && gx * gx + gy * gy + gz * gz < rle2) {
            const int cx0 = max(0, (int)floorf((lx - rl) * d.icw[0]) - 1);
            const int cx1 = min(d.ncx - 1, (int)floorf((hx + rl) * d.icw[0]) + 1);
            const int cy0 = max(0, (int)floorf((ly - rl) * d.icw[1]) - 1);
            const int cy1 = min(d.ncy - 1, (int)floorf((hy + rl) * d.icw[1]) + 1);
            const float zmin = lz - rl, zmax = hz + rl;
            // the half list keeps cur > ci (cur == ci only for the
            // zero and "positive" shifts)
            const int lo_c = shift >= SHIFT_ZERO ? ci : ci + 1;
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
                    // columns numbered wholly below ci hold no candidate
                    if (b0 <= lo_c) continue;
                    const float cl_per_z = (float)(b0 - a0) * izl;
                    const int a =
                        max(lo_c, window_bound<true>(d.bb, a0, b0, zmin, a0 + (int)(zmin * cl_per_z)));
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
                        unsigned long long m = (cur == ci && shift == SHIFT_ZERO) ? s_diag : ~0ull;
                        m &= rmask_i & s_colmask[(int)lj.w];
                        if ((x_filter >> (cur & 63)) & 1ull) {
                            for (int k = 0; k < n_xc; ++k)
                                if (s_xc[k][threadIdx.x] == cur) m &= ~s_xm[k][threadIdx.x];
                        }
                        if (x_slow && ((x_filter >> (cur & 63)) & 1ull)) {
                            for (int ii = 0; ii < nri; ++ii) {
                                const int aa = d.perm[ci * CL + ii];
                                for (int e = d.excl_index[aa]; e < d.excl_index[aa + 1]; ++e) {
                                    const int p = d.iperm[d.excl_atoms[e]];
                                    if ((p >> 3) == cur) m &= ~(1ull << rot_bit(ii, p & 7));
                                }
                            }
                        }
                        // entries whose boxes are not clearly inside the
                        // list radius get their atom pairs tested by the prune
                        const int cv = g2 < rbb2 ? cur : (cur | PRUNE_CHECK);
                        const int q = w_e & 3;
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (k == q) {
                                bc[k] = cv;
                                bm[k] = m;
                            }
                        ++w_e;
                        if (q == 3 && w_e <= ce) ts_store4(list, ebase + w_e - 4, bc, bm);
                    }
                }
            }
        }
        // the run of this image as items of at most max_entries
        // entries, clipped to the slab; one reservation per warp
        const int r0 = min(run0, ce), r1 = min(w_e, ce);
        const int n_it = r1 > r0 ? (r1 - r0 + max_entries - 1) / max_entries : 0;
        int incl = n_it;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += t;
        }
        const int wtot = __shfl_sync(FULL, incl, 31);
        if (wtot > 0) {
            int ib = 0;
            if (lane == 31) {
                ib = atomicAdd(list.counters + CNT_ITEMS, wtot);
                if ((long long)ib + wtot > list.item_cap) atomicOr(list.counters + CNT_OVERFLOW, 1);
            }
            ib = __shfl_sync(FULL, ib, 31) + incl - n_it;
            const int w = (sid << 5) | shift;
            for (int x = r0; x < r1; x += max_entries, ++ib) {
                if (ib >= list.item_cap) break;
                list.items[ib] = make_int4(ci, (int)(ebase + x), (int)(ebase + min(r1, x + max_entries)), w);
            }
        }
    }
    // the last partial group of four (the slab has room: ce is a multiple of 8)
    if ((w_e & 3) != 0 && w_e < ce) ts_store4(list, ebase + (w_e & ~3), bc, bm);
    // the list's entry count, and the largest count of a cluster
    int tot = w_e;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(FULL, tot, off);
    const int mx = __reduce_max_sync(FULL, (unsigned)w_e);
    if (lane == 0) {
        if (tot > 0) atomicAdd(list.counters + CNT_ENTRIES, tot);
        atomicMax(list.counters + CNT_NEED, mx);
        if (mx > ce) atomicOr(list.counters + CNT_OVERFLOW, 2);
    }
}

constexpr int PRUNE_WARPS = 8;
// checks in flight per lane (8 per round of independent j-atom loads).  On
// the 3M-atom box, 2 at three blocks per SM ran faster than 4 at two blocks
// (0.98 vs 1.05 ms) and than 4 at three blocks, which spills.
constexpr int PRUNE_U = 2;

// Prune (Section 3.3): drop the entries of which no atom pair whose mask bit
// is set lies within the list radius.  A warp takes one work item at a time.
// Per chunk of 32 entries, lane k loads entry k's j-atoms' slots and mask
// (coalesced).  Entries the search marked as certain are kept as they are;
// the others are tested 4 * PRUNE_U at a time, lane = 8 g + j holding j-atom j
// of PRUNE_U of them (independent coalesced loads in flight) against the
// eight i-atoms of the item, which every lane keeps in registers.  Kept
// entries are compacted in place, in order, without the mark; a write never
// passes the entries still to be read.
//
// With POUT (a list of the 8 x 4 geometry, ListDev::jgeo) the entries are
// kept per 4-atom half of their j-atoms: a tested entry keeps the halves with
// a pair within the radius, a certain one the halves with an unmasked pair.
// The kept halves are packed two by two into the entries of the item (each
// half's mask bits moved to its new side), and an odd last half is paired
// with itself under a zero mask.  PIN: the source entries are of that packed
// form already (the inner list of such a list).
//
// The same kernel prunes out of place (dst != src, the inner list of
// nb_pairlist_prune): it then tests every entry against the radius rl2_inner
// and writes the kept entries to the same positions of dst, with dst's items,
// counters and order.
constexpr int PRUNE_UNITS = 2 * 32 + 1;  // halves of one chunk, plus one carried over

// The mask bits of a half moved from j-slots 4 s + t to 4 s' + t (s != s'):
// the nibbles of every byte swap.
__device__ __forceinline__ unsigned long long half_to_side(unsigned long long m, int from, int to) {
    return from == to ? m : (((m >> 4) & 0x0F0F0F0F0F0F0F0Full) | ((m << 4) & 0xF0F0F0F0F0F0F0F0ull));
}

template <bool PIN, bool POUT>
__global__ void __launch_bounds__(PRUNE_WARPS * 32, 3)
k_prune(const SysDev* __restrict__ sys, ListDev src, ListDev dst, KParams kp, float rl2_inner) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned char s_rank[PRUNE_WARPS][32];
    // POUT: the kept halves of a chunk (first slot, mask bits, side), in order
    __shared__ int s_ub[POUT ? PRUNE_WARPS : 1][POUT ? PRUNE_UNITS : 1];
    __shared__ unsigned long long s_um[POUT ? PRUNE_WARPS : 1][POUT ? PRUNE_UNITS : 1];
    __shared__ unsigned char s_us[POUT ? PRUNE_WARPS : 1][POUT ? PRUNE_UNITS : 1];
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
        // Distances relative to c, the shifted i-cluster's first atom: with
        // a' = a - c for both atoms of a pair (the shift cancels on the i
        // side), r^2 = |i'|^2 + |j'|^2 - 2 i'.j', so r^2 < rl2 becomes
        // |i'|^2 - 2 i'.j' < rl2 - |j'|^2: three paired multiply-adds per
        // two i-atoms.  The primed coordinates stay within a few nm, so the
        // float32 rounding of the terms (~1e-6 nm^2) lies far inside the
        // padding of the list radius.  Fillers, 10^6 nm away, stay far.
        // The i-atoms in pairs (2k, 2k+1): -2 i' and |i'|^2.
        const float4 c0 = d.xq_s[item.x * CL];
        float2 ax[CL / 2], ay[CL / 2], az[CL / 2], a2[CL / 2];
#pragma unroll
        for (int k = 0; k < CL / 2; ++k) {
            const float4 v0 = d.xq_s[item.x * CL + 2 * k], v1 = d.xq_s[item.x * CL + 2 * k + 1];
            const float x0 = v0.x - c0.x, y0 = v0.y - c0.y, z0 = v0.z - c0.z;
            const float x1 = v1.x - c0.x, y1 = v1.y - c0.y, z1 = v1.z - c0.z;
            ax[k] = make_float2(-2.f * x0, -2.f * x1);
            ay[k] = make_float2(-2.f * y0, -2.f * y1);
            az[k] = make_float2(-2.f * z0, -2.f * z1);
            a2[k] = make_float2(fmaf(x0, x0, fmaf(y0, y0, z0 * z0)), fmaf(x1, x1, fmaf(y1, y1, z1 * z1)));
        }
        const float cx = c0.x + Sx, cy = c0.y + Sy, cz = c0.z + Sz;
        // POUT after a search: the shifted i-cluster box and the radii of the
        // half-box decisions
        int write = item.y;
        int carry = 0;  // POUT: a half waiting for its partner (unit 0 of s_u*)
        // each chunk's entries are loaded while the previous chunk is tested
        int c_next = 0, b_next = 0;
        unsigned long long m_next = 0ull;
        if (lane < item.z - item.y) {
            c_next = src.cj[item.y + lane];
            if (PIN) b_next = src.cjb[item.y + lane];
            m_next = src.mask[item.y + lane];
        }
        for (int base = item.y; base < item.z; base += 32) {
            const int n = min(32, item.z - base);
            int cjv = 0, lo = 0, hi = 0;
            unsigned long long m = 0ull;
            bool chk = false;
            if (lane < n) {
                const int c = c_next;
                chk = inner || (c & PRUNE_CHECK) != 0;
                cjv = c & ~PRUNE_CHECK;
                if (PIN) {
                    lo = cjv;
                    hi = b_next;
                } else {
                    lo = hi = cjv * CL;
                }
                m = m_next;
            }
            if (base + 32 + lane < item.z) {
                c_next = src.cj[base + 32 + lane];
                if (PIN) b_next = src.cjb[base + 32 + lane];
                m_next = src.mask[base + 32 + lane];
            }
            const unsigned chk_bal = __ballot_sync(FULL, chk);
            unsigned keep = __ballot_sync(FULL, lane < n && !chk);  // bit k: entry base + k is kept
            const int nchk = __popc(chk_bal);
            if (chk) s_rank[w][__popc(chk_bal & ((1u << lane) - 1u))] = (unsigned char)lane;
            __syncwarp();
            // bit k of a lane's word: checked entry base + k has an unmasked
            // pair within the radius (any lane of its group may set it); with
            // POUT bits 2k and 2k + 1 of found2 stand for its two halves
            unsigned found = 0u;
            unsigned long long found2 = 0ull;
            for (int q0 = 0; q0 < nchk; q0 += 4 * PRUNE_U) {
                float4 xj[PRUNE_U];
                unsigned long long mq[PRUNE_U];
                int rk[PRUNE_U];  // the entry's lane in the chunk, -1 past the checked ones
#pragma unroll
                for (int u = 0; u < PRUNE_U; ++u) {
                    const int k = q0 + 4 * u + g;
                    rk[u] = k < nchk ? s_rank[w][k] : -1;
                    const int lok = __shfl_sync(FULL, lo, max(rk[u], 0));
                    const int hik = __shfl_sync(FULL, hi, max(rk[u], 0));
                    mq[u] = __shfl_sync(FULL, m, max(rk[u], 0));
                    xj[u] = rk[u] >= 0 ? d.xq_s[jj + (jj < 4 ? lok : hik)] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < PRUNE_U; ++u) {
                    // j-atom jj of the entry, relative to c
                    const float jx = xj[u].x - cx, jy = xj[u].y - cy, jz = xj[u].z - cz;
                    const float t = rl2 - fmaf(jx, jx, fmaf(jy, jy, jz * jz));
                    const float2 jx2 = dup2(jx), jy2 = dup2(jy), jz2 = dup2(jz);
                    bool near = false;
                    if (__any_sync(FULL, mq[u] != ~0ull)) {
                        // one of the four entries has a partial mask: bit ii of
                        // nb8 is i-atom ii within the radius, masked by the
                        // entry's column of j-slot jj (bit ii = pair (ii, jj))
                        unsigned nb8 = 0;
#pragma unroll
                        for (int k = 0; k < CL / 2; ++k) {
                            const float2 q = fma2(ax[k], jx2, fma2(ay[k], jy2, fma2(az[k], jz2, a2[k])));
                            nb8 |= (q.x < t ? 1u : 0u) << (2 * k);
                            nb8 |= (q.y < t ? 1u : 0u) << (2 * k + 1);
                        }
                        const unsigned lo32 = (unsigned)mq[u], hi32 = (unsigned)(mq[u] >> 32);
                        unsigned col = 0;
#pragma unroll
                        for (int ii = 0; ii < CL; ++ii)
                            col |= (((ii < 4 ? lo32 : hi32) >> (8 * (ii & 3) + (ii ^ jj))) & 1u) << ii;
                        near = (nb8 & col) != 0u;
                    } else {
#pragma unroll
                        for (int k = 0; k < CL / 2; ++k) {
                            const float2 q = fma2(ax[k], jx2, fma2(ay[k], jy2, fma2(az[k], jz2, a2[k])));
                            near = near || q.x < t || q.y < t;
                        }
                    }
                    if (near && rk[u] >= 0) {
                        if (POUT)
                            found2 |= 1ull << (2 * rk[u] + (jj >> 2));
                        else
                            found |= 1u << rk[u];
                    }
                }
            }
            if (!POUT) {
                keep |= __reduce_or_sync(FULL, found);
                __syncwarp();
                if (lane < n && ((keep >> lane) & 1u)) {
                    const int idx = write + __popc(keep & ((1u << lane) - 1u));
                    dst.cj[idx] = cjv;
                    dst.mask[idx] = m;
                }
                write += __popc(keep);
            } else {
                const unsigned f_lo = __reduce_or_sync(FULL, (unsigned)found2);
                const unsigned f_hi = __reduce_or_sync(FULL, (unsigned)(found2 >> 32));
                const unsigned long long f = ((unsigned long long)f_hi << 32) | f_lo;
                // an entry the search marked as certain keeps both halves
                // that have an unmasked pair
                const bool k0 = lane < n && (chk ? ((f >> (2 * lane)) & 1ull) != 0ull : (m & MASK_JLO) != 0ull);
                const bool k1 = lane < n && (chk ? ((f >> (2 * lane + 1)) & 1ull) != 0ull : (m & ~MASK_JLO) != 0ull);
                // the chunk's kept halves go to shared memory in list order,
                // after a half left over from the previous chunk (unit 0);
                // lane k then writes packed entry k from units 2k and 2k + 1,
                // and an odd last unit waits for the next chunk
                const unsigned b0 = __ballot_sync(FULL, k0), b1 = __ballot_sync(FULL, k1);
                const unsigned lt = (1u << lane) - 1u;
                int q = carry + __popc(b0 & lt) + __popc(b1 & lt);
                if (k0) {
                    s_ub[w][q] = lo;
                    s_um[w][q] = m & MASK_JLO;
                    s_us[w][q] = 0;
                    ++q;
                }
                if (k1) {
                    s_ub[w][q] = hi + 4;
                    s_um[w][q] = m & ~MASK_JLO;
                    s_us[w][q] = 1;
                }
                const int units = carry + __popc(b0) + __popc(b1);
                const int npk = units >> 1;  // at most 32
                __syncwarp();
                if (lane < npk) {
                    const int a = 2 * lane, b = 2 * lane + 1;
                    dst.cj[write + lane] = s_ub[w][a];
                    dst.cjb[write + lane] = s_ub[w][b] - 4;
                    dst.mask[write + lane] =
                        half_to_side(s_um[w][a], s_us[w][a], 0) | half_to_side(s_um[w][b], s_us[w][b], 1);
                }
                write += npk;
                carry = units & 1;
                __syncwarp();
                if (carry && lane == 0) {
                    s_ub[w][0] = s_ub[w][units - 1];
                    s_um[w][0] = s_um[w][units - 1];
                    s_us[w][0] = s_us[w][units - 1];
                }
                __syncwarp();
            }
        }
        if (POUT && carry) {
            // the item's odd last half, paired with itself under a zero mask
            if (lane == 0) {
                dst.cj[write] = s_ub[w][0];
                dst.cjb[write] = s_ub[w][0] - 4;
                dst.mask[write] = half_to_side(s_um[w][0], s_us[w][0], 0);
            }
            ++write;
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
        __syncwarp();
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
        return launch_pdl(k_tsearch, blocks, TS_BLOCK, 0, st, p.d_sys, p.d_cl_off, p.nsys, p.tot_clcap,
                          slab_stride(p.list.entry_cap, p.tot_clcap), p.list, p.kp);
    }
    unsigned blocks = (unsigned)((p.tot_clcap + SEARCH_WARPS - 1) / SEARCH_WARPS);
    return launch_pdl(k_search, blocks, SEARCH_WARPS * 32, 0, st, p.d_sys, p.d_cl_off, p.nsys, p.tot_clcap, p.list,
                      p.kp);
}

// The prune of a list just searched (always of the 8 x 8 form) into the
// list's own geometry, in place.
cudaError_t launch_prune(const PlanLaunch& p, cudaStream_t st) {
    unsigned blocks = (unsigned)(p.num_sms * 8);
    if (p.list.jgeo)
        return launch_pdl(k_prune<false, true>, blocks, PRUNE_WARPS * 32, 0, st, p.d_sys, p.list, p.list, p.kp, -1.f);
    return launch_pdl(k_prune<false, false>, blocks, PRUNE_WARPS * 32, 0, st, p.d_sys, p.list, p.list, p.kp, -1.f);
}

// The prune of a pruned list into another (dst takes src's geometry).
cudaError_t launch_prune_into(const PlanLaunch& p, const ListDev& src, const ListDev& dst, float rl2_inner,
                              cudaStream_t st) {
    unsigned blocks = (unsigned)(p.num_sms * 8);
    if (src.jgeo != dst.jgeo) return cudaErrorInvalidValue;
    if (src.jgeo)
        return launch_pdl(k_prune<true, true>, blocks, PRUNE_WARPS * 32, 0, st, p.d_sys, src, dst, p.kp, rl2_inner);
    return launch_pdl(k_prune<false, false>, blocks, PRUNE_WARPS * 32, 0, st, p.d_sys, src, dst, p.kp, rl2_inner);
}

}  // namespace nbgb
