// nb_grid.cu -- grid put (Section 3.2, "SIMD parallelism"): atoms are placed
// on a grid of x-y columns, binned (sorted) along z inside each column, and
// each column is cut into clusters of exactly CL = 8 atom slots; the last
// cluster of a column is padded with filler slots that never interact.
//
// Stages (all batch-aware: one launch covers every system of a plan):
//   k_zero_cols   column counters <- 0
//   k_bin         wrap x into [0, L), column of each atom, arrival slot
//   k_col_scan    clusters per column and their prefix (one block per system)
//   k_scatter     (z, atom) sort keys into the column's slot range
//   k_col_sort    bitonic sort of each column by (z, atom) (shared memory up
//                 to COL_MAX atoms, global memory beyond), write sorted
//                 coordinates, types, the permutation and fillers
//   k_bbox        float32 bounding box of the real atoms of each cluster
#include "nb_internal.cuh"

namespace nbgb {

__device__ __forceinline__ int find_sys(const int* __restrict__ off, int nsys, int idx) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Wrap one coordinate into [0, L); returns the wrapped value and the number
// of box lengths k with wrapped = x - k L.
__device__ __forceinline__ float wrap1(float x, float L, int& k) {
    float f = floorf(x / L);
    float w = x - f * L;
    int kk = (int)f;
    if (w >= L) { w -= L; kk += 1; }
    if (w < 0.f) { w += L; kk -= 1; }
    if (w >= L) w = 0.f;  // x just below a multiple of L can round up to L
    k = kk;
    return w + 0.0f;      // turns -0 into +0
}

// Wrap a point into the cell [0, ax) x [0, by) x [0, cz) of the lattice a =
// (ax,0,0), b = (bx,by,0), c = (cx,cy,cz): z by c first, then y by b, then x
// by a (for a rectangular box, each coordinate by its own edge).  Returns the
// multiples with wrapped = x - kx a - ky b - kz c.
__device__ __forceinline__ void wrap_point(const SysDev& d, float4 v, float& x, float& y, float& z, int& kx,
                                           int& ky, int& kz) {
    z = wrap1(v.z, d.L[2], kz);
    const float fz = (float)kz;
    y = wrap1(fmaf(-fz, d.T[2], v.y), d.L[1], ky);
    x = wrap1(fmaf(-(float)ky, d.T[0], fmaf(-fz, d.T[1], v.x)), d.L[0], kx);
}

__device__ __forceinline__ int pack_wrap(int kx, int ky, int kz) {
    kx = max(-127, min(127, kx));
    ky = max(-127, min(127, ky));
    kz = max(-127, min(127, kz));
    return (kx & 0xff) | ((ky & 0xff) << 8) | ((kz & 0xff) << 16);
}

__global__ void k_zero_cols(const SysDev* __restrict__ sys, const int* __restrict__ col_off,
                            int nsys, int tot_cols) {
    pdl_wait();
    pdl_trigger();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tot_cols) return;
    int s = find_sys(col_off, nsys, t);
    sys[s].col_count[t - col_off[s]] = 0;
}

__global__ void k_bin(const SysDev* __restrict__ sys, const int* __restrict__ atom_off, int nsys,
                      int tot_atoms) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = t < tot_atoms;
    int* cc = nullptr;  // the atom's column counter
    int* slot = nullptr;
    if (ok) {
        const int s = find_sys(atom_off, nsys, t);
        const SysDev& d = sys[s];
        const int a = t - atom_off[s];
        float4 v = d.xq_in[a];
        int kx, ky, kz;
        float x, y, z;
        wrap_point(d, v, x, y, z, kx, ky, kz);
        int cx = max(0, min(d.ncx - 1, (int)(x * d.icw[0])));  // max(): NaN input
        int cy = max(0, min(d.ncy - 1, (int)(y * d.icw[1])));
        int col = cx * d.ncy + cy;
        d.atom_col[a] = col;
        cc = d.col_count + col;
        slot = d.atom_slot + a;
    }
    // one atomic per column and warp: consecutive atoms (a molecule, a run of
    // neighbours) mostly share a column, and the lanes of a column take
    // consecutive arrival slots from it (the z sort orders them anyway)
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(0xffffffffu, (unsigned long long)cc);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (ok && lane == leader) base = atomicAdd(cc, __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (ok) *slot = base + __popc(grp & ((1u << lane) - 1u));
}

// One block per system: exclusive prefix over clusters per column.
__global__ void k_col_scan(const SysDev* __restrict__ sys) {
    pdl_wait();
    pdl_trigger();
    const SysDev& d = sys[blockIdx.x];
    __shared__ int s_part[1024];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < d.ncol; base += blockDim.x) {
        int c = base + threadIdx.x;
        int cnt = c < d.ncol ? d.col_count[c] : 0;
        int v = (cnt + CL - 1) / CL;
        s_part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < blockDim.x; off <<= 1) {
            int add = threadIdx.x >= off ? s_part[threadIdx.x - off] : 0;
            __syncthreads();
            s_part[threadIdx.x] += add;
            __syncthreads();
        }
        if (c < d.ncol) d.col_cl0[c] = s_carry + s_part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += s_part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) d.col_cl0[d.ncol] = s_carry;
}

__global__ void k_scatter(const SysDev* __restrict__ sys, const int* __restrict__ atom_off, int nsys,
                          int tot_atoms) {
    pdl_wait();
    pdl_trigger();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tot_atoms) return;
    int s = find_sys(atom_off, nsys, t);
    const SysDev& d = sys[s];
    int a = t - atom_off[s];
    int col = d.atom_col[a];
    int slot = d.atom_slot[a];
    int k;
    float z = wrap1(d.xq_in[a].z, d.L[2], k);
    unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)a;
    d.keys[(size_t)d.col_cl0[col] * CL + slot] = key;
}

// Sort a[0..n) ascending with the direction-free bitonic network (every
// compare-exchange puts the smaller key at the lower index), so indices at or
// beyond n act as +infinity and are never touched.  Block-wide; `a` may live
// in shared or global memory.
template <typename K>
__device__ void block_sort(K* a, int n) {
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int size = 2; size <= p2; size <<= 1) {
        int half = size >> 1;
        for (int k = threadIdx.x; k < (p2 >> 1); k += blockDim.x) {
            int blk = (k / half) * size;
            int lo = blk + (k % half);
            int hi = blk + size - 1 - (k % half);
            if (hi < n) {
                K x = a[lo], y = a[hi];
                if (y < x) { a[lo] = y; a[hi] = x; }
            }
        }
        __syncthreads();
        for (int stride = half >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < (p2 >> 1); k += blockDim.x) {
                int lo = 2 * k - (k & (stride - 1));
                int hi = lo + stride;
                if (hi < n) {
                    K x = a[lo], y = a[hi];
                    if (y < x) { a[lo] = y; a[hi] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// One block per column: sort the column's keys by (z, atom) and write the
// sorted arrays.  Columns longer than COL_MAX are sorted in global memory.
__global__ void __launch_bounds__(256) k_col_sort(const SysDev* __restrict__ sys,
                                                  const int* __restrict__ col_off, int nsys) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_key[COL_MAX];
    int s = find_sys(col_off, nsys, blockIdx.x);
    const SysDev& d = sys[s];
    int c = blockIdx.x - col_off[s];
    int n = d.col_count[c];
    int start = d.col_cl0[c] * CL;
    int nslot = (n + CL - 1) / CL * CL;
    unsigned long long* keys = s_key;
    if (n <= COL_MAX) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) s_key[k] = d.keys[start + k];
        __syncthreads();
    } else {
        keys = d.keys + start;
    }
    block_sort(keys, n);
    for (int k = threadIdx.x; k < nslot; k += blockDim.x) {
        int slot = start + k;
        if (k < n) {
            int a = (int)(keys[k] & 0xffffffffull);
            float4 v = d.xq_in[a];
            int kx, ky, kz;
            float x, y, z;
            wrap_point(d, v, x, y, z, kx, ky, kz);
            d.xq_s[slot] = make_float4(x, y, z, v.w);
            d.type_s[slot] = d.type_in[a];
            d.perm[slot] = a;
            d.iperm[a] = slot;
            d.wrapk[slot] = pack_wrap(kx, ky, kz);
        } else {
            // filler: far outside every box, pairwise far apart, no charge
            float fx = -1.0e6f - 16.0f * (float)(slot & 1023);
            float fy = -1.0e6f - 16.0f * (float)((slot >> 10) & 1023);
            float fz = -1.0e6f - 16.0f * (float)(slot >> 20);
            d.xq_s[slot] = make_float4(fx, fy, fz, 0.f);
            d.type_s[slot] = 0;
            d.perm[slot] = -1;
            d.wrapk[slot] = 0;
        }
    }
}

__global__ void k_bbox(const SysDev* __restrict__ sys, const int* __restrict__ cl_off, int nsys,
                       int tot_clcap) {
    pdl_wait();
    pdl_trigger();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tot_clcap) return;
    int s = find_sys(cl_off, nsys, t);
    const SysDev& d = sys[s];
    int c = t - cl_off[s];
    if (c >= d.col_cl0[d.ncol]) return;
    float3 lo = make_float3(3.0e38f, 3.0e38f, 3.0e38f);
    float3 hi = make_float3(-3.0e38f, -3.0e38f, -3.0e38f);
    int nreal = 0;
#pragma unroll
    for (int k = 0; k < CL; ++k) {
        int slot = c * CL + k;
        if (d.perm[slot] < 0) continue;
        float4 v = d.xq_s[slot];
        lo.x = fminf(lo.x, v.x); lo.y = fminf(lo.y, v.y); lo.z = fminf(lo.z, v.z);
        hi.x = fmaxf(hi.x, v.x); hi.y = fmaxf(hi.y, v.y); hi.z = fmaxf(hi.z, v.z);
        ++nreal;
    }
    d.bb[2 * c] = make_float4(lo.x, lo.y, lo.z, (float)nreal);
    d.bb[2 * c + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
}

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_grid_put(const PlanLaunch& p, cudaStream_t st) {
    const int bs = 256;
    cudaError_t e = cudaSuccess;
    if (p.tot_cols > 0)
        e = launch_pdl(k_zero_cols, blocks_for(p.tot_cols, bs), bs, 0, st, p.d_sys, p.d_col_off, p.nsys, p.tot_cols);
    if (e == cudaSuccess && p.tot_atoms > 0)
        e = launch_pdl(k_bin, blocks_for(p.tot_atoms, bs), bs, 0, st, p.d_sys, p.d_atom_off, p.nsys, p.tot_atoms);
    if (e == cudaSuccess) e = launch_pdl(k_col_scan, (unsigned)p.nsys, 1024, 0, st, p.d_sys);
    if (e == cudaSuccess && p.tot_atoms > 0)
        e = launch_pdl(k_scatter, blocks_for(p.tot_atoms, bs), bs, 0, st, p.d_sys, p.d_atom_off, p.nsys, p.tot_atoms);
    if (e == cudaSuccess && p.tot_cols > 0)
        e = launch_pdl(k_col_sort, (unsigned)p.tot_cols, 256, 0, st, p.d_sys, p.d_col_off, p.nsys);
    if (e == cudaSuccess && p.tot_clcap > 0)
        e = launch_pdl(k_bbox, blocks_for(p.tot_clcap, bs), bs, 0, st, p.d_sys, p.d_cl_off, p.nsys, p.tot_clcap);
    return e;
}

}  // namespace nbgb
