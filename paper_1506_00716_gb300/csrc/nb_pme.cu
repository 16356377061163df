// nb_pme.cu -- long-range electrostatics by smooth particle-mesh Ewald (PME).
//
// The paper evaluates the long-range part of the Ewald electrostatics with
// PME next to the short-range cluster-pair kernel (Section 1 and the
// multi-level parallelism of Section 2: PME on its own ranks or on the CPU).
// Here it runs on the same GPU, after the short-range kernels, on the same
// sorted atom slots, and adds into the same force buffer and accumulators:
//
//   spread   Q(n) = sum_j q_j M_p(u_jx - n_x) M_p(u_jy - n_y) M_p(u_jz - n_z),
//            u_jd = K_d x_jd / L_d, indices modulo K_d (cardinal B-splines
//            M_p of order p, weights from the de Boor recursion)
//   FFT      real-to-complex along z, complex along y and x
//   solve    F(m) <- G(m) F(m),  G = |b(m)|^2 f exp(-pi^2 m^2 / beta^2) / (pi V m^2),
//            E_rec = 1/2 sum_m G |F|^2 and the virial
//            Xi = -1/2 sum_m E_m (delta - 2 (1 + pi^2 m^2 / beta^2) m m / m^2)
//   FFT      back (unnormalised), giving the potential mesh phi
//   gather   F_j = -q_j sum_n phi(n) grad_j [M_p M_p M_p]
//   self     E_self = -f beta / sqrt(pi) sum q^2
//   excluded E_excl = -f sum_excluded q_i q_j erf(beta r) / r with its forces
//            (the reciprocal sum includes those pairs; float64)
//
// Design for sm_103a.  The mesh is small next to the atom data (a 256^3 mesh
// of float32 is 67 MB), so every FFT pass is one read and one write of the
// mesh through shared memory: a block loads a tile of whole lines (16 lines
// side by side for the strided y and x passes, so that each row of the tile
// is a 128-byte segment), transforms them with a Stockham autosort FFT of
// radix 4, 2, 3 and 5 stages in shared memory (line stride n + 1 to avoid
// bank conflicts), and writes them back.  The z pass packs two real lines
// into one complex transform and separates them afterwards.  The x pass
// holds complete x lines of the spectrum, so the solve is fused into it
// between the forward and the inverse transform: the spectrum is never
// written in the forward direction.  Spreading and gathering use P lanes per
// atom (P = spline order, one z index each), so the P atomics of one (x, y)
// row of an atom hit adjacent words; the atoms come in the grid's spatial
// order, which keeps the mesh rows they touch in L2.  Fractional mesh
// coordinates are formed in float64 (a float32 product of x and K/L would
// move an atom by up to 1e-5 mesh units at L = 30 nm), the splines, mesh and
// transforms are float32, energies and virial are summed in float64.
#include "nb_device.cuh"

namespace nbgb {

namespace {

constexpr unsigned FULL = FULL_MASK;
constexpr int FFT_THREADS = 256;
constexpr int PME_THREADS = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// -i z (forward direction) or +i z (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 z) {
    return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

// r-point DFTs y_t = sum_s v_s w^(t s), w = exp(-+2 pi i / r); the constants
// are cos and sin of 2 pi / 3, 2 pi / 5 and 4 pi / 5.
template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}
template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
    constexpr float S3 = 0.866025403784438647f;  // sin(2 pi / 3)
    const float2 s = cadd(v[1], v[2]);
    const float2 d = mul_mi<INV>(csub(v[1], v[2]));
    const float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
    v[0] = cadd(v[0], s);
    v[1] = make_float2(m.x + S3 * d.x, m.y + S3 * d.y);
    v[2] = make_float2(m.x - S3 * d.x, m.y - S3 * d.y);
}
template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
    constexpr float C1 = 0.309016994374947424f;   // cos(2 pi / 5)
    constexpr float C2 = -0.809016994374947424f;  // cos(4 pi / 5)
    constexpr float S1 = 0.951056516295153572f;   // sin(2 pi / 5)
    constexpr float S2 = 0.587785252292473129f;   // sin(4 pi / 5)
    const float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    const float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    const float2 r1 = make_float2(v[0].x + C1 * a1.x + C2 * a2.x, v[0].y + C1 * a1.y + C2 * a2.y);
    const float2 r2 = make_float2(v[0].x + C2 * a1.x + C1 * a2.x, v[0].y + C2 * a1.y + C1 * a2.y);
    const float2 i1 = mul_mi<INV>(make_float2(S1 * b1.x + S2 * b2.x, S1 * b1.y + S2 * b2.y));
    const float2 i2 = mul_mi<INV>(make_float2(S2 * b1.x - S1 * b2.x, S2 * b1.y - S1 * b2.y));
    v[0] = make_float2(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
    v[1] = cadd(r1, i1);
    v[4] = csub(r1, i1);
    v[2] = cadd(r2, i2);
    v[3] = csub(r2, i2);
}

// One Stockham stage of radix R over nl lines (line stride ls) from src to dst.
template <int R, bool INV>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst, int ls,
                                               int nl, int n, int ns, const float2* __restrict__ tw) {
    const int m = n / R;
    const int step = n / (ns * R);
    for (int idx = threadIdx.x; idx < nl * m; idx += blockDim.x) {
        const int line = idx / m;
        const int j = idx - line * m;
        const float2* s = src + line * ls;
        float2* d = dst + line * ls;
        const int k = j % ns;
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = s[j + t * m];
        if (ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w = __ldg(tw + t * k * step);
                if (INV) w.y = -w.y;
                v[t] = cmul(v[t], w);
            }
        }
        if (R == 2) dft2<INV>(v);
        if (R == 3) dft3<INV>(v);
        if (R == 4) dft4<INV>(v);
        if (R == 5) dft5<INV>(v);
        const int o = (j - k) * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) d[o + t * ns] = v[t];
    }
}

// Transform nl lines held in a (stride ls); b is scratch of the same size.
// Returns the buffer that holds the result.  Every thread of the block calls it.
template <bool INV>
__device__ float2* fft_lines(float2* a, float2* b, int ls, int nl, const FftAxis& ax) {
    int ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int r = ax.rad[s];
        if (r == 4) stockham_stage<4, INV>(a, b, ls, nl, ax.n, ns, ax.tw);
        else if (r == 2) stockham_stage<2, INV>(a, b, ls, nl, ax.n, ns, ax.tw);
        else if (r == 3) stockham_stage<3, INV>(a, b, ls, nl, ax.n, ns, ax.tw);
        else stockham_stage<5, INV>(a, b, ls, nl, ax.n, ns, ax.tw);
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        ns *= r;
    }
    return a;
}

// Lines per block of the strided passes and real-line pairs per block of the
// z pass.
__host__ __device__ inline int tile_lines(int n) { return n <= 512 ? 16 : 8; }
__host__ __device__ inline int z_pairs(int n) { return n >= 2048 ? 1 : (2048 / n > 16 ? 16 : 2048 / n); }

// Forward z pass: real lines (K0 K1 of length n = K2) of Q to half spectra
// in S, two lines per complex transform, z = a + i b, then
// A(k) = (Z(k) + conj Z(-k)) / 2, B(k) = (Z(k) - conj Z(-k)) / (2 i).
__global__ void __launch_bounds__(FFT_THREADS) k_fft_z_r2c(PmeDev pm, long long nlines) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[2];
    const int n = ax.n, ls = n + 1, nh = pm.Kzh, ppb = z_pairs(n);
    float2* a = sm;
    float2* b = sm + ppb * ls;
    const long long line0 = (long long)blockIdx.x * 2 * ppb;
    const int nlb = (int)min((long long)2 * ppb, nlines - line0);
    const int np = (nlb + 1) >> 1;
    const float* __restrict__ q = pm.Q + line0 * n;
    float* af = reinterpret_cast<float*>(a);
    for (int f = threadIdx.x; f < 2 * np * n; f += blockDim.x) {
        const int l = f / n, e = f - l * n;
        af[2 * ((l >> 1) * ls + e) + (l & 1)] = l < nlb ? q[f] : 0.f;
    }
    __syncthreads();
    const float2* z = fft_lines<false>(a, b, ls, np, ax);
    float2* __restrict__ out = pm.S + line0 * nh;
    for (int f = threadIdx.x; f < nlb * nh; f += blockDim.x) {
        const int l = f / nh, k = f - l * nh;
        const float2* zp = z + (l >> 1) * ls;
        const float2 zk = zp[k], zm = zp[k == 0 ? 0 : n - k];
        out[f] = (l & 1) ? make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x))
                         : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    }
}

// Inverse z pass: half spectra of S back to real lines of Q, two per complex
// transform: Z(k) = A(k) + i B(k) over the full range, the upper half from
// the Hermitian symmetry A(n - k) = conj A(k).
__global__ void __launch_bounds__(FFT_THREADS) k_fft_z_c2r(PmeDev pm, long long nlines) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[2];
    const int n = ax.n, ls = n + 1, nh = pm.Kzh, ppb = z_pairs(n);
    float2* a = sm;
    float2* b = sm + ppb * ls;
    const long long line0 = (long long)blockIdx.x * 2 * ppb;
    const int nlb = (int)min((long long)2 * ppb, nlines - line0);
    const int np = (nlb + 1) >> 1;
    const float2* __restrict__ in = pm.S + line0 * nh;
    for (int f = threadIdx.x; f < np * nh; f += blockDim.x) {
        const int p = f / nh, k = f - p * nh;
        const float2 A = in[(2 * p) * nh + k];
        const float2 B = 2 * p + 1 < nlb ? in[(2 * p + 1) * nh + k] : make_float2(0.f, 0.f);
        a[p * ls + k] = make_float2(A.x - B.y, A.y + B.x);
        if (k > 0 && n - k >= nh) a[p * ls + n - k] = make_float2(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    const float2* z = fft_lines<true>(a, b, ls, np, ax);
    float* __restrict__ q = pm.Q + line0 * n;
    for (int f = threadIdx.x; f < nlb * n; f += blockDim.x) {
        const int l = f / n, e = f - l * n;
        const float2 v = z[(l >> 1) * ls + e];
        q[f] = (l & 1) ? v.y : v.x;
    }
}

// Strided complex pass: for each outer index o, lines of n = ax.n elements at
// data[o * os + e * es + i], i in [0, n_inner); a block takes tile_lines(n)
// consecutive i, so that each row of its tile is one contiguous segment.
template <bool INV>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_strided(PmeDev pm, int axis, float2* __restrict__ data,
                                                             int n_inner, long long es, long long os) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[axis];
    const int n = ax.n, ls = n + 1, tb = tile_lines(n);
    float2* a = sm;
    float2* b = sm + tb * ls;
    const int i0 = blockIdx.x * tb;
    const int nlb = min(tb, n_inner - i0);
    float2* base = data + blockIdx.y * os + i0;
    for (int f = threadIdx.x; f < nlb * n; f += blockDim.x) {
        const int e = f / nlb, l = f - e * nlb;
        a[l * ls + e] = base[e * es + l];
    }
    __syncthreads();
    const float2* z = fft_lines<INV>(a, b, ls, nlb, ax);
    for (int f = threadIdx.x; f < nlb * n; f += blockDim.x) {
        const int e = f / nlb, l = f - e * nlb;
        base[e * es + l] = z[l * ls + e];
    }
}

// Sum of NV doubles over the block, added to dst[slot[c]] by one thread.
template <int NV>
__device__ __forceinline__ void block_add(double (&v)[NV], double* __restrict__ acc, const int (&slot)[NV]) {
    __shared__ double red[FFT_THREADS / 32][NV];
#pragma unroll
    for (int c = 0; c < NV; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(FULL, v[c], off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) red[w][c] = v[c];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][threadIdx.x];
        if (s != 0.0) atomicAdd(acc + slot[threadIdx.x], s);
    }
}

// x pass with the solve: complete x lines of the spectrum (i = ky * Kzh + kz),
// forward transform, multiplication by G(m) (with EV, the energy and virial
// of each wave vector, kz in (0, K2/2) counted twice for its mirror image),
// inverse transform, store.
template <bool EV>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_solve(PmeDev pm, double* __restrict__ acc) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[0];
    const int n = ax.n, ls = n + 1, tb = tile_lines(n);
    const int n_inner = pm.K[1] * pm.Kzh;
    const long long es = n_inner;
    float2* a = sm;
    float2* b = sm + tb * ls;
    const int i0 = blockIdx.x * tb;
    const int nlb = min(tb, n_inner - i0);
    float2* base = pm.S + i0;
    for (int f = threadIdx.x; f < nlb * n; f += blockDim.x) {
        const int e = f / nlb, l = f - e * nlb;
        a[l * ls + e] = base[e * es + l];
    }
    __syncthreads();
    float2* z = fft_lines<false>(a, b, ls, nlb, ax);
    float2* other = z == a ? b : a;
    double ev[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int kz_mid = (pm.K[2] & 1) ? -1 : pm.K[2] / 2;
    for (int f = threadIdx.x; f < nlb * n; f += blockDim.x) {
        const int l = f / n, kx = f - l * n;
        const int i = i0 + l;
        const int ky = i / pm.Kzh, kz = i - ky * pm.Kzh;
        const float2 tx = __ldg(pm.tab[0] + kx), ty = __ldg(pm.tab[1] + ky), tz = __ldg(pm.tab[2] + kz);
        const float m2 = tx.x * tx.x + ty.x * ty.x + tz.x * tz.x;
        const float g = m2 > 0.f ? pm.cpre * (tx.y * ty.y * tz.y) / m2 : 0.f;
        float2 v = z[l * ls + kx];
        if (EV && m2 > 0.f) {
            const float wz = (kz == 0 || kz == kz_mid) ? 0.5f : 1.f;  // 1/2 of the mirrored pair
            const double em = (double)(wz * g * (v.x * v.x + v.y * v.y));
            const float s = 2.f * (1.f + pm.pi2_b2 * m2) / m2;
            ev[0] += em;
            ev[1] += em * (double)(1.f - s * tx.x * tx.x);
            ev[2] += em * (double)(1.f - s * ty.x * ty.x);
            ev[3] += em * (double)(1.f - s * tz.x * tz.x);
            ev[4] += em * (double)(-s * tx.x * ty.x);
            ev[5] += em * (double)(-s * tx.x * tz.x);
            ev[6] += em * (double)(-s * ty.x * tz.x);
        }
        v.x *= g;
        v.y *= g;
        z[l * ls + kx] = v;
    }
    __syncthreads();
    z = fft_lines<true>(z, other, ls, nlb, ax);
    for (int f = threadIdx.x; f < nlb * n; f += blockDim.x) {
        const int e = f / nlb, l = f - e * nlb;
        base[e * es + l] = z[l * ls + e];
    }
    if (EV) {
        // em is the energy of wave vector m together with its mirror -m, which
        // the half spectrum does not hold (of m alone on the planes kz = 0
        // and kz = K2 / 2, which hold their own mirrors); the accumulators
        // take -2 Xi = sum_m E_m (delta - s m m)
        const int slot[7] = {ACC_EREC, ACC_VXX, ACC_VYY, ACC_VZZ, ACC_VXY, ACC_VXZ, ACC_VYZ};
        block_add<7>(ev, acc, slot);
    }
}

// Cardinal B-spline weights of order P at fractional offset w in [0, 1):
// th[j] = M_P(w + j), the weight of mesh point base - j, and dth[j] its
// derivative M_{P-1}(w + j) - M_{P-1}(w + j - 1), by the recursion
// M_k(x) = (x M_{k-1}(x) + (k - x) M_{k-1}(x - 1)) / (k - 1) from M_2.
template <int P, bool DERIV>
__device__ __forceinline__ void bspline_weights(float w, float (&th)[P], float (&dth)[P]) {
#pragma unroll
    for (int j = 0; j < P; ++j) th[j] = 0.f;
    th[0] = w;
    th[1] = 1.f - w;
#pragma unroll
    for (int k = 3; k <= P; ++k) {
        if (DERIV && k == P) {
#pragma unroll
            for (int j = 0; j < P; ++j) dth[j] = th[j] - (j > 0 ? th[j - 1] : 0.f);
        }
        // divide by k - 1: a multiplication by a rounded reciprocal would
        // scale every weight of every atom by the same error (for p = 8 it
        // moves E_rec by 1e-6); powers of two are exact either way
        const bool pow2 = ((k - 1) & (k - 2)) == 0;
        const float inv = 1.f / (float)(k - 1);
#pragma unroll
        for (int j = k - 1; j >= 0; --j) {
            const float num = (w + (float)j) * th[j] + ((float)(k - j) - w) * (j > 0 ? th[j - 1] : 0.f);
            th[j] = pow2 ? num * inv : num / (float)(k - 1);
        }
    }
}

// Mesh index and offset of one coordinate: u = x K / L in float64.
__device__ __forceinline__ void mesh_coord(float x, double kl, int K, int& base, float& w) {
    const double u = (double)x * kl;
    const double fl = floor(u);
    w = (float)(u - fl);
    int b = (int)fl % K;
    base = b < 0 ? b + K : b;
}

__device__ __forceinline__ int wrap_down(int i, int K) { return i < 0 ? i + K : i; }

// Lanes per atom of the spread and gather kernels.
__host__ __device__ constexpr int pme_lanes(int P) { return P <= 4 ? 4 : 8; }

// Spread: lane c of an atom's group adds q th_x[a] th_y[b] th_z[c] to the
// mesh point (base_x - a, base_y - b, base_z - c) for all a, b.  With ENER
// also the self energy -f beta / sqrt(pi) sum q^2.
template <int P, bool ENER>
__global__ void __launch_bounds__(PME_THREADS) k_pme_spread(const SysDev* __restrict__ sys, PmeDev pm,
                                                            double* __restrict__ acc) {
    pdl_wait();
    pdl_trigger();
    constexpr int LPA = pme_lanes(P);
    const SysDev& d = sys[0];
    const int nslots = d.col_cl0[d.ncol] * CL;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = (int)(gt / LPA), c = (int)(gt % LPA);
    float4 xq = make_float4(0.f, 0.f, 0.f, 0.f);
    if (slot < nslots && d.perm[slot] >= 0) xq = d.xq_s[slot];
    if (xq.w != 0.f && c < P) {
        int bx, by, bz;
        float wx, wy, wz;
        mesh_coord(xq.x, pm.kl[0], pm.K[0], bx, wx);
        mesh_coord(xq.y, pm.kl[1], pm.K[1], by, wy);
        mesh_coord(xq.z, pm.kl[2], pm.K[2], bz, wz);
        float tx[P], ty[P], tz[P], dummy[P];
        bspline_weights<P, false>(wx, tx, dummy);
        bspline_weights<P, false>(wy, ty, dummy);
        bspline_weights<P, false>(wz, tz, dummy);
        float thz = tz[0];
#pragma unroll
        for (int j = 1; j < P; ++j)
            if (c == j) thz = tz[j];
        const long long iz = wrap_down(bz - c, pm.K[2]);
        const float qz = xq.w * thz;
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const long long ix = wrap_down(bx - a, pm.K[0]);
            const float qa = qz * tx[a];
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const long long iy = wrap_down(by - b, pm.K[1]);
                atomicAdd(pm.Q + (ix * pm.K[1] + iy) * pm.K[2] + iz, qa * ty[b]);
            }
        }
    }
    if (ENER) {
        double q2[1] = {c == 0 ? (double)xq.w * (double)xq.w * pm.self_pre : 0.0};
        const int slot_e[1] = {ACC_ESELF};
        block_add<1>(q2, acc, slot_e);
    }
}

// Gather: the force on each atom from the potential mesh, the P lanes of its
// group summing over their z index and reducing by shuffles.
template <int P>
__global__ void __launch_bounds__(PME_THREADS) k_pme_gather(const SysDev* __restrict__ sys, PmeDev pm) {
    pdl_wait();
    pdl_trigger();
    constexpr int LPA = pme_lanes(P);
    const SysDev& d = sys[0];
    const int nslots = d.col_cl0[d.ncol] * CL;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = (int)(gt / LPA), c = (int)(gt % LPA);
    float4 xq = make_float4(0.f, 0.f, 0.f, 0.f);
    if (slot < nslots && d.perm[slot] >= 0) xq = d.xq_s[slot];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (xq.w != 0.f && c < P) {
        int bx, by, bz;
        float wx, wy, wz;
        mesh_coord(xq.x, pm.kl[0], pm.K[0], bx, wx);
        mesh_coord(xq.y, pm.kl[1], pm.K[1], by, wy);
        mesh_coord(xq.z, pm.kl[2], pm.K[2], bz, wz);
        float tx[P], ty[P], tz[P], dx[P], dy[P], dz[P];
        bspline_weights<P, true>(wx, tx, dx);
        bspline_weights<P, true>(wy, ty, dy);
        bspline_weights<P, true>(wz, tz, dz);
        float thz = tz[0], dthz = dz[0];
#pragma unroll
        for (int j = 1; j < P; ++j)
            if (c == j) {
                thz = tz[j];
                dthz = dz[j];
            }
        const long long iz = wrap_down(bz - c, pm.K[2]);
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const long long ix = wrap_down(bx - a, pm.K[0]);
            float rx = 0.f, ry = 0.f;
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const long long iy = wrap_down(by - b, pm.K[1]);
                const float ph = __ldg(pm.Q + (ix * pm.K[1] + iy) * pm.K[2] + iz);
                rx = fmaf(ty[b], ph, rx);
                ry = fmaf(dy[b], ph, ry);
            }
            sx = fmaf(dx[a], rx, sx);  // sum dth_x th_y phi
            sy = fmaf(tx[a], ry, sy);  // sum th_x dth_y phi
            sz = fmaf(tx[a], rx, sz);  // sum th_x th_y phi
        }
        fx = -xq.w * (float)pm.kl[0] * thz * sx;
        fy = -xq.w * (float)pm.kl[1] * thz * sy;
        fz = -xq.w * (float)pm.kl[2] * dthz * sz;
    }
#pragma unroll
    for (int off = LPA / 2; off > 0; off >>= 1) {
        fx += __shfl_xor_sync(FULL, fx, off);
        fy += __shfl_xor_sync(FULL, fy, off);
        fz += __shfl_xor_sync(FULL, fz, off);
    }
    if (c == 0 && xq.w != 0.f) atomicAdd(d.f_s + slot, make_float4(fx, fy, fz, 0.f));
}

// Excluded-pair correction of the reciprocal sum: every excluded pair
// (i, j), each unordered pair once, minimum image of the rectangular box,
// V = -f qi qj erf(beta r) / r, F_i = (F/r) d, d = x_i - x_j,
// F/r = f qi qj (2 beta / sqrt(pi) exp(-beta^2 r^2) - erf(beta r) / r) / r^2,
// in float64.  One thread per atom.
template <bool ENER, bool VIR>
__global__ void __launch_bounds__(PME_THREADS) k_excl_ewald(const SysDev* __restrict__ sys, PmeDev pm,
                                                            double* __restrict__ acc) {
    pdl_wait();
    pdl_trigger();
    const SysDev& d = sys[0];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (a < d.natoms && d.excl_index) {
        const int sa = d.iperm[a];
        const float4 xa = d.xq_s[sa];
        const double Lx = d.L[0], Ly = d.L[1], Lz = d.L[2];
        const double b2sp = 2.0 * pm.beta * 0.564189583547756287;  // 2 beta / sqrt(pi)
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int k = d.excl_index[a]; k < d.excl_index[a + 1]; ++k) {
            const int b = d.excl_atoms[k];
            if (b <= a) continue;
            const int sb = d.iperm[b];
            const float4 xb = d.xq_s[sb];
            if (xa.w == 0.f || xb.w == 0.f) continue;
            double dx = (double)xa.x - (double)xb.x, dy = (double)xa.y - (double)xb.y,
                   dz = (double)xa.z - (double)xb.z;
            dx -= Lx * rint(dx / Lx);
            dy -= Ly * rint(dy / Ly);
            dz -= Lz * rint(dz / Lz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double r = sqrt(r2);
            const double qq = pm.fq * (double)xa.w * (double)xb.w;
            const double ef = erf(pm.beta * r);
            const double fr = qq * (b2sp * exp(-pm.beta * pm.beta * r2) - ef / r) / r2;
            if (ENER) e -= qq * ef / r;
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
    if (ENER) {
        double ee[1] = {e};
        const int slot_e[1] = {ACC_EEXCL};
        block_add<1>(ee, acc, slot_e);
    }
    if (VIR) {
        const int slot_v[6] = {ACC_VXX, ACC_VYY, ACC_VZZ, ACC_VXY, ACC_VXZ, ACC_VYZ};
        block_add<6>(v, acc, slot_v);
    }
}

size_t strided_smem(int n) { return 2 * (size_t)tile_lines(n) * (n + 1) * sizeof(float2); }
size_t z_smem(int n) { return 2 * (size_t)z_pairs(n) * (n + 1) * sizeof(float2); }

template <int P>
cudaError_t launch_pme_p(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags, cudaStream_t st) {
    const bool en = flags & NB_F_ENERGY, vi = flags & NB_F_VIRIAL;
    const SysDev* sys = p.d_sys;
    cudaError_t e;
    const size_t nq = (size_t)pm.K[0] * pm.K[1] * pm.K[2];
    e = cudaMemsetAsync(pm.Q, 0, sizeof(float) * nq, st);
    if (e != cudaSuccess) return e;
    const long long threads = (long long)p.tot_clcap * CL * pme_lanes(P);
    const unsigned ablocks = (unsigned)((threads + PME_THREADS - 1) / PME_THREADS);
    e = en ? launch_pdl(k_pme_spread<P, true>, ablocks, PME_THREADS, 0, st, sys, pm, acc)
           : launch_pdl(k_pme_spread<P, false>, ablocks, PME_THREADS, 0, st, sys, pm, acc);
    if (e != cudaSuccess) return e;
    const long long zlines = (long long)pm.K[0] * pm.K[1];
    const unsigned zblocks = (unsigned)((zlines + 2 * z_pairs(pm.K[2]) - 1) / (2 * z_pairs(pm.K[2])));
    e = launch_pdl(k_fft_z_r2c, zblocks, FFT_THREADS, z_smem(pm.K[2]), st, pm, zlines);
    if (e != cudaSuccess) return e;
    const int ty = tile_lines(pm.K[1]);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((pm.Kzh + ty - 1) / ty, pm.K[0]);
    cfg.blockDim = dim3(FFT_THREADS);
    cfg.dynamicSmemBytes = strided_smem(pm.K[1]);
    cfg.stream = st;
    const long long es_y = pm.Kzh, os_y = (long long)pm.K[1] * pm.Kzh;
    e = cudaLaunchKernelEx(&cfg, k_fft_strided<false>, pm, 1, pm.S, pm.Kzh, es_y, os_y);
    if (e != cudaSuccess) return e;
    const int tx = tile_lines(pm.K[0]);
    const unsigned xblocks = (unsigned)(((long long)pm.K[1] * pm.Kzh + tx - 1) / tx);
    e = (en || vi) ? launch_pdl(k_fft_x_solve<true>, xblocks, FFT_THREADS, strided_smem(pm.K[0]), st, pm, acc)
                   : launch_pdl(k_fft_x_solve<false>, xblocks, FFT_THREADS, strided_smem(pm.K[0]), st, pm, acc);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, k_fft_strided<true>, pm, 1, pm.S, pm.Kzh, es_y, os_y);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_fft_z_c2r, zblocks, FFT_THREADS, z_smem(pm.K[2]), st, pm, zlines);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_pme_gather<P>, ablocks, PME_THREADS, 0, st, sys, pm);
    if (e != cudaSuccess) return e;
    const unsigned eblocks = (unsigned)((p.tot_atoms + PME_THREADS - 1) / PME_THREADS);
    if (en && vi) return launch_pdl(k_excl_ewald<true, true>, eblocks, PME_THREADS, 0, st, sys, pm, acc);
    if (en) return launch_pdl(k_excl_ewald<true, false>, eblocks, PME_THREADS, 0, st, sys, pm, acc);
    if (vi) return launch_pdl(k_excl_ewald<false, true>, eblocks, PME_THREADS, 0, st, sys, pm, acc);
    return launch_pdl(k_excl_ewald<false, false>, eblocks, PME_THREADS, 0, st, sys, pm, acc);
}

template <typename K>
cudaError_t allow_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t pme_prepare_kernels(const PmeDev& pm) {
    // the device's opt-in maximum, so that no later mesh lowers the limit
    // another system's launches rely on
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((size_t)optin < pme_smem_need(pm.K)) return cudaErrorInvalidValue;
    const size_t lim = (size_t)optin - 1024;  // room for the kernels' static shared memory
    e = allow_smem(k_fft_z_r2c, lim);
    if (e == cudaSuccess) e = allow_smem(k_fft_z_c2r, lim);
    if (e == cudaSuccess) e = allow_smem(k_fft_strided<false>, lim);
    if (e == cudaSuccess) e = allow_smem(k_fft_strided<true>, lim);
    if (e == cudaSuccess) e = allow_smem(k_fft_x_solve<false>, lim);
    if (e == cudaSuccess) e = allow_smem(k_fft_x_solve<true>, lim);
    return e;
}

size_t pme_smem_need(const int K[3]) {
    size_t m = z_smem(K[2]);
    if (strided_smem(K[1]) > m) m = strided_smem(K[1]);
    if (strided_smem(K[0]) > m) m = strided_smem(K[0]);
    return m;
}

cudaError_t launch_pme(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags, cudaStream_t st) {
    switch (pm.order) {
        case 4: return launch_pme_p<4>(p, pm, acc, flags, st);
        case 6: return launch_pme_p<6>(p, pm, acc, flags, st);
        default: return launch_pme_p<8>(p, pm, acc, flags, st);
    }
}

}  // namespace nbgb
