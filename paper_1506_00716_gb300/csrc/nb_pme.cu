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
//            (the reciprocal sum includes those pairs; double-float)
//
// Design for sm_103a.  The mesh is small next to the atom data (a 256^3 mesh
// of float32 is 67 MB, mostly L2-resident), so every FFT pass reads and
// writes the mesh once: a block takes a tile of whole lines (16 lines side
// by side for the strided y and x passes, so that each row of the tile is a
// 128-byte segment) and transforms them with a Stockham autosort FFT of
// radix 16 (4 x 4 in registers), 4, 2, 3 and 5 stages.  The first stage
// reads global memory and the last writes it, so a 256-point line makes one
// round trip through shared memory (lines padded by one slot every 16
// elements against bank conflicts).  The z pass packs two real lines into
// one complex transform and separates them afterwards.  The x pass holds
// complete x lines of the spectrum, so the solve is fused into it between
// the forward and the inverse transform: the spectrum is never written in
// the forward direction.  Spreading and gathering compute each atom's
// splines once into shared memory and use P lanes per atom (P = spline
// order, one z index each), so the P atomics of one (x, y) row of an atom hit
// adjacent words; the atoms come in the grid's spatial order, which keeps
// the mesh rows they touch in L2.  Nothing on the per-atom or per-point paths
// uses the (narrow) float64 pipe: fractional mesh coordinates are formed in
// double-float on the float32 pipes (a float32 product of x and K/L would
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

// 16-point DFT as 4 x 4: DFT4 over n1 of x[4 n1 + n2], twiddle w16^(n2 k1),
// DFT4 over n2; output k = k1 + 4 k2.  The constants are cos and sin of
// multiples of pi / 8.
template <bool INV>
__device__ __forceinline__ float2 tw16(float2 v, float c, float s) {
    // v * exp(-+ i theta) with c = cos theta, s = sin theta
    return INV ? make_float2(v.x * c - v.y * s, v.x * s + v.y * c) : make_float2(v.x * c + v.y * s, v.y * c - v.x * s);
}
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
    constexpr float C1 = 0.923879532511286756f;  // cos(pi / 8)
    constexpr float S1 = 0.382683432365089772f;  // sin(pi / 8)
    constexpr float R2 = 0.707106781186547524f;  // cos(pi / 4)
    float2 a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        float2 t[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
        dft4<INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
    }
    a[1][1] = tw16<INV>(a[1][1], C1, S1);    // w^1
    a[1][2] = tw16<INV>(a[1][2], R2, R2);    // w^2
    a[1][3] = tw16<INV>(a[1][3], S1, C1);    // w^3
    a[2][1] = tw16<INV>(a[2][1], R2, R2);    // w^2
    a[2][2] = mul_mi<INV>(a[2][2]);          // w^4
    a[2][3] = tw16<INV>(a[2][3], -R2, R2);   // w^6
    a[3][1] = tw16<INV>(a[3][1], S1, C1);    // w^3
    a[3][2] = tw16<INV>(a[3][2], -R2, R2);   // w^6
    a[3][3] = tw16<INV>(a[3][3], -C1, -S1);  // w^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        dft4<INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}

// (q, r) = divmod(f, d) while f advances by a fixed stride: one division at
// the start, then additions only (the index loops below would otherwise
// spend most of their issue slots on integer division).
struct DivWalk {
    int q, r, dq, dr, d;
    __device__ __forceinline__ DivWalk(int f0, int stride, int d_) : d(d_) {
        q = f0 / d;
        r = f0 - q * d;
        dq = stride / d;
        dr = stride - dq * d;
    }
    __device__ __forceinline__ void next() {
        q += dq;
        r += dr;
        if (r >= d) {
            r -= d;
            ++q;
        }
    }
};

// Element e of a line sits at pad16(e): one padding slot every 16 elements,
// so that the stride-R accesses of the first stages spread over the banks.
__host__ __device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }
// Line stride in float2 (odd, so that lines start on different banks).
__host__ __device__ __forceinline__ int line_stride(int n) { return (pad16(n) + 1) | 1; }

// Where a stage reads and writes element e of line l: shared memory (line
// major, padded), a strided tile of the spectrum (element e of line l at
// base[e * es + l], lines side by side), or pairs of real z lines (line p of
// the transform is z = a + i b of the real lines 2p and 2p + 1).
struct SmemAcc {
    float2* p;
    int ls;
    __device__ __forceinline__ float2 ld(int l, int e) const { return p[l * ls + pad16(e)]; }
    __device__ __forceinline__ void st(int l, int e, float2 v) const { p[l * ls + pad16(e)] = v; }
};
struct StridedAcc {
    float2* base;
    long long es;
    __device__ __forceinline__ float2 ld(int l, int e) const { return base[e * es + l]; }
    __device__ __forceinline__ void st(int l, int e, float2 v) const { base[e * es + l] = v; }
};
struct RealPairAcc {
    float* q;  // first real line of the block
    int n;     // line length
    int nlb;   // real lines of the block
    __device__ __forceinline__ float2 ld(int p, int e) const {
        const float a = q[(long long)(2 * p) * n + e];
        const float b = 2 * p + 1 < nlb ? q[(long long)(2 * p + 1) * n + e] : 0.f;
        return make_float2(a, b);
    }
    __device__ __forceinline__ void st(int p, int e, float2 v) const {
        q[(long long)(2 * p) * n + e] = v.x;
        if (2 * p + 1 < nlb) q[(long long)(2 * p + 1) * n + e] = v.y;
    }
};

// One Stockham stage of radix R over nl lines, from src to dst (which must
// not be the same buffer).  LF: consecutive threads take consecutive lines
// (for tiles whose lines lie side by side in global memory), else
// consecutive butterflies of a line (lines contiguous in global memory).
template <int R, bool INV, bool LF, class Src, class Dst>
__device__ __forceinline__ void stockham_stage(const Src& src, const Dst& dst, int nl, int n, int ns,
                                               const float2* __restrict__ tw) {
    const int m = n / R;
    const int step = n / (ns * R);
    const bool ns_pow2 = (ns & (ns - 1)) == 0;
    DivWalk w(threadIdx.x, blockDim.x, LF ? nl : m);
    for (int idx = threadIdx.x; idx < nl * m; idx += blockDim.x, w.next()) {
        const int line = LF ? w.r : w.q;
        const int j = LF ? w.q : w.r;
        const int k = ns_pow2 ? (j & (ns - 1)) : j % ns;
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = src.ld(line, j + t * m);
        if (ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 tf = __ldg(tw + t * k * step);
                if (INV) tf.y = -tf.y;
                v[t] = cmul(v[t], tf);
            }
        }
        if (R == 2) dft2<INV>(v);
        if (R == 3) dft3<INV>(v);
        if (R == 4) dft4<INV>(v);
        if (R == 5) dft5<INV>(v);
        if (R == 16) dft16<INV>(v);
        const int o = (j - k) * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) dst.st(line, o + t * ns, v[t]);
    }
}

template <bool INV, bool LF, class Src, class Dst>
__device__ __forceinline__ void stage_r(int r, const Src& src, const Dst& dst, int nl, int n, int ns,
                                        const float2* tw) {
    if (r == 16) stockham_stage<16, INV, LF>(src, dst, nl, n, ns, tw);
    else if (r == 4) stockham_stage<4, INV, LF>(src, dst, nl, n, ns, tw);
    else if (r == 2) stockham_stage<2, INV, LF>(src, dst, nl, n, ns, tw);
    else if (r == 3) stockham_stage<3, INV, LF>(src, dst, nl, n, ns, tw);
    else stockham_stage<5, INV, LF>(src, dst, nl, n, ns, tw);
}

// Transform nl lines from src to dst through the shared-memory buffers a and
// b (stride ls): the first stage reads src, the last writes dst, the stages
// between run in shared memory, so a two-stage transform (n = 256 = 16 x 16)
// makes one shared-memory round trip per element.  src and dst may be the
// same global lines (the first stage has read everything before the last
// writes: a barrier separates every stage).  The first stage writes a, so src
// must not be a; with more than two stages the stages in between alternate
// between a and b, and dst must not be the buffer the last stage reads (a
// after an even number of stages in between, else b).  Every thread of the
// block calls it.
template <bool INV, bool LF, class Src, class Dst>
__device__ void fft_run(const Src& src, const Dst& dst, float2* a, float2* b, int ls, int nl, const FftAxis& ax) {
    if (ax.nst == 1) {
        // one stage: through a, so that src and dst may be the same lines
        stage_r<INV, LF>(ax.rad[0], src, SmemAcc{a, ls}, nl, ax.n, 1, ax.tw);
        __syncthreads();
        DivWalk w(threadIdx.x, blockDim.x, LF ? nl : ax.n);
        for (int idx = threadIdx.x; idx < nl * ax.n; idx += blockDim.x, w.next()) {
            const int line = LF ? w.r : w.q, e = LF ? w.q : w.r;
            dst.st(line, e, a[line * ls + pad16(e)]);
        }
        __syncthreads();
        return;
    }
    stage_r<INV, LF>(ax.rad[0], src, SmemAcc{a, ls}, nl, ax.n, 1, ax.tw);
    __syncthreads();
    int ns = ax.rad[0];
    for (int s = 1; s < ax.nst - 1; ++s) {
        stage_r<INV, LF>(ax.rad[s], SmemAcc{a, ls}, SmemAcc{b, ls}, nl, ax.n, ns, ax.tw);
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        ns *= ax.rad[s];
    }
    stage_r<INV, LF>(ax.rad[ax.nst - 1], SmemAcc{a, ls}, dst, nl, ax.n, ns, ax.tw);
    __syncthreads();
}

// Single-buffer variant, for transforms where every stage has at most one
// butterfly per thread (nl * n / R <= blockDim; 256-point lines of 16 side
// by side, for instance): each stage reads its inputs into registers, waits
// for the whole block, and writes its outputs in place, so one shared buffer
// serves the whole transform and twice as many blocks fit an SM.
template <int R, bool INV, bool LF, class Src, class Dst>
__device__ __forceinline__ void stockham_stage_1(const Src& src, const Dst& dst, int nl, int n, int ns,
                                                 const float2* __restrict__ tw) {
    const int m = n / R;
    const int step = n / (ns * R);
    const int idx = threadIdx.x;
    const bool act = idx < nl * m;
    const int q = LF ? idx / nl : idx / m;
    const int line = LF ? idx - q * nl : q;
    const int j = LF ? q : idx - q * m;
    const int k = (ns & (ns - 1)) == 0 ? (j & (ns - 1)) : j % ns;
    float2 v[R];
    if (act) {
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = src.ld(line, j + t * m);
        if (ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 tf = __ldg(tw + t * k * step);
                if (INV) tf.y = -tf.y;
                v[t] = cmul(v[t], tf);
            }
        }
        if (R == 2) dft2<INV>(v);
        if (R == 3) dft3<INV>(v);
        if (R == 4) dft4<INV>(v);
        if (R == 5) dft5<INV>(v);
        if (R == 16) dft16<INV>(v);
    }
    __syncthreads();
    if (act) {
        const int o = (j - k) * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) dst.st(line, o + t * ns, v[t]);
    }
}

template <bool INV, bool LF, class Src, class Dst>
__device__ __forceinline__ void stage1_r(int r, const Src& src, const Dst& dst, int nl, int n, int ns,
                                         const float2* tw) {
    if (r == 16) stockham_stage_1<16, INV, LF>(src, dst, nl, n, ns, tw);
    else if (r == 4) stockham_stage_1<4, INV, LF>(src, dst, nl, n, ns, tw);
    else if (r == 2) stockham_stage_1<2, INV, LF>(src, dst, nl, n, ns, tw);
    else if (r == 3) stockham_stage_1<3, INV, LF>(src, dst, nl, n, ns, tw);
    else stockham_stage_1<5, INV, LF>(src, dst, nl, n, ns, tw);
}

// The transform with one shared buffer a (stride ls): first stage from src,
// stages in between in place in a, last stage to dst (which may be a, or the
// global lines src came from).  Every thread of the block calls it.
template <bool INV, bool LF, class Src, class Dst>
__device__ void fft_run_1(const Src& src, const Dst& dst, float2* a, int ls, int nl, const FftAxis& ax) {
    const SmemAcc sa{a, ls};
    if (ax.nst == 1) {
        stage1_r<INV, LF>(ax.rad[0], src, dst, nl, ax.n, 1, ax.tw);
        __syncthreads();
        return;
    }
    stage1_r<INV, LF>(ax.rad[0], src, sa, nl, ax.n, 1, ax.tw);
    __syncthreads();
    int ns = ax.rad[0];
    for (int s = 1; s < ax.nst - 1; ++s) {
        stage1_r<INV, LF>(ax.rad[s], sa, sa, nl, ax.n, ns, ax.tw);
        __syncthreads();
        ns *= ax.rad[s];
    }
    stage1_r<INV, LF>(ax.rad[ax.nst - 1], sa, dst, nl, ax.n, ns, ax.tw);
    __syncthreads();
}

// Whether every stage of the axis has at most one butterfly per thread for
// nl lines (then one shared buffer suffices).
__host__ __device__ inline bool one_buffer(const FftAxis& ax, int nl) {
    for (int s = 0; s < ax.nst; ++s)
        if (nl * (ax.n / ax.rad[s]) > FFT_THREADS) return false;
    return true;
}

// Lines per block of the strided passes and real-line pairs per block of the
// z pass.
__host__ __device__ inline int tile_lines(int n) { return n <= 256 ? 16 : (n <= 512 ? 8 : 4); }
__host__ __device__ inline int z_pairs(int n) { return n >= 4096 ? 1 : (4096 / n > 16 ? 16 : 4096 / n); }

// Forward z pass: real lines (K0 K1 of length n = K2) of Q to half spectra
// in S, two lines per complex transform, z = a + i b, then
// A(k) = (Z(k) + conj Z(-k)) / 2, B(k) = (Z(k) - conj Z(-k)) / (2 i).
// The transform lands in shared memory (buffer c); the separation writes S.
__global__ void __launch_bounds__(FFT_THREADS, 4) k_fft_z_r2c(PmeDev pm, long long nlines) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[2];
    const int n = ax.n, ls = line_stride(n), nh = pm.Kzh, ppb = z_pairs(n);
    float2* a = sm;
    float2* b = sm + ppb * ls;
    const long long line0 = (long long)blockIdx.x * 2 * ppb;
    const int nlb = (int)min((long long)2 * ppb, nlines - line0);
    const int np = (nlb + 1) >> 1;
    float2* c;
    if (one_buffer(ax, ppb)) {
        c = a;
        fft_run_1<false, false>(RealPairAcc{pm.Q + line0 * n, n, nlb}, SmemAcc{a, ls}, a, ls, np, ax);
    } else {
        // the result must not land in the buffer the last stage reads: with an
        // even stage count the stages end in a, so the result goes to b, and
        // vice versa
        c = (ax.nst & 1) ? a : b;
        fft_run<false, false>(RealPairAcc{pm.Q + line0 * n, n, nlb}, SmemAcc{c, ls}, a, b, ls, np, ax);
    }
    float2* __restrict__ out = pm.S + line0 * nh;
    DivWalk wlk(threadIdx.x, blockDim.x, nh);
    for (int f = threadIdx.x; f < nlb * nh; f += blockDim.x, wlk.next()) {
        const int l = wlk.q, k = wlk.r;
        const float2* zp = c + (l >> 1) * ls;
        const float2 zk = zp[pad16(k)], zm = zp[pad16(k == 0 ? 0 : n - k)];
        out[f] = (l & 1) ? make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x))
                         : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    }
}

// Inverse z pass: half spectra of S back to real lines of Q, two per complex
// transform: Z(k) = A(k) + i B(k) over the full range, the upper half from
// the Hermitian symmetry A(n - k) = conj A(k), built in shared memory; the
// transform's last stage writes the real lines.
__global__ void __launch_bounds__(FFT_THREADS, 4) k_fft_z_c2r(PmeDev pm, long long nlines) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[2];
    const int n = ax.n, ls = line_stride(n), nh = pm.Kzh, ppb = z_pairs(n);
    float2* a = sm;
    float2* b = sm + ppb * ls;
    const long long line0 = (long long)blockIdx.x * 2 * ppb;
    const int nlb = (int)min((long long)2 * ppb, nlines - line0);
    const int np = (nlb + 1) >> 1;
    // the Hermitian fill goes to the buffer the first stage does not write
    // (with one buffer, to that buffer: its first stage works in place)
    const bool one = one_buffer(ax, ppb);
    float2* c = one ? a : b;
    const float2* __restrict__ in = pm.S + line0 * nh;
    DivWalk wpk(threadIdx.x, blockDim.x, nh);
    for (int f = threadIdx.x; f < np * nh; f += blockDim.x, wpk.next()) {
        const int p = wpk.q, k = wpk.r;
        const float2 A = in[(2 * p) * nh + k];
        const float2 B = 2 * p + 1 < nlb ? in[(2 * p + 1) * nh + k] : make_float2(0.f, 0.f);
        c[p * ls + pad16(k)] = make_float2(A.x - B.y, A.y + B.x);
        if (k > 0 && n - k >= nh) c[p * ls + pad16(n - k)] = make_float2(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    if (one) {
        fft_run_1<true, false>(SmemAcc{a, ls}, RealPairAcc{pm.Q + line0 * n, n, nlb}, a, ls, np, ax);
    } else {
        // the first stage reads c = b and writes a; b is free after it
        fft_run<true, false>(SmemAcc{c, ls}, RealPairAcc{pm.Q + line0 * n, n, nlb}, a, b, ls, np, ax);
    }
}

// Strided complex pass: for each outer index o, lines of n = ax.n elements at
// data[o * os + e * es + i], i in [0, n_inner); a block takes tile_lines(n)
// consecutive i, so that each row of its tile is one contiguous segment.  The
// first stage reads global memory, the last writes it back in place.
template <bool INV>
__global__ void __launch_bounds__(FFT_THREADS, 4) k_fft_strided(PmeDev pm, int axis, float2* __restrict__ data,
                                                             int n_inner, long long es, long long os) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[axis];
    const int n = ax.n, ls = line_stride(n), tb = tile_lines(n);
    const int i0 = blockIdx.x * tb;
    const int nlb = min(tb, n_inner - i0);
    const StridedAcc g{data + blockIdx.y * os + i0, es};
    if (one_buffer(ax, tb)) fft_run_1<INV, true>(g, g, sm, ls, nlb, ax);
    else fft_run<INV, true>(g, g, sm, sm + tb * ls, ls, nlb, ax);
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

// The solve at one stored point of a triclinic cell's half spectrum.  With k'
// the signed indices, m = k R^T and G(k) = |b(k)|^2 f exp(-pi^2 m^2 / beta^2)
// / (pi V m^2).  The point's mirror -k (indices mod K, a Nyquist index its
// own mirror) has m' = k'' R^T, k''_d = k'_d at a Nyquist index and -k'_d
// otherwise, and in a skewed cell G(mirror) may differ from G(k).  The
// spectrum is multiplied by (G(k) + G(mirror)) / 2, which keeps it Hermitian
// and gives the real part of the full inverse transform of G F.  Energy and
// virial take the point with its own m and, inside (0, K2/2) in kz, its
// unstored mirror with m'; a point on the planes kz = 0, K2/2 counts alone
// (its mirror is stored too).
template <bool EV>
__device__ __forceinline__ void tri_solve(const PmeDev& pm, float2 tx, float4 ln, bool nx, bool ny, bool plane,
                                          float2* __restrict__ z, double (&ev)[7]) {
    const float k0 = tx.x, k1 = ln.x, k2 = ln.y;
    const float bb = tx.y * ln.w;
    const float j0 = nx ? k0 : -k0, j1 = ny ? k1 : -k1, j2 = plane ? k2 : -k2;
    const float ma = k0 * pm.rd[0], mb = fmaf(k0, pm.ro[0], k1 * pm.rd[1]),
                mc = fmaf(k0, pm.ro[1], fmaf(k1, pm.ro[2], k2 * pm.rd[2]));
    const float na = j0 * pm.rd[0], nb = fmaf(j0, pm.ro[0], j1 * pm.rd[1]),
                nc = fmaf(j0, pm.ro[1], fmaf(j1, pm.ro[2], j2 * pm.rd[2]));
    const float m2 = ma * ma + mb * mb + mc * mc, n2 = na * na + nb * nb + nc * nc;
    const float g1 = m2 > 0.f ? pm.cpre * bb * expf(-pm.pi2_b2 * m2) / m2 : 0.f;
    const float g2 = n2 > 0.f ? pm.cpre * bb * expf(-pm.pi2_b2 * n2) / n2 : 0.f;
    float2 v = *z;
    if (EV && m2 > 0.f) {
        const float f2 = v.x * v.x + v.y * v.y;
        const double e1 = (double)(0.5f * g1 * f2);
        const float s1 = 2.f * (1.f + pm.pi2_b2 * m2) / m2;
        ev[0] += e1;
        ev[1] += e1 * (double)(1.f - s1 * ma * ma);
        ev[2] += e1 * (double)(1.f - s1 * mb * mb);
        ev[3] += e1 * (double)(1.f - s1 * mc * mc);
        ev[4] += e1 * (double)(-s1 * ma * mb);
        ev[5] += e1 * (double)(-s1 * ma * mc);
        ev[6] += e1 * (double)(-s1 * mb * mc);
        if (!plane) {
            const double e2 = (double)(0.5f * g2 * f2);
            const float s2 = 2.f * (1.f + pm.pi2_b2 * n2) / n2;
            ev[0] += e2;
            ev[1] += e2 * (double)(1.f - s2 * na * na);
            ev[2] += e2 * (double)(1.f - s2 * nb * nb);
            ev[3] += e2 * (double)(1.f - s2 * nc * nc);
            ev[4] += e2 * (double)(-s2 * na * nb);
            ev[5] += e2 * (double)(-s2 * na * nc);
            ev[6] += e2 * (double)(-s2 * nb * nc);
        }
    }
    const float gb = 0.5f * (g1 + g2);
    v.x *= gb;
    v.y *= gb;
    *z = v;
}

// x pass with the solve: complete x lines of the spectrum (i = ky * Kzh + kz),
// forward transform, multiplication by G(m) (with EV, the energy and virial
// of each wave vector, kz in (0, K2/2) counted twice for its mirror image),
// inverse transform, store.
template <bool EV>
__global__ void __launch_bounds__(FFT_THREADS, 4) k_fft_x_solve(PmeDev pm, double* __restrict__ acc) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const FftAxis& ax = pm.ax[0];
    const int n = ax.n, ls = line_stride(n), tb = tile_lines(n);
    const int n_inner = pm.K[1] * pm.Kzh;
    float2* a = sm;
    float2* b = sm + tb * ls;
    const int i0 = blockIdx.x * tb;
    const int nlb = min(tb, n_inner - i0);
    const StridedAcc spec{pm.S + i0, n_inner};
    // per line: (m_y, m_z, m_y^2 + m_z^2, B_y E_y B_z E_z), and the weight of
    // the line's kz plane (1/2 on kz = 0 and K2/2, which hold their own mirrors)
    // Also whether the line's ky is the Nyquist index K1/2 (even K1).
    __shared__ float4 s_line[16];
    __shared__ float s_wz[16];
    __shared__ bool s_nyq[16];
    // (In a triclinic cell the tables hold signed frequencies, and the line
    // record is (k_y', k_z', 0, |b_y|^2 |b_z|^2).)
    if (threadIdx.x < nlb) {
        const int i = i0 + threadIdx.x;
        const int ky = i / pm.Kzh, kz = i - ky * pm.Kzh;
        const float2 ty = __ldg(pm.tab[1] + ky), tz = __ldg(pm.tab[2] + kz);
        s_line[threadIdx.x] = make_float4(ty.x, tz.x, pm.tri ? 0.f : ty.x * ty.x + tz.x * tz.x, ty.y * tz.y);
        s_wz[threadIdx.x] = (kz == 0 || 2 * kz == pm.K[2]) ? 0.5f : 1.f;
        s_nyq[threadIdx.x] = 2 * ky == pm.K[1];
    }
    // forward transform from the spectrum into shared memory (buffer z, the
    // one the last stage does not read), solve there, inverse back
    const bool one = one_buffer(ax, tb);
    float2* z = one ? a : ((ax.nst & 1) ? a : b);
    float2* other = z == a ? b : a;
    if (one) fft_run_1<false, true>(spec, SmemAcc{z, ls}, z, ls, nlb, ax);
    else fft_run<false, true>(spec, SmemAcc{z, ls}, a, b, ls, nlb, ax);
    double ev[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    DivWalk wlkx(threadIdx.x, blockDim.x, n);
    for (int f = threadIdx.x; f < nlb * n; f += blockDim.x, wlkx.next()) {
        const int l = wlkx.q, kx = wlkx.r;
        const float2 tx = __ldg(pm.tab[0] + kx);
        const float4 ln = s_line[l];
        if (pm.tri) {
            tri_solve<EV>(pm, tx, ln, 2 * kx == n, s_nyq[l], s_wz[l] != 1.f, z + l * ls + pad16(kx), ev);
            continue;
        }
        const float m2 = tx.x * tx.x + ln.z;
        const float g = m2 > 0.f ? pm.cpre * (tx.y * ln.w) / m2 : 0.f;
        float2 v = z[l * ls + pad16(kx)];
        if (EV && m2 > 0.f) {
            const float wz = s_wz[l];
            const double em = (double)(wz * g * (v.x * v.x + v.y * v.y));
            const float s = 2.f * (1.f + pm.pi2_b2 * m2) / m2;
            // The Nyquist index K/2 stands for +K/2 in every wave vector, so
            // the unstored mirror of a point with kz inside (0, K2/2) has -m
            // except in a Nyquist component, where it keeps the sign: its
            // off-diagonal products m_a m_b then cancel the stored point's
            // where exactly one of a, b is a Nyquist component.
            const bool inner = wz == 1.f, nx = 2 * kx == n, ny = s_nyq[l];
            const float cxy = (inner && nx != ny) ? 0.f : 1.f;
            const float cxz = (inner && nx) ? 0.f : 1.f;
            const float cyz = (inner && ny) ? 0.f : 1.f;
            ev[0] += em;
            ev[1] += em * (double)(1.f - s * tx.x * tx.x);
            ev[2] += em * (double)(1.f - s * ln.x * ln.x);
            ev[3] += em * (double)(1.f - s * ln.y * ln.y);
            ev[4] += em * (double)(-cxy * s * tx.x * ln.x);
            ev[5] += em * (double)(-cxz * s * tx.x * ln.y);
            ev[6] += em * (double)(-cyz * s * ln.x * ln.y);
        }
        v.x *= g;
        v.y *= g;
        z[l * ls + pad16(kx)] = v;
    }
    __syncthreads();
    if (one) fft_run_1<true, true>(SmemAcc{z, ls}, spec, z, ls, nlb, ax);
    else fft_run<true, true>(SmemAcc{z, ls}, spec, other, z, ls, nlb, ax);
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

// Mesh index and offset of one coordinate, u = x K / L, to float64 accuracy
// on the float32 pipes (the float64 pipe of sm_103a is narrow): K / L =
// klh + kll, x klh = ph + pe exactly, u = ph + (pe + x kll); ph - floor(ph)
// is exact, so the offset w is u's fractional part rounded once.
__device__ __forceinline__ void mesh_coord(float x, float klh, float kll, int K, int& base, float& w) {
    float ph, pe;
    two_prod(x, klh, ph, pe);
    const float pl = fmaf(x, kll, pe);
    float fl = floorf(ph);
    float fr = (ph - fl) + pl;
    if (fr < 0.f) {
        fr += 1.f;
        fl -= 1.f;
    } else if (fr >= 1.f) {
        fr -= 1.f;
        fl += 1.f;
    }
    w = fr;
    const int b = (int)fl % K;
    base = b < 0 ? b + K : b;
}

__device__ __forceinline__ int wrap_down(int i, int K) { return i < 0 ? i + K : i; }

// Mesh coordinate of dimension d in a triclinic cell, u_d = sum_a x_a M[a][d]
// (M lower-triangular: u_0 = x M00 + y M10 + z M20, u_1 = y M11 + z M21,
// u_2 = z M22), each product exact as hi + lo and the terms summed
// error-free before the fractional part is taken (as mesh_coord does for one
// term).
__device__ __forceinline__ void mesh_coord_tri(const float4& xq, int d, const PmeDev& pm, int& base, float& w) {
    const float xs[3] = {xq.x, xq.y, xq.z};
    const float x0 = d == 0 ? xs[0] : (d == 1 ? xs[1] : xs[2]);
    const float dh = d == 0 ? pm.kl_h[0] : (d == 1 ? pm.kl_h[1] : pm.kl_h[2]);
    const float dl = d == 0 ? pm.kl_l[0] : (d == 1 ? pm.kl_l[1] : pm.kl_l[2]);
    float uh, ue;
    two_prod(x0, dh, uh, ue);
    float ul = fmaf(x0, dl, ue);
    // off-diagonal terms: d = 0 takes y M10 and z M20, d = 1 takes z M21
    const int nt = d == 0 ? 2 : (d == 1 ? 1 : 0);
    for (int t = 0; t < nt; ++t) {
        const float xv = (d == 0 && t == 0) ? xs[1] : xs[2];
        const int mi = d == 0 ? t : 2;
        const float mh = mi == 0 ? pm.mo_h[0] : (mi == 1 ? pm.mo_h[1] : pm.mo_h[2]);
        const float ml = mi == 0 ? pm.mo_l[0] : (mi == 1 ? pm.mo_l[1] : pm.mo_l[2]);
        float ph, pe, sh, se;
        two_prod(xv, mh, ph, pe);
        two_sum(uh, ph, sh, se);
        uh = sh;
        ul += se + fmaf(xv, ml, pe);
    }
    float hi, lo;
    fast_two_sum(uh, ul, hi, lo);
    float fl = floorf(hi);
    float fr = (hi - fl) + lo;
    if (fr < 0.f) {
        fr += 1.f;
        fl -= 1.f;
    } else if (fr >= 1.f) {
        fr -= 1.f;
        fl += 1.f;
    }
    w = fr;
    const int K = d == 0 ? pm.K[0] : (d == 1 ? pm.K[1] : pm.K[2]);
    const int b = (int)fl % K;
    base = b < 0 ? b + K : b;
}

// Lanes per atom of the spread and gather kernels.
__host__ __device__ constexpr int pme_lanes(int P) { return P <= 4 ? 4 : 8; }

// Spline weights of the block's atoms, computed once per (atom, dimension)
// by one thread each and kept in shared memory for the P lanes of the atom
// (which would otherwise each recompute all three).  Atoms are the block's
// APB consecutive sorted slots; fillers and uncharged atoms get q = 0.
template <int P, bool DERIV>
struct SplineTile {
    static constexpr int APB = PME_THREADS / pme_lanes(P);
    float w[APB][3][P];
    float dw[DERIV ? APB : 1][3][P];
    int base[APB][3];
    float q[APB];
};

template <int P, bool DERIV>
__device__ __forceinline__ void spline_tile(const SysDev& d, const PmeDev& pm, int slot0, int nslots,
                                            SplineTile<P, DERIV>& st) {
    constexpr int APB = SplineTile<P, DERIV>::APB;
    for (int t = threadIdx.x; t < APB * 3; t += blockDim.x) {
        const int at = t / 3, dim = t - 3 * at;
        const int slot = slot0 + at;
        float4 xq = make_float4(0.f, 0.f, 0.f, 0.f);
        if (slot < nslots && d.perm[slot] >= 0) xq = d.xq_s[slot];
        const float x = dim == 0 ? xq.x : (dim == 1 ? xq.y : xq.z);
        const float klh = dim == 0 ? pm.kl_h[0] : (dim == 1 ? pm.kl_h[1] : pm.kl_h[2]);
        const float kll = dim == 0 ? pm.kl_l[0] : (dim == 1 ? pm.kl_l[1] : pm.kl_l[2]);
        const int K = dim == 0 ? pm.K[0] : (dim == 1 ? pm.K[1] : pm.K[2]);
        int b;
        float w;
        if (pm.tri) mesh_coord_tri(xq, dim, pm, b, w);
        else mesh_coord(x, klh, kll, K, b, w);
        float th[P], dth[P];
        bspline_weights<P, DERIV>(w, th, dth);
#pragma unroll
        for (int j = 0; j < P; ++j) {
            st.w[at][dim][j] = th[j];
            if (DERIV) st.dw[at][dim][j] = dth[j];
        }
        st.base[at][dim] = b;
        if (dim == 0) st.q[at] = xq.w;
    }
    __syncthreads();
}

// Spread: lane c of an atom's group adds q th_x[a] th_y[b] th_z[c] to the
// mesh point (base_x - a, base_y - b, base_z - c) for all a, b.  With ENER
// also the self energy -f beta / sqrt(pi) sum q^2.  The P lanes of an atom
// hit P adjacent words of one mesh row, so each warp instruction's atomics
// reach the L2 as few sector operations.  (Summing a block's contributions
// in a shared-memory window first and adding the window with vector atomics
// was 1.8x slower, with four lanes per atom or with a warp per atom.)
template <int P, bool ENER>
__global__ void __launch_bounds__(PME_THREADS) k_pme_spread(const SysDev* __restrict__ sys, PmeDev pm,
                                                            double* __restrict__ acc) {
    pdl_wait();
    pdl_trigger();
    constexpr int LPA = pme_lanes(P);
    constexpr int APB = SplineTile<P, false>::APB;
    __shared__ SplineTile<P, false> st;
    const SysDev& d = sys[0];
    const int nslots = d.col_cl0[d.ncol] * CL;
    spline_tile<P, false>(d, pm, blockIdx.x * APB, nslots, st);
    const int at = threadIdx.x / LPA, c = threadIdx.x % LPA;
    const float q = st.q[at];
    const int K2 = pm.K[2];
    if (q != 0.f && (K2 & 1) == 0) {
        // Even z extent: the atom's P z points, zl .. zl + P - 1 (mod K2),
        // go out as 8-byte reductions of aligned pairs (2k, 2k + 1), which
        // never straddle a mesh row; lane c takes the c-th pair from zl
        // rounded down to even, and a pair half outside the atom's points
        // adds zero.  About 40% fewer L2 atomic operations than one per point.
        const int zl = wrap_down(st.base[at][2] - (P - 1), K2);
        const int lo = zl & 1;
        if (c < P / 2 + lo) {
            const int bx = st.base[at][0], by = st.base[at][1];
            const int d0 = 2 * c - lo;  // offset of the pair's first point from zl
            // the point at offset d from zl has the weight of index P - 1 - d
            const float w0 = d0 >= 0 ? st.w[at][2][P - 1 - d0] : 0.f;
            const float w1 = d0 + 1 < P ? st.w[at][2][P - 2 - d0] : 0.f;
            int iz0 = zl - lo + 2 * c;
            if (iz0 >= K2) iz0 -= K2;
            const long long iz = iz0;
            const float2 qz = make_float2(q * w0, q * w1);
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const long long ix = wrap_down(bx - a, pm.K[0]);
                const float wa = st.w[at][0][a];
                const float2 qa = make_float2(qz.x * wa, qz.y * wa);
#pragma unroll
                for (int b = 0; b < P; ++b) {
                    const long long iy = wrap_down(by - b, pm.K[1]);
                    const float wb = st.w[at][1][b];
                    atomicAdd(reinterpret_cast<float2*>(pm.Q + (ix * pm.K[1] + iy) * K2 + iz),
                              make_float2(qa.x * wb, qa.y * wb));
                }
            }
        }
    } else if (q != 0.f && c < P) {
        const int bx = st.base[at][0], by = st.base[at][1];
        const long long iz = wrap_down(st.base[at][2] - c, K2);
        const float qz = q * st.w[at][2][c];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const long long ix = wrap_down(bx - a, pm.K[0]);
            const float qa = qz * st.w[at][0][a];
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const long long iy = wrap_down(by - b, pm.K[1]);
                atomicAdd(pm.Q + (ix * pm.K[1] + iy) * K2 + iz, qa * st.w[at][1][b]);
            }
        }
    }
    if (ENER) {
        double q2[1] = {c == 0 ? (double)q * (double)q * pm.self_pre : 0.0};
        const int slot_e[1] = {ACC_ESELF};
        block_add<1>(q2, acc, slot_e);
    }
}

// Gather: the force on each atom from the potential mesh, the P lanes of its
// group summing over their z index and reducing by shuffles.  The mesh is
// read directly: neighbouring atoms of a block share most mesh lines in L1.
// (Copying the block's box of mesh points into shared memory first was 2x
// slower: the copy loads every point of the box from L2 once per block.)
template <int P>
__global__ void __launch_bounds__(PME_THREADS) k_pme_gather(const SysDev* __restrict__ sys, PmeDev pm) {
    pdl_wait();
    pdl_trigger();
    constexpr int LPA = pme_lanes(P);
    constexpr int APB = SplineTile<P, true>::APB;
    __shared__ SplineTile<P, true> st;
    const SysDev& d = sys[0];
    const int nslots = d.col_cl0[d.ncol] * CL;
    spline_tile<P, true>(d, pm, blockIdx.x * APB, nslots, st);
    const int at = threadIdx.x / LPA, c = threadIdx.x % LPA;
    const float q = st.q[at];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (q != 0.f && c < P) {
        const int bx = st.base[at][0], by = st.base[at][1];
        const long long iz = wrap_down(st.base[at][2] - c, pm.K[2]);
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const long long ix = wrap_down(bx - a, pm.K[0]);
            float rx = 0.f, ry = 0.f;
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const long long iy = wrap_down(by - b, pm.K[1]);
                const float ph = __ldg(pm.Q + (ix * pm.K[1] + iy) * pm.K[2] + iz);
                rx = fmaf(st.w[at][1][b], ph, rx);
                ry = fmaf(st.dw[at][1][b], ph, ry);
            }
            sx = fmaf(st.dw[at][0][a], rx, sx);  // sum dth_x th_y phi
            sy = fmaf(st.w[at][0][a], ry, sy);   // sum th_x dth_y phi
            sz = fmaf(st.w[at][0][a], rx, sz);   // sum th_x th_y phi
        }
        // F = -q (dE/du) M^T with M lower-triangular (diagonal K_d / L_d,
        // off-diagonals zero in a rectangular cell)
        const float g0 = st.w[at][2][c] * sx, g1 = st.w[at][2][c] * sy, g2 = st.dw[at][2][c] * sz;
        fx = -q * (pm.kl_h[0] * g0);
        fy = -q * fmaf(pm.mo_h[0], g0, pm.kl_h[1] * g1);
        fz = -q * fmaf(pm.mo_h[1], g0, fmaf(pm.mo_h[2], g1, pm.kl_h[2] * g2));
    }
#pragma unroll
    for (int off = LPA / 2; off > 0; off >>= 1) {
        fx += __shfl_xor_sync(FULL, fx, off);
        fy += __shfl_xor_sync(FULL, fy, off);
        fz += __shfl_xor_sync(FULL, fz, off);
    }
    if (c == 0 && q != 0.f) atomicAdd(d.f_s + blockIdx.x * APB + at, make_float4(fx, fy, fz, 0.f));
}

// Excluded-pair correction of the reciprocal sum: every excluded pair
// (i, j), each unordered pair once, minimum image of the rectangular box,
// V = -f qi qj erf(x) / r, x = beta r, F_i = (F/r) d, d = x_i - x_j,
// F/r = -f qi qj (erf(x) - 2 x / sqrt(pi) exp(-x^2)) / r^3.
//
// The pairs are bonded neighbours (x well below 1 in water), where both
// expressions cancel badly in floating point, and their forces are large
// (~5000 kJ/mol/nm) next to the total long-range force (~60), which the
// reciprocal force cancels down to: the pair terms need about 30 bits.
// With y = x^2 the Taylor series of erf and exp give, without cancellation,
//   erf(x) / r = 2 beta / sqrt(pi) (1 + e(y)),
//     e(y) = sum_{n>=1} (-1)^n y^n / (n! (2n + 1)),
//   F/r = -f qi qj 4 beta^3 / (3 sqrt(pi)) (1 + h(y)),
//     h(y) = sum_{n>=1} (-1)^n (3 / 2) 2 (n + 1) / ((n + 1)! (2n + 3)) y^n,
// whose small corrections e, h are summed in float32 (absolute error
// ~5e-8 for y < 1, ~2e-9 at the bond lengths of water).  The rest is
// double-float arithmetic on the float32 pipes: the exact difference d as
// hi + lo, the prefactors as hi + lo, the force components to ~2^-44.
// Pairs with y >= 1 (exclusions across more than 1 / beta, rare) take the
// float64 library erf and exp.  One thread per atom.
__device__ __forceinline__ float excl_series_e(float y) {
    float t = (float)(-1.0 / 76204800.0);          // n = 10 ... 1, Horner in y
    t = fmaf(t, y, (float)(1.0 / 6894720.0));
    t = fmaf(t, y, (float)(-1.0 / 685440.0));
    t = fmaf(t, y, (float)(1.0 / 75600.0));
    t = fmaf(t, y, (float)(-1.0 / 9360.0));
    t = fmaf(t, y, (float)(1.0 / 1320.0));
    t = fmaf(t, y, (float)(-1.0 / 216.0));
    t = fmaf(t, y, (float)(1.0 / 42.0));
    t = fmaf(t, y, (float)(-1.0 / 10.0));
    t = fmaf(t, y, (float)(1.0 / 3.0));
    return -y * t;  // -y/3 + y^2/10 - ...
}
__device__ __forceinline__ float excl_series_h(float y) {
    // coefficients (3/2) 2(n+1) / ((n+1)! (2n+3)), n = 1..12
    float t = (float)(1.0 / 4311014400.0);                        // n = 12
    t = fmaf(t, y, (float)(-1.0 / 332640000.0));                  // n = 11
    t = fmaf(t, y, (float)(1.0 / 27820800.0));                    // n = 10
    t = fmaf(t, y, (float)(-1.0 / 2540160.0));                    // n = 9
    t = fmaf(t, y, (float)(1.0 / 255360.0));                      // n = 8
    t = fmaf(t, y, (float)(-1.0 / 28560.0));                      // n = 7
    t = fmaf(t, y, (float)(1.0 / 3600.0));                        // n = 6
    t = fmaf(t, y, (float)(-1.0 / 520.0));                        // n = 5
    t = fmaf(t, y, (float)(1.0 / 88.0));                          // n = 4
    t = fmaf(t, y, (float)(-1.0 / 18.0));                         // n = 3
    t = fmaf(t, y, (float)(3.0 / 14.0));                          // n = 2
    t = fmaf(t, y, (float)(-0.6));                                // n = 1
    return y * t;
}

// (h, l) -= v for a double-float and a float v, error-free but for the
// rounding of the low part
__device__ __forceinline__ void sub_df(float& h, float& l, float v) {
    float t, e;
    two_sum(h, -v, t, e);
    fast_two_sum(t, e + l, h, l);
}

// a + b for double-floats (hi, lo), renormalised
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    fast_two_sum(s, e, sh, sl);
}

template <bool ENER, bool VIR>
__global__ void __launch_bounds__(PME_THREADS) k_excl_ewald(const SysDev* __restrict__ sys, PmeDev pm,
                                                            double* __restrict__ acc) {
    pdl_wait();
    pdl_trigger();
    const SysDev& d = sys[0];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    float eh = 0.f, el = 0.f;  // energy of this thread's pairs, hi + lo
    double e_far = 0.0;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (a < d.natoms && d.excl_index) {
        const int sa = d.iperm[a];
        const float4 xa = d.xq_s[sa];
        const float L[3] = {d.L[0], d.L[1], d.L[2]};
        const float T[3] = {d.T[0], d.T[1], d.T[2]};  // bx, cx, cy
        const float iL[3] = {1.f / d.L[0], 1.f / d.L[1], 1.f / d.L[2]};
        float fh[3] = {0.f, 0.f, 0.f}, fl[3] = {0.f, 0.f, 0.f};
        for (int k = d.excl_index[a]; k < d.excl_index[a + 1]; ++k) {
            const int b = d.excl_atoms[k];
            if (b <= a) continue;
            const int sb = d.iperm[b];
            const float4 xb = d.xq_s[sb];
            if (xa.w == 0.f || xb.w == 0.f) continue;
            // d = x_a - x_b minus lattice vectors, exactly as hi + lo: z by c,
            // then y by b, then x by a (the c and b rows carry the cell's
            // off-diagonal components cx, cy, bx, zero in a rectangular box)
            const float xav[3] = {xa.x, xa.y, xa.z}, xbv[3] = {xb.x, xb.y, xb.z};
            float dh[3], dl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) two_sum(xav[c], -xbv[c], dh[c], dl[c]);
            const float sz = rintf(dh[2] * iL[2]);
            if (sz != 0.f) {
                sub_df(dh[2], dl[2], sz * L[2]);
                if (T[2] != 0.f) sub_df(dh[1], dl[1], sz * T[2]);
                if (T[1] != 0.f) sub_df(dh[0], dl[0], sz * T[1]);
            }
            const float sy = rintf(dh[1] * iL[1]);
            if (sy != 0.f) {
                sub_df(dh[1], dl[1], sy * L[1]);
                if (T[0] != 0.f) sub_df(dh[0], dl[0], sy * T[0]);
            }
            const float sx = rintf(dh[0] * iL[0]);
            if (sx != 0.f) sub_df(dh[0], dl[0], sx * L[0]);
            const float r2 = dh[0] * dh[0] + dh[1] * dh[1] + dh[2] * dh[2];
            const float y = pm.beta2 * r2;
            // f qi qj as hi + lo
            float qh, ql, fqh, fql;
            two_prod(xa.w, xb.w, qh, ql);
            dd_mul(pm.fq_h, pm.fq_l, qh, ql, fqh, fql);
            float frh, frl;  // F/r
            if (y < 1.f) {
                float oh, ol;
                two_sum(1.f, excl_series_h(y), oh, ol);
                float th, tl;
                dd_mul(pm.kf_h, pm.kf_l, oh, ol, th, tl);
                dd_mul(fqh, fql, th, tl, frh, frl);
                frh = -frh;
                frl = -frl;
                if (ENER) {
                    two_sum(1.f, excl_series_e(y), oh, ol);
                    dd_mul(pm.ke_h, pm.ke_l, oh, ol, th, tl);
                    float ph, pl;
                    dd_mul(fqh, fql, th, tl, ph, pl);
                    df_add(eh, el, -ph, -pl, eh, el);
                }
            } else {
                const double r2d = (double)dh[0] * dh[0] + (double)dh[1] * dh[1] + (double)dh[2] * dh[2];
                const double r = sqrt(r2d);
                const double qq = (double)fqh + (double)fql;
                const double ef = erf(pm.beta * r);
                const double fr = qq * ((double)pm.ke_h * exp(-pm.beta * pm.beta * r2d) - ef / r) / r2d;
                frh = (float)fr;
                frl = (float)(fr - (double)frh);
                if (ENER) e_far -= qq * ef / r;
            }
            float gh[3], gl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dd_mul(frh, frl, dh[c], dl[c], gh[c], gl[c]);
                df_add(fh[c], fl[c], gh[c], gl[c], fh[c], fl[c]);
            }
            if (VIR) {
                v[0] += frh * dh[0] * dh[0];
                v[1] += frh * dh[1] * dh[1];
                v[2] += frh * dh[2] * dh[2];
                v[3] += frh * dh[0] * dh[1];
                v[4] += frh * dh[0] * dh[2];
                v[5] += frh * dh[1] * dh[2];
            }
            atomicAdd(d.f_s + sb, make_float4(-(gh[0] + gl[0]), -(gh[1] + gl[1]), -(gh[2] + gl[2]), 0.f));
        }
        const float ox = fh[0] + fl[0], oy = fh[1] + fl[1], oz = fh[2] + fl[2];
        if (ox != 0.f || oy != 0.f || oz != 0.f) atomicAdd(d.f_s + sa, make_float4(ox, oy, oz, 0.f));
    }
    if (ENER) {
        double ee[1] = {(double)eh + (double)el + e_far};
        const int slot_e[1] = {ACC_EEXCL};
        block_add<1>(ee, acc, slot_e);
    }
    if (VIR) {
        double vv[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) vv[c] = (double)v[c];
        const int slot_v[6] = {ACC_VXX, ACC_VYY, ACC_VZZ, ACC_VXY, ACC_VXZ, ACC_VYZ};
        block_add<6>(vv, acc, slot_v);
    }
}

// Upper bounds (two buffers), for the size check of a mesh.
size_t strided_smem(int n) { return 2 * (size_t)tile_lines(n) * line_stride(n) * sizeof(float2); }
size_t z_smem(int n) { return 2 * (size_t)z_pairs(n) * line_stride(n) * sizeof(float2); }
// What each pass launches with: one buffer where every stage has at most one
// butterfly per thread, and for the strided pass also with at most two
// stages (global -> shared -> global); else two.
size_t strided_pass_smem(const FftAxis& ax) {
    const int nb = (one_buffer(ax, tile_lines(ax.n)) || ax.nst <= 2) ? 1 : 2;
    return nb * (size_t)tile_lines(ax.n) * line_stride(ax.n) * sizeof(float2);
}
size_t x_pass_smem(const FftAxis& ax) {
    return (one_buffer(ax, tile_lines(ax.n)) ? 1 : 2) * (size_t)tile_lines(ax.n) * line_stride(ax.n) * sizeof(float2);
}
size_t z_pass_smem(const FftAxis& ax) {
    return (one_buffer(ax, z_pairs(ax.n)) ? 1 : 2) * (size_t)z_pairs(ax.n) * line_stride(ax.n) * sizeof(float2);
}

template <int P>
cudaError_t launch_spread_p(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags, cudaStream_t st) {
    const size_t nq = (size_t)pm.K[0] * pm.K[1] * pm.K[2];
    cudaError_t e = cudaMemsetAsync(pm.Q, 0, sizeof(float) * nq, st);
    if (e != cudaSuccess) return e;
    constexpr int APB = PME_THREADS / pme_lanes(P);
    const unsigned blocks = (unsigned)(((long long)p.tot_clcap * CL + APB - 1) / APB);
    return (flags & NB_F_ENERGY) ? launch_pdl(k_pme_spread<P, true>, blocks, PME_THREADS, 0, st, p.d_sys, pm, acc)
                                 : launch_pdl(k_pme_spread<P, false>, blocks, PME_THREADS, 0, st, p.d_sys, pm, acc);
}

template <int P>
cudaError_t launch_gather_p(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags, cudaStream_t st) {
    constexpr int APB = PME_THREADS / pme_lanes(P);
    const unsigned blocks = (unsigned)(((long long)p.tot_clcap * CL + APB - 1) / APB);
    cudaError_t e = launch_pdl(k_pme_gather<P>, blocks, PME_THREADS, 0, st, p.d_sys, pm);
    if (e != cudaSuccess) return e;
    const bool en = flags & NB_F_ENERGY, vi = flags & NB_F_VIRIAL;
    const unsigned eblocks = (unsigned)((p.tot_atoms + PME_THREADS - 1) / PME_THREADS);
    if (en && vi) return launch_pdl(k_excl_ewald<true, true>, eblocks, PME_THREADS, 0, st, p.d_sys, pm, acc);
    if (en) return launch_pdl(k_excl_ewald<true, false>, eblocks, PME_THREADS, 0, st, p.d_sys, pm, acc);
    if (vi) return launch_pdl(k_excl_ewald<false, true>, eblocks, PME_THREADS, 0, st, p.d_sys, pm, acc);
    return launch_pdl(k_excl_ewald<false, false>, eblocks, PME_THREADS, 0, st, p.d_sys, pm, acc);
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

cudaError_t launch_pme_spread(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags,
                              cudaStream_t st) {
    switch (pm.order) {
        case 4: return launch_spread_p<4>(p, pm, acc, flags, st);
        case 6: return launch_spread_p<6>(p, pm, acc, flags, st);
        default: return launch_spread_p<8>(p, pm, acc, flags, st);
    }
}

cudaError_t launch_pme_gather(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags,
                              cudaStream_t st) {
    switch (pm.order) {
        case 4: return launch_gather_p<4>(p, pm, acc, flags, st);
        case 6: return launch_gather_p<6>(p, pm, acc, flags, st);
        default: return launch_gather_p<8>(p, pm, acc, flags, st);
    }
}

cudaError_t launch_pme_fft(const PlanLaunch& p, const PmeDev& pm, double* acc, unsigned flags, cudaStream_t st) {
    (void)p;
    const bool ev = flags & (NB_F_ENERGY | NB_F_VIRIAL);
    const long long zlines = (long long)pm.K[0] * pm.K[1];
    const unsigned zblocks = (unsigned)((zlines + 2 * z_pairs(pm.K[2]) - 1) / (2 * z_pairs(pm.K[2])));
    cudaError_t e = launch_pdl(k_fft_z_r2c, zblocks, FFT_THREADS, z_pass_smem(pm.ax[2]), st, pm, zlines);
    if (e != cudaSuccess) return e;
    // y pass: a 2D grid (z tiles, x planes)
    const int ty = tile_lines(pm.K[1]);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((pm.Kzh + ty - 1) / ty, pm.K[0]);
    cfg.blockDim = dim3(FFT_THREADS);
    cfg.dynamicSmemBytes = strided_pass_smem(pm.ax[1]);
    cfg.stream = st;
    const long long es_y = pm.Kzh, os_y = (long long)pm.K[1] * pm.Kzh;
    e = cudaLaunchKernelEx(&cfg, k_fft_strided<false>, pm, 1, pm.S, pm.Kzh, es_y, os_y);
    if (e != cudaSuccess) return e;
    const int tx = tile_lines(pm.K[0]);
    const unsigned xblocks = (unsigned)(((long long)pm.K[1] * pm.Kzh + tx - 1) / tx);
    e = ev ? launch_pdl(k_fft_x_solve<true>, xblocks, FFT_THREADS, x_pass_smem(pm.ax[0]), st, pm, acc)
           : launch_pdl(k_fft_x_solve<false>, xblocks, FFT_THREADS, x_pass_smem(pm.ax[0]), st, pm, acc);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, k_fft_strided<true>, pm, 1, pm.S, pm.Kzh, es_y, os_y);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_fft_z_c2r, zblocks, FFT_THREADS, z_pass_smem(pm.ax[2]), st, pm, zlines);
}

}  // namespace nbgb
