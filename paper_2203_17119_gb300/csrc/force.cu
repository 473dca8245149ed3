// Link force of the fermion bilinear Re <X, D Y>: the insertion of delta D
// between two solved fields that the DD-HMC forces of Sec. 2.3 (the
// variations of R^-1 = P - P D^-1 D_partialbar and of the two-flavour and
// ratio actions built from it) consist of.
//
// D depends on the links only through the hop of D_W = (4 - M5) - Dh / 2 and
// D = D_W B + 1 - S5 with B = b5 + c5 S5, so with Z = B Y the link U_mu(x)
// enters Re <X, D Y> through
//     -1/2 Re { X(x)^+ (1 - g_mu) U Z(x + mu) + X(x + mu)^+ (1 + g_mu) U^+ Z(x) }.
// Both projectors have rank two: with h = the upper half spinor of (1 - g_mu) X(x)
// and g that of (1 - g_mu) Z(x + mu) (and h', g' of (1 + g_mu) applied to
// X(x + mu), Z(x)), the colour matrix
//     M = sum_{lanes, k = 0, 1} g_k h_k^+ + (g'_k h'_k^+)^+
// gives the change under U -> U + i eps H U as Re tr[i eps H U M] (times -1/2),
// and the force is F_mu(x) = -1/2 TA(U_mu(x) M), TA the traceless
// anti-Hermitian part: d/d eps Re <X, D(exp(i eps H) U) Y> = Re tr[i H F].
// In the chiral basis g_mu = [[0, A], [A^+, 0]] with A = -i sigma_mu (mu < 3)
// or 1 (mu = 3); the upper half of (1 -+ g_mu) v is v_up -+ A v_low.
//
// Work split: four threads per site (of both parities) share the site's
// lanes (lane = rhs * Ls + s, thread t takes lanes t, t + 4, ...); for each
// direction the four partial matrices are summed by shuffles and thread mu
// keeps M_mu, so after the (unrolled) direction loop thread t writes the force
// of link t of its site.  Each thread reads its own site's rows once per
// direction (L1 hits after the first) and the neighbour's rows once.
#include <algorithm>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

namespace {

template <class R>
struct Cx {
    R re, im;
};

template <class S, class R>
__device__ __forceinline__ Cx<R> ld(const S* p);
template <>
__device__ __forceinline__ Cx<float> ld<float, float>(const float* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return Cx<float>{v.x, v.y};
}
template <>
__device__ __forceinline__ Cx<double> ld<double, double>(const double* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return Cx<double>{v.x, v.y};
}

// upper half spinor of (1 + SG g_mu) v from the four spin rows v[4] (one colour)
template <int MU, int SG, class R>
__device__ __forceinline__ void proj(const Cx<R> (&v)[4], Cx<R> (&o)[2]) {
    // A v_low: mu 0: (-i v3, -i v2); mu 1: (-v3, v2); mu 2: (-i v2, i v3); mu 3: (v2, v3)
    Cx<R> a0, a1;
    if (MU == 0) { a0 = {v[3].im, -v[3].re}; a1 = {v[2].im, -v[2].re}; }
    if (MU == 1) { a0 = {-v[3].re, -v[3].im}; a1 = {v[2].re, v[2].im}; }
    if (MU == 2) { a0 = {v[2].im, -v[2].re}; a1 = {-v[3].im, v[3].re}; }
    if (MU == 3) { a0 = v[2]; a1 = v[3]; }
    o[0] = {v[0].re + SG * a0.re, v[0].im + SG * a0.im};
    o[1] = {v[1].re + SG * a1.re, v[1].im + SG * a1.im};
}

// half spinors (2 spins x 3 colours) of one lane of a site's rows
template <int MU, int SG, class S, class R>
__device__ __forceinline__ void half(const S* __restrict__ base, int N5, int lane, Cx<R> (&o)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Cx<R> v[4];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) v[sp] = ld<S, R>(base + ((sp * 3 + c) * N5 + lane) * 2);
        Cx<R> p[2];
        proj<MU, SG, R>(v, p);
        o[0][c] = p[0];
        o[1][c] = p[1];
    }
}

struct ForceArgs {
    const void* X[2];        // per parity: cb field of X
    const void* Z[2];        // per parity: cb field of Z = B Y
    const void* links[2];    // per parity: [site][8][9] complex, k < 4 forward U_mu(x)
    const int* nbr[2];       // per parity: [site][8] neighbour in the other parity
    const int64_t* gidx[2];  // per parity: [site][8], k < 4: canonical link index lex * 4 + mu
    double* out;             // canonical [lex][mu][3][3] complex
    int64_t ns0, ns;         // sites of parity 0, total sites
    int N5;
    int accumulate;
    int use_box;
    int L[4], org[4], ext[4];
};

__device__ __forceinline__ bool in_box(const ForceArgs& a, const int* x) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int d = (x[mu] - a.org[mu]) % a.L[mu];
        if (d < 0) d += a.L[mu];
        if (d >= a.ext[mu]) return false;
    }
    return true;
}

// F = -1/2 TA(U_t(x) M) for link t of site i of parity p, written to (or
// added into) the canonical force array; links outside the active box get 0.
template <class SL, class R>
__device__ __forceinline__ void link_out(const ForceArgs& a, int p, int64_t i, int t, const Cx<R> (&Mt)[3][3]) {
    const SL* U = reinterpret_cast<const SL*>(a.links[p]) + (i * 8 + t) * 18;
    Cx<R> F[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R re = 0, im = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const R ur = (R)U[(r * 3 + k) * 2], ui = (R)U[(r * 3 + k) * 2 + 1];
                re += ur * Mt[k][c].re - ui * Mt[k][c].im;
                im += ur * Mt[k][c].im + ui * Mt[k][c].re;
            }
            F[r][c] = Cx<R>{re, im};
        }
    const int64_t g = a.gidx[p][i * 8 + t];   // lex * 4 + mu
    if (g < 0) return;
    bool active = true;
    if (a.use_box) {
        const int64_t lex = g >> 2;
        int x[4] = {(int)(lex % a.L[0]), (int)((lex / a.L[0]) % a.L[1]),
                    (int)((lex / ((int64_t)a.L[0] * a.L[1])) % a.L[2]),
                    (int)(lex / ((int64_t)a.L[0] * a.L[1] * a.L[2]))};
        active = in_box(a, x);
        x[t] = (x[t] + 1) % a.L[t];
        active = active && in_box(a, x);
    }
    double* o = a.out + g * 18;
    // -1/2 TA(F) = -1/4 (F - F^+) + tr(F - F^+)/12, in the arithmetic precision
    const R tr = (F[0][0].im + F[1][1].im + F[2][2].im) * (R)(1.0 / 3.0);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R re = (R)-0.25 * (F[r][c].re - F[c][r].re);
            R im = (R)-0.25 * (F[r][c].im + F[c][r].im);
            if (r == c) im += (R)0.5 * tr;
            if (!active) re = im = (R)0;
            if (a.accumulate) {
                o[(r * 3 + c) * 2] += re;
                o[(r * 3 + c) * 2 + 1] += im;
            } else {
                o[(r * 3 + c) * 2] = re;
                o[(r * 3 + c) * 2 + 1] = im;
            }
        }
}

template <int MU, class S, class R>
__device__ __forceinline__ void dir_matrix(const ForceArgs& a, int p, int64_t i, int t, Cx<R> (&M)[3][3]) {
    const int q = 1 - p;
    const int n = a.nbr[p][i * 8 + MU];
    const int64_t site_el = (int64_t)12 * a.N5 * 2;
    const S* Xx = reinterpret_cast<const S*>(a.X[p]) + i * site_el;
    const S* Zx = reinterpret_cast<const S*>(a.Z[p]) + i * site_el;
    const S* Xn = reinterpret_cast<const S*>(a.X[q]) + (int64_t)(n < 0 ? 0 : n) * site_el;
    const S* Zn = reinterpret_cast<const S*>(a.Z[q]) + (int64_t)(n < 0 ? 0 : n) * site_el;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r][c] = Cx<R>{(R)0, (R)0};
    // (a cut neighbour adds nothing; the shuffles below still run on every lane)
    const int lend = n < 0 ? 0 : a.N5;
    for (int l = t; l < lend; l += 4) {
        Cx<R> g[2][3], h[2][3];
        // g h^+ with g = (1 - g_mu) Z(x + mu), h = (1 - g_mu) X(x)
        half<MU, -1, S, R>(Zn, a.N5, l, g);
        half<MU, -1, S, R>(Xx, a.N5, l, h);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    M[r][c].re += g[k][r].re * h[k][c].re + g[k][r].im * h[k][c].im;
                    M[r][c].im += g[k][r].im * h[k][c].re - g[k][r].re * h[k][c].im;
                }
        // (g' h'^+)^+ = h' g'^+ with g' = (1 + g_mu) Z(x), h' = (1 + g_mu) X(x + mu)
        half<MU, 1, S, R>(Zx, a.N5, l, g);
        half<MU, 1, S, R>(Xn, a.N5, l, h);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    M[r][c].re += h[k][r].re * g[k][c].re + h[k][r].im * g[k][c].im;
                    M[r][c].im += h[k][r].im * g[k][c].re - h[k][r].re * g[k][c].im;
                }
    }
    // sum over the four threads of the site
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                M[r][c].re += __shfl_xor_sync(0xffffffffu, M[r][c].re, o);
                M[r][c].im += __shfl_xor_sync(0xffffffffu, M[r][c].im, o);
            }
}

template <class S, class SL, class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_force(const ForceArgs a) {
    const int64_t nthreads = a.ns * 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every thread of a warp runs the same number of iterations (the
    // shuffles need all 32 lanes); threads past the end compute on a clamped
    // site and store nothing
    const int64_t span = (nthreads + stride - 1) / stride * stride;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < span; id += stride) {
        const bool live = id < nthreads;
        const int64_t site = live ? id >> 2 : a.ns - 1;
        const int t = (int)(id & 3);
        const int p = site >= a.ns0 ? 1 : 0;
        const int64_t i = site - (p ? a.ns0 : 0);
        Cx<R> M[3][3], Mt[3][3];
        dir_matrix<0, S, R>(a, p, i, t, M);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Mt[r][c] = M[r][c];
#define DWF_FORCE_DIR(MU)                                                         \
    dir_matrix<MU, S, R>(a, p, i, t, M);                                          \
    if (t == MU) {                                                                \
        _Pragma("unroll") for (int r = 0; r < 3; ++r)                             \
            _Pragma("unroll") for (int c = 0; c < 3; ++c) Mt[r][c] = M[r][c];     \
    }
        DWF_FORCE_DIR(1)
        DWF_FORCE_DIR(2)
        DWF_FORCE_DIR(3)
#undef DWF_FORCE_DIR
        if (!live) continue;
        link_out<SL, R>(a, p, i, t, Mt);
    }
}



// ---------------------------------------------------------------------------
// FP32, N5 <= 16: sixteen threads per site (one lane each, lanes past N5
// idle), two sites per warp.  A site's own X and Z rows are loaded once into
// registers and serve all four directions; each row load of a warp is two
// contiguous runs of N5 complex.  Per direction the 18 reals of M are summed
// over the 16 lanes by a reduce-scatter (each halving step keeps half the
// values and exchanges the other half: 9 + 5 + 3 + 2 shuffles), the lanes
// park their sums in shared memory, and nine threads form U M and its
// traceless anti-Hermitian part.
constexpr int FW_THREADS = 256;

// one halving step of the reduce-scatter: n values (n even) -> n / 2
template <int N>
__device__ __forceinline__ void rs_step(float (&v)[N], int (&idx)[N], int bit) {
    constexpr int H = N / 2;
    const bool hi = (threadIdx.x & bit) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float mine = hi ? v[H + i] : v[i];
        const float other = hi ? v[i] : v[H + i];
        v[i] = mine + __shfl_xor_sync(0xffffffffu, other, bit);
        idx[i] = hi ? idx[H + i] : idx[i];
    }
}

template <int SRC, int DST>
__device__ __forceinline__ void rs_pad(const float (&a)[SRC], const int (&ia)[SRC], float (&b)[DST], int (&ib)[DST]) {
#pragma unroll
    for (int i = 0; i < DST; ++i) {
        b[i] = i < SRC ? a[i < SRC ? i : 0] : 0.f;
        ib[i] = i < SRC ? ia[i < SRC ? i : 0] : -1;
    }
}

// the upper half spinor of (1 + SG g_mu) v of one lane, all three colours
template <int MU, int SG>
__device__ __forceinline__ void half_reg(const float2 (&v)[12], Cx<float> (&o)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Cx<float> w[4], pr[2];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) w[sp] = Cx<float>{v[sp * 3 + c].x, v[sp * 3 + c].y};
        proj<MU, SG, float>(w, pr);
        o[0][c] = pr[0];
        o[1][c] = pr[1];
    }
}

template <int MU>
__device__ __forceinline__ void dir_lane(const ForceArgs& a, int p, int64_t i, int l, bool on, bool store,
                                         const float2 (&xo)[12], const float2 (&zo)[12], float* sM, float* sF,
                                         int g16) {
    const int N5 = a.N5;
    const int n = a.nbr[p][i * 8 + MU];
    float m[18];
#pragma unroll
    for (int e = 0; e < 18; ++e) m[e] = 0.f;
    if (on && n >= 0) {
        const float2* Xn = reinterpret_cast<const float2*>(a.X[1 - p]) + (int64_t)n * 12 * N5 + l;
        const float2* Zn = reinterpret_cast<const float2*>(a.Z[1 - p]) + (int64_t)n * 12 * N5 + l;
        float2 xn[12], zn[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            xn[c] = __ldg(Xn + c * N5);
            zn[c] = __ldg(Zn + c * N5);
        }
        Cx<float> g[2][3], h[2][3];
        half_reg<MU, -1>(zn, g);   // g = (1 - g_mu) Z(x + mu)
        half_reg<MU, -1>(xo, h);   // h = (1 - g_mu) X(x)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    m[(r * 3 + c) * 2] += g[k][r].re * h[k][c].re + g[k][r].im * h[k][c].im;
                    m[(r * 3 + c) * 2 + 1] += g[k][r].im * h[k][c].re - g[k][r].re * h[k][c].im;
                }
        half_reg<MU, 1>(zo, g);    // g' = (1 + g_mu) Z(x)
        half_reg<MU, 1>(xn, h);    // h' = (1 + g_mu) X(x + mu)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    m[(r * 3 + c) * 2] += h[k][r].re * g[k][c].re + h[k][r].im * g[k][c].im;
                    m[(r * 3 + c) * 2 + 1] += h[k][r].im * g[k][c].re - h[k][r].re * g[k][c].im;
                }
    }
    // reduce-scatter over the 16 lanes of the site: 18 -> 9 -> 5 -> 3 -> 2
    int id18[18];
#pragma unroll
    for (int e = 0; e < 18; ++e) id18[e] = e;
    rs_step<18>(m, id18, 8);
    float v10[10];
    int i10[10];
    {
        float t9[9];
        int j9[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) { t9[e] = m[e]; j9[e] = id18[e]; }
        rs_pad<9, 10>(t9, j9, v10, i10);
    }
    rs_step<10>(v10, i10, 4);
    float v6[6];
    int i6[6];
    {
        float t5[5];
        int j5[5];
#pragma unroll
        for (int e = 0; e < 5; ++e) { t5[e] = v10[e]; j5[e] = i10[e]; }
        rs_pad<5, 6>(t5, j5, v6, i6);
    }
    rs_step<6>(v6, i6, 2);
    float v4[4];
    int i4[4];
    {
        float t3[3];
        int j3[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) { t3[e] = v6[e]; j3[e] = i6[e]; }
        rs_pad<3, 4>(t3, j3, v4, i4);
    }
    rs_step<4>(v4, i4, 1);
    // park the two sums of this lane, then nine lanes form F = U M and TA(F)
    float* Mg = sM + g16 * 18;
    float* Fg = sF + g16 * 18;
#pragma unroll
    for (int e = 0; e < 2; ++e)
        if (i4[e] >= 0) Mg[i4[e]] = v4[e];
    __syncwarp();
    const int lq = threadIdx.x & 15;
    if (lq < 9) {
        const int r = lq / 3, c = lq % 3;
        const float* U = reinterpret_cast<const float*>(a.links[p]) + (i * 8 + MU) * 18;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float ur = U[(r * 3 + k) * 2], ui = U[(r * 3 + k) * 2 + 1];
            const float mr = Mg[(k * 3 + c) * 2], mi = Mg[(k * 3 + c) * 2 + 1];
            re += ur * mr - ui * mi;
            im += ur * mi + ui * mr;
        }
        Fg[lq * 2] = re;
        Fg[lq * 2 + 1] = im;
    }
    __syncwarp();
    if (lq < 9 && store) {   // a cut link (n < 0) has M = 0 and gets F = 0
        const int r = lq / 3, c = lq % 3;
        const int64_t gl = a.gidx[p][i * 8 + MU];
        if (gl >= 0) {
            bool act = true;
            if (a.use_box) {
                const int64_t lex = gl >> 2;
                int x[4] = {(int)(lex % a.L[0]), (int)((lex / a.L[0]) % a.L[1]),
                            (int)((lex / ((int64_t)a.L[0] * a.L[1])) % a.L[2]),
                            (int)(lex / ((int64_t)a.L[0] * a.L[1] * a.L[2]))};
                act = in_box(a, x);
                x[MU] = (x[MU] + 1) % a.L[MU];
                act = act && in_box(a, x);
            }
            const float tr = (Fg[1] + Fg[(1 * 3 + 1) * 2 + 1] + Fg[(2 * 3 + 2) * 2 + 1]) * (1.f / 3.f);
            float re = -0.25f * (Fg[(r * 3 + c) * 2] - Fg[(c * 3 + r) * 2]);
            float im = -0.25f * (Fg[(r * 3 + c) * 2 + 1] + Fg[(c * 3 + r) * 2 + 1]);
            if (r == c) im += 0.5f * tr;
            if (!act) re = im = 0.f;
            double* o = a.out + gl * 18 + (r * 3 + c) * 2;
            if (a.accumulate) {
                o[0] += re;
                o[1] += im;
            } else {
                o[0] = re;
                o[1] = im;
            }
        }
    }
    __syncwarp();   // Mg, Fg are reused by the next direction
}

__global__ void __launch_bounds__(FW_THREADS, 2) k_force_w16(const ForceArgs a) {
    __shared__ float sM[FW_THREADS / 16 * 18];
    __shared__ float sF[FW_THREADS / 16 * 18];
    const int g16 = threadIdx.x >> 4;          // site group in the block
    const int l = threadIdx.x & 15;            // lane of the site
    const bool on = l < a.N5;
    const int64_t ngroups = (int64_t)gridDim.x * (FW_THREADS / 16);
    // the two groups of a warp run the same number of iterations (shuffles)
    const int64_t span = (a.ns + ngroups - 1) / ngroups * ngroups;
    for (int64_t site0 = blockIdx.x * (int64_t)(FW_THREADS / 16) + g16; site0 < span; site0 += ngroups) {
        const int64_t site = site0 < a.ns ? site0 : a.ns - 1;
        const int p = site >= a.ns0 ? 1 : 0;
        const int64_t i = site - (p ? a.ns0 : 0);
        float2 xo[12], zo[12];
        if (on) {
            const float2* Xs = reinterpret_cast<const float2*>(a.X[p]) + i * 12 * a.N5 + l;
            const float2* Zs = reinterpret_cast<const float2*>(a.Z[p]) + i * 12 * a.N5 + l;
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                xo[c] = __ldg(Xs + c * a.N5);
                zo[c] = __ldg(Zs + c * a.N5);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 12; ++c) xo[c] = zo[c] = make_float2(0.f, 0.f);
        }
        // a clamped site past the end only joins the shuffles and stores nothing
        const bool store = site0 < a.ns;
        dir_lane<0>(a, p, i, l, on, store, xo, zo, sM, sF, g16);
        dir_lane<1>(a, p, i, l, on, store, xo, zo, sM, sF, g16);
        dir_lane<2>(a, p, i, l, on, store, xo, zo, sM, sF, g16);
        dir_lane<3>(a, p, i, l, on, store, xo, zo, sM, sF, g16);
    }
}

}  // namespace

dwf_status force_bilinear(dwf_handle* h, double* out, const void* X, const void* Y, dwf_prec prec, int nrhs,
                          const dwf_box* active, int accumulate, cudaStream_t s) {
    if (h->dirichlet) {
        set_error("force: needs a whole-lattice handle (fields supported in a box give its Dirichlet force)");
        return DWF_ERR_ARG;
    }
    if (out == nullptr || X == nullptr || Y == nullptr || nrhs < 1 || nrhs > h->nrhs_max ||
        (prec != DWF_FP64 && prec != DWF_FP32)) {
        set_error("force: bad arguments (device fields, 1 <= nrhs <= nrhs_max, FP64 or FP32)");
        return DWF_ERR_ARG;
    }
    if (!h->have_gauge) {
        set_error("force: no gauge field loaded");
        return DWF_ERR_ARG;
    }
    ForceArgs a{};
    for (int mu = 0; mu < 4; ++mu) {
        a.L[mu] = h->p.dims[mu];
        if (active) {
            if (active->extent[mu] < 1 || active->extent[mu] > a.L[mu]) {
                set_error("force: active box extent out of range");
                return DWF_ERR_ARG;
            }
            a.org[mu] = active->origin[mu];
            a.ext[mu] = active->extent[mu];
        }
    }
    a.use_box = active != nullptr;
    const size_t ps = prec_size(prec) * 2;
    const size_t off1 = cb_elems(h, 0, nrhs) * ps;
    a.X[0] = X;
    a.X[1] = (const char*)X + off1;
    if (h->p.c5 == 0.0 && h->p.b5 == 1.0) {   // Shamir: B = 1
        a.Z[0] = Y;
        a.Z[1] = (const char*)Y + off1;
    } else {
        DWF_TRY(op_local(h, L_B, h->d_tmp, Y, nullptr, 0, 0, prec, prec, prec, nrhs, 1.0, nullptr, s));
        DWF_TRY(op_local(h, L_B, h->d_tmp2, (const char*)Y + off1, nullptr, 1, 0, prec, prec, prec, nrhs, 1.0,
                         nullptr, s));
        a.Z[0] = h->d_tmp;
        a.Z[1] = h->d_tmp2;
    }
    for (int p = 0; p < 2; ++p) {
        a.links[p] = h->d_links[prec == DWF_FP64 ? 0 : 1][p];
        a.nbr[p] = h->d_nbr[p];
        a.gidx[p] = h->d_link_src[p];
    }
    a.out = out;
    a.ns0 = h->nsite[0];
    a.ns = h->nsite[0] + h->nsite[1];
    a.N5 = h->p.Ls * nrhs;
    a.accumulate = accumulate;
    const int64_t nthreads = a.ns * 4;
    const int64_t want = (nthreads + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 8));
    if (prec == DWF_FP64) {
        k_force<double, double, double><<<grid, 256, 0, s>>>(a);
    } else if (a.N5 <= 16) {
        const int64_t wgroups = (a.ns + FW_THREADS / 16 - 1) / (FW_THREADS / 16);
        const int wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgroups, 152 * 8));
        k_force_w16<<<wgrid, FW_THREADS, 0, s>>>(a);
    } else {
        k_force<float, float, float><<<grid, 256, 0, s>>>(a);
    }
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

}  // namespace dwf
