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
    if (prec == DWF_FP64)
        k_force<double, double, double><<<grid, 256, 0, s>>>(a);
    else
        k_force<float, float, float><<<grid, 256, 0, s>>>(a);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

}  // namespace dwf
