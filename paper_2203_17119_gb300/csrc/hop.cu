// Wilson hop over all fifth-dimension (and right-hand-side) lanes.
//
//   (Dh psi)(x, l) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu, l) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu, l)
//
// (the hopping term of D_W = (4 - M5) - Dh/2; the dagger swaps the two
// projectors).  The operator is identical on every lane l = r * Ls + s, so a
// CTA takes a tile of 4D sites of one parity and all of their lanes: the
// 8 links and 8 neighbour indices of every site of the tile are copied once
// into shared memory by one bulk (TMA) copy and reused by all lanes.  Each
// thread owns VL consecutive lanes of one site; spinor loads and stores are
// VL-wide vectors of the [site][12][lanes] layout, so a warp reads whole
// contiguous lane rows.  The spin projection to a half spinor uses the
// chiral-basis structure of (1 -+ g_mu): two colour vectors are transported
// per direction and the lower spins are rebuilt from them.
//
// Epilogues: PLAIN   out = scale * Dh in
//            MOO     out = M_oo x + scale * Dh in  (+ per-tile |out|^2),
//            the last step of the Schur operator M_pc = M_oo - M_oe M_ee^-1 M_eo.
#include <algorithm>
#include <cstdio>
#include <type_traits>
#include <map>
#include <utility>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

struct HopArgs {
    const void* in;
    void* out;
    const void* xmoo;
    const void* links;   // parity table [site][8][9] complex (site-major)
    const int* nbr;      // [site][8]
    const int4* tiles;
    int T, N5, Ls, nrhs, ntiles;
    int chunk;           // consecutive tiles a CTA takes before striding: neighbouring rows of
                         // the lattice on one SM, so y-neighbours are re-read from L1
    double scale, d, e, mf, b5, c5;
    double fa, inv_d, inv_den;   // EPI_BMINV: a = -e/d, 1/d, 1/(d (1 + mf a^Ls))
    double* partial;
    int* err;
    // EPI_POST: CG vectors (FP32) and per-system scalars
    void* cg_x;
    void* cg_r;
    const void* cg_p;
    const double* alpha;
    const int* run;
};

// Scans across the lanes of one right-hand side (Ls lanes held by Ls / VL
// consecutive threads of a warp) for the fifth-dimension factor between the
// hops of M_pc, B M^-1 = (b5 + c5 S)(d + e S)^-1 per chirality, S the
// twisted shift S_- (reads lane s - 1, wall -mf) or S_+ (s + 1).  With
// a = -e/d, S_-^Ls = -mf and (1 - a S)^-1 = sum_{k<Ls} (a S)^k / (1 + mf a^Ls):
//   (d + e S_-)^-1 x |_s = P_s / d - mf a^(s+1) P_(Ls-1) / (d (1 + mf a^Ls)),
//   P_s = sum_{t<=s} a^(s-t) x_t,
// a decayed prefix sum (in-thread, then across threads by shuffles); S_+ is
// the mirror image with suffix sums Q_s = sum_{t>=s} a^(t-s) x_t and
// a^(Ls-s) Q_0.
template <int VL>
struct ScanCtx {
    unsigned mask;          // the site group's threads
    int j, nthr, seg0;      // thread index in the rhs segment, threads per segment, its first lane
    float a, inv_d, wc;     // a, 1/d, mf / (d (1 + mf a^Ls))
    float mf, b5, c5;
    float astep[5];         // a^(VL o) for scan strides o = 1, 2, 4, 8, 16
    float pdn[VL], pup[VL]; // a^(s+1), a^(Ls-s) per lane
    float cdn[VL], cup[VL]; // carry factors a^(v+1), a^(VL-v)
};

template <int VL, bool DN>
__device__ __forceinline__ void scan_bminv(const ScanCtx<VL>& k, float (&x)[VL]) {
    float p[VL];
    if (DN) {
        p[0] = x[0];
#pragma unroll
        for (int v = 1; v < VL; ++v) p[v] = fmaf(k.a, p[v - 1], x[v]);
    } else {
        p[VL - 1] = x[VL - 1];
#pragma unroll
        for (int v = VL - 2; v >= 0; --v) p[v] = fmaf(k.a, p[v + 1], x[v]);
    }
    // inclusive scan of the thread totals over the segment (Hillis-Steele)
    const int me = k.seg0 + k.j;
    float tot = DN ? p[VL - 1] : p[0];
    // unrolled over the five possible strides (compile-time index into astep:
    // the context stays in registers); strides beyond the segment are skipped
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
        const int o = 1 << lvl;
        if (o < k.nthr) {
            const bool has = DN ? k.j >= o : k.j + o < k.nthr;
            const float v = __shfl_sync(k.mask, tot, has ? (DN ? me - o : me + o) : me);
            if (has) tot = fmaf(k.astep[lvl], v, tot);
        }
    }
    // carry in from the neighbouring thread's inclusive total
    const bool hc = DN ? k.j > 0 : k.j + 1 < k.nthr;
    const float carry = __shfl_sync(k.mask, tot, hc ? (DN ? me - 1 : me + 1) : me);
    if (hc) {
#pragma unroll
        for (int v = 0; v < VL; ++v) p[v] = fmaf(DN ? k.cdn[v] : k.cup[v], carry, p[v]);
    }
    // the wall term: P at the segment's last lane (Q at its first)
    const float T = __shfl_sync(k.mask, DN ? p[VL - 1] : p[0], DN ? k.seg0 + k.nthr - 1 : k.seg0);
    float y[VL];
#pragma unroll
    for (int v = 0; v < VL; ++v) y[v] = fmaf(-k.wc * (DN ? k.pdn[v] : k.pup[v]), T, p[v] * k.inv_d);
    // (b5 + c5 S) y
    float nb;
    if (DN) {
        const bool in = k.j > 0;
        nb = __shfl_sync(k.mask, y[VL - 1], in ? me - 1 : k.seg0 + k.nthr - 1) * (in ? 1.f : -k.mf);
    } else {
        const bool in = k.j + 1 < k.nthr;
        nb = __shfl_sync(k.mask, y[0], in ? me + 1 : k.seg0) * (in ? 1.f : -k.mf);
    }
#pragma unroll
    for (int v = 0; v < VL; ++v) {
        const float sv = DN ? (v > 0 ? y[(v + VL - 1) % VL] : nb) : (v < VL - 1 ? y[(v + 1) % VL] : nb);
        x[v] = fmaf(k.c5, sv, k.b5 * y[v]);
    }
}

// Lanes next to the first and last lane of this thread within its site
// group, for S5 across threads: the thread holding the lane above the last
// one (as its first lane) and the one holding the lane below the first one
// (as its last lane), with the wall factor -mf where the shift wraps.
struct LaneNbrs {
    int src_up, src_dn;
    unsigned mask;     // the site group's threads in the warp
    float f_up, f_dn;
};

// One direction K (0..3: +mu, 4..7: -mu) for the VL lanes of one site; src
// points at lane0 of the neighbour's spinor ([12][N5] complex), in global or
// shared memory.
template <int K, bool DAG, class Sin, class SL, class R, int VL>
__device__ __forceinline__ void hop_dir_src(const Sin* __restrict__ src, const SL* s_link, int N5,
                                            R (&ar)[12][VL], R (&ai)[12][VL]) {
    constexpr int MU = K & 3;
    constexpr bool FWD = K < 4;
    constexpr int SGI = (FWD != DAG) ? 1 : -1;   // (1 - SG g_mu) projector
    const R SG = (R)SGI;
    R ur[2][3][VL], ui[2][3][VL], lr[2][3][VL], li[2][3][VL];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            load_lanes<Sin, VL, R>(src + (int64_t)((sp * 3 + c) * N5) * 2, ur[sp][c], ui[sp][c]);
            load_lanes<Sin, VL, R>(src + (int64_t)(((sp + 2) * 3 + c) * N5) * 2, lr[sp][c],
                                   li[sp][c]);
        }
    // half spinor h = u - SG A_mu l
    R hr[2][3][VL], hi[2][3][VL];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int v = 0; v < VL; ++v) {
            if (MU == 0) {
                hr[0][c][v] = ur[0][c][v] - SG * li[1][c][v];
                hi[0][c][v] = ui[0][c][v] + SG * lr[1][c][v];
                hr[1][c][v] = ur[1][c][v] - SG * li[0][c][v];
                hi[1][c][v] = ui[1][c][v] + SG * lr[0][c][v];
            } else if (MU == 1) {
                hr[0][c][v] = ur[0][c][v] + SG * lr[1][c][v];
                hi[0][c][v] = ui[0][c][v] + SG * li[1][c][v];
                hr[1][c][v] = ur[1][c][v] - SG * lr[0][c][v];
                hi[1][c][v] = ui[1][c][v] - SG * li[0][c][v];
            } else if (MU == 2) {
                hr[0][c][v] = ur[0][c][v] - SG * li[0][c][v];
                hi[0][c][v] = ui[0][c][v] + SG * lr[0][c][v];
                hr[1][c][v] = ur[1][c][v] + SG * li[1][c][v];
                hi[1][c][v] = ui[1][c][v] - SG * lr[1][c][v];
            } else {
                hr[0][c][v] = ur[0][c][v] - SG * lr[0][c][v];
                hi[0][c][v] = ui[0][c][v] - SG * li[0][c][v];
                hr[1][c][v] = ur[1][c][v] - SG * lr[1][c][v];
                hi[1][c][v] = ui[1][c][v] - SG * li[1][c][v];
            }
        }
    // g = W h (two colour vectors)
    const SL* w = s_link + K * 18;
    R gr[2][3][VL], gi[2][3][VL];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R wr[3], wi[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) link_c<SL, R>(w, a * 3 + b, wr[b], wi[b]);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int v = 0; v < VL; ++v) {
                R sr = wr[0] * hr[sp][0][v] - wi[0] * hi[sp][0][v];
                R si = wr[0] * hi[sp][0][v] + wi[0] * hr[sp][0][v];
                sr = fma(wr[1], hr[sp][1][v], sr); sr = fma(-wi[1], hi[sp][1][v], sr);
                si = fma(wr[1], hi[sp][1][v], si); si = fma(wi[1], hr[sp][1][v], si);
                sr = fma(wr[2], hr[sp][2][v], sr); sr = fma(-wi[2], hi[sp][2][v], sr);
                si = fma(wr[2], hi[sp][2][v], si); si = fma(wi[2], hr[sp][2][v], si);
                gr[sp][a][v] = sr;
                gi[sp][a][v] = si;
            }
    }
    // reconstruct: upper += g, lower += -SG A_mu^+ g
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int v = 0; v < VL; ++v) {
            ar[c][v] += gr[0][c][v];
            ai[c][v] += gi[0][c][v];
            ar[3 + c][v] += gr[1][c][v];
            ai[3 + c][v] += gi[1][c][v];
            if (MU == 0) {
                ar[6 + c][v] += SG * gi[1][c][v];
                ai[6 + c][v] -= SG * gr[1][c][v];
                ar[9 + c][v] += SG * gi[0][c][v];
                ai[9 + c][v] -= SG * gr[0][c][v];
            } else if (MU == 1) {
                ar[6 + c][v] -= SG * gr[1][c][v];
                ai[6 + c][v] -= SG * gi[1][c][v];
                ar[9 + c][v] += SG * gr[0][c][v];
                ai[9 + c][v] += SG * gi[0][c][v];
            } else if (MU == 2) {
                ar[6 + c][v] += SG * gi[0][c][v];
                ai[6 + c][v] -= SG * gr[0][c][v];
                ar[9 + c][v] -= SG * gi[1][c][v];
                ai[9 + c][v] += SG * gr[1][c][v];
            } else {
                ar[6 + c][v] -= SG * gr[0][c][v];
                ai[6 + c][v] -= SG * gi[0][c][v];
                ar[9 + c][v] -= SG * gr[1][c][v];
                ai[9 + c][v] -= SG * gi[1][c][v];
            }
        }
}

// The same direction for two lanes in FP32 with paired-FP32 instructions
// (fma/mul .f32x2 on sm_100 and later): each float2 holds one real or
// imaginary component of both lanes, so every operation of the scalar form
// above is one instruction for the pair.  Same formulas, same order.  Used
// for BF16 operands, whose conversion already yields separate components
// (15% faster at 32^4 x 16); for FP32 operands the regrouping of the loaded
// (re, im, re, im) quads and the extra register pressure made it slower.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int K, bool DAG, class Sin, class SL>
__device__ __forceinline__ void hop_dir_x2(const Sin* __restrict__ src, const SL* s_link, int N5,
                                           float2 (&ar)[12], float2 (&ai)[12]) {
    constexpr int MU = K & 3;
    constexpr bool FWD = K < 4;
    constexpr float SG = (FWD != DAG) ? 1.f : -1.f;   // (1 - SG g_mu) projector
    const float2 P = f2(SG), M = f2(-SG);
    float2 ur[2][3], ui[2][3], lr[2][3], li[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float re[2], im[2];
            load_lanes<Sin, 2, float>(src + (int64_t)((sp * 3 + c) * N5) * 2, re, im);
            ur[sp][c] = make_float2(re[0], re[1]);
            ui[sp][c] = make_float2(im[0], im[1]);
            load_lanes<Sin, 2, float>(src + (int64_t)(((sp + 2) * 3 + c) * N5) * 2, re, im);
            lr[sp][c] = make_float2(re[0], re[1]);
            li[sp][c] = make_float2(im[0], im[1]);
        }
    // half spinor h = u - SG A_mu l
    float2 hr[2][3], hi[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) {
            hr[0][c] = fma2(M, li[1][c], ur[0][c]);
            hi[0][c] = fma2(P, lr[1][c], ui[0][c]);
            hr[1][c] = fma2(M, li[0][c], ur[1][c]);
            hi[1][c] = fma2(P, lr[0][c], ui[1][c]);
        } else if (MU == 1) {
            hr[0][c] = fma2(P, lr[1][c], ur[0][c]);
            hi[0][c] = fma2(P, li[1][c], ui[0][c]);
            hr[1][c] = fma2(M, lr[0][c], ur[1][c]);
            hi[1][c] = fma2(M, li[0][c], ui[1][c]);
        } else if (MU == 2) {
            hr[0][c] = fma2(M, li[0][c], ur[0][c]);
            hi[0][c] = fma2(P, lr[0][c], ui[0][c]);
            hr[1][c] = fma2(P, li[1][c], ur[1][c]);
            hi[1][c] = fma2(M, lr[1][c], ui[1][c]);
        } else {
            hr[0][c] = fma2(M, lr[0][c], ur[0][c]);
            hi[0][c] = fma2(M, li[0][c], ui[0][c]);
            hr[1][c] = fma2(M, lr[1][c], ur[1][c]);
            hi[1][c] = fma2(M, li[1][c], ui[1][c]);
        }
    }
    // g = W h (two colour vectors)
    const SL* w = s_link + K * 18;
    float2 gr[2][3], gi[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float wr[3], wi[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) link_c<SL, float>(w, a * 3 + b, wr[b], wi[b]);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            float2 sr = __fmul2_rn(f2(wr[0]), hr[sp][0]);
            float2 si = __fmul2_rn(f2(wr[0]), hi[sp][0]);
            sr = fma2(f2(-wi[0]), hi[sp][0], sr);
            si = fma2(f2(wi[0]), hr[sp][0], si);
            sr = fma2(f2(wr[1]), hr[sp][1], sr); sr = fma2(f2(-wi[1]), hi[sp][1], sr);
            si = fma2(f2(wr[1]), hi[sp][1], si); si = fma2(f2(wi[1]), hr[sp][1], si);
            sr = fma2(f2(wr[2]), hr[sp][2], sr); sr = fma2(f2(-wi[2]), hi[sp][2], sr);
            si = fma2(f2(wr[2]), hi[sp][2], si); si = fma2(f2(wi[2]), hr[sp][2], si);
            gr[sp][a] = sr;
            gi[sp][a] = si;
        }
    }
    // reconstruct: upper += g, lower += -SG A_mu^+ g
    const float2 one = f2(1.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ar[c] = fma2(one, gr[0][c], ar[c]);
        ai[c] = fma2(one, gi[0][c], ai[c]);
        ar[3 + c] = fma2(one, gr[1][c], ar[3 + c]);
        ai[3 + c] = fma2(one, gi[1][c], ai[3 + c]);
        if (MU == 0) {
            ar[6 + c] = fma2(P, gi[1][c], ar[6 + c]);
            ai[6 + c] = fma2(M, gr[1][c], ai[6 + c]);
            ar[9 + c] = fma2(P, gi[0][c], ar[9 + c]);
            ai[9 + c] = fma2(M, gr[0][c], ai[9 + c]);
        } else if (MU == 1) {
            ar[6 + c] = fma2(M, gr[1][c], ar[6 + c]);
            ai[6 + c] = fma2(M, gi[1][c], ai[6 + c]);
            ar[9 + c] = fma2(P, gr[0][c], ar[9 + c]);
            ai[9 + c] = fma2(P, gi[0][c], ai[9 + c]);
        } else if (MU == 2) {
            ar[6 + c] = fma2(P, gi[0][c], ar[6 + c]);
            ai[6 + c] = fma2(M, gr[0][c], ai[6 + c]);
            ar[9 + c] = fma2(M, gi[1][c], ar[9 + c]);
            ai[9 + c] = fma2(P, gr[1][c], ai[9 + c]);
        } else {
            ar[6 + c] = fma2(M, gr[0][c], ar[6 + c]);
            ai[6 + c] = fma2(M, gi[0][c], ai[6 + c]);
            ar[9 + c] = fma2(M, gr[1][c], ar[9 + c]);
            ai[9 + c] = fma2(M, gi[1][c], ai[9 + c]);
        }
    }
}

template <int K, bool DAG, class Sin, class SL>
__device__ __forceinline__ void hop_dir2(const Sin* __restrict__ in, const int* s_nbr,
                                         const SL* s_link, int N5, int lane0, float2 (&ar)[12],
                                         float2 (&ai)[12]) {
    const int n = s_nbr[K];
    if (n < 0) return;   // link cut by a Dirichlet boundary
    hop_dir_x2<K, DAG, Sin, SL>(in + ((int64_t)n * 12 * N5 + lane0) * 2, s_link, N5, ar, ai);
}

template <int K, bool DAG, class Sin, class SL, class R, int VL>
__device__ __forceinline__ void hop_dir(const Sin* __restrict__ in, const int* s_nbr,
                                        const SL* s_link, int N5, int lane0, R (&ar)[12][VL],
                                        R (&ai)[12][VL]) {
    const int n = s_nbr[K];
    if (n < 0) return;   // link cut by a Dirichlet boundary
    hop_dir_src<K, DAG, Sin, SL, R, VL>(in + ((int64_t)n * 12 * N5 + lane0) * 2, s_link, N5, ar, ai);
}

// Output of one site's VL lanes: PLAIN out = scale * acc; MOO out = M_oo x +
// scale * acc, returning the lanes' |out|^2 (FP32 arithmetic: summed in FP32
// per site, one FP64 add per site, off GB300's slow FP64 pipe).
// Site groups (N5 / VL threads) known at compile time to divide a warp: the
// epilogues take a site's neighbouring fifth-dimension lane by shuffle.
template <int VL, int CN5>
constexpr bool kLaneShfl = CN5 > 0 && CN5 % VL == 0 && CN5 / VL <= 32 && 32 % (CN5 / VL) == 0;

template <class Sout, class R, int VL, bool DAG, int EPI, int CN5>
__device__ __forceinline__ double hop_store(const HopArgs& a, int N5, int64_t site, int lane0,
                                            const R (&ar)[12][VL], const R (&ai)[12][VL],
                                            const LaneNbrs& nb, int box, const ScanCtx<VL>& sk) {
    const R sc = (R)a.scale;
    if constexpr (EPI == EPI_BMINV) {
        // out = scale B M^-1 acc: non-adjoint upper spins see S_-, lower S_+
        Sout* out = reinterpret_cast<Sout*>(a.out) + (site * 12 * N5 + lane0) * 2;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            float xr[VL], xi[VL];
#pragma unroll
            for (int v = 0; v < VL; ++v) { xr[v] = (float)ar[c][v]; xi[v] = (float)ai[c][v]; }
            if ((c < 6) != DAG) {
                scan_bminv<VL, true>(sk, xr);
                scan_bminv<VL, true>(sk, xi);
            } else {
                scan_bminv<VL, false>(sk, xr);
                scan_bminv<VL, false>(sk, xi);
            }
#pragma unroll
            for (int v = 0; v < VL; ++v) { xr[v] *= (float)sc; xi[v] *= (float)sc; }
            store_lanes<Sout, VL, float, true>(out + (int64_t)c * N5 * 2, xr, xi);
        }
        return 0.0;
    }
    if constexpr (EPI == EPI_POST) {
        static_assert(DAG, "the fused M_pc^+ tail follows the adjoint hop");
        // B^+ acc = b5 acc + c5 S5^+ acc on this site's lanes: S5^+ takes
        // lane s + 1 for the upper spins and s - 1 for the lower ones (walls
        // -mf); the lanes beyond this thread's come from its neighbours in
        // the site group
        const R b5 = (R)a.b5, c5 = (R)a.c5;
        R br[12][VL], bi[12][VL];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            if (c < 6) {
                const R nr = __shfl_sync(nb.mask, ar[c][0], nb.src_up) * (R)nb.f_up;
                const R ni = __shfl_sync(nb.mask, ai[c][0], nb.src_up) * (R)nb.f_up;
#pragma unroll
                for (int v = 0; v < VL; ++v) {
                    const R sr = v < VL - 1 ? ar[c][(v + 1) % VL] : nr;
                    const R si = v < VL - 1 ? ai[c][(v + 1) % VL] : ni;
                    br[c][v] = b5 * ar[c][v] + c5 * sr;
                    bi[c][v] = b5 * ai[c][v] + c5 * si;
                }
            } else {
                const R nr = __shfl_sync(nb.mask, ar[c][VL - 1], nb.src_dn) * (R)nb.f_dn;
                const R ni = __shfl_sync(nb.mask, ai[c][VL - 1], nb.src_dn) * (R)nb.f_dn;
#pragma unroll
                for (int v = 0; v < VL; ++v) {
                    const R sr = v > 0 ? ar[c][(v + VL - 1) % VL] : nr;
                    const R si = v > 0 ? ai[c][(v + VL - 1) % VL] : ni;
                    br[c][v] = b5 * ar[c][v] + c5 * sr;
                    bi[c][v] = b5 * ai[c][v] + c5 * si;
                }
            }
        }
        // Ap = M_oo^+ t + scale B^+ acc (t = xmoo; M_oo^+ = d + e S5^+ from
        // memory), then x += alpha p, r -= alpha Ap and |r|^2
        const int Ls = a.Ls;
        const int s0 = lane0 % Ls;
        const int rbase = lane0 - s0;
        const int sys = box * a.nrhs + lane0 / Ls;
        const R alpha = (R)a.alpha[sys];
        const bool live = a.run == nullptr || a.run[sys] != 0;
        const bool hi_wrap = (s0 + VL == Ls), lo_wrap = (s0 == 0);
        const int l_above = hi_wrap ? rbase : lane0 + VL;
        const int l_below = lo_wrap ? rbase + Ls - 1 : lane0 - 1;
        const R mf = (R)a.mf, d = (R)a.d, e = (R)a.e;
        // distinct fields: no aliasing, so the loads of later components can
        // be issued ahead of the stores of earlier ones
        const Sout* __restrict__ tb = reinterpret_cast<const Sout*>(a.xmoo) + (site * 12 * N5) * 2;
        float* __restrict__ xb = reinterpret_cast<float*>(a.cg_x) + (site * 12 * N5 + lane0) * 2;
        float* __restrict__ rb = reinterpret_cast<float*>(a.cg_r) + (site * 12 * N5 + lane0) * 2;
        const float* __restrict__ pb = reinterpret_cast<const float*>(a.cg_p) + (site * 12 * N5 + lane0) * 2;
        float nrm = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            R tr[VL], ti[VL];
            load_lanes<Sout, VL, R>(tb + (int64_t)(c * N5 + lane0) * 2, tr, ti);
            const bool up = c < 6;   // S5^+: upper spins read s + 1
            R nr, ni, fn;
            if constexpr (kLaneShfl<VL, CN5>) {
                nr = __shfl_sync(nb.mask, up ? tr[0] : tr[VL - 1], up ? nb.src_up : nb.src_dn);
                ni = __shfl_sync(nb.mask, up ? ti[0] : ti[VL - 1], up ? nb.src_up : nb.src_dn);
                fn = (R)(up ? nb.f_up : nb.f_dn);
            } else {
                load_c1<Sout, R>(tb + (int64_t)(c * N5 + (up ? l_above : l_below)) * 2, nr, ni);
                fn = up ? (hi_wrap ? -mf : (R)1) : (lo_wrap ? -mf : (R)1);
            }
            float rr[VL], ri[VL];
            load_lanes<float, VL, float>(rb + (int64_t)c * N5 * 2, rr, ri);
            if (live) {
                float xr[VL], xi[VL], pr[VL], pi[VL];
                load_lanes<float, VL, float>(xb + (int64_t)c * N5 * 2, xr, xi);
                load_lanes<float, VL, float>(pb + (int64_t)c * N5 * 2, pr, pi);
#pragma unroll
                for (int v = 0; v < VL; ++v) {
                    R sr, si;
                    if (up) {
                        sr = v == VL - 1 ? fn * nr : tr[(v + 1) % VL];
                        si = v == VL - 1 ? fn * ni : ti[(v + 1) % VL];
                    } else {
                        sr = v == 0 ? fn * nr : tr[(v + VL - 1) % VL];
                        si = v == 0 ? fn * ni : ti[(v + VL - 1) % VL];
                    }
                    const R apr = d * tr[v] + e * sr + sc * br[c][v];
                    const R api = d * ti[v] + e * si + sc * bi[c][v];
                    xr[v] = fmaf((float)alpha, pr[v], xr[v]);
                    xi[v] = fmaf((float)alpha, pi[v], xi[v]);
                    rr[v] = fmaf(-(float)alpha, (float)apr, rr[v]);
                    ri[v] = fmaf(-(float)alpha, (float)api, ri[v]);
                }
                store_lanes<float, VL, float>(xb + (int64_t)c * N5 * 2, xr, xi);
                store_lanes<float, VL, float>(rb + (int64_t)c * N5 * 2, rr, ri);
            }
#pragma unroll
            for (int v = 0; v < VL; ++v) nrm = fmaf(rr[v], rr[v], fmaf(ri[v], ri[v], nrm));
        }
        return (double)nrm;
    }
    Sout* __restrict__ out = reinterpret_cast<Sout*>(a.out) + (site * 12 * N5 + lane0) * 2;
    if (EPI == EPI_PLAIN) {
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            R orr[VL], oi[VL];
#pragma unroll
            for (int v = 0; v < VL; ++v) {
                orr[v] = sc * ar[c][v];
                oi[v] = sc * ai[c][v];
            }
            store_lanes<Sout, VL, R, true>(out + (int64_t)c * N5 * 2, orr, oi);
        }
        return 0.0;
    }
    // M_oo x = d x + e S5 x on this site's lanes; S5 (non-dagger):
    // upper spins x_{s-1}, lower spins x_{s+1}, walls -mf.
    const Sout* __restrict__ xb = reinterpret_cast<const Sout*>(a.xmoo) + (site * 12 * N5) * 2;
    const int Ls = a.Ls;
    const int s0 = lane0 % Ls;
    const int rbase = lane0 - s0;
    const R d = (R)a.d, e = (R)a.e, mf = (R)a.mf;
    // neighbouring lanes below and above this thread's block
    const bool lo_wrap = (s0 == 0);
    const bool hi_wrap = (s0 + VL == Ls);
    const int l_below = lo_wrap ? rbase + Ls - 1 : lane0 - 1;
    const int l_above = hi_wrap ? rbase : lane0 + VL;
    const R f_below = lo_wrap ? -mf : (R)1;
    const R f_above = hi_wrap ? -mf : (R)1;
    double nrm = 0.0;
    float nrm_f = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        R xr[VL], xi[VL];
        load_lanes<Sout, VL, R>(xb + (int64_t)(c * N5 + lane0) * 2, xr, xi);
        // upper spins use S_- (x_{s-1}) unless dagger, lower S_+
        const bool use_below = (c < 6) != DAG;
        R nr, ni, fn;
        if constexpr (kLaneShfl<VL, CN5>) {
            // the neighbouring lane is held by the adjacent thread of the site group
            nr = __shfl_sync(nb.mask, use_below ? xr[VL - 1] : xr[0], use_below ? nb.src_dn : nb.src_up);
            ni = __shfl_sync(nb.mask, use_below ? xi[VL - 1] : xi[0], use_below ? nb.src_dn : nb.src_up);
            fn = (R)(use_below ? nb.f_dn : nb.f_up);
        } else {
            load_c1<Sout, R>(xb + (int64_t)(c * N5 + (use_below ? l_below : l_above)) * 2, nr, ni);
            fn = use_below ? f_below : f_above;
        }
        R orr[VL], oi[VL];
        float part = 0.f;
#pragma unroll
        for (int v = 0; v < VL; ++v) {
            R sr, si;
            if (use_below) {
                sr = (v == 0) ? fn * nr : xr[v - 1];
                si = (v == 0) ? fn * ni : xi[v - 1];
            } else {
                sr = (v == VL - 1) ? fn * nr : xr[(v + 1) % VL];
                si = (v == VL - 1) ? fn * ni : xi[(v + 1) % VL];
            }
            orr[v] = d * xr[v] + e * sr + sc * ar[c][v];
            oi[v] = d * xi[v] + e * si + sc * ai[c][v];
            part += (float)(orr[v] * orr[v] + oi[v] * oi[v]);
            if (sizeof(R) == 8) nrm += (double)orr[v] * orr[v] + (double)oi[v] * oi[v];
        }
        if (sizeof(R) != 8) nrm_f += part;
        store_lanes<Sout, VL, R, true>(out + (int64_t)c * N5 * 2, orr, oi);
    }
    return sizeof(R) == 8 ? nrm : (double)nrm_f;
}

// Persistent kernel: CTA b takes tiles b, b + gridDim, ...; the links and
// neighbour indices of a tile arrive by bulk copy into one half of a double
// buffer.  There is no CTA-wide barrier in the tile loop: each warp waits for
// its tile's copy on the buffer's mbarrier, and the last warp to finish with
// a buffer (a shared-memory arrival counter) sums the per-warp norm partials
// in warp order and issues the copy of the tile two steps ahead into it, so
// fast warps run on into the next tile.
// CN5 > 0 fixes N5 = Ls * nrhs at compile time (the common single-rhs
// cases), so the row offsets of every spinor load and store are immediates.
template <class Sin, class Sout, class SL, class R, int VL, bool DAG, int EPI, int CN5>
__global__ void __launch_bounds__(256, (VL == 1 && sizeof(R) == 4) ? 3 : 2) k_hop(const HopArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int N5 = CN5 > 0 ? CN5 : a.N5;
    const int TPS = N5 / VL;
    const size_t link_bytes = (size_t)a.T * 144 * sizeof(SL);
    const size_t buf_bytes = link_bytes + (size_t)a.T * 32;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * buf_bytes);
    int* done = reinterpret_cast<int*>(bar + 2);              // [2] warps finished with a buffer
    double* s_red = reinterpret_cast<double*>(bar + 3);       // [2][nwarps][nrhs]
    const int nt = a.ntiles;
    const int nwarps = (int)(blockDim.x >> 5), warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // k-th tile of this CTA: chunks of `chunk` consecutive tiles, strided by the grid
    const int ck = a.chunk;
    auto tile_of = [&](int k) { return ((k / ck) * (int)gridDim.x + (int)blockIdx.x) * ck + k % ck; };

    auto issue = [&](int tile, int b) {
        const int4 t = a.tiles[tile];
        const uint32_t lb = (uint32_t)t.z * 144u * (uint32_t)sizeof(SL);
        const uint32_t nb = (uint32_t)t.z * 32u;
        unsigned char* base = smem + b * buf_bytes;
        // order the generic-proxy reads of this buffer before the async write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[b], lb + nb);
        bulk_g2s(base, reinterpret_cast<const SL*>(a.links) + (int64_t)t.y * 144, lb, &bar[b]);
        bulk_g2s(base + link_bytes, a.nbr + (int64_t)t.y * 8, nb, &bar[b]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        done[0] = done[1] = 0;
        fence_mbar_init();
        if (tile_of(0) < nt) issue(tile_of(0), 0);
        if (tile_of(1) < nt) issue(tile_of(1), 1);
    }
    __syncthreads();

    const int G = blockDim.x / TPS;
    const int sg = threadIdx.x / TPS;
    const int lane0 = (threadIdx.x - sg * TPS) * VL;
    const int rhs = lane0 / a.Ls;   // of this thread's lanes (threads without sites add 0)
    const bool part = (EPI == EPI_MOO || EPI == EPI_POST) && a.partial != nullptr;
    ScanCtx<VL> sk{};
    if constexpr (EPI == EPI_BMINV) {
        const int wl = threadIdx.x & 31;
        const int Ls = a.Ls;
        const int tig = lane0 / VL;
        const int gb = wl - tig;
        sk.mask = TPS >= 32 ? 0xffffffffu : (((1u << TPS) - 1u) << gb);
        sk.nthr = Ls / VL;
        sk.j = (lane0 % Ls) / VL;
        sk.seg0 = wl - sk.j;
        sk.a = (float)a.fa;
        sk.inv_d = (float)a.inv_d;
        sk.wc = (float)(a.mf * a.inv_den);
        sk.mf = (float)a.mf;
        sk.b5 = (float)a.b5;
        sk.c5 = (float)a.c5;
        float av = 1.f;
#pragma unroll
        for (int v = 0; v < VL; ++v) av *= sk.a;
#pragma unroll
        for (int l = 0; l < 5; ++l) { sk.astep[l] = av; av *= av; }
        const int s0 = lane0 % Ls;
#pragma unroll
        for (int v = 0; v < VL; ++v) {
            float pd = 1.f, pu = 1.f, cd = 1.f, cu = 1.f;
            for (int q = 0; q < s0 + v + 1; ++q) pd *= sk.a;
            for (int q = 0; q < Ls - s0 - v; ++q) pu *= sk.a;
            for (int q = 0; q < v + 1; ++q) cd *= sk.a;
            for (int q = 0; q < VL - v; ++q) cu *= sk.a;
            sk.pdn[v] = pd; sk.pup[v] = pu; sk.cdn[v] = cd; sk.cup[v] = cu;
        }
    }
    LaneNbrs nbrs{};
    if constexpr (EPI == EPI_POST || (EPI == EPI_MOO && kLaneShfl<VL, CN5>)) {
        // site groups are warp-aligned here (TPS divides 32, checked on the host)
        const int wl = threadIdx.x & 31;
        const int tig = lane0 / VL;
        const int gb = wl - tig;
        const int s_first = lane0 % a.Ls, s_last = (lane0 + VL - 1) % a.Ls;
        const int rb = lane0 - s_first;
        const int above = s_last == a.Ls - 1 ? rb : lane0 + VL;
        const int below = s_first == 0 ? rb + a.Ls - 1 : lane0 - 1;
        nbrs.src_up = gb + above / VL;
        nbrs.src_dn = gb + below / VL;
        nbrs.f_up = s_last == a.Ls - 1 ? -(float)a.mf : 1.f;
        nbrs.f_dn = s_first == 0 ? -(float)a.mf : 1.f;
        nbrs.mask = TPS >= 32 ? 0xffffffffu : (((1u << TPS) - 1u) << gb);
    }

    int k = 0;
    for (int tile = tile_of(0); tile < nt; tile = tile_of(++k)) {
        const int b = k & 1;
        const uint32_t ph = (uint32_t)((k >> 1) & 1);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[b], ph))) {
            // a lost copy: record it, let it land, stop
            if (lane == 0) {
                atomicOr(a.err, kErrBulkTimeout);
                mbar_wait_bounded(&bar[b], ph);
            }
            return;
        }
        const int4 tl = a.tiles[tile];
        const int begin = tl.y, count = tl.z;
        const SL* s_link_t = reinterpret_cast<const SL*>(smem + b * buf_bytes);
        const int* s_nbr_t = reinterpret_cast<const int*>(smem + b * buf_bytes + link_bytes);
        double tile_norm = 0.0;
        for (int sl = sg; sg < G && sl < count; sl += G) {
            // the M_oo input of this site's lanes, into L1 while the last two
            // directions run (earlier, the lines are evicted by the neighbour
            // traffic before the epilogue reads them)
            auto prefetch_moo = [&]() {
                if (EPI == EPI_MOO || EPI == EPI_POST) {
                    const Sout* xb = reinterpret_cast<const Sout*>(a.xmoo) + ((int64_t)(begin + sl) * 12 * N5 + lane0) * 2;
#pragma unroll
                    for (int c = 0; c < 12; ++c)
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(xb + (int64_t)c * N5 * 2));
                }
            };
            R ar[12][VL], ai[12][VL];
            const Sin* in = reinterpret_cast<const Sin*>(a.in);
            const int* nb = s_nbr_t + sl * 8;
            const SL* lk = s_link_t + (size_t)sl * 144;
            // +mu and -mu back to back: the row that is the +x neighbour of
            // one site is the -x neighbour of the next, still in L1
            if constexpr (std::is_same<R, float>::value && VL == 2 && std::is_same<Sin, bf16>::value) {
                float2 pr[12], pi[12];
#pragma unroll
                for (int c = 0; c < 12; ++c) pr[c] = pi[c] = make_float2(0.f, 0.f);
                hop_dir2<0, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
                hop_dir2<4, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
                hop_dir2<1, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
                hop_dir2<5, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
                hop_dir2<2, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
                hop_dir2<6, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
                prefetch_moo();
                hop_dir2<3, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
                hop_dir2<7, DAG, Sin, SL>(in, nb, lk, N5, lane0, pr, pi);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    ar[c][0] = pr[c].x; ar[c][VL - 1] = pr[c].y;
                    ai[c][0] = pi[c].x; ai[c][VL - 1] = pi[c].y;
                }
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c)
#pragma unroll
                    for (int v = 0; v < VL; ++v) ar[c][v] = ai[c][v] = (R)0;
                hop_dir<0, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
                hop_dir<4, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
                hop_dir<1, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
                hop_dir<5, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
                hop_dir<2, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
                hop_dir<6, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
                prefetch_moo();
                hop_dir<3, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
                hop_dir<7, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
            }
            tile_norm += hop_store<Sout, R, VL, DAG, EPI, CN5>(a, N5, begin + sl, lane0, ar, ai, nbrs, tl.x, sk);
        }
        double* red = s_red + (size_t)b * nwarps * a.nrhs;
        if (part) {
            for (int r = 0; r < a.nrhs; ++r) {
                double v = rhs == r ? tile_norm : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) red[warp * a.nrhs + r] = v;
            }
        }
        __syncwarp();   // this warp's reads of buffer b are done
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&done[b], 1) == nwarps - 1) {   // the last warp out
                __threadfence_block();
                if (part)
                    for (int r = 0; r < a.nrhs; ++r) {
                        double sum = 0.0;
                        for (int w = 0; w < nwarps; ++w) sum += red[w * a.nrhs + r];
                        a.partial[(size_t)tile * a.nrhs + r] = sum;
                    }
                done[b] = 0;
                const int next2 = tile_of(k + 2);
                if (next2 < nt) issue(next2, b);
            }
        }
    }
}

// ------------------------------------------------------------- launcher
template <class Sin, class Sout, class SL, class R, int VL, int CN5 = 0>
static dwf_status launch_t(dwf_handle* h, const HopCall& c, const TileSet& ts, cudaStream_t s) {
    const int p = c.out_parity;
    HopArgs a;
    a.in = c.in;
    a.out = c.out;
    a.xmoo = c.xmoo;
    a.links = h->d_links[c.prec_link][p];
    a.nbr = h->d_nbr[p];
    a.tiles = ts.d_tiles[p];
    a.T = ts.T;
    a.Ls = h->p.Ls;
    a.nrhs = c.nrhs;
    a.N5 = h->p.Ls * c.nrhs;
    a.scale = c.scale;
    a.d = h->f5[0].d;
    a.e = h->f5[0].e;
    a.mf = h->p.mf;
    a.partial = c.partial;
    a.err = h->d_err;
    a.chunk = c.chunk > 0 ? c.chunk : 1;
    a.b5 = h->p.b5;
    a.c5 = h->p.c5;
    a.fa = h->f5[0].a;
    a.inv_d = h->f5[0].inv_d;
    a.inv_den = h->f5[0].inv_den;
    a.cg_x = c.cg_x;
    a.cg_r = c.cg_r;
    a.cg_p = c.cg_p;
    a.alpha = c.alpha;
    a.run = c.run;
    const int TPS = a.N5 / VL;
    // site groups per CTA: as many as fit in 256 threads, at most T
    int groups = 256 / TPS;
    if (groups > ts.T) groups = ts.T;
    if (groups < 1) {
        set_error("hop: %d threads per site exceed 256", TPS);
        return DWF_ERR_ARG;
    }
    int threads = (groups * TPS + 31) / 32 * 32;
    const size_t smem = hop_smem(ts.T, sizeof(SL), threads / 32, c.nrhs);
    const int nt = ts.ntiles[p];
    if (nt == 0) return DWF_OK;
    a.ntiles = nt;
    void (*kern)(const HopArgs);
    const bool moo = c.xmoo != nullptr;
    if (c.post) {
        if constexpr (std::is_same<R, float>::value && std::is_same<Sout, float>::value) {
            if (!c.dagger || !moo || 32 % TPS != 0 || c.cg_x == nullptr || c.cg_r == nullptr ||
                c.cg_p == nullptr || c.alpha == nullptr) {
                set_error("hop: fused M_pc^+ tail needs the adjoint, t, the CG vectors and "
                          "site groups that divide a warp");
                return DWF_ERR_ARG;
            }
            kern = k_hop<Sin, Sout, SL, R, VL, true, EPI_POST, CN5>;
        } else {
            set_error("hop: fused M_pc^+ tail needs FP32 arithmetic and FP32 vectors");
            return DWF_ERR_UNSUPPORTED;
        }
    } else if (c.bminv) {
        if constexpr (std::is_same<R, float>::value) {
            if (moo || 32 % TPS != 0) {
                set_error("hop: fused B M_ee^-1 needs site groups that divide a warp");
                return DWF_ERR_ARG;
            }
            kern = c.dagger ? k_hop<Sin, Sout, SL, R, VL, true, EPI_BMINV, CN5>
                            : k_hop<Sin, Sout, SL, R, VL, false, EPI_BMINV, CN5>;
        } else {
            set_error("hop: fused B M_ee^-1 needs FP32 arithmetic");
            return DWF_ERR_UNSUPPORTED;
        }
    } else if (c.dagger)
        kern = moo ? k_hop<Sin, Sout, SL, R, VL, true, EPI_MOO, CN5>
                   : k_hop<Sin, Sout, SL, R, VL, true, EPI_PLAIN, CN5>;
    else
        kern = moo ? k_hop<Sin, Sout, SL, R, VL, false, EPI_MOO, CN5>
                   : k_hop<Sin, Sout, SL, R, VL, false, EPI_PLAIN, CN5>;
    if (smem > kHopMaxSmem) {
        set_error("hop: tile of %d sites needs %zu bytes of shared memory", ts.T, smem);
        return DWF_ERR_ARG;
    }
    // persistent grid: as many CTAs as are resident at once, at most one per tile
    int grid = 0;
    DWF_TRY(persistent_grid((const void*)kern, threads, smem, nt, &grid));
    kern<<<grid, threads, smem, s>>>(a);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

// FP32-arithmetic hop: two lanes per thread unless the call asks for one
// (FP32 links only).
template <class Sin, class Sout, class SL>
static dwf_status launch_f32(dwf_handle* h, const HopCall& c, const TileSet& ts, cudaStream_t s) {
    const int N5 = h->p.Ls * c.nrhs;
    if constexpr (std::is_same<SL, float>::value) {
        if (c.VL == 1) {
            if (N5 == 12) return launch_t<Sin, Sout, SL, float, 1, 12>(h, c, ts, s);
            if (N5 == 16) return launch_t<Sin, Sout, SL, float, 1, 16>(h, c, ts, s);
            return launch_t<Sin, Sout, SL, float, 1>(h, c, ts, s);
        }
    }
    constexpr bool spec = (std::is_same<SL, float>::value && std::is_same<Sin, float>::value &&
                           std::is_same<Sout, float>::value) ||
                          (std::is_same<Sin, bf16>::value && std::is_same<Sout, bf16>::value);
    if constexpr (spec) {
        if (N5 == 12) return launch_t<Sin, Sout, SL, float, 2, 12>(h, c, ts, s);
        if (N5 == 16) return launch_t<Sin, Sout, SL, float, 2, 16>(h, c, ts, s);
    }
    return launch_t<Sin, Sout, SL, float, 2>(h, c, ts, s);
}

// Raise the dynamic shared-memory limit of every hop instantiation once, so
// that launches recorded into a CUDA graph never need a host-side call.
template <class Sin, class Sout, class SL, class R, int VL, int CN5 = 0>
static cudaError_t hop_attr() {
    cudaError_t e = cudaSuccess;
    void (*k[4])(const HopArgs) = {k_hop<Sin, Sout, SL, R, VL, false, EPI_PLAIN, CN5>,
                                   k_hop<Sin, Sout, SL, R, VL, false, EPI_MOO, CN5>,
                                   k_hop<Sin, Sout, SL, R, VL, true, EPI_PLAIN, CN5>,
                                   k_hop<Sin, Sout, SL, R, VL, true, EPI_MOO, CN5>};
    for (auto f : k) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kHopMaxSmem);
        if (r != cudaSuccess) e = r;
    }
    if constexpr (std::is_same<R, float>::value && std::is_same<Sout, float>::value) {
        cudaError_t r = cudaFuncSetAttribute(k_hop<Sin, Sout, SL, R, VL, true, EPI_POST, CN5>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kHopMaxSmem);
        if (r != cudaSuccess) e = r;
    }
    if constexpr (std::is_same<R, float>::value) {
        cudaError_t r = cudaFuncSetAttribute(k_hop<Sin, Sout, SL, R, VL, false, EPI_BMINV, CN5>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kHopMaxSmem);
        if (r != cudaSuccess) e = r;
        r = cudaFuncSetAttribute(k_hop<Sin, Sout, SL, R, VL, true, EPI_BMINV, CN5>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kHopMaxSmem);
        if (r != cudaSuccess) e = r;
    }
    return e;
}

dwf_status init_hop_kernels() {
    DWF_CUDA((hop_attr<double, double, double, double, 1>()));
    DWF_CUDA((hop_attr<float, float, float, float, 2>()));
    DWF_CUDA((hop_attr<float, float, float, float, 1>()));
    DWF_CUDA((hop_attr<bf16, bf16, bf16, float, 2>()));
    DWF_CUDA((hop_attr<bf16, float, bf16, float, 2>()));
    DWF_CUDA((hop_attr<float, bf16, bf16, float, 2>()));
    DWF_CUDA((hop_attr<float, float, bf16, float, 2>()));
    DWF_CUDA((hop_attr<float, float, float, float, 2, 12>()));
    DWF_CUDA((hop_attr<float, float, float, float, 2, 16>()));
    DWF_CUDA((hop_attr<float, float, float, float, 1, 12>()));
    DWF_CUDA((hop_attr<float, float, float, float, 1, 16>()));
    DWF_CUDA((hop_attr<bf16, bf16, bf16, float, 2, 12>()));
    DWF_CUDA((hop_attr<bf16, bf16, bf16, float, 2, 16>()));
    return DWF_OK;
}

bool hop_post_ok(const dwf_handle* h, dwf_prec op, dwf_prec vec, int nrhs, int VL) {
    if (vec != DWF_FP32 || (op != DWF_FP32 && op != DWF_BF16)) return false;
    const int n5 = h->p.Ls * nrhs;
    const int vl = op == DWF_BF16 ? 2 : (VL == 1 ? 1 : 2);
    const int tps = n5 / vl;
    return n5 % vl == 0 && tps <= 32 && 32 % tps == 0;
}

bool hop_bminv_ok(const dwf_handle* h, dwf_prec op, int nrhs, int VL) {
    if (op != DWF_FP32 && op != DWF_BF16) return false;
    const int n5 = h->p.Ls * nrhs;
    const int vl = op == DWF_BF16 ? 2 : (VL == 1 ? 1 : 2);
    const int tps = n5 / vl;
    return n5 % vl == 0 && tps <= 32 && 32 % tps == 0;
}

dwf_status launch_hop(dwf_handle* h, const HopCall& c, cudaStream_t s) {
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, tile_or_default(c.T), &tsp));
    const TileSet& ts = *tsp;
    if (c.prec_link == DWF_FP64) {
        if (c.prec_in != DWF_FP64 || c.prec_out != DWF_FP64) return DWF_ERR_UNSUPPORTED;
        return launch_t<double, double, double, double, 1>(h, c, ts, s);
    }
    if (c.prec_link == DWF_FP32) {
        if (c.prec_in != DWF_FP32 || c.prec_out != DWF_FP32) return DWF_ERR_UNSUPPORTED;
        return launch_f32<float, float, float>(h, c, ts, s);
    }
    // BF16 links: FP32 arithmetic, operands FP32 or BF16
    if (c.tc) return launch_hop_tc(h, c, ts, s);
    if (c.prec_in == DWF_BF16 && c.prec_out == DWF_BF16) return launch_f32<bf16, bf16, bf16>(h, c, ts, s);
    if (c.prec_in == DWF_BF16 && c.prec_out == DWF_FP32) return launch_f32<bf16, float, bf16>(h, c, ts, s);
    if (c.prec_in == DWF_FP32 && c.prec_out == DWF_BF16) return launch_f32<float, bf16, bf16>(h, c, ts, s);
    if (c.prec_in == DWF_FP32 && c.prec_out == DWF_FP32) return launch_f32<float, float, bf16>(h, c, ts, s);
    return DWF_ERR_UNSUPPORTED;
}

}  // namespace dwf
