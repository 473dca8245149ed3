// Right-preconditioned flexible GCR(k) on the normal equations of the Schur
// system, A x_o = M_pc^+ b'_o with A = M_pc^+ M_pc, with the learned
// preconditioner K (or none), all boxes and right-hand sides at once.  (On
// M_pc itself restarted GCR stalls for Moebius DWF: the field of values of
// the Schur operator contains the origin.)
//
//   z_j = K r;  q_j = A z_j;
//   modified Gram-Schmidt: for i < j: beta = <q_i, q_j>, q_j -= beta q_i, z_j -= beta z_i;
//   q_j, z_j /= |q_j|;  a = <q_j, r>;  x += a z_j;  r -= a q_j;
//   restart after k steps (or when |r| reaches the target) with the residual
//   recomputed in FP64 from the FP64 solution.
//
// The inner vectors and operator are FP32; solution increments flush into
// the FP64 solution at every restart; inner products are deterministic FP64
// reductions.  x_e is reconstructed and |b - D x| recomputed in FP64 at the
// end, as for CGNE.
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

// partial[tile][rhs] = Re <a, b>, partial_im[tile][rhs] = Im <a, b>  (FP32 fields)
__global__ void __launch_bounds__(512) k_cdot_partial(const int4* __restrict__ tiles, int nrhs, int Ls,
                                                      const float* __restrict__ a,
                                                      const float* __restrict__ b, double* pre,
                                                      double* pim) {
    __shared__ double s_red[512];
    const int4 tl = tiles[blockIdx.x];
    const int rows = tl.z * 12 * nrhs;
    const int64_t off = (int64_t)tl.y * 12 * nrhs * Ls;
    double accr = 0.0, acci = 0.0;
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const float* pa = a + 2 * (off + (int64_t)row * Ls);
        const float* pb = b + 2 * (off + (int64_t)row * Ls);
        float sr = 0.f, si = 0.f;
        for (int s = 0; s < Ls; ++s) {
            const float ar = pa[2 * s], ai = pa[2 * s + 1], br = pb[2 * s], bi = pb[2 * s + 1];
            sr += ar * br + ai * bi;     // conj(a) b
            si += ar * bi - ai * br;
        }
        accr += sr;
        acci += si;
    }
    const int nr = nrhs;
    auto rhs = [&](int t) { return t < rows ? t % nr : -1; };
    block_rhs_reduce(accr, s_red, nrhs, rhs, pre + (size_t)blockIdx.x * nrhs);
    block_rhs_reduce(acci, s_red, nrhs, rhs, pim + (size_t)blockIdx.x * nrhs);
}

// y += c x with complex c per system (cre, cim arrays), FP32 fields
__global__ void k_caxpy(const int4* __restrict__ tiles, int nrhs, int Ls, const double* cre,
                        const double* cim, const float* __restrict__ x, float* __restrict__ y) {
    const int4 tl = tiles[blockIdx.x];
    const int n = tl.z * 12 * nrhs * Ls;
    const int64_t off = (int64_t)tl.y * 12 * nrhs * Ls;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int sys = tl.x * nrhs + (i / Ls) % nrhs;
        const float cr = (float)cre[sys], ci = (float)cim[sys];
        const float2 xv = reinterpret_cast<const float2*>(x)[off + i];
        float2 yv = reinterpret_cast<float2*>(y)[off + i];
        yv.x += cr * xv.x - ci * xv.y;
        yv.y += cr * xv.y + ci * xv.x;
        reinterpret_cast<float2*>(y)[off + i] = yv;
    }
}

// Partial sums per (i, tile, rhs) of <Q_i, v>: the inner products of
// classical Gram-Schmidt against all previous directions at once.  A CTA
// takes one tile and up to kDotGroup directions i = kDotGroup * blockIdx.y + g,
// so v is read once per group instead of once per direction; each thread
// walks rows (one (site, colour-spin, rhs) row holds Ls contiguous complex
// lanes) in 16-byte steps of two lanes.
constexpr int kDotGroup = 8;
__global__ void __launch_bounds__(512) k_multi_cdot_partial(const int4* __restrict__ tiles, int ntiles, int nrhs,
                                                            int Ls, int nq, const float* __restrict__ Q,
                                                            size_t fstride, const float* __restrict__ v,
                                                            double* pre, double* pim) {
    __shared__ double s_red[512];
    const int i0 = blockIdx.y * kDotGroup;
    const int ng = min(kDotGroup, nq - i0);
    const int4 tl = tiles[blockIdx.x];
    const int rows = tl.z * 12 * nrhs;
    const int64_t off = (int64_t)tl.y * 12 * nrhs * Ls;
    double accr[kDotGroup], acci[kDotGroup];
#pragma unroll
    for (int g = 0; g < kDotGroup; ++g) accr[g] = acci[g] = 0.0;
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const int64_t base = 2 * (off + (int64_t)row * Ls);
        float sr[kDotGroup], si[kDotGroup];
#pragma unroll
        for (int g = 0; g < kDotGroup; ++g) sr[g] = si[g] = 0.f;
        for (int s2 = 0; s2 < Ls; s2 += 2) {
            const float4 b = *reinterpret_cast<const float4*>(v + base + 2 * s2);
#pragma unroll
            for (int g = 0; g < kDotGroup; ++g) {
                if (g < ng) {
                    const float4 a =
                        *reinterpret_cast<const float4*>(Q + (size_t)(i0 + g) * fstride + base + 2 * s2);
                    // conj(a) b for the two lanes
                    sr[g] += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
                    si[g] += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
                }
            }
        }
#pragma unroll
        for (int g = 0; g < kDotGroup; ++g) {
            accr[g] += sr[g];
            acci[g] += si[g];
        }
    }
    const int nr = nrhs;
    auto rhs = [&](int t) { return t < rows ? t % nr : -1; };
    for (int g = 0; g < ng; ++g) {
        const size_t o = ((size_t)(i0 + g) * ntiles + blockIdx.x) * nrhs;
        block_rhs_reduce(accr[g], s_red, nrhs, rhs, pre + o);
        block_rhs_reduce(acci[g], s_red, nrhs, rhs, pim + o);
    }
}

// c[i][sys] = sgn * sum over the box's tiles of the partials (0 for systems
// that are not active), i = blockIdx.y; fixed-order tree.
__global__ void k_multi_reduce(const double* __restrict__ pre, const double* __restrict__ pim,
                               const int* __restrict__ box_tb, int ntiles, int nrhs, const int* __restrict__ act,
                               double sgn, double* cre, double* cim) {
    __shared__ double sr[256], si[256];
    const int sys = blockIdx.x, i = blockIdx.y;
    const int nsys = gridDim.x;
    const int box = sys / nrhs, r = sys % nrhs;
    const int t0 = box_tb[box], t1 = box_tb[box + 1];
    double ar = 0.0, ai = 0.0;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const size_t o = ((size_t)i * ntiles + t) * nrhs + r;
        ar += pre[o];
        ai += pim[o];
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            si[threadIdx.x] += si[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool on = act[sys] != 0;
        cre[(size_t)i * nsys + sys] = on ? sgn * sr[0] : 0.0;
        cim[(size_t)i * nsys + sys] = on ? sgn * si[0] : 0.0;
    }
}

// y -= sum_{i<j} c_i Q_i and z -= sum_{i<j} c_i Z_i (complex c per system).
constexpr int kAxpyGroup = 8;
__global__ void k_multi_caxpy(const int4* __restrict__ tiles, int nrhs, int Ls, int nsys, int j,
                              const double* __restrict__ cre, const double* __restrict__ cim,
                              const float* __restrict__ Q, const float* __restrict__ Z, size_t fstride,
                              float* __restrict__ y, float* __restrict__ z) {
    const int4 tl = tiles[blockIdx.x];
    const int n = tl.z * 12 * nrhs * Ls;
    const int64_t off = (int64_t)tl.y * 12 * nrhs * Ls;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int sys = tl.x * nrhs + (e / Ls) % nrhs;
        float2 yv = reinterpret_cast<float2*>(y)[off + e];
        float2 zv = reinterpret_cast<float2*>(z)[off + e];
        // directions in groups of 8 with all their loads issued before the
        // updates (more loads in flight per thread); the updates keep the
        // order i = 0, 1, ..., so the result does not depend on the grouping
        int i = 0;
        for (; i + kAxpyGroup <= j; i += kAxpyGroup) {
            float2 q[kAxpyGroup], w[kAxpyGroup];
            float cr[kAxpyGroup], ci[kAxpyGroup];
#pragma unroll
            for (int u = 0; u < kAxpyGroup; ++u) {
                cr[u] = (float)cre[(size_t)(i + u) * nsys + sys];
                ci[u] = (float)cim[(size_t)(i + u) * nsys + sys];
                q[u] = reinterpret_cast<const float2*>(Q + (size_t)(i + u) * fstride)[off + e];
                w[u] = reinterpret_cast<const float2*>(Z + (size_t)(i + u) * fstride)[off + e];
            }
#pragma unroll
            for (int u = 0; u < kAxpyGroup; ++u) {
                yv.x -= cr[u] * q[u].x - ci[u] * q[u].y;
                yv.y -= cr[u] * q[u].y + ci[u] * q[u].x;
                zv.x -= cr[u] * w[u].x - ci[u] * w[u].y;
                zv.y -= cr[u] * w[u].y + ci[u] * w[u].x;
            }
        }
        for (; i < j; ++i) {
            const float cr = (float)cre[(size_t)i * nsys + sys], ci = (float)cim[(size_t)i * nsys + sys];
            const float2 q = reinterpret_cast<const float2*>(Q + (size_t)i * fstride)[off + e];
            const float2 w = reinterpret_cast<const float2*>(Z + (size_t)i * fstride)[off + e];
            yv.x -= cr * q.x - ci * q.y;
            yv.y -= cr * q.y + ci * q.x;
            zv.x -= cr * w.x - ci * w.y;
            zv.y -= cr * w.y + ci * w.x;
        }
        reinterpret_cast<float2*>(y)[off + e] = yv;
        reinterpret_cast<float2*>(z)[off + e] = zv;
    }
}

// inv[sys] = active and n2 > 0 ? 1 / sqrt(n2) : 0
__global__ void k_inv_norm(const double* __restrict__ n2, const int* __restrict__ act, int nsys, double* inv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsys) inv[i] = (act[i] != 0 && n2[i] > 0.0) ? 1.0 / sqrt(n2[i]) : 0.0;
}

struct GcrWS {
    int nrhs = 0, k = 0;
    float* q = nullptr;   // k fields
    float* zz = nullptr;  // k fields
    float* r = nullptr;
    float* xlo = nullptr;
    void* tA = nullptr;
    void* tB = nullptr;
    double* x64 = nullptr;
    double* bp64 = nullptr;
    double* t64a = nullptr;
    double* t64b = nullptr;
    double* t64c = nullptr;
    double* full64 = nullptr;
    double* t64d = nullptr;
    float* t32 = nullptr;
    double* part = nullptr;
    double* scal = nullptr;   // per-system scalars [8][nsys]
    double* mpart = nullptr;  // Gram-Schmidt partials [2][k][ntiles][nrhs]
    double* mcoef = nullptr;  // Gram-Schmidt coefficients [2][k][nsys]
    int* act = nullptr;       // per-system active flags (device)
};

static std::map<dwf_handle*, GcrWS> g_gcr;

void free_gcr_ws(dwf_handle* h) {
    auto it = g_gcr.find(h);
    if (it == g_gcr.end()) return;
    GcrWS& w = it->second;
    void* p[] = {w.q, w.zz, w.r, w.xlo, w.tA, w.tB, w.x64, w.bp64, w.t64a, w.t64b, w.t64c, w.full64,
                 w.t64d, w.t32, w.part, w.scal, w.mpart, w.mcoef, w.act};
    for (void* q : p) cudaFree(q);
    g_gcr.erase(it);
}

static dwf_status gcr_ws(dwf_handle* h, int nrhs, int k, GcrWS** out) {
    GcrWS& w = g_gcr[h];
    if (w.nrhs != nrhs || w.k != k) {
        free_gcr_ws(h);
        GcrWS& v = g_gcr[h];
        const size_t no = cb_elems(h, 1, nrhs), ne = cb_elems(h, 0, nrhs);
        const size_t nm = no > ne ? no : ne;
        DWF_CUDA(dev_malloc(&v.q, (size_t)k * no * 8));
        DWF_CUDA(dev_malloc(&v.zz, (size_t)k * no * 8));
        DWF_CUDA(dev_malloc(&v.r, no * 8));
        DWF_CUDA(dev_malloc(&v.xlo, no * 8));
        DWF_CUDA(dev_malloc(&v.tA, nm * 16));
        DWF_CUDA(dev_malloc(&v.tB, nm * 16));
        DWF_CUDA(dev_malloc(&v.x64, no * 16));
        DWF_CUDA(dev_malloc(&v.bp64, no * 16));
        DWF_CUDA(dev_malloc(&v.t64a, nm * 16));
        DWF_CUDA(dev_malloc(&v.t64b, nm * 16));
        DWF_CUDA(dev_malloc(&v.t64c, nm * 16));
        DWF_CUDA(dev_malloc(&v.full64, (no + ne) * 16));
        DWF_CUDA(dev_malloc(&v.t64d, no * 16));
        DWF_CUDA(dev_malloc(&v.t32, no * 8));
        const int64_t nsmax = h->nsite[0] > h->nsite[1] ? h->nsite[0] : h->nsite[1];
        DWF_CUDA(dev_malloc(&v.part, (size_t)2 * (nsmax / kMinTile + h->nbox + 1) * nrhs * 8));
        DWF_CUDA(dev_malloc(&v.scal, (size_t)8 * h->nbox * nrhs * 8));
        DWF_CUDA(dev_malloc(&v.mpart, (size_t)2 * k * (nsmax / kMinTile + h->nbox + 1) * nrhs * 8));
        DWF_CUDA(dev_malloc(&v.mcoef, (size_t)2 * k * h->nbox * nrhs * 8));
        DWF_CUDA(dev_malloc(&v.act, (size_t)h->nbox * nrhs * sizeof(int)));
        v.nrhs = nrhs;
        v.k = k;
        *out = &v;
        return DWF_OK;
    }
    *out = &w;
    return DWF_OK;
}

dwf_status nn_apply_internal(dwf_nn* K, dwf_handle* h, float* out, const float* in, int nrhs,
                             cudaStream_t s);
dwf_status mg_apply(dwf_mg* mg, float* z, const float* r, cudaStream_t s);

dwf_status gcr_solve(dwf_handle* h, double* x, const double* b, int nrhs, dwf_nn* K, dwf_mg* mg,
                     const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t user) {
    auto t0 = std::chrono::steady_clock::now();
    if (!h->have_gauge || !x || !b || !sp || nrhs < 1 || nrhs > h->nrhs_max || !(sp->tol > 0)) {
        set_error("dwf_gcr_solve: bad arguments");
        return DWF_ERR_ARG;
    }
    const int k = sp->restart > 0 ? sp->restart : 16;
    GcrWS* wp;
    DWF_TRY(gcr_ws(h, nrhs, k, &wp));
    GcrWS& w = *wp;
    cudaStream_t s = user;
    const int nsys = h->nbox * nrhs;
    const int T = tile_for(h, nrhs);
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, T, &tsp));
    const TileSet& ts = *tsp;
    const size_t ne = cb_elems(h, 0, nrhs), no = cb_elems(h, 1, nrhs);
    const double* be = b;
    const double* bo = b + 2 * ne;
    double* xe = x;
    double* xo = x + 2 * ne;
    double* pre = w.part;
    double* pim = w.part + (ts.ntiles[1] + 1) * (size_t)nrhs;
    double* s_re = w.scal;
    double* s_im = w.scal + nsys;
    double* s_c2 = w.scal + 2 * nsys;   // coefficients
    double* s_c3 = w.scal + 3 * nsys;
    std::vector<double> hre(nsys), him(nsys), hc(2 * nsys);
    int cdot_threads = 32;
    while (cdot_threads % nrhs) cdot_threads += 32;    // lcm(32, nrhs): fixed rhs per thread
    if (cdot_threads > 512) {
        set_error("dwf_gcr_solve: nrhs = %d unsupported", nrhs);
        return DWF_ERR_UNSUPPORTED;
    }
    if (cdot_threads < 256) cdot_threads *= 256 / cdot_threads;
    auto norm2 = [&](int parity, const void* f, dwf_prec pr, std::vector<double>& out) -> dwf_status {
        DWF_TRY(launch_dot_partial(h, parity, f, f, pr, pr, nrhs, pre, T, s));
        DWF_TRY(launch_reduce_sys(h, parity, pre, nrhs, s_re, T, s));
        DWF_CUDA(cudaMemcpyAsync(out.data(), s_re, nsys * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        return DWF_OK;
    };
    auto cdot = [&](const float* a, const float* bb) -> dwf_status {
        k_cdot_partial<<<ts.ntiles[1], cdot_threads, 0, s>>>(ts.d_tiles[1], nrhs, h->p.Ls, a, bb, pre, pim);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_TRY(launch_reduce_sys(h, 1, pre, nrhs, s_re, T, s));
        DWF_TRY(launch_reduce_sys(h, 1, pim, nrhs, s_im, T, s));
        DWF_CUDA(cudaMemcpyAsync(hre.data(), s_re, nsys * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaMemcpyAsync(him.data(), s_im, nsys * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        return DWF_OK;
    };
    auto caxpy = [&](const std::vector<std::complex<double>>& c, const float* xx, float* yy) -> dwf_status {
        for (int i = 0; i < nsys; ++i) { hc[i] = c[i].real(); hc[nsys + i] = c[i].imag(); }
        DWF_CUDA(cudaMemcpyAsync(s_c2, hc.data(), nsys * 8, cudaMemcpyHostToDevice, s));
        DWF_CUDA(cudaMemcpyAsync(s_c3, hc.data() + nsys, nsys * 8, cudaMemcpyHostToDevice, s));
        k_caxpy<<<ts.ntiles[1], 256, 0, s>>>(ts.d_tiles[1], nrhs, h->p.Ls, s_c2, s_c3, xx, yy);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_CUDA(cudaStreamSynchronize(s));   // hc is reused by the next call
        return DWF_OK;
    };

    // |b| per system, b'_o, initial x
    std::vector<double> bn2(nsys), tmp(nsys);
    DWF_TRY(norm2(0, be, DWF_FP64, tmp));
    DWF_TRY(norm2(1, bo, DWF_FP64, bn2));
    std::vector<double> bnorm(nsys);
    for (int i = 0; i < nsys; ++i) bnorm[i] = std::sqrt(bn2[i] + tmp[i]);
    DWF_TRY(op_local(h, L_MINV, w.t64a, be, nullptr, 0, 0, DWF_FP64, DWF_FP64, DWF_FP64, nrhs, 1.0, nullptr, s));
    DWF_TRY(op_dslash_eo(h, w.t64b, w.t64a, 1, 0, DWF_FP64, nrhs, w.t64c, s));
    DWF_CUDA(cudaMemcpyAsync(w.bp64, bo, no * 16, cudaMemcpyDeviceToDevice, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, -1.0, w.t64b, DWF_FP64, nullptr, 1.0, w.bp64, DWF_FP64, nullptr, T, s));
    if (sp->use_x0) DWF_CUDA(cudaMemcpyAsync(w.x64, xo, no * 16, cudaMemcpyDeviceToDevice, s));
    else DWF_CUDA(cudaMemsetAsync(w.x64, 0, no * 16, s));

    std::vector<int> active(nsys, 1), status(nsys, DWF_ERR_NOT_CONVERGED), iters(nsys, 0), restarts(nsys, 0);
    std::vector<double> tres(nsys, 1.0);
    int total_iters = 0;
    bool timed_out = false;
    std::vector<double> target(nsys, 0.0), best(nsys, 1e300);
    std::vector<int> stall(nsys, 0);
    bool fallback = false;
    for (;;) {
        // res = b' - M_pc x (FP64): the true residual test; r = M_pc^+ res
        DWF_TRY(op_mpc(h, w.t64c, w.x64, 0, DWF_FP64, DWF_FP64, nrhs, w.t64a, w.t64b, nullptr, nullptr, s));
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, w.bp64, DWF_FP64, nullptr, -1.0, w.t64c, DWF_FP64, nullptr, T, s));
        std::vector<double> rn2(nsys), nn2(nsys);
        DWF_TRY(norm2(1, w.t64c, DWF_FP64, rn2));
        DWF_TRY(op_mpc(h, w.t64d, w.t64c, 1, DWF_FP64, DWF_FP64, nrhs, w.t64a, w.t64b, nullptr, nullptr, s));
        DWF_TRY(norm2(1, w.t64d, DWF_FP64, nn2));
        bool any = false;
        for (int i = 0; i < nsys; ++i) {
            const double bn = bnorm[i] > 0 ? bnorm[i] : 1.0;
            tres[i] = std::sqrt(rn2[i]) / bn;
            if (!(tres[i] == tres[i])) { status[i] = DWF_ERR_NAN; active[i] = 0; }
            if (active[i] && tres[i] <= 0.9 * sp->tol) { status[i] = DWF_OK; active[i] = 0; }
            if (active[i] && iters[i] >= sp->maxiter) active[i] = 0;
            // a preconditioner that stops reducing the true residual for two
            // restarts hands the system to the CG fallback
            if (active[i]) {
                if (tres[i] < 0.99 * best[i]) { best[i] = tres[i]; stall[i] = 0; }
                else if (++stall[i] >= 2) { fallback = true; active[i] = 0; }
            }
            if (active[i]) {
                // inner target for |A e| from the observed |M^+ res| / |res|
                const double ratio = rn2[i] > 0 ? std::sqrt(nn2[i] / rn2[i]) : 1.0;
                const double tg = 0.5 * sp->tol * bn * ratio;
                target[i] = target[i] > 0 ? std::min(0.3 * target[i], tg) : tg;
            }
            any |= active[i] != 0;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (sp->max_seconds > 0 && el > sp->max_seconds) { timed_out = true; break; }
        if (!any) break;
        DWF_TRY(launch_convert(w.r, DWF_FP32, w.t64d, DWF_FP64, no, s));
        DWF_CUDA(cudaMemsetAsync(w.xlo, 0, no * 8, s));
        // inner GCR cycle: Gram-Schmidt, normalisation and the x, r updates run
        // with device-side coefficients; the host reads |r|^2 once per step
        {
            std::vector<int> a(active.begin(), active.end());
            DWF_CUDA(cudaMemcpyAsync(w.act, a.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, s));
            DWF_CUDA(cudaStreamSynchronize(s));   // a is a host temporary
        }
        const size_t fs = no * 2;                 // floats per field
        const int ntl = ts.ntiles[1];
        const int* box_tb = ts.d_box_tile_begin[1];
        double* mre = w.mcoef;
        double* mim = w.mcoef + (size_t)k * nsys;
        double* ppre = w.mpart;
        double* ppim = w.mpart + (size_t)k * ntl * nrhs;
        double* a_re = w.scal + 4 * (size_t)nsys;   // <q_j, r> and its negative
        double* a_im = w.scal + 5 * (size_t)nsys;
        double* an_re = w.scal + 6 * (size_t)nsys;
        double* an_im = w.scal + 7 * (size_t)nsys;
        // one classical Gram-Schmidt pass of (q_j, z_j) against the j previous pairs
        auto project = [&](int j, float* qj, float* zj) -> dwf_status {
            k_multi_cdot_partial<<<dim3(ntl, (j + kDotGroup - 1) / kDotGroup), cdot_threads, 0, s>>>(
                ts.d_tiles[1], ntl, nrhs, h->p.Ls, j, w.q, fs, qj, ppre, ppim);
            note_launch();
            k_multi_reduce<<<dim3(nsys, j), 256, 0, s>>>(ppre, ppim, box_tb, ntl, nrhs, w.act, 1.0, mre, mim);
            note_launch();
            k_multi_caxpy<<<ntl, 256, 0, s>>>(ts.d_tiles[1], nrhs, h->p.Ls, nsys, j, mre, mim, w.q, w.zz, fs, qj, zj);
            note_launch();
            DWF_CUDA(cudaGetLastError());
            return DWF_OK;
        };
        for (int j = 0; j < k; ++j) {
            float* qj = w.q + (size_t)j * no * 2;
            float* zj = w.zz + (size_t)j * no * 2;
            if (mg) DWF_TRY(mg_apply(mg, zj, w.r, s));
            else if (K) DWF_TRY(nn_apply_internal(K, h, zj, w.r, nrhs, s));
            else DWF_CUDA(cudaMemcpyAsync(zj, w.r, no * 8, cudaMemcpyDeviceToDevice, s));
            DWF_TRY(op_mpc(h, w.t32, zj, 0, DWF_FP32, DWF_FP32, nrhs, w.tA, w.tB, nullptr, nullptr, s));
            DWF_TRY(op_mpc(h, qj, w.t32, 1, DWF_FP32, DWF_FP32, nrhs, w.tA, w.tB, nullptr, nullptr, s));
            if (j > 0) {
                // classical Gram-Schmidt with all inner products at once, and a
                // second pass where the first lost orthogonality: the criterion of
                // Daniel, Gragg, Kaufman and Stewart (1976), repeat when the pass
                // shrank |q_j| by more than 1/sqrt(2) (any active system decides)
                std::vector<double> n0(nsys), n1(nsys);
                DWF_TRY(norm2(1, qj, DWF_FP32, n0));
                DWF_TRY(project(j, qj, zj));
                DWF_TRY(norm2(1, qj, DWF_FP32, n1));
                bool again = false;
                for (int m = 0; m < nsys; ++m)
                    if (active[m] && !(n1[m] >= 0.5 * n0[m])) again = true;
                if (again) DWF_TRY(project(j, qj, zj));
            }
            // q_j, z_j /= |q_j|
            DWF_TRY(launch_dot_partial(h, 1, qj, qj, DWF_FP32, DWF_FP32, nrhs, pre, T, s));
            DWF_TRY(launch_reduce_sys(h, 1, pre, nrhs, s_re, T, s));
            k_inv_norm<<<(nsys + 127) / 128, 128, 0, s>>>(s_re, w.act, nsys, s_c2);
            note_launch();
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 0.0, nullptr, DWF_FP32, s_c2, 0.0, qj, DWF_FP32, nullptr, T, s));
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 0.0, nullptr, DWF_FP32, s_c2, 0.0, zj, DWF_FP32, nullptr, T, s));
            // a = <q_j, r>: x += a z_j, r -= a q_j
            k_multi_cdot_partial<<<dim3(ntl, 1), cdot_threads, 0, s>>>(ts.d_tiles[1], ntl, nrhs, h->p.Ls, 1, qj, fs,
                                                                      w.r, ppre, ppim);
            note_launch();
            k_multi_reduce<<<dim3(nsys, 1), 256, 0, s>>>(ppre, ppim, box_tb, ntl, nrhs, w.act, 1.0, a_re, a_im);
            note_launch();
            k_multi_reduce<<<dim3(nsys, 1), 256, 0, s>>>(ppre, ppim, box_tb, ntl, nrhs, w.act, -1.0, an_re, an_im);
            note_launch();
            k_caxpy<<<ntl, 256, 0, s>>>(ts.d_tiles[1], nrhs, h->p.Ls, a_re, a_im, zj, w.xlo);
            note_launch();
            k_caxpy<<<ntl, 256, 0, s>>>(ts.d_tiles[1], nrhs, h->p.Ls, an_re, an_im, qj, w.r);
            note_launch();
            DWF_CUDA(cudaGetLastError());
            total_iters++;
            std::vector<double> rr(nsys);
            DWF_TRY(norm2(1, w.r, DWF_FP32, rr));
            bool cont = false;
            for (int m = 0; m < nsys; ++m)
                if (active[m]) {
                    iters[m]++;
                    const double bn = bnorm[m] > 0 ? bnorm[m] : 1.0;
                    (void)bn;
                    if (std::sqrt(rr[m]) > target[m] && iters[m] < sp->maxiter) cont = true;
                }
            if (!cont) break;
        }
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, w.xlo, DWF_FP32, nullptr, 1.0, w.x64, DWF_FP64, nullptr, T, s));
        for (int m = 0; m < nsys; ++m) if (active[m]) restarts[m]++;
    }
    // x_o, x_e and the FP64 residual of the full system
    DWF_CUDA(cudaMemcpyAsync(xo, w.x64, no * 16, cudaMemcpyDeviceToDevice, s));
    DWF_TRY(op_dslash_eo(h, w.t64a, xo, 0, 0, DWF_FP64, nrhs, w.t64c, s));
    DWF_TRY(launch_axpby(h, 0, nrhs, nullptr, 1.0, be, DWF_FP64, nullptr, -1.0, w.t64a, DWF_FP64, nullptr, T, s));
    DWF_TRY(op_local(h, L_MINV, xe, w.t64a, nullptr, 0, 0, DWF_FP64, DWF_FP64, DWF_FP64, nrhs, 1.0, nullptr, s));
    DWF_TRY(op_apply_d(h, w.full64, x, 0, DWF_FP64, nrhs, w.t64c, s));
    DWF_TRY(launch_axpby(h, 0, nrhs, nullptr, 1.0, be, DWF_FP64, nullptr, -1.0, w.full64, DWF_FP64, nullptr, T, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, bo, DWF_FP64, nullptr, -1.0, w.full64 + 2 * ne, DWF_FP64, nullptr, T, s));
    std::vector<double> f0(nsys), f1(nsys);
    DWF_TRY(norm2(0, w.full64, DWF_FP64, f0));
    DWF_TRY(norm2(1, w.full64 + 2 * ne, DWF_FP64, f1));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    dwf_status result = DWF_OK;
    for (int i = 0; i < nsys; ++i) {
        const double bn = bnorm[i] > 0 ? bnorm[i] : 1.0;
        const double tr = std::sqrt(f0[i] + f1[i]) / bn;
        if (timed_out && status[i] != DWF_OK) status[i] = DWF_ERR_TIMEOUT;
        if (status[i] == DWF_OK && !(tr <= sp->tol)) status[i] = DWF_ERR_NOT_CONVERGED;
        if (stats) {
            stats[i].iters = iters[i];
            stats[i].reliable_updates = restarts[i];
            stats[i].op_applies = iters[i] + restarts[i] + 1;
            stats[i].status = status[i];
            stats[i].true_resid = tr;
            stats[i].seconds = secs;
            stats[i].recorded = 0;
        }
        if (status[i] != DWF_OK && result == DWF_OK) result = (dwf_status)status[i];
    }
    if (fallback && result != DWF_OK && !timed_out) {
        // plain red-black CG from the current x (mixed precision, FP64 updates)
        dwf_solver_params cp = *sp;
        cp.use_x0 = 1;
        cp.inner_prec = DWF_FP32;
        cp.record_x = nullptr;
        std::vector<dwf_solver_stats> cst(nsys);
        const dwf_status r2 = cgne_solve(h, x, b, nrhs, &cp, cst.data(), s);
        const double secs2 = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < nsys && stats; ++i) {
            stats[i].iters += cst[i].iters;
            stats[i].reliable_updates += cst[i].reliable_updates;
            stats[i].op_applies += cst[i].op_applies;
            stats[i].status = cst[i].status;
            stats[i].true_resid = cst[i].true_resid;
            stats[i].seconds = secs2;
            stats[i].recorded = -1;   // marks a solve finished by the CG fallback
        }
        return r2;
    }
    if (result != DWF_OK) set_error("dwf_gcr_solve: not every system reached tol");
    return result;
}

}  // namespace dwf
