// Two-level aggregation multigrid for the normal Schur operator
// A = M_pc^+ M_pc of a handle's domain (the whole lattice, or each Dirichlet
// box: the local systems of Sec. 4), set up from Chebyshev-filtered vectors
// (dwf_chebyshev_filter), the set-up Sec. 4 proposes in place of inverse
// iteration.  The rest of the method is standard aggregation multigrid:
//
//   aggregates  4D blocks of the odd sites of each box (all Ls and spin-colour
//               components of a block together)
//   P           the near-null vectors restricted to each block and
//               orthonormalised there in vector order (classical Gram-Schmidt
//               with reorthogonalisation, P^+ P = 1)
//   A_c         P^+ A P (Galerkin), dense, inverted once (Gauss-Jordan on the device)
//   M^-1 r      V(1,1) cycle: z = S r; z += P A_c^-1 P^+ (r - A z);
//               z += S (r - A z), smoother S none, a Chebyshev iteration on
//               [lo, hi] or the learned network K
//
// used as the preconditioner of flexible GCR on A x = M_pc^+ b' (gcr.cu).
//
// Layouts: the basis is one odd cb FP32 field with nvec lanes per site,
// [site][12][k][s] complex (the layout of nvec right-hand sides), coarse
// vectors are complex FP64 c[r][block][k], A_c^-1 is row-major complex FP64.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {
dwf_status nn_apply_internal(dwf_nn* K, dwf_handle* h, float* out, const float* in, int nrhs,
                             cudaStream_t s);
}

struct dwf_mg {
    dwf_handle* h = nullptr;
    int block[4] = {0, 0, 0, 0};
    int nvec = 0, nb = 0, nc = 0;
    int* d_site_block = nullptr;   // [odd site] -> block
    int* d_blk_off = nullptr;      // [nb + 1] CSR offsets into d_blk_sites
    int* d_blk_sites = nullptr;    // odd sites of each block, in domain order
    float2* d_basis = nullptr;     // [site][12][nvec][Ls]
    double2* d_cinv = nullptr;     // nc x nc
    double2* d_c = nullptr;        // coarse vectors: 2 x nc (nrhs = 1) or nvec x nc (set-up)
    double2* d_ac = nullptr;       // set-up: A_c
    // odd cb FP32 scratch: [0] residual (nvec lanes in the set-up), [1] the
    // middle field of A (nvec lanes), [2..4] Chebyshev d, res, A d, [5] the
    // post-smoothing correction
    float* d_f[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void* d_ta = nullptr;          // operator temporaries (FP32, max(ne, no))
    void* d_tb = nullptr;
    bool ready = false;
    int smoother = 0;              // 0 none, 1 Chebyshev iteration, 2 learned K
    int steps = 0;
    double lo = 0.0, hi = 0.0;
    dwf_nn* K = nullptr;
};

namespace dwf {

static constexpr int kMgThreads = 256;

// Deterministic block sum of one double2 per thread (all threads call it).
__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();   // sh may still be read from the previous call
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t.x += sh[w].x; t.y += sh[w].y; }
    return t;
}

// Element e of a block (sites of the block in order, then 12 components, then s).
__device__ __forceinline__ size_t mg_elem(const int* sites, int e, int Ls, int nlane, int lane, int& site) {
    const int q = e / (12 * Ls);
    const int rem = e - q * 12 * Ls;
    const int c = rem / Ls, s = rem - c * Ls;
    site = sites[q];
    return ((size_t)((size_t)site * 12 + c) * nlane + lane) * Ls + s;
}

// out[b][j] = <B_j, B_k> over block b for j0 <= j < j0 + gridDim.y (one CTA
// per (block, j)): the inner products of Gram-Schmidt, all blocks at once.
__global__ void __launch_bounds__(kMgThreads) k_mg_bdot(const float2* __restrict__ basis, const int* __restrict__ off,
                                                        const int* __restrict__ sites, int nvec, int Ls, int k,
                                                        int j0, double2* out) {
    __shared__ double2 sh[32];
    const int b = blockIdx.x, j = j0 + blockIdx.y;
    const int* bs = sites + off[b];
    const int nel = (off[b + 1] - off[b]) * 12 * Ls;
    double2 acc = make_double2(0.0, 0.0);
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        int site;
        const float2 u = basis[mg_elem(bs, e, Ls, nvec, j, site)];
        const float2 w = basis[mg_elem(bs, e, Ls, nvec, k, site)];
        acc.x += (double)(u.x * w.x + u.y * w.y);     // conj(u) w
        acc.y += (double)(u.x * w.y - u.y * w.x);
    }
    const double2 d = block_sum2(acc, sh);
    if (threadIdx.x == 0) out[(size_t)b * nvec + j] = d;
}

// B_k -= sum_{j<k} d[b][j] B_j on every odd site (b its block): one
// classical Gram-Schmidt projection (thread per complex element of B_k).
__global__ void k_mg_bproj(float2* basis, const int* __restrict__ site_block, const double2* __restrict__ d,
                           int64_t nsites, int nvec, int Ls, int k) {
    const int64_t n = nsites * 12 * Ls;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ls);
        const int64_t sc = i / Ls;                      // site * 12 + component
        const int b = site_block[sc / 12];
        float2* row = basis + (size_t)sc * nvec * Ls + s;
        float2 w = row[(size_t)k * Ls];
        for (int j = 0; j < k; ++j) {
            const double2 c = d[(size_t)b * nvec + j];
            const float2 u = row[(size_t)j * Ls];
            w.x -= (float)c.x * u.x - (float)c.y * u.y;
            w.y -= (float)c.x * u.y + (float)c.y * u.x;
        }
        row[(size_t)k * Ls] = w;
    }
}

// B_k /= |B_k| per block (d[b][k] holds |B_k|^2 on block b); a vanishing
// norm sets the error word and leaves the vector.
__global__ void k_mg_bscale(float2* basis, const int* __restrict__ site_block, const double2* __restrict__ d,
                            int64_t nsites, int nvec, int Ls, int k, int* err) {
    const int64_t n = nsites * 12 * Ls;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ls);
        const int64_t sc = i / Ls;
        const int b = site_block[sc / 12];
        const double n2 = d[(size_t)b * nvec + k].x;
        if (!(n2 > 0.0)) {
            atomicOr(err, 1);
            continue;
        }
        const float inv = (float)(1.0 / sqrt(n2));
        float2* w = basis + ((size_t)sc * nvec + k) * Ls + s;
        w->x *= inv;
        w->y *= inv;
    }
}

// c[r][b][k] = <B_k on block b, f_r>: one CTA per (block, k, rhs).
__global__ void __launch_bounds__(kMgThreads) k_mg_restrict(const float2* __restrict__ basis,
                                                            const float2* __restrict__ f,
                                                            const int* __restrict__ off,
                                                            const int* __restrict__ sites, int nvec,
                                                            int nrhs, int Ls, int nb, double2* c) {
    __shared__ double2 sh[32];
    const int b = blockIdx.x, k = blockIdx.y, r = blockIdx.z;
    const int* bs = sites + off[b];
    const int nel = (off[b + 1] - off[b]) * 12 * Ls;
    double2 acc = make_double2(0.0, 0.0);
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        int site;
        const float2 u = basis[mg_elem(bs, e, Ls, nvec, k, site)];
        const int q = e / (12 * Ls);
        const int rem = e - q * 12 * Ls;
        const int cc = rem / Ls, s = rem - cc * Ls;
        const float2 w = f[((size_t)((size_t)site * 12 + cc) * nrhs + r) * Ls + s];
        acc.x += (double)(u.x * w.x + u.y * w.y);
        acc.y += (double)(u.x * w.y - u.y * w.x);
    }
    const double2 d = block_sum2(acc, sh);
    if (threadIdx.x == 0) c[((size_t)r * nb + b) * nvec + k] = d;
}

// f_r (+)= sum_k c[r][block(site)][k] B_k  (thread per complex element).
__global__ void k_mg_prolong(const float2* __restrict__ basis, const double2* __restrict__ c,
                             const int* __restrict__ site_block, int64_t nsites, int nvec, int nrhs,
                             int Ls, int nb, int add, float2* f) {
    const int64_t n = nsites * 12 * nrhs * Ls;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ls);
        const int r = (int)((i / Ls) % nrhs);
        const int64_t sc = i / ((int64_t)Ls * nrhs);          // site * 12 + component
        const int b = site_block[sc / 12];
        float xr = 0.f, xi = 0.f;
        if (b >= 0) {
            const double2* cb = c + ((size_t)r * nb + b) * nvec;
            const float2* u = basis + (size_t)sc * nvec * Ls + s;
            double ar = 0.0, ai = 0.0;
            for (int k = 0; k < nvec; ++k) {
                const float2 v = u[(size_t)k * Ls];
                const double2 ck = cb[k];
                ar += ck.x * v.x - ck.y * v.y;
                ai += ck.x * v.y + ck.y * v.x;
            }
            xr = (float)ar;
            xi = (float)ai;
        }
        if (add) {
            float2 o = f[i];
            o.x += xr;
            o.y += xi;
            f[i] = o;
        } else {
            f[i] = make_float2(xr, xi);
        }
    }
}

// f = basis lanes on block b0 only (k -> lane k), zero elsewhere: the
// prolongations of the coarse unit vectors (b0, k), k < nvec, as nvec lanes.
__global__ void k_mg_block_lanes(const float2* __restrict__ basis, const int* __restrict__ site_block,
                                 int64_t nsites, int nvec, int Ls, int b0, float2* f) {
    const int64_t n = nsites * 12 * nvec * Ls;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t site = i / ((int64_t)12 * nvec * Ls);
        f[i] = site_block[site] == b0 ? basis[i] : make_float2(0.f, 0.f);
    }
}

// y = M x, M row-major n x n complex (one warp per row, fixed order).
__global__ void k_mg_matvec(const double2* __restrict__ M, const double2* __restrict__ x, int n,
                            double2* y) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    double ar = 0.0, ai = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double2 m = M[(size_t)row * n + j], v = x[j];
        ar += m.x * v.x - m.y * v.y;
        ai += m.x * v.y + m.y * v.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_down_sync(0xffffffffu, ar, o);
        ai += __shfl_down_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) y[row] = make_double2(ar, ai);
}

static int mg_grid(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

static dwf_status mg_restrict(dwf_mg* mg, double2* c, const float* f, int nrhs, cudaStream_t s) {
    k_mg_restrict<<<dim3(mg->nb, mg->nvec, nrhs), kMgThreads, 0, s>>>(
        mg->d_basis, reinterpret_cast<const float2*>(f), mg->d_blk_off, mg->d_blk_sites, mg->nvec, nrhs,
        mg->h->p.Ls, mg->nb, c);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

static dwf_status mg_prolong(dwf_mg* mg, float* f, const double2* c, int nrhs, bool add, cudaStream_t s) {
    const int64_t ns = mg->h->nsite[1];
    k_mg_prolong<<<mg_grid(ns * 12 * nrhs * mg->h->p.Ls), 256, 0, s>>>(
        mg->d_basis, c, mg->d_site_block, ns, mg->nvec, nrhs, mg->h->p.Ls, mg->nb, add ? 1 : 0,
        reinterpret_cast<float2*>(f));
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

// dst = A src = M_pc^+ M_pc src, FP32, nrhs lanes
static dwf_status mg_A(dwf_mg* mg, float* dst, const float* src, float* mid, int nrhs, cudaStream_t s) {
    DWF_TRY(op_mpc(mg->h, mid, src, 0, DWF_FP32, DWF_FP32, nrhs, mg->d_ta, mg->d_tb, nullptr, nullptr, s));
    return op_mpc(mg->h, dst, mid, 1, DWF_FP32, DWF_FP32, nrhs, mg->d_ta, mg->d_tb, nullptr, nullptr, s);
}

// z = S r for the chosen smoother (z, r distinct; scratch d_f[2..4])
static dwf_status mg_smooth(dwf_mg* mg, float* z, const float* r, cudaStream_t s) {
    dwf_handle* h = mg->h;
    const int T = tile_for(h, 1);
    const size_t bytes = cb_elems(h, 1, 1) * 8;
    if (mg->smoother == 2) return nn_apply_internal(mg->K, h, z, r, 1, s);
    // Chebyshev iteration on [lo, hi] from z = 0 (steps - 1 applications of A)
    const double theta = 0.5 * (mg->hi + mg->lo), delta = 0.5 * (mg->hi - mg->lo);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    float* d = mg->d_f[2];
    float* res = mg->d_f[3];
    float* ad = mg->d_f[4];
    DWF_CUDA(cudaMemcpyAsync(res, r, bytes, cudaMemcpyDeviceToDevice, s));
    DWF_CUDA(cudaMemsetAsync(z, 0, bytes, s));
    DWF_TRY(launch_axpby(h, 1, 1, nullptr, 1.0 / theta, r, DWF_FP32, nullptr, 0.0, d, DWF_FP32, nullptr, T, s));
    for (int k = 0; k < mg->steps; ++k) {
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, 1.0, d, DWF_FP32, nullptr, 1.0, z, DWF_FP32, nullptr, T, s));
        if (k == mg->steps - 1) break;
        DWF_TRY(mg_A(mg, ad, d, mg->d_f[1], 1, s));
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, -1.0, ad, DWF_FP32, nullptr, 1.0, res, DWF_FP32, nullptr, T, s));
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, 2.0 * rho_new / delta, res, DWF_FP32, nullptr, rho_new * rho, d,
                             DWF_FP32, nullptr, T, s));
        rho = rho_new;
    }
    return DWF_OK;
}

dwf_status mg_apply(dwf_mg* mg, float* z, const float* r, cudaStream_t s) {
    dwf_handle* h = mg->h;
    const int T = tile_for(h, 1);
    const size_t bytes = cb_elems(h, 1, 1) * 8;
    float* t = mg->d_f[0];
    if (mg->smoother != 0) {
        DWF_TRY(mg_smooth(mg, z, r, s));
        DWF_TRY(mg_A(mg, t, z, mg->d_f[1], 1, s));
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, 1.0, r, DWF_FP32, nullptr, -1.0, t, DWF_FP32, nullptr, T, s));
    } else {
        DWF_CUDA(cudaMemsetAsync(z, 0, bytes, s));
        DWF_CUDA(cudaMemcpyAsync(t, r, bytes, cudaMemcpyDeviceToDevice, s));
    }
    DWF_TRY(mg_restrict(mg, mg->d_c, t, 1, s));
    const int nc = mg->nc;
    k_mg_matvec<<<(nc * 32 + 255) / 256, 256, 0, s>>>(mg->d_cinv, mg->d_c, nc, mg->d_c + nc);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    DWF_TRY(mg_prolong(mg, z, mg->d_c + nc, 1, true, s));
    if (mg->smoother != 0) {
        DWF_TRY(mg_A(mg, t, z, mg->d_f[1], 1, s));
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, 1.0, r, DWF_FP32, nullptr, -1.0, t, DWF_FP32, nullptr, T, s));
        float* u = mg->d_f[5];
        DWF_TRY(mg_smooth(mg, u, t, s));
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, 1.0, u, DWF_FP32, nullptr, 1.0, z, DWF_FP32, nullptr, T, s));
    }
    return DWF_OK;
}

// In-place inverse of a dense complex matrix (Gauss-Jordan, partial pivoting).
// Gauss-Jordan inversion with partial pivoting of the dense coarse operator on
// the device, FP64: the augmented rows [A | 1] (n x 2n, row-major), per
// column c the pivot (largest |a_rc|, r >= c, the smallest such r), the row
// swap and scaling, the column's factors, then every other row minus its
// factor times the pivot row.  n <= 4096.
__global__ void k_gj_identity(double2* M, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        M[(size_t)i * 2 * n + n + i] = make_double2(1.0, 0.0);
}

// the pivot row index and the pivot value (read here, before any row changes)
__global__ void k_gj_pivot(const double2* __restrict__ M, int n, int c, int* piv, double2* pval) {
    __shared__ double sv[256];
    __shared__ int si[256];
    double best = -1.0;
    int bi = n;
    for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
        const double2 v = M[(size_t)r * 2 * n + c];
        const double m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi = r; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const double o = sv[threadIdx.x + w];
            const int oi = si[threadIdx.x + w];
            if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool ok = sv[0] > 0.0 && si[0] < n;
        piv[0] = ok ? si[0] : -1;
        pval[0] = ok ? M[(size_t)si[0] * 2 * n + c] : make_double2(1.0, 0.0);
    }
}

// swap rows c and piv, scale row c by 1 / a_cc, and keep the column-c factors
// of every row (read before the elimination writes them)
__global__ void k_gj_swap_scale(double2* M, int n, int c, const int* __restrict__ piv,
                                const double2* __restrict__ pval, int* err) {
    const int p = piv[0];
    if (p < 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *err = 1;
        return;
    }
    const size_t ld = 2 * (size_t)n;
    const double2 d = pval[0];
    const double den = d.x * d.x + d.y * d.y;
    const double2 inv = make_double2(d.x / den, -d.y / den);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += gridDim.x * blockDim.x) {
        const double2 vp = M[(size_t)p * ld + j], vc = M[(size_t)c * ld + j];
        M[(size_t)c * ld + j] = make_double2(vp.x * inv.x - vp.y * inv.y, vp.x * inv.y + vp.y * inv.x);
        if (p != c) M[(size_t)p * ld + j] = vc;
    }
}

__global__ void k_gj_factors(const double2* __restrict__ M, int n, int c, const int* __restrict__ piv,
                             double2* fac) {
    if (piv[0] < 0) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        fac[r] = r == c ? make_double2(0.0, 0.0) : M[(size_t)r * 2 * n + c];
}

__global__ void k_gj_eliminate(double2* M, int n, int c, const int* __restrict__ piv,
                               const double2* __restrict__ fac) {
    if (piv[0] < 0) return;
    const size_t ld = 2 * (size_t)n;
    const int r = blockIdx.y;
    const double2 f = fac[r];
    if (f.x == 0.0 && f.y == 0.0) return;
    for (int j = c + blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += gridDim.x * blockDim.x) {
        const double2 pc = M[(size_t)c * ld + j];
        double2 v = M[(size_t)r * ld + j];
        v.x -= f.x * pc.x - f.y * pc.y;
        v.y -= f.x * pc.y + f.y * pc.x;
        M[(size_t)r * ld + j] = v;
    }
}

// d_out = A^-1 for the n x n complex matrix at A (device); false if singular.
static dwf_status invert_device(const double2* A, int n, double2* d_out, int* singular, cudaStream_t s) {
    double2* M = nullptr;
    double2* fac = nullptr;   // n factors, then the pivot value
    int* iw = nullptr;        // [0] pivot, [1] singular flag
    dwf_status st = DWF_OK;
    auto fail = [&](cudaError_t e) {
        if (e != cudaSuccess) {
            set_error("dwf_mg_setup: coarse inversion: %s", cudaGetErrorString(e));
            st = DWF_ERR_CUDA;
        }
        return e != cudaSuccess;
    };
    if (!fail(dev_malloc(&M, (size_t)n * 2 * n * sizeof(double2))) && !fail(dev_malloc(&fac, (size_t)(n + 1) * sizeof(double2))) &&
        !fail(dev_malloc(&iw, 2 * sizeof(int))) && !fail(cudaMemsetAsync(iw, 0, 2 * sizeof(int), s)) &&
        !fail(cudaMemsetAsync(M, 0, (size_t)n * 2 * n * sizeof(double2), s)) &&
        !fail(cudaMemcpy2DAsync(M, 2 * n * sizeof(double2), A, n * sizeof(double2), n * sizeof(double2), n,
                                cudaMemcpyDeviceToDevice, s))) {
        k_gj_identity<<<(n + 255) / 256, 256, 0, s>>>(M, n);   // the right half: element (i, n + i)
        note_launch();
        for (int c = 0; c < n && st == DWF_OK; ++c) {
            k_gj_pivot<<<1, 256, 0, s>>>(M, n, c, iw, fac + n);
            k_gj_swap_scale<<<(2 * n + 255) / 256, 256, 0, s>>>(M, n, c, iw, fac + n, iw + 1);
            k_gj_factors<<<(n + 255) / 256, 256, 0, s>>>(M, n, c, iw, fac);
            k_gj_eliminate<<<dim3((2 * n - c + 255) / 256, n), 256, 0, s>>>(M, n, c, iw, fac);
            note_launch();
            note_launch();
            note_launch();
            note_launch();
            fail(cudaGetLastError());
        }
        if (st == DWF_OK)
            fail(cudaMemcpy2DAsync(d_out, n * sizeof(double2), M + n, 2 * n * sizeof(double2), n * sizeof(double2), n,
                                   cudaMemcpyDeviceToDevice, s));
        if (st == DWF_OK) fail(cudaMemcpyAsync(singular, iw + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (st == DWF_OK) fail(cudaStreamSynchronize(s));
    }
    cudaStreamSynchronize(s);
    cudaFree(M);
    cudaFree(fac);
    cudaFree(iw);
    return st;
}

void free_mg(dwf_mg* mg) {
    cudaFree(mg->d_site_block);
    cudaFree(mg->d_blk_off);
    cudaFree(mg->d_blk_sites);
    cudaFree(mg->d_basis);
    cudaFree(mg->d_cinv);
    cudaFree(mg->d_c);
    cudaFree(mg->d_ac);
    for (float* f : mg->d_f) cudaFree(f);
    cudaFree(mg->d_ta);
    cudaFree(mg->d_tb);
}

}  // namespace dwf

using namespace dwf;

extern "C" {

dwf_status dwf_mg_create(dwf_mg** out, dwf_handle* h, const int block[4], int nvec) {
    DWF_TRY(check_handle(h));
    if (!out || !block || nvec < 1 || nvec > h->nrhs_max) {
        set_error("dwf_mg_create: bad argument (1 <= nvec <= the handle's nrhs_max)");
        return DWF_ERR_ARG;
    }
    *out = nullptr;
    // blocks per box; box-local lexicographic block order, boxes in order
    std::vector<int> box_nb(h->nbox), box_b0(h->nbox + 1, 0);
    for (int b = 0; b < h->nbox; ++b) {
        int n = 1;
        for (int mu = 0; mu < 4; ++mu) {
            const int e = h->boxes[b].extent[mu];
            if (block[mu] < 1 || e % block[mu]) {
                set_error("dwf_mg_create: block extent %d does not divide box %d extent %d (direction %d)",
                          block[mu], b, e, mu);
                return DWF_ERR_ARG;
            }
            n *= e / block[mu];
        }
        box_nb[b] = n;
        box_b0[b + 1] = box_b0[b] + n;
    }
    const int nb = box_b0[h->nbox];
    // odd sites in domain order: per box, box-local lex, those of global parity 1
    std::vector<int> site_block;
    site_block.reserve(h->nsite[1]);
    for (int b = 0; b < h->nbox; ++b) {
        const int* o = h->boxes[b].origin;
        const int* e = h->boxes[b].extent;
        const int nbx = e[0] / block[0], nby = e[1] / block[1], nbz = e[2] / block[2];
        const int64_t vol = (int64_t)e[0] * e[1] * e[2] * e[3];
        for (int64_t l = 0; l < vol; ++l) {
            const int lc[4] = {(int)(l % e[0]), (int)((l / e[0]) % e[1]), (int)((l / ((int64_t)e[0] * e[1])) % e[2]),
                               (int)(l / ((int64_t)e[0] * e[1] * e[2]))};
            int par = 0;
            for (int mu = 0; mu < 4; ++mu) par += (o[mu] + lc[mu]) % h->p.dims[mu];
            if ((par & 1) == 0) continue;
            const int bc = lc[0] / block[0] + nbx * (lc[1] / block[1] + nby * (lc[2] / block[2] + nbz * (lc[3] / block[3])));
            site_block.push_back(box_b0[b] + bc);
        }
    }
    if ((int64_t)site_block.size() != h->nsite[1]) {
        set_error("dwf_mg_create: site enumeration mismatch");
        return DWF_ERR_ARG;
    }
    std::vector<int> off(nb + 1, 0), sites(site_block.size());
    for (int b : site_block) off[b + 1]++;
    for (int b = 0; b < nb; ++b) {
        if (off[b + 1] == 0) {
            set_error("dwf_mg_create: block %d holds no odd site", b);
            return DWF_ERR_ARG;
        }
        off[b + 1] += off[b];
    }
    {
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (int i = 0; i < (int)site_block.size(); ++i) sites[fill[site_block[i]]++] = i;
    }
    const int nc = nb * nvec;
    if (nc > 4096) {
        set_error("dwf_mg_create: %d coarse unknowns (blocks x nvec) exceed the dense coarse solve's 4096", nc);
        return DWF_ERR_ARG;
    }
    dwf_mg* mg = new dwf_mg();
    mg->h = h;
    for (int mu = 0; mu < 4; ++mu) mg->block[mu] = block[mu];
    mg->nvec = nvec;
    mg->nb = nb;
    mg->nc = nc;
    auto fail = [&](dwf_status st) {
        free_mg(mg);
        delete mg;
        return st;
    };
    const size_t no = cb_elems(h, 1, 1), ne = cb_elems(h, 0, 1);
    const size_t nm = (no > ne ? no : ne) * (size_t)nvec;
    cudaError_t e = dev_malloc(&mg->d_site_block, site_block.size() * sizeof(int));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_blk_off, off.size() * sizeof(int));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_blk_sites, sites.size() * sizeof(int));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_basis, no * nvec * sizeof(float2));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_cinv, (size_t)nc * nc * sizeof(double2));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_ac, (size_t)nc * nc * sizeof(double2));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_c, (size_t)nvec * nc * sizeof(double2) + 2 * nc * sizeof(double2));
    for (int i = 0; i < 6 && e == cudaSuccess; ++i)
        e = dev_malloc(&mg->d_f[i], no * (i == 1 || i == 0 ? (size_t)nvec : 1) * sizeof(float2));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_ta, nm * sizeof(float2));
    if (e == cudaSuccess) e = dev_malloc(&mg->d_tb, nm * sizeof(float2));
    if (e == cudaSuccess)
        e = cudaMemcpy(mg->d_site_block, site_block.data(), site_block.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mg->d_blk_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(mg->d_blk_sites, sites.data(), sites.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("dwf_mg_create: %s", cudaGetErrorString(e));
        return fail(DWF_ERR_CUDA);
    }
    *out = mg;
    return DWF_OK;
}

dwf_status dwf_mg_destroy(dwf_mg* mg) {
    if (mg == nullptr) return DWF_OK;
    free_mg(mg);
    delete mg;
    return DWF_OK;
}

dwf_status dwf_mg_setup(dwf_mg* mg, const float* V, void* stream) {
    DWF_RANGE("dwf_mg_setup");
    if (mg == nullptr || V == nullptr) {
        set_error("dwf_mg_setup: null argument");
        return DWF_ERR_ARG;
    }
    dwf_handle* h = mg->h;
    DWF_TRY(check_handle(h));
    if (!h->have_gauge) {
        set_error("dwf_mg_setup: no gauge field loaded");
        return DWF_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nvec = mg->nvec, nb = mg->nb, nc = mg->nc, Ls = h->p.Ls;
    const size_t no = cb_elems(h, 1, 1);
    mg->ready = false;
    DWF_CUDA(cudaMemcpyAsync(mg->d_basis, V, no * nvec * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    DWF_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
    // block Gram-Schmidt in vector order: for each k two classical projections
    // against B_0..B_{k-1} (as stable as the modified form), then the norm
    double2* dots = mg->d_c;   // nb x nvec complex (set-up scratch)
    const int64_t ns = h->nsite[1];
    const int g = mg_grid(ns * 12 * Ls);
    for (int k = 0; k < nvec; ++k) {
        for (int pass = 0; pass < 2 && k > 0; ++pass) {
            k_mg_bdot<<<dim3(nb, k), kMgThreads, 0, s>>>(mg->d_basis, mg->d_blk_off, mg->d_blk_sites, nvec, Ls, k, 0,
                                                         dots);
            k_mg_bproj<<<g, 256, 0, s>>>(mg->d_basis, mg->d_site_block, dots, ns, nvec, Ls, k);
            note_launch();
            note_launch();
        }
        k_mg_bdot<<<dim3(nb, 1), kMgThreads, 0, s>>>(mg->d_basis, mg->d_blk_off, mg->d_blk_sites, nvec, Ls, k, k, dots);
        k_mg_bscale<<<g, 256, 0, s>>>(mg->d_basis, mg->d_site_block, dots, ns, nvec, Ls, k, h->d_err);
        note_launch();
        note_launch();
    }
    DWF_CUDA(cudaGetLastError());
    // Galerkin A_c, nvec columns (b0, k) at a time as the lanes of one A application
    float* F = mg->d_f[0];
    float* G = mg->d_f[1];
    float* mid = reinterpret_cast<float*>(h->d_tmp);   // FP64-sized scratch holds the FP32 middle field
    double2* cols = mg->d_c;                           // [k][b][k'] = A_c[(b, k'), (b0, k)]
    std::vector<double2> hc((size_t)nvec * nc), hac((size_t)nc * nc);
    for (int b0 = 0; b0 < nb; ++b0) {
        k_mg_block_lanes<<<mg_grid(h->nsite[1] * 12 * nvec * Ls), 256, 0, s>>>(
            mg->d_basis, mg->d_site_block, h->nsite[1], nvec, Ls, b0, reinterpret_cast<float2*>(F));
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_TRY(op_mpc(h, mid, F, 0, DWF_FP32, DWF_FP32, nvec, mg->d_ta, mg->d_tb, nullptr, nullptr, s));
        DWF_TRY(op_mpc(h, G, mid, 1, DWF_FP32, DWF_FP32, nvec, mg->d_ta, mg->d_tb, nullptr, nullptr, s));
        DWF_TRY(mg_restrict(mg, cols, G, nvec, s));
        DWF_CUDA(cudaMemcpyAsync(hc.data(), cols, hc.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nvec; ++k)
            for (int row = 0; row < nc; ++row) hac[(size_t)row * nc + b0 * nvec + k] = hc[(size_t)k * nc + row];
    }
    int herr = 0;
    DWF_CUDA(cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        set_error("dwf_mg_setup: a near-null vector vanishes on a block after orthogonalisation "
                  "(linearly dependent vectors)");
        return DWF_ERR_ARG;
    }
    DWF_CUDA(cudaMemcpy(mg->d_ac, hac.data(), hac.size() * sizeof(double2), cudaMemcpyHostToDevice));
    int singular = 0;
    DWF_TRY(invert_device(mg->d_ac, nc, mg->d_cinv, &singular, s));
    if (singular) {
        set_error("dwf_mg_setup: the coarse operator is singular");
        return DWF_ERR_ARG;
    }
    mg->ready = true;
    return DWF_OK;
}

dwf_status dwf_mg_set_smoother(dwf_mg* mg, int kind, int steps, double lo, double hi, dwf_nn* K) {
    if (mg == nullptr || kind < 0 || kind > 2 || (kind == 1 && (steps < 1 || !(hi > lo) || !(lo > 0))) ||
        (kind == 2 && K == nullptr)) {
        set_error("dwf_mg_set_smoother: kind 0 (none), 1 (Chebyshev: steps >= 1, 0 < lo < hi) or 2 (K)");
        return DWF_ERR_ARG;
    }
    mg->smoother = kind;
    mg->steps = steps;
    mg->lo = lo;
    mg->hi = hi;
    mg->K = K;
    return DWF_OK;
}

dwf_status dwf_mg_apply(dwf_mg* mg, float* z, const float* r, void* stream) {
    DWF_RANGE("dwf_mg_apply");
    if (mg == nullptr || z == nullptr || r == nullptr || z == r) {
        set_error("dwf_mg_apply: null or aliasing argument");
        return DWF_ERR_ARG;
    }
    DWF_TRY(check_handle(mg->h));
    if (!mg->ready) {
        set_error("dwf_mg_apply: dwf_mg_setup has not succeeded");
        return DWF_ERR_ARG;
    }
    return mg_apply(mg, z, r, (cudaStream_t)stream);
}

dwf_status dwf_mg_restrict(dwf_mg* mg, double* c, const float* f, void* stream) {
    if (mg == nullptr || c == nullptr || f == nullptr) {
        set_error("dwf_mg_restrict: null argument");
        return DWF_ERR_ARG;
    }
    DWF_TRY(check_handle(mg->h));
    return mg_restrict(mg, reinterpret_cast<double2*>(c), f, 1, (cudaStream_t)stream);
}

dwf_status dwf_mg_prolong(dwf_mg* mg, float* f, const double* c, void* stream) {
    if (mg == nullptr || c == nullptr || f == nullptr) {
        set_error("dwf_mg_prolong: null argument");
        return DWF_ERR_ARG;
    }
    DWF_TRY(check_handle(mg->h));
    return mg_prolong(mg, f, reinterpret_cast<const double2*>(c), 1, false, (cudaStream_t)stream);
}

dwf_status dwf_mg_handle(const dwf_mg* mg, dwf_handle** h) {
    if (mg == nullptr || h == nullptr) {
        set_error("dwf_mg_handle: null argument");
        return DWF_ERR_ARG;
    }
    if (!mg->ready) {
        set_error("dwf_mg_handle: dwf_mg_setup has not succeeded");
        return DWF_ERR_ARG;
    }
    *h = mg->h;
    return DWF_OK;
}

dwf_status dwf_mg_info(const dwf_mg* mg, int* nblocks, int* ncoarse) {
    if (mg == nullptr) {
        set_error("dwf_mg_info: null argument");
        return DWF_ERR_ARG;
    }
    if (nblocks) *nblocks = mg->nb;
    if (ncoarse) *ncoarse = mg->nc;
    return DWF_OK;
}

dwf_status dwf_mg_copy(const dwf_mg* mg, int what, void* dst, void* stream) {
    if (mg == nullptr || dst == nullptr || (what != 0 && what != 1)) {
        set_error("dwf_mg_copy: what = 0 (basis) or 1 (coarse operator), non-null destination");
        return DWF_ERR_ARG;
    }
    if (!mg->ready) {
        set_error("dwf_mg_copy: dwf_mg_setup has not succeeded");
        return DWF_ERR_ARG;
    }
    DWF_TRY(check_handle(mg->h));
    const size_t bytes = what == 0 ? cb_elems(mg->h, 1, 1) * mg->nvec * sizeof(float2)
                                   : (size_t)mg->nc * mg->nc * sizeof(double2);
    DWF_CUDA(cudaMemcpyAsync(dst, what == 0 ? (const void*)mg->d_basis : (const void*)mg->d_ac, bytes,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DWF_OK;
}

}  // extern "C"
