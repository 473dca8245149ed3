// Gauge-covariant parallel-transport convolutional preconditioner K: forward,
// backward and Adam kernels (FP32 arithmetic, BF16 weights for the forward
// pass, FP32 master weights for training).
//
//   T_0 = 1;  T_{1+mu} f(x) = U_mu(x) f(x+mu);  T_{5+mu} f(x) = U_mu(x-mu)^+ f(x-mu);
//   T_9 f(x,s) = f(x,s+1), T_10 f(x,s) = f(x,s-1)  (zero outside [0, Ls));
//   layer 1 (1 -> C):  R_d = T_d r,            phi^a = sum_d W1[a][d] R_d
//   layer 2 (C -> 1):  psi_d = sum_b W2[d][b] phi^b,   z = sum_d T_d psi_d
//
// W[o][i] are complex 4x4 spin matrices (they commute with colour and with
// the transports, so the order of mixing and transport within a layer is
// free).  K acts on the odd checkerboard: the input is embedded with zero on
// even sites and the output is read on odd sites.  Backward: g_psi_d =
// T_d^+ g_z, gW2[d][b] = sum g_psi_d phi_b^+, g_phi_b = sum_d W2[d][b]^+ g_psi_d,
// gW1[a][d] = sum g_phi_a R_d^+ (sums over sites, colour and lanes).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

constexpr int kNDir = 11;
constexpr int kAdj[kNDir] = {0, 5, 6, 7, 8, 1, 2, 3, 4, 10, 9};

struct TransArgs {
    const float* in;           // full field (both parities)
    float* out;                // out fields, stride `fstride` floats
    const float* const* ins;   // transport-sum: input field per direction
    const float* links;        // FP32 doubled link table of parity p
    const int* nbr;
    const int4* tiles;
    int dirs[kNDir];           // direction applied for output j
    int ndir, N5, Ls, parity;
    int64_t off_p, off_q;      // float offsets of parity p / 1-p blocks in a full field
    int64_t fstride;           // floats per full field
};

// f = U v (3x3 complex times colour vector) for 4 spins
__device__ __forceinline__ void su3_spinor(const float* __restrict__ w, const float (&vr)[12],
                                           const float (&vi)[12], float (&orr)[12], float (&oi)[12]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float wr = w[2 * (a * 3 + b)], wi = w[2 * (a * 3 + b) + 1];
                sr = fmaf(wr, vr[sp * 3 + b], sr);
                sr = fmaf(-wi, vi[sp * 3 + b], sr);
                si = fmaf(wr, vi[sp * 3 + b], si);
                si = fmaf(wi, vr[sp * 3 + b], si);
            }
            orr[sp * 3 + a] = sr;
            oi[sp * 3 + a] = si;
        }
}

// Value of T_d f at (site, lane) of parity p: 12 complex.
__device__ __forceinline__ void transport_at(const TransArgs& a, const float* __restrict__ f, int d,
                                             int64_t site, int tsite_nb_k, int lane,
                                             float (&orr)[12], float (&oi)[12]) {
    const int N5 = a.N5;
    if (d == 0 || d == 9 || d == 10) {
        int l = lane;
        if (d != 0) {
            const int s = lane % a.Ls;
            if ((d == 9 && s == a.Ls - 1) || (d == 10 && s == 0)) {
#pragma unroll
                for (int c = 0; c < 12; ++c) orr[c] = oi[c] = 0.f;
                return;
            }
            l = d == 9 ? lane + 1 : lane - 1;
        }
        const float* p = f + a.off_p + (site * 12 * N5 + l) * 2;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const float2 v = *reinterpret_cast<const float2*>(p + (int64_t)c * N5 * 2);
            orr[c] = v.x;
            oi[c] = v.y;
        }
        return;
    }
    const int k = d <= 4 ? d - 1 : d - 5 + 4;     // neighbour / link slot
    const int n = a.nbr[site * 8 + k];
    if (n < 0) {
#pragma unroll
        for (int c = 0; c < 12; ++c) orr[c] = oi[c] = 0.f;
        return;
    }
    (void)tsite_nb_k;
    float vr[12], vi[12];
    const float* p = f + a.off_q + ((int64_t)n * 12 * N5 + lane) * 2;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float2 v = *reinterpret_cast<const float2*>(p + (int64_t)c * N5 * 2);
        vr[c] = v.x;
        vi[c] = v.y;
    }
    su3_spinor(a.links + (site * 8 + k) * 18, vr, vi, orr, oi);
}

// out[j] = T_{dirs[j]} in on the sites of parity p (one thread per site x lane)
__global__ void __launch_bounds__(256) k_transport_multi(const TransArgs a) {
    const int4 tl = a.tiles[blockIdx.x];
    const int N5 = a.N5;
    for (int t = threadIdx.x; t < tl.z * N5; t += blockDim.x) {
        const int64_t site = tl.y + t / N5;
        const int lane = t % N5;
        for (int j = 0; j < a.ndir; ++j) {
            float orr[12], oi[12];
            transport_at(a, a.in, a.dirs[j], site, 0, lane, orr, oi);
            float* o = a.out + j * a.fstride + a.off_p + (site * 12 * N5 + lane) * 2;
#pragma unroll
            for (int c = 0; c < 12; ++c)
                *reinterpret_cast<float2*>(o + (int64_t)c * N5 * 2) = make_float2(orr[c], oi[c]);
        }
    }
}

// out = sum_j T_{dirs[j]} ins[j] on the sites of parity p
__global__ void __launch_bounds__(256) k_transport_sum(const TransArgs a) {
    const int4 tl = a.tiles[blockIdx.x];
    const int N5 = a.N5;
    for (int t = threadIdx.x; t < tl.z * N5; t += blockDim.x) {
        const int64_t site = tl.y + t / N5;
        const int lane = t % N5;
        float ar[12], ai[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) ar[c] = ai[c] = 0.f;
        for (int j = 0; j < a.ndir; ++j) {
            float orr[12], oi[12];
            transport_at(a, a.ins[j], a.dirs[j], site, 0, lane, orr, oi);
#pragma unroll
            for (int c = 0; c < 12; ++c) { ar[c] += orr[c]; ai[c] += oi[c]; }
        }
        float* o = a.out + a.off_p + (site * 12 * N5 + lane) * 2;
#pragma unroll
        for (int c = 0; c < 12; ++c)
            *reinterpret_cast<float2*>(o + (int64_t)c * N5 * 2) = make_float2(ar[c], ai[c]);
    }
}

// Pointwise mixing: out[o][so] = sum_{i,si} W[o][so][i][si] in[i][si] at every
// pixel (site, colour, lane) of a full field.  W: [nout][4][nin][4] complex
// (FP32 in shared memory).  One thread per pixel, NOUT*4 accumulators.
template <int NOUT>
__global__ void __launch_bounds__(128) k_mix(const float* __restrict__ in, int nin, float* __restrict__ out,
                                             const float* __restrict__ W, int64_t npix, int N5,
                                             int64_t fstride) {
    extern __shared__ float sW[];
    const int nw = NOUT * 4 * nin * 4 * 2;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) sW[i] = W[i];
    __syncthreads();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(p % N5);
        const int64_t sc = p / N5;              // site * 3 + colour
        const int colour = (int)(sc % 3);
        const int64_t site = sc / 3;
        const int64_t base = (site * 12 + colour) * N5 + lane;   // complex index of spin 0
        float accr[NOUT][4], acci[NOUT][4];
#pragma unroll
        for (int o = 0; o < NOUT; ++o)
#pragma unroll
            for (int so = 0; so < 4; ++so) accr[o][so] = acci[o][so] = 0.f;
        for (int i = 0; i < nin; ++i) {
            float xr[4], xi[4];
#pragma unroll
            for (int si = 0; si < 4; ++si) {
                const float2 v = *reinterpret_cast<const float2*>(
                    in + i * fstride + 2 * (base + (int64_t)si * 3 * N5));
                xr[si] = v.x;
                xi[si] = v.y;
            }
#pragma unroll
            for (int o = 0; o < NOUT; ++o)
#pragma unroll
                for (int so = 0; so < 4; ++so) {
                    const float* w = sW + 2 * (((o * 4 + so) * nin + i) * 4);
#pragma unroll
                    for (int si = 0; si < 4; ++si) {
                        const float wr = w[2 * si], wi = w[2 * si + 1];
                        accr[o][so] = fmaf(wr, xr[si], fmaf(-wi, xi[si], accr[o][so]));
                        acci[o][so] = fmaf(wr, xi[si], fmaf(wi, xr[si], acci[o][so]));
                    }
                }
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o)
#pragma unroll
            for (int so = 0; so < 4; ++so)
                *reinterpret_cast<float2*>(out + o * fstride + 2 * (base + (int64_t)so * 3 * N5)) =
                    make_float2(accr[o][so], acci[o][so]);
    }
}

// Weight gradient: g[o][so][i][si] = sum_pixels gout[o][so] conj(in[i][si]).
// One thread per (o, i) pair with a 4x4 complex accumulator; the CTA walks
// (site, colour) chunks of N5 lanes staged in shared memory; per-CTA FP64
// partials are summed in a fixed order by k_wgrad_reduce.
__global__ void __launch_bounds__(512) k_wgrad(const float* __restrict__ gout, int nout,
                                               const float* __restrict__ in, int nin,
                                               int64_t nchunks, int N5, int64_t fstride,
                                               double* __restrict__ partial) {
    extern __shared__ float sm[];
    float* sg = sm;                              // [nout][4][N5] complex
    float* sx = sm + (size_t)nout * 4 * N5 * 2;  // [nin][4][N5] complex
    const int pairs = nout * nin;
    const int t = threadIdx.x;
    const int o = t / nin, i = t % nin;
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = 0.f;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t site = ch / 3;
        const int colour = (int)(ch % 3);
        __syncthreads();
        const int ng = nout * 4 * N5, nx = nin * 4 * N5;
        for (int e = t; e < ng + nx; e += blockDim.x) {
            const bool isg = e < ng;
            const int ee = isg ? e : e - ng;
            const int fld = ee / (4 * N5), sp = (ee / N5) % 4, lane = ee % N5;
            const float* src = (isg ? gout : in) + fld * fstride +
                               2 * ((site * 12 + sp * 3 + colour) * N5 + lane);
            const float2 v = *reinterpret_cast<const float2*>(src);
            float* dst = (isg ? sg : sx) + 2 * ee;
            dst[0] = v.x;
            dst[1] = v.y;
        }
        __syncthreads();
        if (t < pairs) {
            for (int l = 0; l < N5; ++l) {
                float gr[4], gi[4], xr[4], xi[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    gr[a] = sg[2 * ((o * 4 + a) * N5 + l)];
                    gi[a] = sg[2 * ((o * 4 + a) * N5 + l) + 1];
                    xr[a] = sx[2 * ((i * 4 + a) * N5 + l)];
                    xi[a] = sx[2 * ((i * 4 + a) * N5 + l) + 1];
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {   // g_a * conj(x_b)
                        ar[a][b] = fmaf(gr[a], xr[b], fmaf(gi[a], xi[b], ar[a][b]));
                        ai[a][b] = fmaf(gi[a], xr[b], fmaf(-gr[a], xi[b], ai[a][b]));
                    }
            }
        }
    }
    if (t < pairs) {
        double* out = partial + (size_t)blockIdx.x * pairs * 32;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                // layout [o][a][i][b] complex
                const size_t idx = (((size_t)o * 4 + a) * nin + i) * 4 + b;
                out[2 * idx] = (double)ar[a][b];
                out[2 * idx + 1] = (double)ai[a][b];
            }
    }
}

__global__ void k_wgrad_reduce(const double* __restrict__ partial, int nblocks, int nval,
                               double* __restrict__ out) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nval; v += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * nval + v];
        out[v] = s;
    }
}

// Adam on the real and imaginary parts (all arrays of n reals).
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const double* __restrict__ g, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = (float)g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace dwf

// ===================================================================== API
using namespace dwf;

struct dwf_nn {
    int C = 16;
    // master weights (FP32, complex interleaved), layout of the oracle:
    // W1[d][a][0][so][si] and W2[d][0][b][so][si]
    std::vector<float> w1, w2;
    float* d_w1 = nullptr;   // master FP32 (device), oracle layout
    float* d_w2 = nullptr;
    float* d_m = nullptr;    // Adam moments over [w1 | w2]
    float* d_v = nullptr;
    float* d_mix1 = nullptr; // BF16-rounded mixing matrices, kernel layouts
    float* d_mix2 = nullptr;
    float* d_mix2h = nullptr;    // adjoint of layer-2 mixing
    float* d_fold[2] = {nullptr, nullptr};   // W2 W1 on even / odd sites (inference)
    int adam_t = 0;
    bool dirty = true;           // mixing matrices need a refresh
};

namespace dwf {

static size_t w1_len(int C) { return (size_t)kNDir * C * 16 * 2; }
static size_t w2_len(int C) { return (size_t)kNDir * C * 16 * 2; }

// Directions whose R_d = T_d x0 can be nonzero on each parity when x0 vanishes
// on even sites: the link transports reach even sites from odd neighbours, the
// identity and the two s-shifts stay on odd sites.
constexpr int kNFold[2] = {8, 3};
constexpr int kFoldDirs[2][8] = {{1, 2, 3, 4, 5, 6, 7, 8}, {0, 9, 10, 0, 0, 0, 0, 0}};
static size_t fold_len(int p) { return (size_t)kNFold[p] * 4 * kNFold[p] * 4 * 2; }

static float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Rebuild the kernel-layout mixing matrices from the master weights (BF16 rounded).
static dwf_status refresh_mix(dwf_nn* K) {
    if (!K->dirty) return DWF_OK;
    const int C = K->C;
    std::vector<float> w1(w1_len(C)), w2(w2_len(C));
    DWF_CUDA(cudaMemcpy(w1.data(), K->d_w1, w1.size() * 4, cudaMemcpyDeviceToHost));
    DWF_CUDA(cudaMemcpy(w2.data(), K->d_w2, w2.size() * 4, cudaMemcpyDeviceToHost));
    // mix1: [o = a][so][i = d][si]  <- W1[d][a][so][si]
    std::vector<float> m1((size_t)C * 4 * kNDir * 4 * 2), m2((size_t)kNDir * 4 * C * 4 * 2),
        m2h((size_t)C * 4 * kNDir * 4 * 2);
    for (int d = 0; d < kNDir; ++d)
        for (int a = 0; a < C; ++a)
            for (int so = 0; so < 4; ++so)
                for (int si = 0; si < 4; ++si) {
                    const size_t src1 = (((size_t)d * C + a) * 4 + so) * 4 + si;
                    const size_t dst1 = (((size_t)a * 4 + so) * kNDir + d) * 4 + si;
                    m1[2 * dst1] = bf16_round(w1[2 * src1]);
                    m1[2 * dst1 + 1] = bf16_round(w1[2 * src1 + 1]);
                    // W2[d][0][b = a][so][si] -> mix2 [o = d][so][i = b][si]
                    const size_t dst2 = (((size_t)d * 4 + so) * C + a) * 4 + si;
                    const float r2 = bf16_round(w2[2 * src1]), i2 = bf16_round(w2[2 * src1 + 1]);
                    m2[2 * dst2] = r2;
                    m2[2 * dst2 + 1] = i2;
                    // adjoint: g_phi[b][si] = sum_{d,so} conj(W2[d][b][so][si]) g_psi[d][so]
                    //   -> mix2h [o = b][so' = si][i = d][si' = so] = conj(W2[d][b][so][si])
                    const size_t dsth = (((size_t)a * 4 + si) * kNDir + d) * 4 + so;
                    m2h[2 * dsth] = r2;
                    m2h[2 * dsth + 1] = -i2;
                }
    DWF_CUDA(cudaMemcpy(K->d_mix1, m1.data(), m1.size() * 4, cudaMemcpyHostToDevice));
    DWF_CUDA(cudaMemcpy(K->d_mix2, m2.data(), m2.size() * 4, cudaMemcpyHostToDevice));
    DWF_CUDA(cudaMemcpy(K->d_mix2h, m2h.data(), m2h.size() * 4, cudaMemcpyHostToDevice));
    // folded layers for inference: M[d][d'] = sum_b W2[d][b] W1[d'][b] (4x4 complex
    // spin blocks, FP64 products of the BF16-rounded weights, stored FP32) in the
    // mixing layout [o = d][so][i = d'][si], restricted to each parity's directions
    for (int p = 0; p < 2; ++p) {
        const int n = kNFold[p];
        std::vector<float> fm(fold_len(p));
        for (int o = 0; o < n; ++o)
            for (int i = 0; i < n; ++i)
                for (int so = 0; so < 4; ++so)
                    for (int si = 0; si < 4; ++si) {
                        const int d = kFoldDirs[p][o], dp = kFoldDirs[p][i];
                        double mr = 0.0, mi = 0.0;
                        for (int b = 0; b < C; ++b)
                            for (int t = 0; t < 4; ++t) {
                                const size_t i2 = (((size_t)d * C + b) * 4 + so) * 4 + t;
                                const size_t i1 = (((size_t)dp * C + b) * 4 + t) * 4 + si;
                                const double ar = bf16_round(w2[2 * i2]), ai = bf16_round(w2[2 * i2 + 1]);
                                const double br = bf16_round(w1[2 * i1]), bi = bf16_round(w1[2 * i1 + 1]);
                                mr += ar * br - ai * bi;
                                mi += ar * bi + ai * br;
                            }
                        const size_t dst = (((size_t)o * 4 + so) * n + i) * 4 + si;
                        fm[2 * dst] = (float)mr;
                        fm[2 * dst + 1] = (float)mi;
                    }
        DWF_CUDA(cudaMemcpy(K->d_fold[p], fm.data(), fm.size() * 4, cudaMemcpyHostToDevice));
    }
    K->dirty = false;
    return DWF_OK;
}

// network workspace of a handle for nrhs lanes
struct NNWS {
    int nrhs = 0, C = 0;
    float* x0 = nullptr;      // embedded input (full field)
    float* R = nullptr;       // 11 full fields
    float* phi = nullptr;     // C full fields
    float* psi = nullptr;     // 11 full fields
    float* z = nullptr;       // full field
    float* gphi = nullptr;    // C full fields (training)
    float* at = nullptr;      // odd FP32 temporaries for the energy-norm loss
    float* aw = nullptr;
    double* wpart = nullptr;  // weight-gradient partials
    double* gw = nullptr;     // [gW1 | gW2]
    int wblocks = 0;
};

static std::map<dwf_handle*, NNWS> g_nnws;

static int64_t full_floats(const dwf_handle* h, int nrhs) {
    return (int64_t)(h->nsite[0] + h->nsite[1]) * 12 * h->p.Ls * nrhs * 2;
}

static dwf_status nn_ws(dwf_handle* h, int nrhs, int C, bool train, NNWS** out) {
    NNWS& w = g_nnws[h];
    if (w.nrhs != nrhs || w.C != C || (train && w.gphi == nullptr)) {
        cudaFree(w.x0); cudaFree(w.R); cudaFree(w.phi); cudaFree(w.psi); cudaFree(w.z);
        cudaFree(w.gphi); cudaFree(w.wpart); cudaFree(w.gw); cudaFree(w.at); cudaFree(w.aw);
        w = NNWS();
        const int64_t f = full_floats(h, nrhs);
        DWF_CUDA(dev_malloc(&w.x0, f * 4));
        DWF_CUDA(dev_malloc(&w.R, (size_t)kNDir * f * 4));
        DWF_CUDA(dev_malloc(&w.phi, (size_t)C * f * 4));
        DWF_CUDA(dev_malloc(&w.psi, (size_t)kNDir * f * 4));
        DWF_CUDA(dev_malloc(&w.z, f * 4));
        if (train) {
            DWF_CUDA(dev_malloc(&w.gphi, (size_t)C * f * 4));
            w.wblocks = 152 * 2;
            DWF_CUDA(dev_malloc(&w.wpart, (size_t)w.wblocks * C * kNDir * 32 * sizeof(double)));
            DWF_CUDA(dev_malloc(&w.gw, (w1_len(C) + w2_len(C)) * sizeof(double)));
            const size_t odd = (size_t)h->nsite[1] * 12 * h->p.Ls * nrhs * 2;
            DWF_CUDA(dev_malloc(&w.at, odd * 4));
            DWF_CUDA(dev_malloc(&w.aw, odd * 4));
        }
        w.nrhs = nrhs;
        w.C = C;
    }
    *out = &w;
    return DWF_OK;
}

void free_nn_ws(dwf_handle* h) {
    auto it = g_nnws.find(h);
    if (it == g_nnws.end()) return;
    NNWS& w = it->second;
    cudaFree(w.x0); cudaFree(w.R); cudaFree(w.phi); cudaFree(w.psi); cudaFree(w.z);
    cudaFree(w.gphi); cudaFree(w.wpart); cudaFree(w.gw); cudaFree(w.at); cudaFree(w.aw);
    g_nnws.erase(it);
}

static TransArgs trans_args(dwf_handle* h, int nrhs, int p) {
    TransArgs a{};
    a.N5 = h->p.Ls * nrhs;
    a.Ls = h->p.Ls;
    a.parity = p;
    const int64_t c0 = h->nsite[0] * 12 * (int64_t)a.N5 * 2;
    a.off_p = p ? c0 : 0;
    a.off_q = p ? 0 : c0;
    a.fstride = full_floats(h, nrhs);
    a.links = (const float*)h->d_links[DWF_FP32][p];
    a.nbr = h->d_nbr[p];
    return a;
}

static dwf_status launch_transport(dwf_handle* h, int nrhs, const float* in, float* out,
                                   const int* dirs, int ndir, bool sum, const float* const* ins,
                                   cudaStream_t s, int only_parity = -1) {
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, tile_for(h, nrhs), &tsp));
    const TileSet& ts = *tsp;
    for (int p = 0; p < 2; ++p) {
        if (ts.ntiles[p] == 0 || (only_parity >= 0 && p != only_parity)) continue;
        TransArgs a = trans_args(h, nrhs, p);
        a.in = in;
        a.out = out;
        a.ins = ins;
        a.tiles = ts.d_tiles[p];
        a.ndir = ndir;
        for (int j = 0; j < ndir; ++j) a.dirs[j] = dirs[j];
        if (sum) k_transport_sum<<<ts.ntiles[p], 256, 0, s>>>(a);
        else k_transport_multi<<<ts.ntiles[p], 256, 0, s>>>(a);
        note_launch();
        DWF_CUDA(cudaGetLastError());
    }
    return DWF_OK;
}

// Mixing on a full field, or (parity 0 / 1) on that parity's block only: `in`
// and `out` then point at the block, fields keep the full-field stride.
static dwf_status launch_mix(dwf_handle* h, int nrhs, const float* in, int nin, float* out, int nout,
                             const float* W, cudaStream_t s, int only_parity = -1) {
    const int64_t nsites = only_parity < 0 ? h->nsite[0] + h->nsite[1] : h->nsite[only_parity];
    const int64_t npix = nsites * 3 * (int64_t)h->p.Ls * nrhs;
    if (npix == 0) return DWF_OK;
    const int64_t fstride = full_floats(h, nrhs);
    const size_t smem = (size_t)nout * 4 * nin * 4 * 2 * sizeof(float);
    int64_t blocks = (npix + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const int N5 = h->p.Ls * nrhs;
    if (nout == 16)
        k_mix<16><<<(int)blocks, 128, smem, s>>>(in, nin, out, W, npix, N5, fstride);
    else if (nout == 11)
        k_mix<11><<<(int)blocks, 128, smem, s>>>(in, nin, out, W, npix, N5, fstride);
    else if (nout == 8)
        k_mix<8><<<(int)blocks, 128, smem, s>>>(in, nin, out, W, npix, N5, fstride);
    else if (nout == 3)
        k_mix<3><<<(int)blocks, 128, smem, s>>>(in, nin, out, W, npix, N5, fstride);
    else {
        set_error("nn: unsupported channel count %d", nout);
        return DWF_ERR_UNSUPPORTED;
    }
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

static dwf_status launch_wgrad(dwf_handle* h, NNWS& w, int nrhs, const float* gout, int nout,
                               const float* in, int nin, double* dst, cudaStream_t s) {
    const int N5 = h->p.Ls * nrhs;
    const int64_t nchunks = (h->nsite[0] + h->nsite[1]) * 3;
    const int64_t fstride = full_floats(h, nrhs);
    int threads = (nout * nin + 31) / 32 * 32;
    const size_t smem = (size_t)(nout + nin) * 4 * N5 * 2 * sizeof(float);
    static bool attr = false;
    if (!attr) {
        DWF_CUDA(cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    if (smem > 200 * 1024) {
        set_error("nn: %d lanes need %zu bytes of shared memory for the weight gradient", N5, smem);
        return DWF_ERR_UNSUPPORTED;
    }
    k_wgrad<<<w.wblocks, threads, smem, s>>>(gout, nout, in, nin, nchunks, N5, fstride, w.wpart);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    const int nval = nout * nin * 32;
    k_wgrad_reduce<<<(nval + 255) / 256, 256, 0, s>>>(w.wpart, w.wblocks, nval, dst);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

static const int kDirsFwd[kNDir] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10};

// z = K x0 (x0 full field with the input on odd sites, zero on even)
static dwf_status nn_forward(dwf_nn* K, dwf_handle* h, NNWS& w, int nrhs, cudaStream_t s) {
    const int C = K->C;
    DWF_TRY(refresh_mix(K));
    DWF_TRY(launch_transport(h, nrhs, w.x0, w.R, kDirsFwd, kNDir, false, nullptr, s));
    DWF_TRY(launch_mix(h, nrhs, w.R, kNDir, w.phi, C, K->d_mix1, s));
    DWF_TRY(launch_mix(h, nrhs, w.phi, C, w.psi, kNDir, K->d_mix2, s));
    const int64_t f = full_floats(h, nrhs);
    const float* ins[kNDir];
    for (int d = 0; d < kNDir; ++d) ins[d] = w.psi + d * f;
    // device array of pointers
    static thread_local const float** d_ins = nullptr;
    if (d_ins == nullptr) DWF_CUDA(dev_malloc(&d_ins, kNDir * sizeof(float*)));
    DWF_CUDA(cudaMemcpyAsync(d_ins, ins, sizeof(ins), cudaMemcpyHostToDevice, s));
    return launch_transport(h, nrhs, nullptr, w.z, kDirsFwd, kNDir, true, d_ins, s);
}

// Inference z = K x on the odd checkerboard.  The same function as
// nn_forward up to rounding, with the work that is exactly zero left out: x0
// vanishes on even sites, so R_d = T_d x0 is zero on odd sites for the link
// directions 1..8 and on even sites for 0, 9 and 10; only odd z is read, which
// takes psi_d on even sites for d = 1..8 and on odd sites for 0, 9, 10; and
// with no nonlinearity between the layers psi = (W2 W1) R.  Per parity the
// folded 4x4-block matrix over that parity's directions (8 x 8 blocks even,
// 3 x 3 odd) replaces the two mixes through the C channels.
dwf_status nn_apply_internal(dwf_nn* K, dwf_handle* h, float* out, const float* in, int nrhs,
                             cudaStream_t s) {
    NNWS* w;
    DWF_TRY(nn_ws(h, nrhs, K->C, false, &w));
    DWF_TRY(refresh_mix(K));
    const int64_t c0 = h->nsite[0] * 12 * (int64_t)h->p.Ls * nrhs * 2;
    const int64_t c1 = h->nsite[1] * 12 * (int64_t)h->p.Ls * nrhs * 2;
    const int64_t f = full_floats(h, nrhs);
    // the even block of x0 is never read below
    DWF_CUDA(cudaMemcpyAsync(w->x0 + c0, in, c1 * 4, cudaMemcpyDeviceToDevice, s));
    for (int p = 0; p < 2; ++p)
        DWF_TRY(launch_transport(h, nrhs, w->x0, w->R, kFoldDirs[p], kNFold[p], false, nullptr, s, p));
    DWF_TRY(launch_mix(h, nrhs, w->R, kNFold[0], w->psi, kNFold[0], K->d_fold[0], s, 0));
    DWF_TRY(launch_mix(h, nrhs, w->R + c0, kNFold[1], w->psi + c0, kNFold[1], K->d_fold[1], s, 1));
    // z on odd sites: psi field j holds direction kFoldDirs[p][j] on parity p
    int dirs[kNDir];
    const float* ins[kNDir];
    int nd = 0;
    for (int p = 1; p >= 0; --p)
        for (int j = 0; j < kNFold[p]; ++j) {
            dirs[nd] = kFoldDirs[p][j];
            ins[nd++] = w->psi + j * f;
        }
    static thread_local const float** d_ins = nullptr;
    if (d_ins == nullptr) DWF_CUDA(dev_malloc(&d_ins, kNDir * sizeof(float*)));
    DWF_CUDA(cudaMemcpyAsync(d_ins, ins, sizeof(ins), cudaMemcpyHostToDevice, s));
    DWF_TRY(launch_transport(h, nrhs, nullptr, w->z, dirs, kNDir, true, d_ins, s, 1));
    DWF_CUDA(cudaMemcpyAsync(out, w->z + c0, c1 * 4, cudaMemcpyDeviceToDevice, s));
    return DWF_OK;
}

}  // namespace dwf

extern "C" {

dwf_status dwf_nn_create(dwf_nn** out, int channels) {
    if (out == nullptr || channels != 16) {
        set_error("dwf_nn_create: channels must be 16");
        return DWF_ERR_ARG;
    }
    dwf_nn* K = new dwf_nn();
    K->C = channels;
    const size_t n1 = w1_len(channels), n2 = w2_len(channels);
    K->w1.assign(n1, 0.f);
    K->w2.assign(n2, 0.f);
    // identity: W1[0][0] = 1, W2[0][0][0] = 1
    for (int so = 0; so < 4; ++so) {
        K->w1[2 * (so * 4 + so)] = 1.f;
        K->w2[2 * (so * 4 + so)] = 1.f;
    }
    if (dev_malloc(&K->d_w1, n1 * 4) != cudaSuccess || dev_malloc(&K->d_w2, n2 * 4) != cudaSuccess ||
        dev_malloc(&K->d_m, (n1 + n2) * 4) != cudaSuccess ||
        dev_malloc(&K->d_v, (n1 + n2) * 4) != cudaSuccess ||
        dev_malloc(&K->d_mix1, n1 * 4) != cudaSuccess || dev_malloc(&K->d_mix2, n2 * 4) != cudaSuccess ||
        dev_malloc(&K->d_mix2h, n2 * 4) != cudaSuccess ||
        dev_malloc(&K->d_fold[0], fold_len(0) * 4) != cudaSuccess ||
        dev_malloc(&K->d_fold[1], fold_len(1) * 4) != cudaSuccess) {
        set_error("dwf_nn_create: cudaMalloc failed");
        return DWF_ERR_CUDA;
    }
    cudaMemcpy(K->d_w1, K->w1.data(), n1 * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(K->d_w2, K->w2.data(), n2 * 4, cudaMemcpyHostToDevice);
    cudaMemset(K->d_m, 0, (n1 + n2) * 4);
    cudaMemset(K->d_v, 0, (n1 + n2) * 4);
    K->dirty = true;
    *out = K;
    return DWF_OK;
}

dwf_status dwf_nn_destroy(dwf_nn* K) {
    if (!K) return DWF_OK;
    cudaFree(K->d_w1); cudaFree(K->d_w2); cudaFree(K->d_m); cudaFree(K->d_v);
    cudaFree(K->d_mix1); cudaFree(K->d_mix2); cudaFree(K->d_mix2h);
    cudaFree(K->d_fold[0]); cudaFree(K->d_fold[1]);
    delete K;
    return DWF_OK;
}

dwf_status dwf_nn_set_weights(dwf_nn* K, const double* w, size_t n) {
    if (!K || !w || n != (w1_len(K->C) + w2_len(K->C)) / 2) {
        set_error("dwf_nn_set_weights: expected %zu complex numbers",
                  K ? (w1_len(K->C) + w2_len(K->C)) / 2 : (size_t)0);
        return DWF_ERR_ARG;
    }
    const size_t n1 = w1_len(K->C);
    std::vector<float> all(2 * n);
    for (size_t i = 0; i < 2 * n; ++i) all[i] = (float)w[i];
    DWF_CUDA(cudaMemcpy(K->d_w1, all.data(), n1 * 4, cudaMemcpyHostToDevice));
    DWF_CUDA(cudaMemcpy(K->d_w2, all.data() + n1, (2 * n - n1) * 4, cudaMemcpyHostToDevice));
    K->dirty = true;
    return DWF_OK;
}

dwf_status dwf_nn_get_weights(const dwf_nn* K, double* w, size_t n) {
    if (!K || !w || n != (w1_len(K->C) + w2_len(K->C)) / 2) {
        set_error("dwf_nn_get_weights: bad buffer");
        return DWF_ERR_ARG;
    }
    const size_t n1 = w1_len(K->C);
    std::vector<float> all(2 * n);
    DWF_CUDA(cudaMemcpy(all.data(), K->d_w1, n1 * 4, cudaMemcpyDeviceToHost));
    DWF_CUDA(cudaMemcpy(all.data() + n1, K->d_w2, (2 * n - n1) * 4, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < 2 * n; ++i) w[i] = all[i];
    return DWF_OK;
}

// Weight file: the 8 bytes "DWFNN001", int32 channels, int32 0, int64 number
// of complex weights n, then n complex128 (re, im) in the order of
// dwf_nn_set_weights, little-endian as written by this host.
static const char kNNMagic[8] = {'D', 'W', 'F', 'N', 'N', '0', '0', '1'};

dwf_status dwf_nn_save(const dwf_nn* K, const char* path) {
    if (!K || !path) {
        set_error("dwf_nn_save: null argument");
        return DWF_ERR_ARG;
    }
    const size_t n = (w1_len(K->C) + w2_len(K->C)) / 2;
    std::vector<double> w(2 * n);
    DWF_TRY(dwf_nn_get_weights(K, w.data(), n));
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("dwf_nn_save: cannot open %s for writing", path);
        return DWF_ERR_ARG;
    }
    const int32_t hdr[2] = {K->C, 0};
    const int64_t nn = (int64_t)n;
    bool ok = fwrite(kNNMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(&nn, sizeof(nn), 1, f) == 1 && fwrite(w.data(), sizeof(double), w.size(), f) == w.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("dwf_nn_save: write to %s failed", path);
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

dwf_status dwf_nn_load(dwf_nn* K, const char* path) {
    if (!K || !path) {
        set_error("dwf_nn_load: null argument");
        return DWF_ERR_ARG;
    }
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("dwf_nn_load: cannot open %s", path);
        return DWF_ERR_ARG;
    }
    char magic[8];
    int32_t hdr[2];
    int64_t nn = 0;
    const size_t n = (w1_len(K->C) + w2_len(K->C)) / 2;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kNNMagic, 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
              fread(&nn, sizeof(nn), 1, f) == 1 && hdr[0] == K->C && nn == (int64_t)n;
    std::vector<double> w(2 * n);
    ok = ok && fread(w.data(), sizeof(double), w.size(), f) == w.size();
    fclose(f);
    if (!ok) {
        set_error("dwf_nn_load: %s is not a weight file of a %d-channel network", path, K->C);
        return DWF_ERR_ARG;
    }
    return dwf_nn_set_weights(K, w.data(), n);
}

// One training pair from an FP64 solve: e = (x* - x_k) / |x* - x_k|,
// r = M_pc^+ M_pc e (FP64 operator), both written in FP32.
dwf_status dwf_nn_make_pair(dwf_handle* h, const double* x_star, const double* x_k, float* r,
                            float* e, double* norm, void* stream) {
    DWF_RANGE("dwf_nn_make_pair");
    DWF_TRY(check_handle(h));
    if (!x_star || !x_k || !r || !e || !norm || !h->have_gauge || h->dirichlet) {
        set_error("dwf_nn_make_pair: bad argument (whole-lattice handle with a gauge field, "
                  "non-null fields)");
        return DWF_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t no = cb_elems(h, 1, 1);
    const int T = tile_for(h, 1);
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, T, &tsp));
    double* buf = nullptr;
    const size_t nd = (size_t)tsp->ntiles[1] + 1;
    DWF_CUDA(dev_malloc(&buf, (3 * no * 2 + nd) * sizeof(double)));
    double* e64 = buf;
    double* t64 = buf + 2 * no;
    double* r64 = buf + 4 * no;
    double* part = buf + 6 * no;
    double* d_n2 = part + tsp->ntiles[1];
    double n2 = 0.0;
    dwf_status st = DWF_OK;
    auto run = [&]() -> dwf_status {
        DWF_CUDA(cudaMemcpyAsync(e64, x_star, no * 16, cudaMemcpyDeviceToDevice, s));
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, -1.0, x_k, DWF_FP64, nullptr, 1.0, e64, DWF_FP64, nullptr, T, s));
        DWF_TRY(launch_dot_partial(h, 1, e64, e64, DWF_FP64, DWF_FP64, 1, part, T, s));
        DWF_TRY(launch_reduce_sys(h, 1, part, 1, d_n2, T, s));
        DWF_CUDA(cudaMemcpyAsync(&n2, d_n2, sizeof(double), cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        *norm = std::sqrt(n2);
        if (!(n2 > 0.0)) return DWF_OK;
        DWF_TRY(launch_axpby(h, 1, 1, nullptr, 0.0, e64, DWF_FP64, nullptr, 1.0 / *norm, e64, DWF_FP64,
                             nullptr, T, s));
        DWF_TRY(op_mpc(h, t64, e64, 0, DWF_FP64, DWF_FP64, 1, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        DWF_TRY(op_mpc(h, r64, t64, 1, DWF_FP64, DWF_FP64, 1, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        DWF_TRY(launch_convert(r, DWF_FP32, r64, DWF_FP64, no, s));
        DWF_TRY(launch_convert(e, DWF_FP32, e64, DWF_FP64, no, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        return DWF_OK;
    };
    st = run();
    cudaFree(buf);
    return st;
}

// out = K in on the odd checkerboard (FP32 cb fields, nrhs lanes)
dwf_status dwf_nn_apply(dwf_nn* K, dwf_handle* h, float* out, const float* in, int nrhs, void* stream) {
    DWF_RANGE("dwf_nn_apply");
    DWF_TRY(check_handle(h));
    if (!K || !out || !in || nrhs < 1 || nrhs > h->nrhs_max || !h->have_gauge) {
        set_error("dwf_nn_apply: bad argument");
        return DWF_ERR_ARG;
    }
    return nn_apply_internal(K, h, out, in, nrhs, (cudaStream_t)stream);
}

// One Adam step on a batch of nrhs (r, e) pairs (odd cb FP32, lanes = pairs):
// loss = mean_k |K r_k - e_k|^2 / |e_k|^2 (returned, before the step).
dwf_status dwf_nn_train_step(dwf_nn* K, dwf_handle* h, const float* r, const float* e, int nrhs,
                             int loss_kind, double lr, double* loss, void* stream) {
    DWF_RANGE("dwf_nn_train_step");
    DWF_TRY(check_handle(h));
    if (!K || !r || !e || nrhs < 1 || nrhs > h->nrhs_max || !h->have_gauge || h->dirichlet) {
        set_error("dwf_nn_train_step: bad argument");
        return DWF_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    NNWS* wp;
    DWF_TRY(nn_ws(h, nrhs, K->C, true, &wp));
    NNWS& w = *wp;
    const int C = K->C;
    const int64_t c0 = h->nsite[0] * 12 * (int64_t)h->p.Ls * nrhs * 2;
    const int64_t c1 = h->nsite[1] * 12 * (int64_t)h->p.Ls * nrhs * 2;
    const int64_t f = full_floats(h, nrhs);
    DWF_CUDA(cudaMemsetAsync(w.x0, 0, c0 * 4, s));
    DWF_CUDA(cudaMemcpyAsync(w.x0 + c0, r, c1 * 4, cudaMemcpyDeviceToDevice, s));
    DWF_TRY(nn_forward(K, h, w, nrhs, s));
    const int T = tile_for(h, nrhs);
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, T, &tsp));
    const TileSet& ts = *tsp;
    std::vector<double> h1(nrhs), h2(nrhs), h3(nrhs);
    double* d_scal;
    DWF_CUDA(dev_malloc(&d_scal, (size_t)(4 * nrhs + (ts.ntiles[1] + 1) * nrhs) * sizeof(double)));
    double* d1 = d_scal;
    double* d2 = d_scal + nrhs;
    double* d_coef = d_scal + 2 * nrhs;
    double* d3 = d_scal + 3 * nrhs;
    double* part = d_scal + 4 * nrhs;
    float* zo = w.z + c0;
    auto dot = [&](const void* x, const void* y, double* dst) -> dwf_status {
        DWF_TRY(launch_dot_partial(h, 1, x, y, DWF_FP32, DWF_FP32, nrhs, part, T, s));
        return launch_reduce_sys(h, 1, part, nrhs, dst, T, s);
    };
    double L = 0.0;
    std::vector<double> coef(nrhs);
    if (loss_kind == 0) {
        // |z - e|^2 / |e|^2: the fit residual overwrites z
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, -1.0, e, DWF_FP32, nullptr, 1.0, zo, DWF_FP32, nullptr, T, s));
        DWF_TRY(dot(e, e, d1));
        DWF_TRY(dot(zo, zo, d2));
        DWF_CUDA(cudaMemcpyAsync(h1.data(), d1, nrhs * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaMemcpyAsync(h2.data(), d2, nrhs * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nrhs; ++k) {
            L += h2[k] / h1[k] / nrhs;
            coef[k] = 2.0 / (h1[k] * nrhs);
        }
    } else if (loss_kind == 2) {
        // A^2 norm: |A z - r|^2 / |r|^2, gradient 2 A (A z - r) / |r|^2, held in z
        DWF_TRY(op_mpc(h, w.at, zo, 0, DWF_FP32, DWF_FP32, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        DWF_TRY(op_mpc(h, w.aw, w.at, 1, DWF_FP32, DWF_FP32, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, -1.0, r, DWF_FP32, nullptr, 1.0, w.aw, DWF_FP32, nullptr, T, s));
        DWF_TRY(dot(w.aw, w.aw, d1));
        DWF_TRY(dot(r, r, d3));
        DWF_CUDA(cudaMemcpyAsync(h1.data(), d1, nrhs * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaMemcpyAsync(h3.data(), d3, nrhs * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nrhs; ++k) {
            L += h1[k] / h3[k] / nrhs;
            coef[k] = 2.0 / (h3[k] * nrhs);
        }
        DWF_TRY(op_mpc(h, w.at, w.aw, 0, DWF_FP32, DWF_FP32, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        DWF_TRY(op_mpc(h, zo, w.at, 1, DWF_FP32, DWF_FP32, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
    } else {
        // energy norm of A = M_pc^+ M_pc: (<z,Az> - 2 Re<z,r> + <e,r>) / <e,r>,
        // gradient 2 (A z - r) / <e,r>, held in z
        DWF_TRY(op_mpc(h, w.at, zo, 0, DWF_FP32, DWF_FP32, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        DWF_TRY(op_mpc(h, w.aw, w.at, 1, DWF_FP32, DWF_FP32, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        DWF_TRY(dot(zo, w.aw, d1));
        DWF_TRY(dot(zo, r, d2));
        DWF_TRY(dot(e, r, d3));
        DWF_CUDA(cudaMemcpyAsync(h1.data(), d1, nrhs * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaMemcpyAsync(h2.data(), d2, nrhs * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaMemcpyAsync(h3.data(), d3, nrhs * 8, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nrhs; ++k) {
            L += (h1[k] - 2.0 * h2[k] + h3[k]) / h3[k] / nrhs;
            coef[k] = 2.0 / (h3[k] * nrhs);
        }
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, -1.0, r, DWF_FP32, nullptr, 1.0, w.aw, DWF_FP32, nullptr, T, s));
        DWF_CUDA(cudaMemcpyAsync(zo, w.aw, (size_t)c1 * 4, cudaMemcpyDeviceToDevice, s));
    }
    if (loss) *loss = L;
    DWF_CUDA(cudaMemcpyAsync(d_coef, coef.data(), nrhs * 8, cudaMemcpyHostToDevice, s));
    // g_z = coef * (held residual) on odd sites, zero on even sites
    DWF_CUDA(cudaMemsetAsync(w.z, 0, c0 * 4, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 0.0, nullptr, DWF_FP32, d_coef, 0.0, zo, DWF_FP32, nullptr, T, s));
    // g_psi_d = T_d^+ g_z  (into psi)
    DWF_TRY(launch_transport(h, nrhs, w.z, w.psi, kAdj, kNDir, false, nullptr, s));
    // gW2[o = d][so][i = b][si] = sum g_psi_d phi_b^+
    DWF_TRY(launch_wgrad(h, w, nrhs, w.psi, kNDir, w.phi, C, w.gw + w1_len(C), s));
    // g_phi = W2^+ g_psi
    DWF_TRY(launch_mix(h, nrhs, w.psi, kNDir, w.gphi, C, K->d_mix2h, s));
    // gW1[o = a][so][i = d][si] = sum g_phi_a R_d^+
    DWF_TRY(launch_wgrad(h, w, nrhs, w.gphi, C, w.R, kNDir, w.gw, s));
    // gradients are in kernel layouts: convert to the master (oracle) layout on the host
    const size_t n1 = w1_len(C), n2 = w2_len(C);
    std::vector<double> gk(n1 + n2), gm(n1 + n2);
    DWF_CUDA(cudaMemcpyAsync(gk.data(), w.gw, (n1 + n2) * 8, cudaMemcpyDeviceToHost, s));
    DWF_CUDA(cudaStreamSynchronize(s));
    for (int d = 0; d < kNDir; ++d)
        for (int a = 0; a < C; ++a)
            for (int so = 0; so < 4; ++so)
                for (int si = 0; si < 4; ++si) {
                    const size_t m = (((size_t)d * C + a) * 4 + so) * 4 + si;          // master
                    const size_t k1 = (((size_t)a * 4 + so) * kNDir + d) * 4 + si;      // gW1 kernel
                    const size_t k2 = (((size_t)d * 4 + so) * C + a) * 4 + si;          // gW2 kernel
                    gm[2 * m] = gk[2 * k1];
                    gm[2 * m + 1] = gk[2 * k1 + 1];
                    gm[n1 + 2 * m] = gk[n1 + 2 * k2];
                    gm[n1 + 2 * m + 1] = gk[n1 + 2 * k2 + 1];
                }
    DWF_CUDA(cudaMemcpyAsync(w.gw, gm.data(), (n1 + n2) * 8, cudaMemcpyHostToDevice, s));
    // Adam (w1 and w2 are separate allocations: two launches over [w1 | w2])
    K->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)K->adam_t), bc2 = 1.f - powf(b2, (float)K->adam_t);
    k_adam<<<(int)((n1 + 255) / 256), 256, 0, s>>>(K->d_w1, K->d_m, K->d_v, w.gw, (int)n1, (float)lr,
                                                    b1, b2, 1e-8f, bc1, bc2);
    note_launch();
    k_adam<<<(int)((n2 + 255) / 256), 256, 0, s>>>(K->d_w2, K->d_m + n1, K->d_v + n1, w.gw + n1,
                                                    (int)n2, (float)lr, b1, b2, 1e-8f, bc1, bc2);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    DWF_CUDA(cudaStreamSynchronize(s));
    cudaFree(d_scal);
    K->dirty = true;
    return DWF_OK;
}

// Debug/training access to the raw gradient of the last train step
// (master layout, doubles): used by the gradient parity test.
dwf_status dwf_nn_last_grad(dwf_handle* h, double* g, size_t n) {
    auto it = g_nnws.find(h);
    if (it == g_nnws.end() || it->second.gw == nullptr || !g) {
        set_error("dwf_nn_last_grad: no training step on this handle");
        return DWF_ERR_ARG;
    }
    const int C = it->second.C;
    if (n != (w1_len(C) + w2_len(C)) / 2) {
        set_error("dwf_nn_last_grad: expected %zu complex numbers", (w1_len(C) + w2_len(C)) / 2);
        return DWF_ERR_ARG;
    }
    DWF_CUDA(cudaMemcpy(g, it->second.gw, 2 * n * sizeof(double), cudaMemcpyDeviceToHost));
    return DWF_OK;
}

}  // extern "C"
