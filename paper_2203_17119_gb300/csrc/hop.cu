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
#include <cstdio>
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
    double scale, d, e, mf;
    double* partial;
    int* err;
};

template <int K, bool DAG, class Sin, class SL, class R, int VL>
__device__ __forceinline__ void hop_dir(const Sin* __restrict__ in, const int* s_nbr,
                                        const SL* s_link, int N5, int lane0, R (&ar)[12][VL],
                                        R (&ai)[12][VL]) {
    constexpr int MU = K & 3;
    constexpr bool FWD = K < 4;
    constexpr int SGI = (FWD != DAG) ? 1 : -1;   // (1 - SG g_mu) projector
    const R SG = (R)SGI;
    const int n = s_nbr[K];
    if (n < 0) return;   // link cut by a Dirichlet boundary
    const Sin* src = in + ((int64_t)n * 12 * N5 + lane0) * 2;
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

// Persistent kernel: CTA b takes tiles b, b + gridDim, ...; the links and
// neighbour indices of the next tile are bulk-copied into the other half of
// a double buffer while the current tile is computed.
template <class Sin, class Sout, class SL, class R, int VL, bool DAG, int EPI>
__global__ void __launch_bounds__(256, (VL == 1 && sizeof(R) == 4) ? 3 : 2) k_hop(const HopArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int TPS = a.N5 / VL;
    const size_t link_bytes = (size_t)a.T * 144 * sizeof(SL);
    const size_t buf_bytes = link_bytes + (size_t)a.T * 32;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * buf_bytes);
    double* s_red = reinterpret_cast<double*>(bar + 2);
    __shared__ int s_ok;
    const int nt = a.ntiles;

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
        fence_mbar_init();
        if ((int)blockIdx.x < nt) issue(blockIdx.x, 0);
    }
    __syncthreads();

    const int G = blockDim.x / TPS;
    const int sg = threadIdx.x / TPS;
    const int lane0 = (threadIdx.x - sg * TPS) * VL;
    const int N5 = a.N5;
    const Sin* in = reinterpret_cast<const Sin*>(a.in);

    int k = 0;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x, ++k) {
        const int b = k & 1;
        if (threadIdx.x == 0) {
            const int next = tile + gridDim.x;
            if (next < nt) issue(next, b ^ 1);   // the other buffer is free
            bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1));
            if (!ok) {
                atomicOr(a.err, kErrBulkTimeout);
                mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1));
            }
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) {
            // a lost copy: let the one in flight land, then stop (uniform)
            if (threadIdx.x == 0 && tile + gridDim.x < nt)
                mbar_wait_bounded(&bar[b ^ 1], (uint32_t)(((k + 1) >> 1) & 1));
            return;
        }
        const int4 tl = a.tiles[tile];
        const int begin = tl.y, count = tl.z;
        const SL* s_link_t = reinterpret_cast<const SL*>(smem + b * buf_bytes);
        const int* s_nbr_t = reinterpret_cast<const int*>(smem + b * buf_bytes + link_bytes);
        double tile_norm = 0.0;

    for (int sl = sg; sg < G && sl < count; sl += G) {
        R ar[12][VL], ai[12][VL];
#pragma unroll
        for (int c = 0; c < 12; ++c)
#pragma unroll
            for (int v = 0; v < VL; ++v) ar[c][v] = ai[c][v] = (R)0;
        const Sin* in = reinterpret_cast<const Sin*>(a.in);
        const int* nb = s_nbr_t + sl * 8;
        const SL* lk = s_link_t + (size_t)sl * 144;
        // +mu and -mu back to back: the row that is the +x neighbour of
        // one site is the -x neighbour of the next, still in L1
        hop_dir<0, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
        hop_dir<4, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
        hop_dir<1, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
        hop_dir<5, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
        hop_dir<2, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
        hop_dir<6, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
        hop_dir<3, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);
        hop_dir<7, DAG, Sin, SL, R, VL>(in, nb, lk, N5, lane0, ar, ai);

        const R sc = (R)a.scale;
        const int64_t site = begin + sl;
        Sout* out = reinterpret_cast<Sout*>(a.out) + (site * 12 * N5 + lane0) * 2;
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
        } else {
            // M_oo x = d x + e S5 x on this site's lanes; S5 (non-dagger):
            // upper spins x_{s-1}, lower spins x_{s+1}, walls -mf.
            const Sout* xb = reinterpret_cast<const Sout*>(a.xmoo) + (site * 12 * N5) * 2;
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
            float nrm_f = 0.f;   // FP32 arithmetic: one FP64 add per site, off the slow FP64 pipe
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                R xr[VL], xi[VL];
                load_lanes<Sout, VL, R>(xb + (int64_t)(c * N5 + lane0) * 2, xr, xi);
                // upper spins use S_- (x_{s-1}) unless dagger, lower S_+
                const bool use_below = (c < 6) != DAG;
                R nr, ni;
                load_c1<Sout, R>(xb + (int64_t)(c * N5 + (use_below ? l_below : l_above)) * 2, nr,
                                 ni);
                const R fn = use_below ? f_below : f_above;
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
            tile_norm += sizeof(R) == 8 ? nrm : (double)nrm_f;
        }
    }
        if (EPI == EPI_MOO && a.partial != nullptr) {
            const int Ls = a.Ls;
            block_rhs_reduce(
                tile_norm, s_red, a.nrhs,
                [&](int t) { return (t / TPS < G && t / TPS < count) ? ((t % TPS) * VL) / Ls : -1; },
                a.partial + (size_t)tile * a.nrhs);
        }
        __syncthreads();   // buffer b is rewritten two tiles from now
    }
}

// ------------------------------------------------------------- launcher
template <class Sin, class Sout, class SL, class R, int VL>
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
    const int TPS = a.N5 / VL;
    // site groups per CTA: as many as fit in 256 threads, at most T
    int groups = 256 / TPS;
    if (groups > ts.T) groups = ts.T;
    if (groups < 1) {
        set_error("hop: %d threads per site exceed 256", TPS);
        return DWF_ERR_ARG;
    }
    int threads = (groups * TPS + 31) / 32 * 32;
    const size_t smem = 2 * (size_t)ts.T * (144 * sizeof(SL) + 32) + 16 + (size_t)threads * 8;
    const int nt = ts.ntiles[p];
    if (nt == 0) return DWF_OK;
    a.ntiles = nt;
    void (*kern)(const HopArgs);
    const bool moo = c.xmoo != nullptr;
    if (c.dagger)
        kern = moo ? k_hop<Sin, Sout, SL, R, VL, true, EPI_MOO>
                   : k_hop<Sin, Sout, SL, R, VL, true, EPI_PLAIN>;
    else
        kern = moo ? k_hop<Sin, Sout, SL, R, VL, false, EPI_MOO>
                   : k_hop<Sin, Sout, SL, R, VL, false, EPI_PLAIN>;
    if (smem > kHopMaxSmem) {
        set_error("hop: tile of %d sites needs %zu bytes of shared memory", ts.T, smem);
        return DWF_ERR_ARG;
    }
    // persistent grid: as many CTAs as are resident at once, at most one per tile
    static std::map<std::pair<const void*, long>, int> occ_cache;
    const auto key = std::make_pair((const void*)kern, (long)threads * 1000000L + (long)smem);
    int per_sm = 0;
    auto it = occ_cache.find(key);
    if (it == occ_cache.end()) {
        DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        occ_cache[key] = per_sm;
    } else {
        per_sm = it->second;
    }
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    int grid = (per_sm > 0 ? per_sm : 1) * n_sm;
    if (grid > nt) grid = nt;
    kern<<<grid, threads, smem, s>>>(a);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

// Raise the dynamic shared-memory limit of every hop instantiation once, so
// that launches recorded into a CUDA graph never need a host-side call.
template <class Sin, class Sout, class SL, class R, int VL>
static cudaError_t hop_attr() {
    cudaError_t e = cudaSuccess;
    void (*k[4])(const HopArgs) = {k_hop<Sin, Sout, SL, R, VL, false, EPI_PLAIN>,
                                   k_hop<Sin, Sout, SL, R, VL, false, EPI_MOO>,
                                   k_hop<Sin, Sout, SL, R, VL, true, EPI_PLAIN>,
                                   k_hop<Sin, Sout, SL, R, VL, true, EPI_MOO>};
    for (auto f : k) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kHopMaxSmem);
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
    return DWF_OK;
}

dwf_status launch_hop(dwf_handle* h, const HopCall& c, cudaStream_t s) {
    const TileSet& ts = get_tiles(h, c.T > 0 ? c.T : 16);
    if (c.prec_link == DWF_FP64) {
        if (c.prec_in != DWF_FP64 || c.prec_out != DWF_FP64) return DWF_ERR_UNSUPPORTED;
        return launch_t<double, double, double, double, 1>(h, c, ts, s);
    }
    if (c.prec_link == DWF_FP32) {
        if (c.prec_in != DWF_FP32 || c.prec_out != DWF_FP32) return DWF_ERR_UNSUPPORTED;
        if (c.VL == 1) return launch_t<float, float, float, float, 1>(h, c, ts, s);
        return launch_t<float, float, float, float, 2>(h, c, ts, s);
    }
    // BF16 links: FP32 arithmetic, operands FP32 or BF16
    if (c.prec_in == DWF_BF16 && c.prec_out == DWF_BF16)
        return launch_t<bf16, bf16, bf16, float, 2>(h, c, ts, s);
    if (c.prec_in == DWF_BF16 && c.prec_out == DWF_FP32)
        return launch_t<bf16, float, bf16, float, 2>(h, c, ts, s);
    if (c.prec_in == DWF_FP32 && c.prec_out == DWF_BF16)
        return launch_t<float, bf16, bf16, float, 2>(h, c, ts, s);
    if (c.prec_in == DWF_FP32 && c.prec_out == DWF_FP32)
        return launch_t<float, float, bf16, float, 2>(h, c, ts, s);
    return DWF_ERR_UNSUPPORTED;
}

}  // namespace dwf
