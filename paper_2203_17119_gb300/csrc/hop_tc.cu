// Wilson hop on the tensor cores, BF16 operator (FP32 accumulation).
//
// For one site and direction the hop is the colour contraction g = U h of
// the link U (3 x 3 complex) with the projected half spinor h on every lane
// (l = r * Ls + s) and both projected spin components, and the reconstructed
// lower spins are fixed multiples (+-1, +-i) of the same products.  So the
// output of a site, rows (lane, spin), columns (colour, re/im), is
//
//     out[(l, spin)][(a, ri)] = sum over directions d, colours b, (re, im) of
//                               v_d[(l, spin)][(b, ri')] * Ureal_d[(b, ri')][(a, ri)]
//
// with v_d the projected (upper spins) or projected-and-multiplied (lower
// spins) neighbour spinor and Ureal_d the real 6 x 6 form of U_d: a dense
// contraction of K = 6 per direction, accumulated over the eight directions
// in one FP32 accumulator.  It maps onto mma.sync m16n8k16 (BF16 in, FP32
// accumulate): M = 16 rows = 8 lanes x 2 spins, K = 16 = the +mu and -mu
// directions of one mu (6 real columns each, padded to 8), N = 8 = 3 colours
// x (re, im) padded.  One warp takes one site; for each group of 8 lanes it
// runs 2 MMAs (upper and lower spins) per mu.  Thread (g, t) of the warp
// (g = lane / 4, t = lane % 4) owns lane 8q + g and colour t: it loads that
// lane's four spin components of colour t from each neighbour, forms the two
// projected components h0, h1 (FP32, then rounded to BF16), and ends with
// the four output spins of its (lane, colour), so the MMA fragments are built
// in registers without any shuffle.  Link tiles arrive by bulk copy as in the
// SIMT hop, with the same barrier-free tile loop.
#include <algorithm>
#include <map>
#include <type_traits>
#include <utility>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

struct HopTcArgs {
    const void* in;
    void* out;
    const void* xmoo;
    const bf16* links;   // parity table [site][8][3][3] complex, BF16
    const int* nbr;      // [site][8]
    const int4* tiles;
    int T, N5, Ls, nrhs, ntiles;
    float scale, d, e, mf;
    double* partial;
    int* err;
};

__device__ __forceinline__ uint32_t pack_bf2(float re, float im) {
    __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <class S>
__device__ __forceinline__ void ld_c(const S* p, float& re, float& im) {
    float r[1], i[1];
    load_lanes<S, 1, float>(p, r, i);
    re = r[0];
    im = i[0];
}

// One direction K for lane l, colour b: the upper A values (spins 0, 1) and
// the lower ones (spins 2, 3) as packed BF16 pairs.  Same projection and
// reconstruction as the SIMT hop: h = u - SG A_mu l, lower = -SG A_mu^+ h.
template <int K, bool DAG, class Sin>
__device__ __forceinline__ void tc_avals(const Sin* __restrict__ nb, int N5, int l, int b,
                                         uint32_t& up0, uint32_t& up1, uint32_t& lo2,
                                         uint32_t& lo3) {
    constexpr int MU = K & 3;
    constexpr bool FWD = K < 4;
    constexpr float SG = (FWD != DAG) ? 1.f : -1.f;
    float ur0, ui0, ur1, ui1, lr0, li0, lr1, li1;
    ld_c<Sin>(nb + (int64_t)((0 * 3 + b) * N5 + l) * 2, ur0, ui0);
    ld_c<Sin>(nb + (int64_t)((1 * 3 + b) * N5 + l) * 2, ur1, ui1);
    ld_c<Sin>(nb + (int64_t)((2 * 3 + b) * N5 + l) * 2, lr0, li0);
    ld_c<Sin>(nb + (int64_t)((3 * 3 + b) * N5 + l) * 2, lr1, li1);
    float hr0, hi0, hr1, hi1;
    if (MU == 0) {
        hr0 = ur0 - SG * li1; hi0 = ui0 + SG * lr1;
        hr1 = ur1 - SG * li0; hi1 = ui1 + SG * lr0;
    } else if (MU == 1) {
        hr0 = ur0 + SG * lr1; hi0 = ui0 + SG * li1;
        hr1 = ur1 - SG * lr0; hi1 = ui1 - SG * li0;
    } else if (MU == 2) {
        hr0 = ur0 - SG * li0; hi0 = ui0 + SG * lr0;
        hr1 = ur1 + SG * li1; hi1 = ui1 - SG * lr1;
    } else {
        hr0 = ur0 - SG * lr0; hi0 = ui0 - SG * li0;
        hr1 = ur1 - SG * lr1; hi1 = ui1 - SG * li1;
    }
    up0 = pack_bf2(hr0, hi0);
    up1 = pack_bf2(hr1, hi1);
    // lower spins: the SIMT reconstruction written as a multiple of h
    if (MU == 0) {          // spin 2 += -i SG h1, spin 3 += -i SG h0
        lo2 = pack_bf2(SG * hi1, -SG * hr1);
        lo3 = pack_bf2(SG * hi0, -SG * hr0);
    } else if (MU == 1) {   // spin 2 += -SG h1, spin 3 += SG h0
        lo2 = pack_bf2(-SG * hr1, -SG * hi1);
        lo3 = pack_bf2(SG * hr0, SG * hi0);
    } else if (MU == 2) {   // spin 2 += -i SG h0, spin 3 += i SG h1
        lo2 = pack_bf2(SG * hi0, -SG * hr0);
        lo3 = pack_bf2(-SG * hi1, SG * hr1);
    } else {                // spin 2 += -SG h0, spin 3 += -SG h1
        lo2 = pack_bf2(-SG * hr0, -SG * hi0);
        lo3 = pack_bf2(-SG * hr1, -SG * hi1);
    }
}

// B fragment of direction K for thread (g, t): column n = g = (a, ro),
// rows (b = t, re / im); real form of U: [Ur -Ui; Ui Ur] by (ri', ri).
__device__ __forceinline__ uint32_t tc_bval(const bf16* lk, int K, int g, int t) {
    if (g >= 6 || t >= 3) return 0u;
    const int a = g >> 1, ro = g & 1;
    const __nv_bfloat162 u = reinterpret_cast<const __nv_bfloat162*>(lk + K * 18)[a * 3 + t];
    const float ur = __bfloat162float(u.x), ui = __bfloat162float(u.y);
    return ro == 0 ? pack_bf2(ur, -ui) : pack_bf2(ui, ur);
}

template <int MU, bool DAG, class Sin>
__device__ __forceinline__ void tc_mu(const Sin* in, const int* nb, const bf16* lk, int N5, int l,
                                      int b, bool act, int g, int t, float (&cu)[4],
                                      float (&cl)[4]) {
    constexpr int K0 = MU, K1 = MU + 4;
    const int n0 = nb[K0], n1 = nb[K1];
    uint32_t u0a = 0, u1a = 0, l2a = 0, l3a = 0, u0b = 0, u1b = 0, l2b = 0, l3b = 0;
    if (act && n0 >= 0)
        tc_avals<K0, DAG, Sin>(in + (int64_t)n0 * 12 * N5 * 2, N5, l, b, u0a, u1a, l2a, l3a);
    if (act && n1 >= 0)
        tc_avals<K1, DAG, Sin>(in + (int64_t)n1 * 12 * N5 * 2, N5, l, b, u0b, u1b, l2b, l3b);
    const uint32_t b0 = n0 >= 0 ? tc_bval(lk, K0, g, t) : 0u;
    const uint32_t b1 = n1 >= 0 ? tc_bval(lk, K1, g, t) : 0u;
    // rows g / g + 8 = spins 0 / 1 (upper) or 2 / 3 (lower); k 0..7 = +mu, 8..15 = -mu
    mma_bf16(cu, u0a, u1a, u0b, u1b, b0, b1);
    mma_bf16(cl, l2a, l3a, l2b, l3b, b0, b1);
}

template <class Sin, class Sout, bool DAG, int EPI>
__global__ void __launch_bounds__(256, 2) k_hop_tc(const HopTcArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const size_t link_bytes = (size_t)a.T * 144 * sizeof(bf16);
    const size_t buf_bytes = link_bytes + (size_t)a.T * 32;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * buf_bytes);
    int* done = reinterpret_cast<int*>(bar + 2);
    double* s_red = reinterpret_cast<double*>(bar + 3);   // [2][nwarps][nrhs]
    const int nt = a.ntiles, N5 = a.N5, Ls = a.Ls;
    const int nwarps = (int)(blockDim.x >> 5), warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const Sin* in = reinterpret_cast<const Sin*>(a.in);
    const bool part = EPI == EPI_MOO && a.partial != nullptr;

    auto issue = [&](int tile, int bf) {
        const int4 tt = a.tiles[tile];
        const uint32_t lb = (uint32_t)tt.z * 144u * (uint32_t)sizeof(bf16);
        const uint32_t nbb = (uint32_t)tt.z * 32u;
        unsigned char* base = smem + bf * buf_bytes;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[bf], lb + nbb);
        bulk_g2s(base, a.links + (int64_t)tt.y * 144, lb, &bar[bf]);
        bulk_g2s(base + link_bytes, a.nbr + (int64_t)tt.y * 8, nbb, &bar[bf]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        done[0] = done[1] = 0;
        fence_mbar_init();
        if ((int)blockIdx.x < nt) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < nt) issue(blockIdx.x + gridDim.x, 1);
    }
    __syncthreads();

    int k = 0;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x, ++k) {
        const int bf = k & 1;
        const uint32_t ph = (uint32_t)((k >> 1) & 1);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[bf], ph))) {
            if (lane == 0) {
                atomicOr(a.err, kErrBulkTimeout);
                mbar_wait_bounded(&bar[bf], ph);
            }
            return;
        }
        const int4 tl = a.tiles[tile];
        const bf16* s_link_t = reinterpret_cast<const bf16*>(smem + bf * buf_bytes);
        const int* s_nbr_t = reinterpret_cast<const int*>(smem + bf * buf_bytes + link_bytes);
        // this warp's |out|^2 per rhs for the tile (lane 0 accumulates)
        double* red = s_red + (size_t)bf * nwarps * a.nrhs;
        if (part) {
            for (int r = lane; r < a.nrhs; r += 32) red[warp * a.nrhs + r] = 0.0;
            __syncwarp();
        }
        for (int sl = warp; sl < tl.z; sl += nwarps) {
            const int* nb = s_nbr_t + sl * 8;
            const bf16* lk = s_link_t + (size_t)sl * 144;
            const int64_t site = (int64_t)tl.y + sl;
            for (int q = 0; q * 8 < N5; ++q) {
                const int l = q * 8 + g;
                const bool act = l < N5 && t < 3;
                const int b = t < 3 ? t : 0;
                float cu[4] = {0.f, 0.f, 0.f, 0.f}, cl[4] = {0.f, 0.f, 0.f, 0.f};
                tc_mu<0, DAG, Sin>(in, nb, lk, N5, l, b, act, g, t, cu, cl);
                tc_mu<1, DAG, Sin>(in, nb, lk, N5, l, b, act, g, t, cu, cl);
                tc_mu<2, DAG, Sin>(in, nb, lk, N5, l, b, act, g, t, cu, cl);
                tc_mu<3, DAG, Sin>(in, nb, lk, N5, l, b, act, g, t, cu, cl);
                // this thread: lane l, colour t; spins 0, 1 in cu rows g, g + 8; spins 2, 3 in cl
                const float sc = a.scale;
                const float vr[4] = {cu[0], cu[2], cl[0], cl[2]}, vi[4] = {cu[1], cu[3], cl[1], cl[3]};
                Sout* ob = reinterpret_cast<Sout*>(a.out) + site * 12 * N5 * 2;
                float pn = 0.f;
                if (act) {
                    if (EPI == EPI_PLAIN) {
#pragma unroll
                        for (int sp = 0; sp < 4; ++sp) {
                            float orr[1] = {sc * vr[sp]}, oi[1] = {sc * vi[sp]};
                            store_lanes<Sout, 1, float, true>(ob + (int64_t)((sp * 3 + t) * N5 + l) * 2, orr, oi);
                        }
                    } else {
                        // M_oo x = d x + e S5 x: upper spins x_{s-1}, lower x_{s+1} (swapped by DAG)
                        const Sout* xb = reinterpret_cast<const Sout*>(a.xmoo) + site * 12 * N5 * 2;
                        const int s0 = l % Ls, rb = l - s0;
                        const int lbw = s0 == 0 ? rb + Ls - 1 : l - 1, lab = s0 == Ls - 1 ? rb : l + 1;
                        const float fbw = s0 == 0 ? -a.mf : 1.f, fab = s0 == Ls - 1 ? -a.mf : 1.f;
#pragma unroll
                        for (int sp = 0; sp < 4; ++sp) {
                            const int row = (sp * 3 + t) * N5;
                            const bool below = (sp < 2) != DAG;
                            float xr, xi, nr, ni;
                            ld_c<Sout>(xb + (int64_t)(row + l) * 2, xr, xi);
                            ld_c<Sout>(xb + (int64_t)(row + (below ? lbw : lab)) * 2, nr, ni);
                            const float fn = below ? fbw : fab;
                            const float o_r = a.d * xr + a.e * fn * nr + sc * vr[sp];
                            const float o_i = a.d * xi + a.e * fn * ni + sc * vi[sp];
                            pn += o_r * o_r + o_i * o_i;
                            float orr[1] = {o_r}, oi[1] = {o_i};
                            store_lanes<Sout, 1, float, true>(ob + (int64_t)(row + l) * 2, orr, oi);
                        }
                    }
                }
                if (part) {
                    // lanes 8q .. 8q + 7 touch rhs r_lo .. r_hi: one warp sum each, in lane order
                    const int r_lo = (q * 8) / Ls, r_hi = (min(q * 8 + 7, N5 - 1)) / Ls;
                    for (int r = r_lo; r <= r_hi; ++r) {
                        double v = (act && l / Ls == r) ? (double)pn : 0.0;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                        if (lane == 0) red[warp * a.nrhs + r] += v;
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&done[bf], 1) == nwarps - 1) {   // the last warp out
                __threadfence_block();
                if (part) {
                    const double* red = s_red + (size_t)bf * nwarps * a.nrhs;
                    for (int r = 0; r < a.nrhs; ++r) {
                        double sum = 0.0;
                        for (int w = 0; w < nwarps; ++w) sum += red[w * a.nrhs + r];
                        a.partial[(size_t)tile * a.nrhs + r] = sum;
                    }
                }
                done[bf] = 0;
                const int next2 = tile + 2 * (int)gridDim.x;
                if (next2 < nt) issue(next2, bf);
            }
        }
    }
}

// ------------------------------------------------------------- launcher
template <class Sin, class Sout>
static dwf_status launch_tc_t(dwf_handle* h, const HopCall& c, const TileSet& ts, cudaStream_t s) {
    const int p = c.out_parity;
    HopTcArgs a;
    a.in = c.in;
    a.out = c.out;
    a.xmoo = c.xmoo;
    a.links = reinterpret_cast<const bf16*>(h->d_links[DWF_BF16][p]);
    a.nbr = h->d_nbr[p];
    a.tiles = ts.d_tiles[p];
    a.T = ts.T;
    a.Ls = h->p.Ls;
    a.nrhs = c.nrhs;
    a.N5 = h->p.Ls * c.nrhs;
    a.scale = (float)c.scale;
    a.d = (float)h->f5[0].d;
    a.e = (float)h->f5[0].e;
    a.mf = (float)h->p.mf;
    a.partial = c.partial;
    a.err = h->d_err;
    const int nt = ts.ntiles[p];
    if (nt == 0) return DWF_OK;
    a.ntiles = nt;
    const int threads = 256;
    const size_t smem = hop_smem(ts.T, sizeof(bf16), threads / 32, c.nrhs);
    if (smem > (size_t)kHopMaxSmem) {
        set_error("hop: tile of %d sites needs %zu bytes of shared memory", ts.T, smem);
        return DWF_ERR_ARG;
    }
    void (*kern)(const HopTcArgs);
    const bool moo = c.xmoo != nullptr;
    if (c.dagger)
        kern = moo ? k_hop_tc<Sin, Sout, true, EPI_MOO> : k_hop_tc<Sin, Sout, true, EPI_PLAIN>;
    else
        kern = moo ? k_hop_tc<Sin, Sout, false, EPI_MOO> : k_hop_tc<Sin, Sout, false, EPI_PLAIN>;
    int grid = 0;
    DWF_TRY(persistent_grid((const void*)kern, threads, smem, nt, &grid));
    kern<<<grid, threads, smem, s>>>(a);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

template <class Sin, class Sout>
static cudaError_t tc_attr() {
    cudaError_t e = cudaSuccess;
    void (*k[4])(const HopTcArgs) = {k_hop_tc<Sin, Sout, false, EPI_PLAIN>, k_hop_tc<Sin, Sout, false, EPI_MOO>,
                                     k_hop_tc<Sin, Sout, true, EPI_PLAIN>, k_hop_tc<Sin, Sout, true, EPI_MOO>};
    for (auto f : k) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kHopMaxSmem);
        if (r != cudaSuccess) e = r;
    }
    return e;
}

dwf_status init_hop_tc_kernels() {
    DWF_CUDA((tc_attr<bf16, bf16>()));
    DWF_CUDA((tc_attr<bf16, float>()));
    DWF_CUDA((tc_attr<float, bf16>()));
    DWF_CUDA((tc_attr<float, float>()));
    return DWF_OK;
}

// BF16-link hop on the tensor cores (operands FP32 or BF16).
dwf_status launch_hop_tc(dwf_handle* h, const HopCall& c, const TileSet& ts, cudaStream_t s) {
    if (c.prec_link != DWF_BF16) return DWF_ERR_UNSUPPORTED;
    if (c.prec_in == DWF_BF16 && c.prec_out == DWF_BF16) return launch_tc_t<bf16, bf16>(h, c, ts, s);
    if (c.prec_in == DWF_BF16 && c.prec_out == DWF_FP32) return launch_tc_t<bf16, float>(h, c, ts, s);
    if (c.prec_in == DWF_FP32 && c.prec_out == DWF_BF16) return launch_tc_t<float, bf16>(h, c, ts, s);
    if (c.prec_in == DWF_FP32 && c.prec_out == DWF_FP32) return launch_tc_t<float, float>(h, c, ts, s);
    return DWF_ERR_UNSUPPORTED;
}

}  // namespace dwf
