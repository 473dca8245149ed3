// Operator compositions built from the hop and site-local kernels.
//
//   M_{p,1-p}        = -Dh_{p,1-p} (b5 + c5 S5) / 2          (off-diagonal block of D)
//   (M_{1-p,p})^+    = -(b5 + c5 S5^+) Dh^+_{p,1-p} / 2
//   M_pc             = M_oo - (1/4) Dh_oe [ (b5 + c5 S5) M_ee^-1 ] Dh_eo (b5 + c5 S5)
//   M_pc^+           = M_oo^+ - (1/4) (b5 + c5 S5^+) Dh^+_oe [ M_ee^-+ (b5 + c5 S5^+) ] Dh^+_eo
//   D                = [[M_ee, M_eo], [M_oe, M_oo]]
//
// (the bracketed site-local factors commute: per chirality both are functions
// of the same twisted shift).  Shamir (c5 = 0) skips the (b5 + c5 S5) passes
// and folds b5 into the hop scale.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

// Sites per tile for every kernel of an operator chain with nrhs right-hand
// sides: the value dwf_autotune or dwf_set_tile chose (never below kMinTile),
// else 32, whose table every handle builds when it is created.
int tile_for(dwf_handle* h, int nrhs) {
    auto it = h->tuned_T.find(nrhs);
    if (it != h->tuned_T.end() && it->second >= kMinTile) return it->second;
    return 32;
}

// Autotuner: for each candidate (tile size, lanes per thread) time what a
// CG iteration applies, M_pc and M_pc^+ with the operator of precision
// `prec` (the hops and the fifth-dimension kernels share the tile table; for
// FP64, whose fields do not fit the scratch twice, the bare hop), with CUDA
// events, median of 7 runs on a private stream with L2 flushed before each,
// on the handle's scratch fields; keep the fastest for every kernel chain
// with this nrhs.
dwf_status autotune(dwf_handle* h, int nrhs, dwf_prec prec, int* best) {
    const int cands[] = {8, 16, 32, 64, 128};
    cudaStream_t s;
    DWF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const size_t bytes = cb_elems(h, 1, nrhs) * 2 * prec_size(prec);
    cudaMemsetAsync(h->d_tmp2, 0, bytes, s);
    // FP32 / BF16 fields: two per FP64-sized scratch field
    unsigned char* t1 = reinterpret_cast<unsigned char*>(h->d_tmp);
    unsigned char* t2 = reinterpret_cast<unsigned char*>(h->d_tmp2);
    const bool chain = prec != DWF_FP64;
    if (chain) cudaMemsetAsync(t2 + bytes, 0, bytes, s);
    const auto saved_T = h->tuned_T;
    const auto saved_vl = h->tuned_vl;
    const auto saved_tc = h->tuned_tc;
    const auto saved_chunk = h->tuned_chunk;
    const auto saved_fuse = h->tuned_fuse;
    // candidates are timed with L2 flushed (solves stream more than L2 holds)
    const size_t flush_bytes = (size_t)256 << 20;
    void* flush = nullptr;
    DWF_CUDA(dev_malloc(&flush, flush_bytes));
    float best_ms = 1e30f;
    int best_T = tile_for(h, nrhs);
    int best_vl = 2;
    dwf_status st = DWF_OK;
    // lanes per thread: FP32 tries both; BF16 the SIMT kernel (0) and the
    // tensor-core one (-1); FP64 has one kernel
    const std::vector<int> vls = prec == DWF_FP32   ? std::vector<int>{2, 1}
                                 : prec == DWF_BF16 ? std::vector<int>{0, -1}
                                                    : std::vector<int>{0};
    const int chunks[] = {1, 8};
    int best_chunk = 1;
    int best_fuse = 0;
    // the fused epilogues exist for FP32-arithmetic chains whose site groups
    // divide a warp: time both forms there
    const bool can_fuse = chain && hop_bminv_ok(h, prec, nrhs, 2);
    int n_sm = 152;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    for (int fu = 0; fu <= (can_fuse ? 1 : 0); ++fu)
    for (int ck : chunks)
    for (int vl : vls)
    for (int T : cands) {
        // chunked tile order only with >= 4 chunks per resident CTA (two per SM):
        // fewer leave the last round unbalanced, by more than L1 reuse gains
        if (ck > 1 && (h->nsite[0] / T) / ck < 4 * 2 * n_sm) continue;
        // the tile table is shared by every precision of an operator chain
        // (FP64 reliable updates included): size the check for FP64 links
        const size_t smem = hop_smem(T, 8, 8, nrhs);
        if (smem > (size_t)kHopMaxSmem) continue;   // double-buffered links + reduction scratch
        HopCall c{};
        c.in = h->d_tmp2;
        c.out = h->d_tmp;
        c.out_parity = 0;
        c.prec_link = c.prec_in = c.prec_out = prec;
        c.nrhs = nrhs;
        c.scale = 1.0;
        c.T = T;
        c.VL = vl > 0 ? vl : 0;
        c.tc = vl < 0 ? 1 : 0;
        c.chunk = ck;
        std::vector<float> ts;
        for (int rep = 0; rep < 9 && st == DWF_OK; ++rep) {
            cudaMemsetAsync(flush, rep & 0xff, flush_bytes, s);
            cudaEventRecord(e0, s);
            if (chain) {
                h->tuned_T[nrhs] = T;
                h->tuned_chunk[nrhs] = ck;
                h->tuned_fuse[nrhs] = fu;
                if (vl > 0) h->tuned_vl[nrhs] = vl;
                if (prec == DWF_BF16) h->tuned_tc[nrhs] = vl < 0 ? 1 : 0;
                st = op_mpc(h, t2 + bytes, t2, 0, prec, prec, nrhs, t1, t1 + bytes, nullptr, nullptr, s);
                if (st == DWF_OK)
                    st = op_mpc(h, t2, t2 + bytes, 1, prec, prec, nrhs, t1, t1 + bytes, nullptr, nullptr, s);
            } else {
                st = launch_hop(h, c, s);
            }
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 2) ts.push_back(ms);
        }
        if (st != DWF_OK) break;
        std::sort(ts.begin(), ts.end());
        const float med = ts[ts.size() / 2];
        if (med < best_ms) { best_ms = med; best_T = T; best_vl = vl; best_chunk = ck; best_fuse = fu; }
    }
    // the handle-wide tile order for the chosen configuration: lexicographic or
    // blocked in (z, t) by 8 x 8 planes, whichever runs the chain faster
    if (st == DWF_OK && h->nbox == 1 && !h->dirichlet) {
        const int order0 = h->tile_order, bz0 = h->order_bz, bt0 = h->order_bt;
        float ord_ms[2] = {0.f, 0.f};
        h->tuned_T[nrhs] = best_T;
        h->tuned_chunk[nrhs] = best_chunk;
        h->tuned_fuse[nrhs] = best_fuse;
        if (best_vl > 0) h->tuned_vl[nrhs] = best_vl;
        if (prec == DWF_BF16) h->tuned_tc[nrhs] = best_vl < 0 ? 1 : 0;
        for (int od = 0; od < 2 && st == DWF_OK; ++od) {
            st = set_tile_order(h, od, 8, 8);
            std::vector<float> ts;
            for (int rep = 0; rep < 9 && st == DWF_OK; ++rep) {
                cudaMemsetAsync(flush, rep & 0xff, flush_bytes, s);
                cudaEventRecord(e0, s);
                if (chain) {
                    st = op_mpc(h, t2 + bytes, t2, 0, prec, prec, nrhs, t1, t1 + bytes, nullptr, nullptr, s);
                    if (st == DWF_OK)
                        st = op_mpc(h, t2, t2 + bytes, 1, prec, prec, nrhs, t1, t1 + bytes, nullptr, nullptr, s);
                } else {
                    HopCall c{};
                    c.in = h->d_tmp2;
                    c.out = h->d_tmp;
                    c.prec_link = c.prec_in = c.prec_out = prec;
                    c.nrhs = nrhs;
                    c.scale = 1.0;
                    c.T = best_T;
                    c.chunk = best_chunk;
                    st = launch_hop(h, c, s);
                }
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep >= 2) ts.push_back(ms);
            }
            if (st == DWF_OK) {
                std::sort(ts.begin(), ts.end());
                ord_ms[od] = ts[ts.size() / 2];
            }
        }
        if (st == DWF_OK) st = set_tile_order(h, ord_ms[1] < ord_ms[0] ? 1 : 0, 8, 8);
        else set_tile_order(h, order0, bz0, bt0);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(flush);
    cudaStreamDestroy(s);
    h->tuned_T = saved_T;
    h->tuned_vl = saved_vl;
    h->tuned_tc = saved_tc;
    h->tuned_chunk = saved_chunk;
    h->tuned_fuse = saved_fuse;
    if (st != DWF_OK) return st;
    h->tuned_T[nrhs] = best_T;
    h->tuned_chunk[nrhs] = best_chunk;
    h->tuned_prec[nrhs] = (int)prec;
    h->tuned_fuse[nrhs] = best_fuse;
    if (prec == DWF_FP32) h->tuned_vl[nrhs] = best_vl;
    if (prec == DWF_BF16) h->tuned_tc[nrhs] = best_vl < 0 ? 1 : 0;
    if (best) *best = best_T;
    return DWF_OK;
}

static int tileT(dwf_handle* h, int, dwf_prec, int nrhs) { return tile_for(h, nrhs); }

// Key of a tuning in the autotune file: the device, the domain (lattice, Ls,
// boxes), the precision and nrhs -- what the measured choice depends on.
std::string tuning_key(const dwf_handle* h, int nrhs, int prec) {
    cudaDeviceProp dp{};
    cudaGetDeviceProperties(&dp, h->device);
    std::string name(dp.name);
    for (char& ch : name)
        if (ch == ' ') ch = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "%s/%d|%d,%d,%d,%d|%d|", name.c_str(), dp.multiProcessorCount, h->p.dims[0],
             h->p.dims[1], h->p.dims[2], h->p.dims[3], h->p.Ls);
    std::string k(buf);
    if (h->dirichlet)
        for (const dwf_box& b : h->boxes) {
            snprintf(buf, sizeof(buf), "%d,%d,%d,%d:%d,%d,%d,%d;", b.origin[0], b.origin[1], b.origin[2], b.origin[3],
                     b.extent[0], b.extent[1], b.extent[2], b.extent[3]);
            k += buf;
        }
    else
        k += "whole";
    for (const dwf_box& b : h->cut) {
        snprintf(buf, sizeof(buf), "%scut%d,%d,%d,%d:%d,%d,%d,%d", &b == &h->cut[0] ? "/" : ";", b.origin[0],
                 b.origin[1], b.origin[2], b.origin[3], b.extent[0], b.extent[1], b.extent[2], b.extent[3]);
        k += buf;
    }
    snprintf(buf, sizeof(buf), "|p%d|n%d", prec, nrhs);
    return k + buf;
}

size_t cb_elems(const dwf_handle* h, int parity, int nrhs) {
    return (size_t)h->nsite[parity] * 12 * h->p.Ls * nrhs;   // complex elements
}

static bool shamir(const dwf_handle* h) { return h->p.c5 == 0.0; }

// Lanes per thread of the FP32-arithmetic hop with nrhs right-hand sides.
static int hop_vl(dwf_handle* h, dwf_prec link, int nrhs) {
    if (link != DWF_FP32) return 2;
    auto it = h->tuned_vl.find(nrhs);
    return it == h->tuned_vl.end() ? 2 : it->second;
}

static HopCall hop_call(dwf_handle* h, const void* in, void* out, int out_parity, int dagger,
                        dwf_prec link, dwf_prec pin, dwf_prec pout, int nrhs, double scale,
                        const void* xmoo, double* partial);

// Whether the chains of nrhs right-hand sides run the site-local factors in
// the hop epilogues (chosen by dwf_autotune or dwf_set_fusion; default off).
static bool fused(const dwf_handle* h, int nrhs) {
    auto it = h->tuned_fuse.find(nrhs);
    return it != h->tuned_fuse.end() && it->second != 0;
}

dwf_status op_hop(dwf_handle* h, void* out, const void* in, int out_parity, int dagger,
                  dwf_prec link, dwf_prec pin, dwf_prec pout, int nrhs, double scale,
                  const void* xmoo, double* partial, cudaStream_t s) {
    return launch_hop(h, hop_call(h, in, out, out_parity, dagger, link, pin, pout, nrhs, scale, xmoo,
                                  partial), s);
}

// The hop launch of an operator chain: tuned tile, lanes, kernel and tile order.
static HopCall hop_call(dwf_handle* h, const void* in, void* out, int out_parity, int dagger,
                        dwf_prec link, dwf_prec pin, dwf_prec pout, int nrhs, double scale,
                        const void* xmoo, double* partial) {
    HopCall c;
    c.in = in;
    c.out = out;
    c.xmoo = xmoo;
    c.out_parity = out_parity;
    c.dagger = dagger;
    c.prec_link = link;
    c.prec_in = pin;
    c.prec_out = pout;
    c.nrhs = nrhs;
    c.scale = scale;
    c.partial = partial;
    c.T = tileT(h, 0, link, nrhs);
    if (link == DWF_FP32) {
        auto it = h->tuned_vl.find(nrhs);
        c.VL = it == h->tuned_vl.end() ? 2 : it->second;
    }
    if (link == DWF_BF16) {
        auto it = h->tuned_tc.find(nrhs);
        c.tc = it == h->tuned_tc.end() ? 0 : it->second;
    }
    {
        auto it = h->tuned_chunk.find(nrhs);
        c.chunk = it == h->tuned_chunk.end() ? 1 : it->second;
    }
    return c;
}

dwf_status op_local(dwf_handle* h, LocalOp op, void* out, const void* in, const void* in2,
                    int parity, int dagger, dwf_prec pin, dwf_prec pin2, dwf_prec pout, int nrhs,
                    double scale, double* partial, cudaStream_t s) {
    LocalCall c{};
    c.op = op;
    c.in = in;
    c.in2 = in2;
    c.out = out;
    c.parity = parity;
    c.dagger = dagger;
    c.prec_in = pin;
    c.prec_in2 = pin2;
    c.prec_out = pout;
    c.nrhs = nrhs;
    c.scale = scale;
    c.partial = partial;
    c.T = tileT(h, 0, pout == DWF_FP64 ? DWF_FP64 : DWF_FP32, nrhs);
    return launch_local(h, c, s);
}

// out = M_{p,1-p} in (dagger: (M_{1-p,p})^+ in); in/out/link precision `prec`.
dwf_status op_dslash_eo(dwf_handle* h, void* out, const void* in, int p, int dagger,
                        dwf_prec prec, int nrhs, void* tmp, cudaStream_t s) {
    const double b5 = h->p.b5;
    if (shamir(h)) return op_hop(h, out, in, p, dagger, prec, prec, prec, nrhs, -0.5 * b5, nullptr, nullptr, s);
    if (!dagger) {
        DWF_TRY(op_local(h, L_B, tmp, in, nullptr, 1 - p, 0, prec, prec, prec, nrhs, 1.0, nullptr, s));
        return op_hop(h, out, tmp, p, 0, prec, prec, prec, nrhs, -0.5, nullptr, nullptr, s);
    }
    DWF_TRY(op_hop(h, tmp, in, p, 1, prec, prec, prec, nrhs, 1.0, nullptr, nullptr, s));
    return op_local(h, L_B, out, tmp, nullptr, p, 1, prec, prec, prec, nrhs, -0.5, nullptr, s);
}

// (b5 + c5 S5)(d + e S5)^-1 Dh_{eo} in (adjoint chain: with S5^+ and Dh^+),
// the first half of M_pc (M_pc^+), into one of the temporaries tmpA, tmpB
// (returned in *res; `in` may be one of them and is never overwritten while
// it is read): one hop with the site-local factor in its epilogue where the
// site's lanes share a warp, else the hop and the separate site-local pass.
static dwf_status hop_then_bminv(dwf_handle* h, const void* in, int dagger, dwf_prec po,
                                 dwf_prec pin, int nrhs, double scale, void* tmpA, void* tmpB,
                                 void** res, cudaStream_t s) {
    void* first = (in == tmpA) ? tmpB : tmpA;
    void* second = (first == tmpA) ? tmpB : tmpA;
    HopCall hc = hop_call(h, in, first, 0, dagger, po, pin, po, nrhs, scale, nullptr, nullptr);
    if (hc.tc == 0 && fused(h, nrhs) && hop_bminv_ok(h, po, nrhs, hop_vl(h, po, nrhs))) {
        hc.bminv = true;
        *res = first;
        return launch_hop(h, hc, s);
    }
    DWF_TRY(launch_hop(h, hc, s));
    *res = second;
    return op_local(h, L_BMINV, second, first, nullptr, 0, dagger, po, po, po, nrhs, 1.0, nullptr, s);
}

// Schur operator on the odd checkerboard.  pv: precision of in/out (and of
// the CG vectors), po: operator precision (links and intermediates).
// tmpA/tmpB: cb temporaries of precision po.  partial: per-tile |out|^2.
// cg: optional fused CG step of the adjoint (x += alpha p, r -= alpha out).

dwf_status op_mpc(dwf_handle* h, void* out, const void* in, int dagger, dwf_prec pv, dwf_prec po,
                  int nrhs, void* tmpA, void* tmpB, double* partial, const CgFuse* cg,
                  cudaStream_t s) {
    const double b5 = h->p.b5;
    if (!dagger) {
        const void* src = in;
        dwf_prec psrc = pv;
        double sc1 = b5;
        if (!shamir(h)) {
            DWF_TRY(op_local(h, L_B, tmpA, in, nullptr, 1, 0, pv, pv, po, nrhs, 1.0, nullptr, s));
            src = tmpA;
            psrc = po;
            sc1 = 1.0;
        }
        void* mid = nullptr;
        DWF_TRY(hop_then_bminv(h, src, 0, po, psrc, nrhs, sc1, tmpA, tmpB, &mid, s));
        return op_hop(h, out, mid, 1, 0, po, po, pv, nrhs, -0.25, in, partial, s);
    }
    void* mid = nullptr;
    DWF_TRY(hop_then_bminv(h, in, 1, po, pv, nrhs, 1.0, tmpA, tmpB, &mid, s));
    void* other = (mid == tmpA) ? tmpB : tmpA;
    HopCall hc = hop_call(h, mid, nullptr, 1, 1, po, po, pv, nrhs, -0.25, in, partial);
    if (cg != nullptr && hc.tc == 0 && fused(h, nrhs) && hop_post_ok(h, po, pv, nrhs, hop_vl(h, po, nrhs))) {
        // the tail M_oo^+ in - (1/4) B^+ (.) and the CG update in the last hop's epilogue
        hc.post = true;
        hc.cg_x = cg->x;
        hc.cg_r = cg->r;
        hc.cg_p = cg->p;
        hc.alpha = cg->alpha;
        hc.run = cg->run;
        return launch_hop(h, hc, s);
    }
    DWF_TRY(op_hop(h, other, mid, 1, 1, po, po, po, nrhs, 1.0, nullptr, nullptr, s));
    LocalCall c{};
    c.op = L_POST;
    c.in = in;
    c.in2 = other;
    c.out = out;
    c.parity = 1;
    c.dagger = 1;
    c.prec_in = pv;
    c.prec_in2 = po;
    c.prec_out = pv;
    c.nrhs = nrhs;
    c.scale = -0.25;
    c.partial = partial;
    c.T = tileT(h, 0, pv == DWF_FP64 ? DWF_FP64 : DWF_FP32, nrhs);
    if (cg) {
        c.cg_x = cg->x;
        c.cg_r = cg->r;
        c.cg_p = cg->p;
        c.alpha = cg->alpha;
        c.run = cg->run;
        c.prec_vec = pv;
    }
    return launch_local(h, c, s);
}

// M_pc p when t1 = (b5 + c5 S5) p has already been formed (by the fused CG
// direction update): out = M_oo p - (1/4) Dh_oe (b5 + c5 S5) M_ee^-1 Dh_eo t1.
dwf_status op_mpc_pre(dwf_handle* h, void* out, const void* p, const void* t1, dwf_prec pv,
                      dwf_prec po, int nrhs, void* tmpA, void* tmpB, double* partial,
                      cudaStream_t s) {
    void* mid = nullptr;
    DWF_TRY(hop_then_bminv(h, t1, 0, po, po, nrhs, 1.0, tmpA, tmpB, &mid, s));
    return op_hop(h, out, mid, 1, 0, po, po, pv, nrhs, -0.25, p, partial, s);
}

// Full operator on full fields (both parities): D or D^+.
dwf_status op_apply_d(dwf_handle* h, void* out, const void* in, int dagger, dwf_prec prec,
                      int nrhs, void* tmp, cudaStream_t s) {
    const size_t ps = prec_size(prec) * 2;
    const size_t off1 = cb_elems(h, 0, nrhs) * ps;
    char* o = (char*)out;
    const char* i = (const char*)in;
    for (int p = 0; p < 2; ++p) {
        char* op = o + (p ? off1 : 0);
        const char* ip = i + (p ? off1 : 0);
        const char* iq = i + (p ? 0 : off1);
        if (!dagger) {
            const void* src = iq;
            double sc = -0.5 * h->p.b5;
            if (!shamir(h)) {
                DWF_TRY(op_local(h, L_B, tmp, iq, nullptr, 1 - p, 0, prec, prec, prec, nrhs, 1.0, nullptr, s));
                src = tmp;
                sc = -0.5;
            }
            DWF_TRY(op_hop(h, op, src, p, 0, prec, prec, prec, nrhs, sc, ip, nullptr, s));
        } else {
            DWF_TRY(op_hop(h, tmp, iq, p, 1, prec, prec, prec, nrhs, 1.0, nullptr, nullptr, s));
            DWF_TRY(op_local(h, L_POST, op, ip, tmp, p, 1, prec, prec, prec, nrhs, -0.5, nullptr, s));
        }
    }
    return DWF_OK;
}

}  // namespace dwf
