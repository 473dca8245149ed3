// Domains: site lists, neighbour and tile tables, link tables, layout kernels.
//
// A handle's domain is a list of boxes (the whole lattice is one box).  The
// Dirichlet block operator D_Omega of a box (Sec. 2.1) is D with every link
// that leaves the box removed (Sec. 2.4); here that removal is done once, when
// the neighbour table is built: a hop that leaves its box gets neighbour -1
// and a zero link, and the kernels skip it.  Sites outside every box are not
// stored at all, so the operator never touches Omega-bar.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char* last_error() { return g_err; }

static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_allocs{0};

void note_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }
uint64_t alloc_count() { return g_allocs.load(); }
static thread_local int g_capturing = 0;
static thread_local int g_captured = 0;

void note_launch() {
    if (g_capturing) ++g_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void capture_begin() { g_capturing = 1; g_captured = 0; }
int capture_end() { g_capturing = 0; return g_captured; }
void note_graph_launch(int kernels) { g_launches.fetch_add((uint64_t)kernels, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(); }

size_t prec_size(dwf_prec p) { return p == DWF_FP64 ? 8 : (p == DWF_FP32 ? 4 : 2); }

dwf_status check_handle(const dwf_handle* h) {
    if (h == nullptr) {
        set_error("null handle");
        return DWF_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) {
        set_error("handle created on device %d used with device %d current", h->device, dev);
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

dwf_status persistent_grid(const void* kern, int threads, size_t smem, int ntiles, int* grid) {
    static std::mutex mu;
    static std::map<int, int> n_sm;                                    // device -> SMs
    static std::map<std::tuple<int, const void*, int, size_t>, int> occ;   // -> blocks per SM
    int dev = 0;
    DWF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto is = n_sm.find(dev);
    if (is == n_sm.end()) {
        int n = 0;
        DWF_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        is = n_sm.emplace(dev, n > 0 ? n : 1).first;
    }
    const auto key = std::make_tuple(dev, kern, threads, smem);
    auto io = occ.find(key);
    if (io == occ.end()) {
        int per_sm = 0;
        DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        io = occ.emplace(key, per_sm > 0 ? per_sm : 1).first;
    }
    const long g = (long)io->second * is->second;
    *grid = (int)(g < ntiles ? g : ntiles);
    return DWF_OK;
}

const TileSet* find_tiles(const dwf_handle* h, int T) {
    auto it = h->tiles.find(T);
    return it == h->tiles.end() ? nullptr : &it->second;
}

static void free_tiles(TileSet& ts) {
    for (int p = 0; p < 2; ++p) {
        cudaFree(ts.d_tiles[p]);
        cudaFree(ts.d_box_tile_begin[p]);
        ts.d_tiles[p] = nullptr;
        ts.d_box_tile_begin[p] = nullptr;
    }
}

// The tiles of parity p for T sites per tile, box by box, and where each box's
// tiles begin.  Within a box the tiles run in lexicographic site order, or
// (tile_order 1) blocked in (z, t): by t / bt, z / bz, then t % bt, z % bz, y,
// x of a tile's first site, so that the two uses of a z or t neighbour row
// (as the +mu neighbour of one plane, the -mu neighbour of the plane two
// steps on) lie a block's planes apart instead of a whole time slice.
static void tile_list(const dwf_handle* h, int T, int p, std::vector<int4>& tl, std::vector<int>& begin) {
    tl.clear();
    begin.assign(h->nbox + 1, 0);
    for (int b = 0; b < h->nbox; ++b) {
        begin[b] = (int)tl.size();
        const int64_t off = h->box_off[p][b], cnt = h->box_cnt[p][b];
        for (int64_t i = 0; i < cnt; i += T)
            tl.push_back(make_int4(b, (int)(off + i), (int)std::min<int64_t>(T, cnt - i), 0));
        if (h->tile_order == 1 && !h->site_local_host[p].empty()) {
            const int* e = h->boxes[b].extent;
            const int bz = h->order_bz, bt = h->order_bt;
            auto key = [&](const int4& t) {
                const int64_t l = h->site_local_host[p][t.y];
                const int64_t x = l % e[0], y = (l / e[0]) % e[1], z = (l / ((int64_t)e[0] * e[1])) % e[2],
                              tt = l / ((int64_t)e[0] * e[1] * e[2]);
                return std::make_tuple(tt / bt, z / bz, tt % bt, z % bz, y, x);
            };
            std::stable_sort(tl.begin() + begin[b], tl.end(),
                             [&](const int4& u, const int4& v) { return key(u) < key(v); });
        }
    }
    begin[h->nbox] = (int)tl.size();
}

dwf_status get_tiles(dwf_handle* h, int T, const TileSet** out) {
    *out = find_tiles(h, T);
    if (*out != nullptr) return DWF_OK;
    if (T < 1) {
        set_error("tile table: %d sites per tile", T);
        return DWF_ERR_ARG;
    }
    TileSet ts;
    ts.T = T;
    for (int p = 0; p < 2; ++p) {
        std::vector<int4> tl;
        tile_list(h, T, p, tl, ts.box_tile_begin[p]);
#ifdef DWF_DEBUG
        for (const int4& t : tl)
            if (t.x < 0 || t.x >= h->nbox || t.y < 0 || t.z < 1 || (int64_t)t.y + t.z > h->nsite[p]) {
                set_error("tile table (debug): tile {%d, %d, %d} outside parity %d's %lld sites", t.x, t.y, t.z, p,
                          (long long)h->nsite[p]);
                free_tiles(ts);
                return DWF_ERR_ARG;
            }
#endif
        ts.ntiles[p] = (int)tl.size();
        cudaError_t e = cudaSuccess;
        if (!tl.empty()) {
            e = dev_malloc(&ts.d_tiles[p], tl.size() * sizeof(int4));
            if (e == cudaSuccess)
                e = cudaMemcpy(ts.d_tiles[p], tl.data(), tl.size() * sizeof(int4), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = dev_malloc(&ts.d_box_tile_begin[p], (h->nbox + 1) * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(ts.d_box_tile_begin[p], ts.box_tile_begin[p].data(), (h->nbox + 1) * sizeof(int),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_tiles(ts);
            set_error("tile table of %d sites per tile: %s", T, cudaGetErrorString(e));
            return DWF_ERR_CUDA;
        }
    }
    *out = &h->tiles.emplace(T, ts).first->second;
    return DWF_OK;
}

// Reorder every existing tile table in place (same tiles, same device
// buffers, so captured graphs and per-tile buffers stay valid) and build later
// ones in the new order.  Waits for the device first.
dwf_status set_tile_order(dwf_handle* h, int order, int bz, int bt) {
    if ((order != 0 && order != 1) || bz < 1 || bt < 1) {
        set_error("dwf_set_tile_order: order must be 0 or 1, block extents >= 1");
        return DWF_ERR_ARG;
    }
    DWF_CUDA(cudaDeviceSynchronize());
    h->tile_order = order;
    h->order_bz = bz;
    h->order_bt = bt;
    for (auto& kv : h->tiles) {
        TileSet& ts = kv.second;
        for (int p = 0; p < 2; ++p) {
            std::vector<int4> tl;
            std::vector<int> begin;
            tile_list(h, ts.T, p, tl, begin);
            if ((int)tl.size() != ts.ntiles[p] || begin != ts.box_tile_begin[p]) {
                set_error("dwf_set_tile_order: tile table changed shape");
                return DWF_ERR_ARG;
            }
            if (!tl.empty())
                DWF_CUDA(cudaMemcpy(ts.d_tiles[p], tl.data(), tl.size() * sizeof(int4), cudaMemcpyHostToDevice));
        }
    }
    return DWF_OK;
}

// ----------------------------------------------------------- link tables
// doubled link table of one parity: [site][k][3][3] complex, k < 4 forward
// U_mu(x), k >= 4 backward U_mu(x - mu)^+; zero where src < 0 (cut).
__global__ void k_gather_links(const double* __restrict__ U, const int64_t* __restrict__ src,
                               int64_t n /* sites * 8 */, double* __restrict__ l64,
                               float* __restrict__ l32, bf16* __restrict__ l16) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * 9;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sk = i / 9;
        const int ab = (int)(i % 9);
        const int a = ab / 3, b = ab % 3;
        const int k = (int)(sk % 8);
        const int64_t g = src[sk];
        double re = 0.0, im = 0.0;
        if (g >= 0) {
            if (k < 4) {
                re = U[(g * 9 + a * 3 + b) * 2];
                im = U[(g * 9 + a * 3 + b) * 2 + 1];
            } else {   // (U^+)_{ab} = conj(U_{ba})
                re = U[(g * 9 + b * 3 + a) * 2];
                im = -U[(g * 9 + b * 3 + a) * 2 + 1];
            }
        }
        l64[2 * i] = re;
        l64[2 * i + 1] = im;
        l32[2 * i] = (float)re;
        l32[2 * i + 1] = (float)im;
        l16[2 * i] = __float2bfloat16_rn((float)re);
        l16[2 * i + 1] = __float2bfloat16_rn((float)im);
    }
}

// --------------------------------------------------------- layout kernels
// canonical [box][r][l][s][spin][colour] <-> full field [parity][site][c][r][s]
template <bool TO_DOMAIN, class S>
__global__ void k_pack(S* __restrict__ dom, double* __restrict__ canon,
                       const int* __restrict__ site_box, const int* __restrict__ site_local,
                       const int64_t* __restrict__ box_vol, const int64_t* __restrict__ box_prefix,
                       int64_t nsite, int64_t dom_off, int nrhs, int Ls) {
    const int64_t n = nsite * 12 * nrhs * Ls;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % Ls);
        const int r = (int)((i / Ls) % nrhs);
        const int c = (int)((i / ((int64_t)Ls * nrhs)) % 12);
        const int64_t site = i / ((int64_t)Ls * nrhs * 12);
        const int b = site_box[site];
        const int64_t l = site_local[site];
        const int64_t cs = nrhs * box_prefix[b] + (int64_t)r * box_vol[b] + l;
        const int64_t ci = (cs * Ls + s) * 12 + c;
        const int64_t di = dom_off + i;
        if (TO_DOMAIN) {
            double re = canon[2 * ci], im = canon[2 * ci + 1];
            if constexpr (std::is_same<S, double>::value) {
                dom[2 * di] = re; dom[2 * di + 1] = im;
            } else if constexpr (std::is_same<S, float>::value) {
                dom[2 * di] = (float)re; dom[2 * di + 1] = (float)im;
            } else {
                dom[2 * di] = __float2bfloat16_rn((float)re);
                dom[2 * di + 1] = __float2bfloat16_rn((float)im);
            }
        } else {
            double re, im;
            if constexpr (std::is_same<S, bf16>::value) {
                re = __bfloat162float(dom[2 * di]); im = __bfloat162float(dom[2 * di + 1]);
            } else {
                re = (double)dom[2 * di]; im = (double)dom[2 * di + 1];
            }
            canon[2 * ci] = re;
            canon[2 * ci + 1] = im;
        }
    }
}

template <bool TO, class S>
static dwf_status pack_t(dwf_handle* h, S* dom, double* canon, int nrhs, cudaStream_t s) {
    int64_t off = 0;
    for (int p = 0; p < 2; ++p) {
        const int64_t n = h->nsite[p] * 12 * nrhs * h->p.Ls;
        if (n > 0) {
            int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 64);
            k_pack<TO, S><<<(int)blocks, 256, 0, s>>>(dom, canon, h->d_site_box[p],
                                                      h->d_site_local[p], h->d_box_canon_vol,
                                                      h->d_box_canon_vol + h->nbox, h->nsite[p],
                                                      off, nrhs, h->p.Ls);
            note_launch();
            DWF_CUDA(cudaGetLastError());
        }
        off += n;
    }
    return DWF_OK;
}

dwf_status pack(dwf_handle* h, void* dst, const double* src, int nrhs, dwf_prec prec,
                cudaStream_t s) {
    double* c = const_cast<double*>(src);
    switch (prec) {
        case DWF_FP64: return pack_t<true, double>(h, (double*)dst, c, nrhs, s);
        case DWF_FP32: return pack_t<true, float>(h, (float*)dst, c, nrhs, s);
        default: return pack_t<true, bf16>(h, (bf16*)dst, c, nrhs, s);
    }
}

dwf_status unpack(dwf_handle* h, double* dst, const void* src, int nrhs, dwf_prec prec,
                  cudaStream_t s) {
    void* d = const_cast<void*>(src);
    switch (prec) {
        case DWF_FP64: return pack_t<false, double>(h, (double*)d, dst, nrhs, s);
        case DWF_FP32: return pack_t<false, float>(h, (float*)d, dst, nrhs, s);
        default: return pack_t<false, bf16>(h, (bf16*)d, dst, nrhs, s);
    }
}

dwf_status set_gauge(dwf_handle* h, const double* U, cudaStream_t s) {
    for (int p = 0; p < 2; ++p) {
        const int64_t n = h->nsite[p] * 8;
        if (n == 0) continue;
        const int64_t blocks = std::min<int64_t>((n * 9 + 255) / 256, 152 * 64);
        k_gather_links<<<(int)blocks, 256, 0, s>>>(U, h->d_link_src[p], n, (double*)h->d_links[0][p],
                                                   (float*)h->d_links[1][p], (bf16*)h->d_links[2][p]);
        note_launch();
        DWF_CUDA(cudaGetLastError());
    }
    DWF_CUDA(cudaStreamSynchronize(s));
    h->have_gauge = true;
    return DWF_OK;
}

// ------------------------------------------------------------ creation
static FiveD make_f5(const dwf_params& p) {
    FiveD f;
    f.Ls = p.Ls;
    f.mf = p.mf;
    f.b5 = p.b5;
    f.c5 = p.c5;
    f.d = p.b5 * (4.0 - p.M5) + 1.0;
    f.e = p.c5 * (4.0 - p.M5) - 1.0;
    f.a = -f.e / f.d;
    f.inv_d = 1.0 / f.d;
    double aL = 1.0;
    for (int i = 0; i < p.Ls; ++i) aL *= f.a;
    f.inv_den = 1.0 / (f.d * (1.0 + p.mf * aL));
    return f;
}

static dwf_status h2d(void* dst, const void* src, size_t bytes) {
    DWF_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
    return DWF_OK;
}

template <class T>
static dwf_status dalloc(T** ptr, size_t n) {
    *ptr = nullptr;
    if (n == 0) n = 1;
    DWF_CUDA(dev_malloc(ptr, n * sizeof(T)));
    return DWF_OK;
}

dwf_status create(dwf_handle** out, const dwf_params* p, const dwf_box* boxes, int nbox,
                  int nrhs_max) {
    if (out == nullptr || p == nullptr) {
        set_error("dwf_create: null argument");
        return DWF_ERR_ARG;
    }
    *out = nullptr;
    for (int mu = 0; mu < 4; ++mu)
        if (p->dims[mu] < 2 || p->dims[mu] % 2) {
            set_error("dwf_create: dims[%d] = %d must be even and >= 2", mu, p->dims[mu]);
            return DWF_ERR_ARG;
        }
    if (p->Ls < 2 || p->Ls > kMaxLs || p->Ls % 2) {
        set_error("dwf_create: Ls = %d must be even, 2 <= Ls <= %d", p->Ls, kMaxLs);
        return DWF_ERR_ARG;
    }
    if (nrhs_max < 1 || p->Ls * nrhs_max > kMaxLanes) {
        set_error("dwf_create: nrhs_max = %d out of range (Ls * nrhs_max <= %d)", nrhs_max, kMaxLanes);
        return DWF_ERR_ARG;
    }
    if (nbox < 0 || (nbox > 0 && boxes == nullptr)) {
        set_error("dwf_create: bad box list");
        return DWF_ERR_ARG;
    }
    const FiveD f5 = make_f5(*p);
    if (!(f5.d != 0.0) || !std::isfinite(f5.inv_den)) {
        set_error("dwf_create: M_ee = d + e S5 is singular for these parameters");
        return DWF_ERR_ARG;
    }
    const int* L = p->dims;
    std::vector<dwf_box> bx;
    if (nbox == 0) {
        dwf_box b;
        for (int mu = 0; mu < 4; ++mu) { b.origin[mu] = 0; b.extent[mu] = L[mu]; }
        bx.push_back(b);
    } else {
        for (int i = 0; i < nbox; ++i) {
            dwf_box b = boxes[i];
            for (int mu = 0; mu < 4; ++mu) {
                if (b.extent[mu] < 1 || b.extent[mu] > L[mu]) {
                    set_error("dwf_create: box %d extent[%d] = %d outside [1, %d]", i, mu,
                              b.extent[mu], L[mu]);
                    return DWF_ERR_ARG;
                }
                b.origin[mu] = ((b.origin[mu] % L[mu]) + L[mu]) % L[mu];
            }
            bx.push_back(b);
        }
    }
    dwf_handle* h = new dwf_handle();
    h->p = *p;
    h->nbox = (int)bx.size();
    h->dirichlet = nbox > 0;
    h->boxes = bx;
    h->nrhs_max = nrhs_max;
    cudaGetDevice(&h->device);
    h->f5[0] = h->f5[1] = f5;
    // site enumeration
    std::vector<int> site_box[2], site_local[2];
    std::vector<int64_t> site_glob[2];
    std::vector<std::vector<int>> loc2idx(h->nbox);
    std::vector<int64_t> prefix(h->nbox + 1, 0);
    for (int q = 0; q < 2; ++q) { h->box_off[q].assign(h->nbox, 0); h->box_cnt[q].assign(h->nbox, 0); }
    h->box_vol.assign(h->nbox, 0);
    for (int b = 0; b < h->nbox; ++b) {
        const int* o = bx[b].origin;
        const int* e = bx[b].extent;
        const int64_t vol = (int64_t)e[0] * e[1] * e[2] * e[3];
        h->box_vol[b] = vol;
        prefix[b + 1] = prefix[b] + vol;
        loc2idx[b].assign(vol, 0);
        for (int q = 0; q < 2; ++q) h->box_off[q][b] = (int64_t)site_box[q].size();
        for (int64_t l = 0; l < vol; ++l) {
            int lc[4] = {(int)(l % e[0]), (int)((l / e[0]) % e[1]), (int)((l / ((int64_t)e[0] * e[1])) % e[2]),
                         (int)(l / ((int64_t)e[0] * e[1] * e[2]))};
            int x[4];
            for (int mu = 0; mu < 4; ++mu) x[mu] = (o[mu] + lc[mu]) % L[mu];
            const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
            loc2idx[b][l] = (int)site_box[par].size();
            site_box[par].push_back(b);
            site_local[par].push_back((int)l);
            site_glob[par].push_back(x[0] + (int64_t)L[0] * (x[1] + (int64_t)L[1] * (x[2] + (int64_t)L[2] * x[3])));
        }
        for (int q = 0; q < 2; ++q) h->box_cnt[q][b] = (int64_t)site_box[q].size() - h->box_off[q][b];
    }
    for (int q = 0; q < 2; ++q) h->nsite[q] = (int64_t)site_box[q].size();
    h->vol = h->nsite[0] + h->nsite[1];
    if (h->vol > (int64_t)1 << 30) {
        set_error("dwf_create: domain too large");
        delete h;
        return DWF_ERR_ARG;
    }
    // neighbour and link-source tables
    dwf_status st = DWF_OK;
    for (int q = 0; q < 2 && st == DWF_OK; ++q) {
        const int64_t ns = h->nsite[q];
        std::vector<int> nbr(ns * 8);
        std::vector<int64_t> lsrc(ns * 8);
        for (int64_t i = 0; i < ns; ++i) {
            const int b = site_box[q][i];
            const int* o = bx[b].origin;
            const int* e = bx[b].extent;
            const int64_t l = site_local[q][i];
            int lc[4] = {(int)(l % e[0]), (int)((l / e[0]) % e[1]), (int)((l / ((int64_t)e[0] * e[1])) % e[2]),
                         (int)(l / ((int64_t)e[0] * e[1] * e[2]))};
            for (int k = 0; k < 8; ++k) {
                const int mu = k & 3;
                const int step = k < 4 ? 1 : -1;
                int nl[4] = {lc[0], lc[1], lc[2], lc[3]};
                nl[mu] += step;
                bool in = true;
                if (e[mu] == L[mu]) nl[mu] = (nl[mu] + L[mu]) % L[mu];
                else if (nl[mu] < 0 || nl[mu] >= e[mu]) in = false;
                if (!in) {
                    nbr[i * 8 + k] = -1;
                    lsrc[i * 8 + k] = -1;
                    continue;
                }
                const int64_t ln = nl[0] + (int64_t)e[0] * (nl[1] + (int64_t)e[1] * (nl[2] + (int64_t)e[2] * nl[3]));
                nbr[i * 8 + k] = loc2idx[b][ln];
                int x[4];
                for (int m = 0; m < 4; ++m) x[m] = (o[m] + lc[m]) % L[m];
                if (k >= 4) x[mu] = (x[mu] - 1 + L[mu]) % L[mu];   // link lives at x - mu
                const int64_t g = x[0] + (int64_t)L[0] * (x[1] + (int64_t)L[1] * (x[2] + (int64_t)L[2] * x[3]));
                lsrc[i * 8 + k] = g * 4 + mu;
            }
        }
#ifdef DWF_DEBUG
        // neighbours index the other parity's site list, links the canonical gauge field
        const int64_t nopp = h->nsite[1 - q], nlink = (int64_t)L[0] * L[1] * L[2] * L[3] * 4;
        for (int64_t e = 0; e < ns * 8 && st == DWF_OK; ++e)
            if (nbr[e] < -1 || nbr[e] >= nopp || lsrc[e] < -1 || lsrc[e] >= nlink || (nbr[e] < 0) != (lsrc[e] < 0)) {
                set_error("dwf_create (debug): table entry %lld of parity %d out of range (neighbour %d of %lld, "
                          "link %lld of %lld)", (long long)e, q, nbr[e], (long long)nopp, (long long)lsrc[e],
                          (long long)nlink);
                st = DWF_ERR_ARG;
            }
        if (st != DWF_OK) break;
#endif
        st = dalloc(&h->d_nbr[q], ns * 8);
        if (st == DWF_OK) st = dalloc(&h->d_link_src[q], ns * 8);
        if (st == DWF_OK) st = dalloc(&h->d_site_box[q], ns);
        if (st == DWF_OK) st = dalloc(&h->d_site_local[q], ns);
        if (st != DWF_OK) break;
        st = h2d(h->d_nbr[q], nbr.data(), ns * 8 * sizeof(int));
        if (st == DWF_OK) st = h2d(h->d_link_src[q], lsrc.data(), ns * 8 * sizeof(int64_t));
        if (st == DWF_OK) st = h2d(h->d_site_box[q], site_box[q].data(), ns * sizeof(int));
        if (st == DWF_OK) st = h2d(h->d_site_local[q], site_local[q].data(), ns * sizeof(int));
        if (st == DWF_OK) h->site_local_host[q] = site_local[q];
        for (int pr = 0; pr < 3 && st == DWF_OK; ++pr)
            st = dalloc((char**)&h->d_links[pr][q], ns * 144 * prec_size((dwf_prec)pr));
    }
    if (st == DWF_OK) {
        std::vector<int64_t> bv(2 * h->nbox);
        for (int b = 0; b < h->nbox; ++b) { bv[b] = h->box_vol[b]; bv[h->nbox + b] = prefix[b]; }
        st = dalloc(&h->d_box_canon_vol, 2 * h->nbox);
        if (st == DWF_OK)
            st = h2d(h->d_box_canon_vol, bv.data(), bv.size() * sizeof(int64_t));
    }
    if (st == DWF_OK) st = init_hop_kernels();
    if (st == DWF_OK) st = init_local_kernels();
    if (st == DWF_OK) st = init_local_mat_kernels();
    if (st == DWF_OK) st = init_hop_tc_kernels();
    if (st == DWF_OK) {
        std::vector<float> mats;
        build_fived_mats(f5, mats);
        st = dalloc(&h->d_mats, mats.size());
        if (st == DWF_OK)
            st = h2d(h->d_mats, mats.data(), mats.size() * sizeof(float));
    }
    if (st == DWF_OK) st = dalloc(&h->d_err, 1);
    if (st == DWF_OK) {
        if (cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess) {
            set_error("dwf_create: clearing the device error word failed");
            st = DWF_ERR_CUDA;
        }
        const size_t nmax = (size_t)std::max(h->nsite[0], h->nsite[1]) * 12 * p->Ls * nrhs_max * 2;
        if (st == DWF_OK) st = dalloc((double**)&h->d_tmp, nmax);
        if (st == DWF_OK) st = dalloc((double**)&h->d_tmp2, nmax);
    }
    if (st == DWF_OK) {   // default tile table, built up front
        const TileSet* ts = nullptr;
        st = get_tiles(h, 32, &ts);
    }
    if (st == DWF_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            set_error("dwf_create: %s", cudaGetErrorString(e));
            st = DWF_ERR_CUDA;
        }
    }
    if (st != DWF_OK) {
        destroy(h);
        return st;
    }
    *out = h;
    return DWF_OK;
}

// D_dirichlet of Sec. 2.3.1 in the whole-lattice layout: a whole-lattice
// handle whose link tables leave out every link U_mu(x) with x and x + mu in
// different domains -- the boxes of `cut` and the rest of the lattice -- the
// Dirichlet wrapper of the gauge field of Sec. 2.4 (the edges of a domain are
// where its mask differs from its shift by one).  Its operators are those of D
// on the cut gauge field, i.e. D_Omega (+) D_Omega-bar on the common site order.
dwf_status create_cut(dwf_handle** out, const dwf_params* p, const dwf_box* cut, int ncut, int nrhs_max) {
    if (out == nullptr || p == nullptr || cut == nullptr || ncut < 1) {
        set_error("dwf_create_cut: null argument or no box");
        return DWF_ERR_ARG;
    }
    *out = nullptr;
    dwf_handle* h = nullptr;
    DWF_TRY(create(&h, p, nullptr, 0, nrhs_max));   // validates the lattice
    const int* L = h->p.dims;
    auto fail = [&](dwf_status st) {
        destroy(h);
        return st;
    };
    for (int i = 0; i < ncut; ++i)
        for (int mu = 0; mu < 4; ++mu)
            if (cut[i].extent[mu] < 1 || cut[i].extent[mu] > L[mu]) {
                set_error("dwf_create_cut: box %d extent[%d] = %d outside [1, %d]", i, mu, cut[i].extent[mu], L[mu]);
                return fail(DWF_ERR_ARG);
            }
    // domain of every site: the box holding it, -1 for the rest; boxes must not overlap
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    std::vector<int> dom(V, -1);
    for (int64_t g = 0; g < V; ++g) {
        const int x[4] = {(int)(g % L[0]), (int)((g / L[0]) % L[1]), (int)((g / ((int64_t)L[0] * L[1])) % L[2]),
                          (int)(g / ((int64_t)L[0] * L[1] * L[2]))};
        for (int i = 0; i < ncut; ++i) {
            bool in = true;
            for (int mu = 0; mu < 4 && in; ++mu) {
                const int o = ((cut[i].origin[mu] % L[mu]) + L[mu]) % L[mu];
                in = ((x[mu] - o + L[mu]) % L[mu]) < cut[i].extent[mu];
            }
            if (!in) continue;
            if (dom[g] >= 0) {
                set_error("dwf_create_cut: boxes %d and %d overlap", dom[g], i);
                return fail(DWF_ERR_ARG);
            }
            dom[g] = i;
        }
    }
    for (int q = 0; q < 2; ++q) {
        const int64_t n = h->nsite[q] * 8;
        std::vector<int64_t> lsrc(n);
        if (cudaMemcpy(lsrc.data(), h->d_link_src[q], n * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("dwf_create_cut: reading the link table failed");
            return fail(DWF_ERR_CUDA);
        }
        for (int64_t e = 0; e < n; ++e) {
            if (lsrc[e] < 0) continue;
            const int64_t g = lsrc[e] / 4;   // the link U_mu(g) joins g and g + mu
            const int mu = (int)(lsrc[e] % 4);
            int x[4] = {(int)(g % L[0]), (int)((g / L[0]) % L[1]), (int)((g / ((int64_t)L[0] * L[1])) % L[2]),
                        (int)(g / ((int64_t)L[0] * L[1] * L[2]))};
            x[mu] = (x[mu] + 1) % L[mu];
            const int64_t gn = x[0] + (int64_t)L[0] * (x[1] + (int64_t)L[1] * (x[2] + (int64_t)L[2] * x[3]));
            if (dom[g] != dom[gn]) lsrc[e] = -1;
        }
#ifdef DWF_DEBUG
        for (int64_t e = 0; e < n; ++e)
            if (lsrc[e] < -1 || lsrc[e] >= 4 * V) {
                set_error("dwf_create_cut (debug): link table entry %lld out of range", (long long)e);
                return fail(DWF_ERR_ARG);
            }
#endif
        const dwf_status st = h2d(h->d_link_src[q], lsrc.data(), n * sizeof(int64_t));
        if (st != DWF_OK) return fail(st);
    }
    h->cut.assign(cut, cut + ncut);
    *out = h;
    return DWF_OK;
}

dwf_status destroy(dwf_handle* h) {
    if (h == nullptr) return DWF_OK;
    for (int q = 0; q < 2; ++q) {
        cudaFree(h->d_nbr[q]);
        cudaFree(h->d_link_src[q]);
        cudaFree(h->d_site_box[q]);
        cudaFree(h->d_site_local[q]);
        for (int pr = 0; pr < 3; ++pr) cudaFree(h->d_links[pr][q]);
    }
    cudaFree(h->d_box_canon_vol);
    cudaFree(h->d_err);
    cudaFree(h->d_tmp);
    cudaFree(h->d_tmp2);
    cudaFree(h->d_mats);
    for (auto& kv : h->tiles)
        for (int q = 0; q < 2; ++q) {
            cudaFree(kv.second.d_tiles[q]);
            cudaFree(kv.second.d_box_tile_begin[q]);
        }
    free_solver_ws(h);
    free_nn_ws(h);
    free_gcr_ws(h);
    free_boundary_cache(h);
    delete h;
    return DWF_OK;
}

}  // namespace dwf
