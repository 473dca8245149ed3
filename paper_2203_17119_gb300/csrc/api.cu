// extern "C" entry points of include/dwf.h: argument checks, then the
// operator compositions of ops.cu, the layout kernels of domain.cu and the
// solver of solver.cu.
#include <cstdio>

#include "dev_common.cuh"
#include <map>
#include <string>
#include <vector>

#include "dwf_internal.cuh"

namespace dwf {
const char* last_error();
std::string tuning_key(const dwf_handle* h, int nrhs, int prec);
}

using namespace dwf;

static bool bad_prec(dwf_prec p) { return p != DWF_FP64 && p != DWF_FP32 && p != DWF_BF16; }

static dwf_status check_op(dwf_handle* h, const void* out, const void* in, dwf_prec prec, int nrhs,
                           const char* who) {
    DWF_TRY(check_handle(h));
    if (out == nullptr || in == nullptr) {
        set_error("%s: null field pointer", who);
        return DWF_ERR_ARG;
    }
    if (out == in) {
        set_error("%s: out and in must not alias", who);
        return DWF_ERR_ARG;
    }
    if (bad_prec(prec)) {
        set_error("%s: bad precision %d", who, (int)prec);
        return DWF_ERR_ARG;
    }
    if (nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("%s: nrhs = %d outside [1, %d]", who, nrhs, h->nrhs_max);
        return DWF_ERR_ARG;
    }
    if (!h->have_gauge) {
        set_error("%s: no gauge field loaded (dwf_set_gauge)", who);
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

extern "C" {

const char* dwf_last_error(void) { return dwf::last_error(); }

dwf_status dwf_create(dwf_handle** h, const dwf_params* p, const dwf_box* boxes, int nbox,
                      int nrhs_max) {
    return dwf::create(h, p, boxes, nbox, nrhs_max);
}

dwf_status dwf_create_cut(dwf_handle** h, const dwf_params* p, const dwf_box* cut, int ncut, int nrhs_max) {
    return dwf::create_cut(h, p, cut, ncut, nrhs_max);
}

dwf_status dwf_destroy(dwf_handle* h) { return dwf::destroy(h); }

dwf_status dwf_domain_sites(const dwf_handle* h, int parity, int64_t* nsites) {
    DWF_TRY(check_handle(h));
    if (nsites == nullptr || (parity != 0 && parity != 1)) {
        set_error("dwf_domain_sites: bad argument");
        return DWF_ERR_ARG;
    }
    *nsites = h->nsite[parity];
    return DWF_OK;
}

dwf_status dwf_box_sites(const dwf_handle* h, int box, int parity, int64_t* offset, int64_t* count) {
    DWF_TRY(check_handle(h));
    if (box < 0 || box >= h->nbox || (parity != 0 && parity != 1) || !offset || !count) {
        set_error("dwf_box_sites: bad argument");
        return DWF_ERR_ARG;
    }
    *offset = h->box_off[parity][box];
    *count = h->box_cnt[parity][box];
    return DWF_OK;
}

dwf_status dwf_set_gauge(dwf_handle* h, const double* U, void* stream) {
    DWF_RANGE("dwf_set_gauge");
    DWF_TRY(check_handle(h));
    if (U == nullptr) {
        set_error("dwf_set_gauge: null gauge pointer");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_set_gauge", {U, link_field_bytes(h), "U"});
    return dwf::set_gauge(h, U, (cudaStream_t)stream);
}

dwf_status dwf_pack(dwf_handle* h, void* dst, const double* src, int nrhs, dwf_prec prec, void* stream) {
    DWF_RANGE("dwf_pack");
    DWF_TRY(check_handle(h));
    if (!dst || !src || bad_prec(prec) || nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("dwf_pack: bad argument");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_pack", {dst, field_bytes(h, 2, prec, nrhs), "dst"},
                     {src, field_bytes(h, 2, DWF_FP64, nrhs), "src"});
    return dwf::pack(h, dst, src, nrhs, prec, (cudaStream_t)stream);
}

dwf_status dwf_unpack(dwf_handle* h, double* dst, const void* src, int nrhs, dwf_prec prec, void* stream) {
    DWF_RANGE("dwf_unpack");
    DWF_TRY(check_handle(h));
    if (!dst || !src || bad_prec(prec) || nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("dwf_unpack: bad argument");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_unpack", {dst, field_bytes(h, 2, DWF_FP64, nrhs), "dst"},
                     {src, field_bytes(h, 2, prec, nrhs), "src"});
    return dwf::unpack(h, dst, src, nrhs, prec, (cudaStream_t)stream);
}

dwf_status dwf_dslash_eo(dwf_handle* h, void* out, const void* in, int out_parity, int dagger,
                         dwf_prec prec, int nrhs, void* stream) {
    DWF_RANGE("dwf_dslash_eo");
    DWF_TRY(check_op(h, out, in, prec, nrhs, "dwf_dslash_eo"));
    if (out_parity != 0 && out_parity != 1) {
        set_error("dwf_dslash_eo: out_parity must be 0 or 1");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_dslash_eo", {out, field_bytes(h, out_parity, prec, nrhs), "out"},
                     {in, field_bytes(h, 1 - out_parity, prec, nrhs), "in"});
    return op_dslash_eo(h, out, in, out_parity, dagger ? 1 : 0, prec, nrhs, h->d_tmp,
                        (cudaStream_t)stream);
}

dwf_status dwf_hop(dwf_handle* h, void* out, const void* in, int out_parity, int dagger, dwf_prec prec,
                   int nrhs, void* stream) {
    DWF_RANGE("dwf_hop");
    DWF_TRY(check_op(h, out, in, prec, nrhs, "dwf_hop"));
    if (out_parity != 0 && out_parity != 1) {
        set_error("dwf_hop: out_parity must be 0 or 1");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_hop", {out, field_bytes(h, out_parity, prec, nrhs), "out"},
                     {in, field_bytes(h, 1 - out_parity, prec, nrhs), "in"});
    return op_hop(h, out, in, out_parity, dagger ? 1 : 0, prec, prec, prec, nrhs, 1.0, nullptr, nullptr,
                  (cudaStream_t)stream);
}

dwf_status dwf_autotune(dwf_handle* h, int nrhs, dwf_prec prec, int* tile_sites) {
    DWF_RANGE("dwf_autotune");
    DWF_TRY(check_handle(h));
    if (bad_prec(prec) || nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("dwf_autotune: bad precision or nrhs");
        return DWF_ERR_ARG;
    }
    if (!h->have_gauge) {
        set_error("dwf_autotune: no gauge field loaded");
        return DWF_ERR_ARG;
    }
    return autotune(h, nrhs, prec, tile_sites);
}

dwf_status dwf_set_tile(dwf_handle* h, int nrhs, int tile_sites, int lanes_per_thread) {
    DWF_TRY(check_handle(h));
    if (nrhs < 1 || nrhs > h->nrhs_max || tile_sites < kMinTile || tile_sites > 256 ||
        (lanes_per_thread != 1 && lanes_per_thread != 2)) {
        set_error("dwf_set_tile: nrhs in [1, nrhs_max], tile_sites in [%d, 256], lanes 1 or 2",
                  kMinTile);
        return DWF_ERR_ARG;
    }
    const size_t smem = hop_smem(tile_sites, 8, 8, nrhs);
    if (smem > (size_t)kHopMaxSmem) {
        set_error("dwf_set_tile: %d sites per tile exceed the FP64 hop's shared memory", tile_sites);
        return DWF_ERR_ARG;
    }
    const TileSet* ts = nullptr;
    DWF_TRY(get_tiles(h, tile_sites, &ts));
    h->tuned_T[nrhs] = tile_sites;
    h->tuned_vl[nrhs] = lanes_per_thread;
    return DWF_OK;
}

dwf_status dwf_autotune_save(const dwf_handle* h, const char* path) {
    DWF_TRY(check_handle(h));
    if (path == nullptr) {
        set_error("dwf_autotune_save: null path");
        return DWF_ERR_ARG;
    }
    // existing lines with other keys are kept; this handle's tunings replace theirs
    std::map<std::string, std::string> lines;
    std::vector<std::string> order;
    if (FILE* f = fopen(path, "r")) {
        char buf[1024];
        while (fgets(buf, sizeof(buf), f)) {
            std::string l(buf);
            while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
            const size_t sp = l.find(' ');
            if (l.empty() || sp == std::string::npos) continue;
            const std::string k = l.substr(0, sp);
            if (!lines.count(k)) order.push_back(k);
            lines[k] = l;
        }
        fclose(f);
    }
    for (const auto& kv : h->tuned_prec) {
        const int nrhs = kv.first;
        const std::string k = tuning_key(h, nrhs, kv.second);
        auto get = [&](const std::map<int, int>& m, int dflt) {
            auto it = m.find(nrhs);
            return it == m.end() ? dflt : it->second;
        };
        char buf[160];
        snprintf(buf, sizeof(buf), " %d %d %d %d %d %d %d %d", get(h->tuned_T, 32), get(h->tuned_vl, 2),
                 get(h->tuned_tc, 0), get(h->tuned_chunk, 1), get(h->tuned_fuse, 0), h->tile_order, h->order_bz,
                 h->order_bt);
        if (!lines.count(k)) order.push_back(k);
        lines[k] = k + buf;
    }
    FILE* f = fopen(path, "w");
    if (!f) {
        set_error("dwf_autotune_save: cannot open %s for writing", path);
        return DWF_ERR_ARG;
    }
    bool ok = true;
    for (const std::string& k : order) ok = ok && fprintf(f, "%s\n", lines[k].c_str()) > 0;
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("dwf_autotune_save: write to %s failed", path);
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

dwf_status dwf_autotune_load(dwf_handle* h, const char* path, int nrhs, dwf_prec prec, int* found) {
    DWF_TRY(check_handle(h));
    if (path == nullptr || found == nullptr || bad_prec(prec) || nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("dwf_autotune_load: bad argument");
        return DWF_ERR_ARG;
    }
    *found = 0;
    FILE* f = fopen(path, "r");
    if (!f) return DWF_OK;   // no file yet: nothing cached
    const std::string key = tuning_key(h, nrhs, (int)prec);
    char buf[1024];
    int T = 0, vl = 0, tc = 0, ck = 0, fu = 0, od = 0, bz = 8, bt = 8;
    while (fgets(buf, sizeof(buf), f)) {
        std::string l(buf);
        const size_t sp = l.find(' ');
        if (sp == std::string::npos || l.compare(0, sp, key) != 0 || sp != key.size()) continue;
        // tile, lanes, tensor cores, chunk, fusion [, tile order, bz, bt]
        int o = 0, z = 8, t = 8;
        const int n = sscanf(l.c_str() + sp, "%d %d %d %d %d %d %d %d", &T, &vl, &tc, &ck, &fu, &o, &z, &t);
        if (n == 5 || n == 8) {
            *found = 1;
            od = n == 8 ? o : 0;
            bz = n == 8 ? z : 8;
            bt = n == 8 ? t : 8;
        }
    }
    fclose(f);
    if (!*found) return DWF_OK;
    if (T < kMinTile || T > 256 || (vl != 1 && vl != 2) || (tc != 0 && tc != 1) || ck < 1 || ck > 64 ||
        (fu != 0 && fu != 1) || (od != 0 && od != 1) || bz < 1 || bt < 1 ||
        hop_smem(T, 8, 8, nrhs) > (size_t)kHopMaxSmem) {
        *found = 0;
        set_error("dwf_autotune_load: entry for this handle in %s is out of range", path);
        return DWF_ERR_ARG;
    }
    const TileSet* ts = nullptr;
    DWF_TRY(get_tiles(h, T, &ts));
    h->tuned_T[nrhs] = T;
    h->tuned_vl[nrhs] = vl;
    h->tuned_tc[nrhs] = tc;
    h->tuned_chunk[nrhs] = ck;
    h->tuned_fuse[nrhs] = fu;
    h->tuned_prec[nrhs] = (int)prec;
    if (od != h->tile_order || bz != h->order_bz || bt != h->order_bt) DWF_TRY(set_tile_order(h, od, bz, bt));
    return DWF_OK;
}

dwf_status dwf_set_hop_kernel(dwf_handle* h, int nrhs, int kernel) {
    DWF_TRY(check_handle(h));
    if (nrhs < 1 || nrhs > h->nrhs_max || (kernel != 0 && kernel != 1)) {
        set_error("dwf_set_hop_kernel: nrhs in [1, nrhs_max], kernel 0 (SIMT) or 1 (tensor cores)");
        return DWF_ERR_ARG;
    }
    h->tuned_tc[nrhs] = kernel;
    return DWF_OK;
}

dwf_status dwf_set_fusion(dwf_handle* h, int nrhs, int fuse) {
    DWF_TRY(check_handle(h));
    if (nrhs < 1 || nrhs > h->nrhs_max || (fuse != 0 && fuse != 1)) {
        set_error("dwf_set_fusion: nrhs in [1, nrhs_max], fuse 0 or 1");
        return DWF_ERR_ARG;
    }
    h->tuned_fuse[nrhs] = fuse;
    return DWF_OK;
}

dwf_status dwf_get_fusion(const dwf_handle* h, int nrhs, int* fuse) {
    DWF_TRY(check_handle(h));
    if (nrhs < 1 || nrhs > h->nrhs_max || fuse == nullptr) {
        set_error("dwf_get_fusion: bad argument");
        return DWF_ERR_ARG;
    }
    auto it = h->tuned_fuse.find(nrhs);
    *fuse = it == h->tuned_fuse.end() ? 0 : it->second;
    return DWF_OK;
}

dwf_status dwf_set_tile_order(dwf_handle* h, int order, int bz, int bt) {
    DWF_TRY(check_handle(h));
    return set_tile_order(h, order, bz, bt);
}

dwf_status dwf_get_tile_order(const dwf_handle* h, int* order, int* bz, int* bt) {
    DWF_TRY(check_handle(h));
    if (order) *order = h->tile_order;
    if (bz) *bz = h->order_bz;
    if (bt) *bt = h->order_bt;
    return DWF_OK;
}

dwf_status dwf_set_hop_chunk(dwf_handle* h, int nrhs, int chunk) {
    DWF_TRY(check_handle(h));
    if (nrhs < 1 || nrhs > h->nrhs_max || chunk < 1 || chunk > 64) {
        set_error("dwf_set_hop_chunk: nrhs in [1, nrhs_max], chunk in [1, 64]");
        return DWF_ERR_ARG;
    }
    h->tuned_chunk[nrhs] = chunk;
    return DWF_OK;
}

dwf_status dwf_get_tuning(const dwf_handle* h, int nrhs, int* tile_sites, int* lanes_per_thread,
                          int* chunk, int* tensor_cores) {
    DWF_TRY(check_handle(h));
    if (nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("dwf_get_tuning: nrhs in [1, nrhs_max]");
        return DWF_ERR_ARG;
    }
    auto get = [&](const std::map<int, int>& m, int dflt) {
        auto it = m.find(nrhs);
        return it == m.end() ? dflt : it->second;
    };
    if (tile_sites) *tile_sites = get(h->tuned_T, 32);
    if (lanes_per_thread) *lanes_per_thread = get(h->tuned_vl, 2);
    if (chunk) *chunk = get(h->tuned_chunk, 1);
    if (tensor_cores) *tensor_cores = get(h->tuned_tc, 0);
    return DWF_OK;
}

dwf_status dwf_launch_count(uint64_t* n) {
    if (n == nullptr) {
        set_error("dwf_launch_count: null pointer");
        return DWF_ERR_ARG;
    }
    *n = launch_count();
    return DWF_OK;
}

dwf_status dwf_alloc_count(uint64_t* n) {
    if (n == nullptr) {
        set_error("dwf_alloc_count: null pointer");
        return DWF_ERR_ARG;
    }
    *n = alloc_count();
    return DWF_OK;
}

dwf_status dwf_mooee(dwf_handle* h, void* out, const void* in, int parity, int dagger, dwf_prec prec,
                     int nrhs, void* stream) {
    DWF_RANGE("dwf_mooee");
    DWF_TRY(check_op(h, out, in, prec, nrhs, "dwf_mooee"));
    if (parity != 0 && parity != 1) {
        set_error("dwf_mooee: parity must be 0 or 1");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_mooee", {out, field_bytes(h, parity, prec, nrhs), "out"},
                     {in, field_bytes(h, parity, prec, nrhs), "in"});
    return op_local(h, L_MOOEE, out, in, nullptr, parity, dagger ? 1 : 0, prec, prec, prec, nrhs, 1.0,
                    nullptr, (cudaStream_t)stream);
}

dwf_status dwf_mooee_inv(dwf_handle* h, void* out, const void* in, int parity, int dagger,
                         dwf_prec prec, int nrhs, void* stream) {
    DWF_RANGE("dwf_mooee_inv");
    DWF_TRY(check_op(h, out, in, prec, nrhs, "dwf_mooee_inv"));
    if (parity != 0 && parity != 1) {
        set_error("dwf_mooee_inv: parity must be 0 or 1");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_mooee_inv", {out, field_bytes(h, parity, prec, nrhs), "out"},
                     {in, field_bytes(h, parity, prec, nrhs), "in"});
    return op_local(h, L_MINV, out, in, nullptr, parity, dagger ? 1 : 0, prec, prec, prec, nrhs, 1.0,
                    nullptr, (cudaStream_t)stream);
}

dwf_status dwf_mpc(dwf_handle* h, void* out, const void* in, int dagger, dwf_prec prec, int nrhs,
                   void* stream) {
    DWF_RANGE("dwf_mpc");
    DWF_TRY(check_op(h, out, in, prec, nrhs, "dwf_mpc"));
    DWF_CHECK_RANGES("dwf_mpc", {out, field_bytes(h, 1, prec, nrhs), "out"},
                     {in, field_bytes(h, 1, prec, nrhs), "in"});
    return op_mpc(h, out, in, dagger ? 1 : 0, prec, prec, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr,
                  (cudaStream_t)stream);
}

dwf_status dwf_apply_d(dwf_handle* h, void* out, const void* in, int dagger, dwf_prec prec, int nrhs,
                       void* stream) {
    DWF_RANGE("dwf_apply_d");
    DWF_TRY(check_op(h, out, in, prec, nrhs, "dwf_apply_d"));
    DWF_CHECK_RANGES("dwf_apply_d", {out, field_bytes(h, 2, prec, nrhs), "out"},
                     {in, field_bytes(h, 2, prec, nrhs), "in"});
    return op_apply_d(h, out, in, dagger ? 1 : 0, prec, nrhs, h->d_tmp, (cudaStream_t)stream);
}

dwf_status dwf_dirichlet_block(dwf_handle* h, void* out, const void* in, int dagger, dwf_prec prec,
                               int nrhs, void* stream) {
    DWF_RANGE("dwf_dirichlet_block");
    DWF_TRY(check_handle(h));
    if (!h->dirichlet) {
        set_error("dwf_dirichlet_block: handle was created for the whole lattice (no boxes)");
        return DWF_ERR_ARG;
    }
    DWF_TRY(check_op(h, out, in, prec, nrhs, "dwf_dirichlet_block"));
    DWF_CHECK_RANGES("dwf_dirichlet_block", {out, field_bytes(h, 2, prec, nrhs), "out"},
                     {in, field_bytes(h, 2, prec, nrhs), "in"});
    return op_apply_d(h, out, in, dagger ? 1 : 0, prec, nrhs, h->d_tmp, (cudaStream_t)stream);
}

dwf_status dwf_cgne_solve(dwf_handle* h, double* x, const double* b, int nrhs,
                          const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_cgne_solve");
    DWF_TRY(check_handle(h));
    if (sp != nullptr && bad_prec(sp->inner_prec)) {
        set_error("dwf_cgne_solve: bad inner precision");
        return DWF_ERR_ARG;
    }
    if (x != nullptr && x == b) {
        set_error("dwf_cgne_solve: x and b must not alias");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_cgne_solve", {x, field_bytes(h, 2, DWF_FP64, nrhs), "x"},
                     {b, field_bytes(h, 2, DWF_FP64, nrhs), "b"});
    return cgne_solve(h, x, b, nrhs, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_gcr_solve(dwf_handle* h, double* x, const double* b, int nrhs, dwf_nn* K,
                         const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_gcr_solve");
    DWF_TRY(check_handle(h));
    if (x != nullptr && x == b) {
        set_error("dwf_gcr_solve: x and b must not alias");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_gcr_solve", {x, field_bytes(h, 2, DWF_FP64, nrhs), "x"},
                     {b, field_bytes(h, 2, DWF_FP64, nrhs), "b"});
    return gcr_solve(h, x, b, nrhs, K, nullptr, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_mg_handle(const dwf_mg* mg, dwf_handle** h);

dwf_status dwf_gcr_solve_mg(dwf_handle* h, double* x, const double* b, dwf_mg* mg,
                            const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_gcr_solve_mg");
    DWF_TRY(check_handle(h));
    dwf_handle* hm = nullptr;
    if (mg == nullptr || dwf_mg_handle(mg, &hm) != DWF_OK || hm != h) {
        set_error("dwf_gcr_solve_mg: the multigrid preconditioner must be set up on this handle");
        return DWF_ERR_ARG;
    }
    if (x != nullptr && x == b) {
        set_error("dwf_gcr_solve_mg: x and b must not alias");
        return DWF_ERR_ARG;
    }
    DWF_CHECK_RANGES("dwf_gcr_solve_mg", {x, field_bytes(h, 2, DWF_FP64, 1), "x"},
                     {b, field_bytes(h, 2, DWF_FP64, 1), "b"});
    return gcr_solve(h, x, b, 1, nullptr, mg, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_multishift_solve(dwf_handle* h, double* x, const double* b, const double* shifts,
                                int nshift, int nrhs, const dwf_solver_params* sp,
                                dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_multishift_solve");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_multishift_solve",
                     {x, nshift > 0 ? (size_t)nshift * field_bytes(h, 1, DWF_FP64, nrhs) : 0, "x"},
                     {b, field_bytes(h, 1, DWF_FP64, nrhs), "b"});
    return multishift_solve(h, x, b, shifts, nshift, nrhs, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_boundary_project(dwf_handle* h, const dwf_box* omega, double* out, const double* in,
                                int nrhs, void* stream) {
    DWF_RANGE("dwf_boundary_project");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_boundary_project", {out, field_bytes(h, 2, DWF_FP64, nrhs), "out"},
                     {in, field_bytes(h, 2, DWF_FP64, nrhs), "in"});
    return boundary_project(h, omega, out, in, nrhs, (cudaStream_t)stream);
}

dwf_status dwf_boundary_rinv(dwf_handle* h, const dwf_box* omega, double* out, const double* in,
                             int nrhs, const dwf_solver_params* sp, dwf_solver_stats* stats,
                             void* stream) {
    DWF_RANGE("dwf_boundary_rinv");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_boundary_rinv", {out, field_bytes(h, 2, DWF_FP64, nrhs), "out"},
                     {in, field_bytes(h, 2, DWF_FP64, nrhs), "in"});
    return boundary_rinv(h, omega, out, in, nrhs, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_boundary_r(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                          const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_boundary_r");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_boundary_r", {out, field_bytes(h, 2, DWF_FP64, nrhs), "out"},
                     {in, field_bytes(h, 2, DWF_FP64, nrhs), "in"});
    return boundary_r(h, omega, out, in, nrhs, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_boundary_ratio_force(dwf_handle* h_light, dwf_handle* h_pv, const dwf_box* omega, double* out,
                                    const double* phi, int nrhs, const dwf_box* active, int accumulate,
                                    const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_boundary_ratio_force");
    DWF_TRY(check_handle(h_light));
    DWF_TRY(check_handle(h_pv));
    DWF_CHECK_RANGES("dwf_boundary_ratio_force", {out, link_field_bytes(h_light), "out"},
                     {phi, field_bytes(h_light, 2, DWF_FP64, nrhs), "phi"});
    return boundary_ratio_force(h_light, h_pv, omega, out, phi, nrhs, active, accumulate, sp, stats,
                                (cudaStream_t)stream);
}

dwf_status dwf_boundary_force(dwf_handle* h, const dwf_box* omega, double* out, const double* phi, int nrhs,
                              const dwf_box* active, int accumulate, const dwf_solver_params* sp,
                              dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_boundary_force");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_boundary_force", {out, link_field_bytes(h), "out"},
                     {phi, field_bytes(h, 2, DWF_FP64, nrhs), "phi"});
    return boundary_force(h, omega, out, phi, nrhs, active, accumulate, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_zolotarev_inv_sqrt(int n, double lo, double hi, double* shifts, double* residues, double* delta) {
    return zolotarev_inv_sqrt(n, lo, hi, shifts, residues, delta);
}

dwf_status dwf_rational_power(double alpha, int n, double lo, double hi, double* a0, double* shifts,
                              double* residues, double* delta) {
    return rational_power(alpha, n, lo, hi, a0, shifts, residues, delta);
}

dwf_status dwf_one_flavour_action(dwf_handle* h, dwf_handle* hd, const double* phi, int nrhs,
                                  const dwf_rational* r1, const dwf_rational* r2, const dwf_solver_params* sp,
                                  double* S, dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_one_flavour_action");
    DWF_TRY(check_handle(h));
    DWF_TRY(check_handle(hd));
    DWF_CHECK_RANGES("dwf_one_flavour_action", {phi, field_bytes(h, 1, DWF_FP64, nrhs), "phi"});
    return one_flavour_action(h, hd, phi, nrhs, r1, r2, sp, S, stats, (cudaStream_t)stream);
}

dwf_status dwf_one_flavour_force(dwf_handle* h, dwf_handle* hd, double* out, const double* phi, int nrhs,
                                 const dwf_rational* r1, const dwf_rational* r2, const dwf_box* active,
                                 int accumulate, const dwf_solver_params* sp, dwf_solver_stats* stats,
                                 void* stream) {
    DWF_RANGE("dwf_one_flavour_force");
    DWF_TRY(check_handle(h));
    DWF_TRY(check_handle(hd));
    DWF_CHECK_RANGES("dwf_one_flavour_force", {out, link_field_bytes(h), "out"},
                     {phi, field_bytes(h, 1, DWF_FP64, nrhs), "phi"});
    return one_flavour_force(h, hd, out, phi, nrhs, r1, r2, active, accumulate, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_one_flavour_heatbath(dwf_handle* h, dwf_handle* hd, double* phi, const double* eta, int nrhs,
                                    const dwf_rational* q1, const dwf_rational* q2, const dwf_solver_params* sp,
                                    dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_one_flavour_heatbath");
    DWF_TRY(check_handle(h));
    DWF_TRY(check_handle(hd));
    DWF_CHECK_RANGES("dwf_one_flavour_heatbath", {phi, field_bytes(h, 1, DWF_FP64, nrhs), "phi"},
                     {eta, field_bytes(h, 1, DWF_FP64, nrhs), "eta"});
    return one_flavour_heatbath(h, hd, phi, eta, nrhs, q1, q2, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_rational_apply(dwf_handle* h, double* out, const double* in, double a0, const double* shifts,
                              const double* residues, int n, int nrhs, const dwf_solver_params* sp,
                              dwf_solver_stats* stats, void* stream) {
    DWF_RANGE("dwf_rational_apply");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_rational_apply", {out, field_bytes(h, 1, DWF_FP64, nrhs), "out"},
                     {in, field_bytes(h, 1, DWF_FP64, nrhs), "in"});
    return rational_apply(h, out, in, a0, shifts, residues, n, nrhs, sp, stats, (cudaStream_t)stream);
}

dwf_status dwf_chebyshev_filter(dwf_handle* h, void* out, const void* in, int order, double lo, double hi,
                                dwf_prec prec, int nrhs, void* stream) {
    DWF_RANGE("dwf_chebyshev_filter");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_chebyshev_filter", {out, field_bytes(h, 1, prec, nrhs), "out"},
                     {in, field_bytes(h, 1, prec, nrhs), "in"});
    return chebyshev_filter(h, out, in, order, lo, hi, prec, nrhs, (cudaStream_t)stream);
}

dwf_status dwf_force(dwf_handle* h, double* out, const void* X, const void* Y, dwf_prec prec, int nrhs,
                     const dwf_box* active, int accumulate, void* stream) {
    DWF_RANGE("dwf_force");
    DWF_TRY(check_handle(h));
    DWF_CHECK_RANGES("dwf_force", {out, link_field_bytes(h), "out"}, {X, field_bytes(h, 2, prec, nrhs), "X"},
                     {Y, field_bytes(h, 2, prec, nrhs), "Y"});
    return force_bilinear(h, out, X, Y, prec, nrhs, active, accumulate, (cudaStream_t)stream);
}

dwf_status dwf_copy(void* dst, const void* src, size_t bytes, void* stream) {
    DWF_RANGE("dwf_copy");
    return copy_sm(dst, src, bytes, (cudaStream_t)stream);
}

dwf_status dwf_check_device(dwf_handle* h) {
    DWF_TRY(check_handle(h));
    int e = 0;
    DWF_CUDA(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        set_error("device error word 0x%x (a bounded wait ran out)", e);
        return DWF_ERR_DEVICE;
    }
    return DWF_OK;
}

}  // extern "C"
