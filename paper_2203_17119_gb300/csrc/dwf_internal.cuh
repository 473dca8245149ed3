// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <initializer_list>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "dwf.h"
#include "nvtx3/nvToolsExt.h"

namespace dwf {

// An NVTX range around one library call (visible to profilers and tracers;
// header-only NVTX v3: without an attached tool it costs a branch).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define DWF_RANGE(name) ::dwf::NvtxRange dwf_range_(name)

using bf16 = __nv_bfloat16;

constexpr int kMaxLanes = 256;   // Ls * nrhs
constexpr int kMaxLs = 32;
constexpr int kHopMaxSmem = 200 * 1024;   // dynamic shared memory cap of the hop
constexpr int kMinTile = 4;               // smallest tile the autotuner may pick

// Dynamic shared memory of the register hop: double-buffered links and
// neighbour indices of T sites, two mbarriers, two arrival counters and the
// per-warp norm partials.
inline size_t hop_smem(int T, size_t link_word, int nwarps, int nrhs) {
    return 2 * (size_t)T * (144 * link_word + 32) + 24 + (size_t)2 * nwarps * nrhs * 8;
}

// ------------------------------------------------------------ errors
void set_error(const char* fmt, ...);

// device allocations made by the library (cudaMalloc through dev_malloc)
void note_alloc();
uint64_t alloc_count();
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
    note_alloc();
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

// kernel launch accounting (graph captures count into the graph instead)
void note_launch();
void capture_begin();
int capture_end();           // kernels recorded since capture_begin
void note_graph_launch(int kernels);
uint64_t launch_count();
#define DWF_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            ::dwf::set_error("%s failed: %s (%s:%d)", #call,                  \
                             cudaGetErrorString(e_), __FILE__, __LINE__);     \
            return DWF_ERR_CUDA;                                              \
        }                                                                     \
    } while (0)
#define DWF_TRY(expr)                                                         \
    do {                                                                      \
        dwf_status s_ = (expr);                                               \
        if (s_ != DWF_OK) return s_;                                          \
    } while (0)

// ------------------------------------------------------- tile tables
// A tile is a contiguous range of one box's sites of one parity:
// {box, begin, count, 0}.  Every kernel walks a tile table.
struct TileSet {
    int T = 0;
    int ntiles[2] = {0, 0};
    int4* d_tiles[2] = {nullptr, nullptr};
    std::vector<int> box_tile_begin[2];          // nbox + 1 entries
    int* d_box_tile_begin[2] = {nullptr, nullptr};
};

// Scalar coefficients of the 5th-dimension operators, host-computed in FP64.
struct FiveD {
    int Ls;
    double mf, b5, c5, d, e;
    double a;        // -e/d
    double inv_d;    // 1/d
    double inv_den;  // 1/(d (1 + mf a^Ls))
};

// Solver workspace of one precision configuration (allocated on first use).
struct SolverWS {
    bool ready = false;
    int nrhs = 0;
    dwf_prec prec = DWF_FP64;
    size_t field_elems = 0;      // complex elements of one odd cb field
    // FP64 state (always)
    double* x64 = nullptr;       // odd x
    double* bp64 = nullptr;      // b'_o
    double* t64a = nullptr;
    double* t64b = nullptr;
    double* t64c = nullptr;
    double* t64d = nullptr;
    double* full64a = nullptr;   // full-field temporaries (both parities)
    // inner-loop vectors (FP32 for mixed, FP64 for plain)
    void* x_lo = nullptr;
    void* r = nullptr;
    void* p = nullptr;
    void* t = nullptr;
    void* tmp1 = nullptr;        // operator intermediates (op precision)
    void* tmp2 = nullptr;
    void* tmp3 = nullptr;
    // reduction partials and per-system scalars
    double* part = nullptr;      // [4][ntiles * nrhs]
    double* sys = nullptr;       // per-system scalars, see solver.cu
    double* h_sys = nullptr;     // pinned host mirror
    int nsys = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_iters = 0;
    int graph_T = 0;
    double graph_delta = -1.0;   // reliable-update threshold captured in the graph
    int graph_kernels = 0;
    cudaStream_t graph_stream = nullptr;
};

}  // namespace dwf

struct dwf_handle {
    dwf_params p;
    int nbox = 1;                 // whole lattice = one box
    bool dirichlet = false;
    std::vector<dwf_box> boxes;
    // whole-lattice handle of D_dirichlet: the links between different
    // domains (each box, and the rest of the lattice) are left out
    std::vector<dwf_box> cut;
    // host copy of every site's box-local lexicographic index (tile ordering)
    std::vector<int> site_local_host[2];
    // order of the tiles within each box: 0 lexicographic, 1 blocked in
    // (z, t) by order_bz x order_bt planes (dwf_set_tile_order)
    int tile_order = 0, order_bz = 8, order_bt = 8;
    int nrhs_max = 1;
    int device = 0;
    int64_t nsite[2] = {0, 0};
    int64_t vol = 0;              // total sites of the domain
    std::vector<int64_t> box_vol;
    std::vector<int64_t> box_off[2], box_cnt[2];
    // device tables
    int* d_nbr[2] = {nullptr, nullptr};        // [nsite][8]
    int* d_site_box[2] = {nullptr, nullptr};   // [nsite]
    int* d_site_local[2] = {nullptr, nullptr}; // [nsite] box-local lex
    int64_t* d_link_src[2] = {nullptr, nullptr}; // [nsite][8] global link or -1
    int64_t* d_box_canon_vol = nullptr;        // [nbox] box volumes
    void* d_links[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    bool have_gauge = false;
    std::map<int, dwf::TileSet> tiles;
    int* d_err = nullptr;
    void* d_tmp = nullptr;        // one FP64 cb field x nrhs_max (operator calls)
    void* d_tmp2 = nullptr;
    dwf::FiveD f5[2];             // [dagger] (identical scalars, kept per use)
    float* d_mats = nullptr;      // fifth-dimension operator matrices [4][2][Ls][Ls]
    std::map<int, dwf::SolverWS> ws;   // keyed by prec * 64 + nrhs
    // autotuned tile sizes: nrhs -> sites per tile
    std::map<int, int> tuned_T;
    // autotuned lanes per thread of the FP32 hop: nrhs -> VL
    std::map<int, int> tuned_vl;
    // BF16-operator hop kernel: nrhs -> 0 (SIMT) or 1 (tensor cores)
    std::map<int, int> tuned_tc;
    // hop tile order: nrhs -> consecutive tiles per CTA before striding by the grid
    std::map<int, int> tuned_chunk;
    // precision the tuning of nrhs was measured with (dwf_autotune)
    std::map<int, int> tuned_prec;
    // nrhs -> 1: the site-local factors of M_pc / M_pc^+ run in the hop
    // epilogues where the site groups allow it (EPI_BMINV, EPI_POST)
    std::map<int, int> tuned_fuse;
    // boundary operator tables of the last Omega (boundary.cu)
    void* boundary_cache = nullptr;
};

namespace dwf {

// ------------------------------------------------------ host helpers
// Sites per tile of a launch: the call's own value, or 16 when it gives none.
inline int tile_or_default(int T) { return T > 0 ? T : 16; }
// The tile table of T sites per tile, built (and allocated) on first use.
dwf_status get_tiles(dwf_handle* h, int T, const TileSet** out);
dwf_status set_tile_order(dwf_handle* h, int order, int bz, int bt);
// The tile table if it exists already (never allocates), else nullptr.
const TileSet* find_tiles(const dwf_handle* h, int T);
// A handle is used on the device it was created on: DWF_ERR_ARG otherwise.
dwf_status check_handle(const dwf_handle* h);

// Byte sizes of the caller's fields: kind 0/1 a cb field of that parity, 2 a
// full field; 0 for an invalid nrhs or precision.  link_field_bytes: the
// canonical gauge (or force) array of the whole lattice.
size_t field_bytes(const dwf_handle* h, int kind, dwf_prec prec, int nrhs);
size_t link_field_bytes(const dwf_handle* h);
struct FieldRange {
    const void* p;
    size_t bytes;
    const char* what;
};
// DWF_CHECK_RANGES(who, {ptr, bytes, name}, ...): in the DWF_DEBUG build,
// DWF_ERR_ARG unless every buffer lies inside one device allocation (null
// pointers and zero sizes are left to the entry point's own checks); nothing
// in the release build.
#ifdef DWF_DEBUG
dwf_status debug_range(const void* p, size_t bytes, const char* who, const char* what);
dwf_status debug_ranges(const char* who, std::initializer_list<FieldRange> r);
#define DWF_CHECK_RANGES(who, ...) DWF_TRY(::dwf::debug_ranges((who), {__VA_ARGS__}))
#else
#define DWF_CHECK_RANGES(who, ...) do { } while (0)
#endif
size_t prec_size(dwf_prec p);   // bytes per real
// Persistent grid of a kernel: the blocks resident at once on the current
// device (occupancy and SM count cached per device), at most one per tile.
dwf_status persistent_grid(const void* kern, int threads, size_t smem, int ntiles, int* grid);

// ------------------------------------------------------ launchers
// hop kinds
enum HopEpi { EPI_PLAIN = 0, EPI_MOO = 1, EPI_POST = 2, EPI_BMINV = 3 };
// site-local operator kinds
enum LocalOp { L_B = 0, L_MOOEE = 1, L_MINV = 2, L_BMINV = 3, L_POST = 4, L_COPY = 5, L_PB = 6 };

struct HopCall {
    const void* in;          // parity 1-p cb field (prec_in)
    void* out;               // parity p cb field (prec_out)
    const void* xmoo;        // EPI_MOO: parity p field of prec_out (M_oo input)
    int out_parity;
    int dagger;
    dwf_prec prec_link;      // links / arithmetic class
    dwf_prec prec_in, prec_out;
    int nrhs;
    double scale;            // out = [M_oo x +] scale * Dh in
    double* partial;         // EPI_MOO: per tile, per rhs |out|^2 (nullable)
    int T;                   // tile size (0 = tuned/default)
    int VL = 0;              // lanes per thread (FP32 links: 1 or 2; 0 = default)
    int tc = 0;              // BF16 links: 1 = tensor-core kernel (hop_tc.cu)
    int chunk = 0;           // consecutive tiles per CTA before striding (0 = 1)
    // EPI_POST (dagger only): the tail of M_pc^+ fused into the hop,
    //   Ap = M_oo^+ xmoo + scale (b5 + c5 S5^+) Dh^+ in,
    // with the CG update x += alpha p, r -= alpha Ap and per-tile |r|^2
    // (FP32 vectors); Ap itself is not stored.  Needs site groups that do
    // not straddle warps: hop_post_ok().
    bool post = false;
    // EPI_BMINV: out = scale (b5 + c5 S5)(d + e S5)^-1 Dh in (adjoint: with
    // S5^+), the site-local factor between the two hops of M_pc applied in the
    // epilogue by scans across the site's lanes; same condition as EPI_POST
    bool bminv = false;
    void* cg_x = nullptr;
    void* cg_r = nullptr;
    const void* cg_p = nullptr;
    const double* alpha = nullptr;
    const int* run = nullptr;
};
dwf_status launch_hop(dwf_handle* h, const HopCall& c, cudaStream_t s);
// The fused M_pc^+ tail is available: FP32 or BF16 operator, FP32 vectors,
// and N5 / (lanes per thread) dividing 32.
bool hop_post_ok(const dwf_handle* h, dwf_prec op, dwf_prec vec, int nrhs, int VL);
// The fused site-local factor between the hops of M_pc is available: FP32
// arithmetic (FP32 or BF16 operator) and N5 / (lanes per thread) dividing 32.
bool hop_bminv_ok(const dwf_handle* h, dwf_prec op, int nrhs, int VL);
dwf_status launch_hop_tc(dwf_handle* h, const HopCall& c, const TileSet& ts, cudaStream_t s);
dwf_status init_hop_tc_kernels();
dwf_status init_hop_kernels();
dwf_status init_local_kernels();
dwf_status init_local_mat_kernels();
void build_fived_mats(const FiveD& f, std::vector<float>& out);
dwf_status autotune(dwf_handle* h, int nrhs, dwf_prec prec, int* best);
dwf_status boundary_project(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                            cudaStream_t s);
void free_boundary_cache(dwf_handle* h);
dwf_status boundary_ratio_force(dwf_handle* hl, dwf_handle* hp, const dwf_box* omega, double* out, const double* phi,
                                int nrhs, const dwf_box* active, int accumulate, const dwf_solver_params* sp,
                                dwf_solver_stats* stats, cudaStream_t s);
dwf_status boundary_r(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                      const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t s);
dwf_status chebyshev_filter(dwf_handle* h, void* out, const void* in, int order, double lo, double hi,
                            dwf_prec prec, int nrhs, cudaStream_t s);
dwf_status boundary_force(dwf_handle* h, const dwf_box* omega, double* out, const double* phi, int nrhs,
                          const dwf_box* active, int accumulate, const dwf_solver_params* sp,
                          dwf_solver_stats* stats, cudaStream_t s);
dwf_status boundary_rinv(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                         const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t s);
dwf_status force_bilinear(dwf_handle* h, double* out, const void* X, const void* Y, dwf_prec prec, int nrhs,
                          const dwf_box* active, int accumulate, cudaStream_t s);
dwf_status zolotarev_inv_sqrt(int n, double lo, double hi, double* shifts, double* residues, double* delta);
// Jacobi sn, cn (parameter m, complementary m1 = 1 - m passed exactly) and K(m)
// by the arithmetic-geometric mean; any output may be null.
void jacobi_sn_cn(double u, double m, double m1, double* sn, double* cn, double* K);
dwf_status rational_power(double alpha, int n, double lo, double hi, double* a0, double* shifts,
                          double* residues, double* delta);
dwf_status rational_apply(dwf_handle* h, double* out, const double* in, double a0, const double* shifts,
                          const double* residues, int n, int nrhs, const dwf_solver_params* sp,
                          dwf_solver_stats* stats, cudaStream_t s);
dwf_status one_flavour_action(dwf_handle* h, dwf_handle* hd, const double* phi, int nrhs, const dwf_rational* r1,
                              const dwf_rational* r2, const dwf_solver_params* sp, double* S,
                              dwf_solver_stats* stats, cudaStream_t s);
dwf_status one_flavour_force(dwf_handle* h, dwf_handle* hd, double* out, const double* phi, int nrhs,
                             const dwf_rational* r1, const dwf_rational* r2, const dwf_box* active, int accumulate,
                             const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t s);
dwf_status one_flavour_heatbath(dwf_handle* h, dwf_handle* hd, double* phi, const double* eta, int nrhs,
                                const dwf_rational* q1, const dwf_rational* q2, const dwf_solver_params* sp,
                                dwf_solver_stats* stats, cudaStream_t s);
dwf_status multishift_solve(dwf_handle* h, double* x, const double* b, const double* shifts,
                            int nshift, int nrhs, const dwf_solver_params* sp,
                            dwf_solver_stats* stats, cudaStream_t s);

struct LocalCall {
    LocalOp op;
    const void* in;          // field of prec_in
    const void* in2;         // L_POST: second input (prec_in2)
    void* out;               // prec_out
    int parity;
    int dagger;
    dwf_prec prec_in, prec_in2, prec_out;
    int nrhs;
    double scale;
    // fused CG update (L_POST only): x += alpha p, r -= alpha * out; |r|^2
    void* cg_x; void* cg_r; const void* cg_p; dwf_prec prec_vec;
    const double* alpha;     // per-system (device); beta for L_PB
    const int* run;          // per-system run flags (device, nullable)
    double* partial;         // per tile, per rhs |result|^2 (nullable)
    int T;
    const FiveD* f5 = nullptr;   // FP64 only: fifth-dimension coefficients other than the handle's
};
dwf_status launch_local(dwf_handle* h, const LocalCall& c, cudaStream_t s);

// elementwise / reduction kernels (blas.cu)
// copy between device and page-locked host memory with SM loads and stores
dwf_status copy_sm(void* dst, const void* src, size_t bytes, cudaStream_t s);
dwf_status launch_convert(void* dst, dwf_prec pd, const void* src, dwf_prec ps,
                          size_t n_complex, cudaStream_t s);
// partial sums per tile and rhs: q0 = Re<a,b> (a == b: |a|^2)
dwf_status launch_dot_partial(dwf_handle* h, int parity, const void* a, const void* b,
                              dwf_prec pa, dwf_prec pb, int nrhs, double* partial,
                              int T, cudaStream_t s);
// per system (box, rhs): out[sys] = sum over the box's tiles of partial
dwf_status launch_reduce_sys(dwf_handle* h, int parity, const double* partial, int nrhs,
                             double* out, int T, cudaStream_t s);
// y = a*x + b*y per system (scalars from device arrays or immediates)
dwf_status launch_axpby(dwf_handle* h, int parity, int nrhs, const double* a_sys, double a_imm,
                        const void* x, dwf_prec px, const double* b_sys, double b_imm,
                        void* y, dwf_prec py, const int* run, int T, cudaStream_t s);

// ------------------------------------------------------ compositions
struct CgFuse {
    void* x;
    void* r;
    const void* p;
    const double* alpha;
    const int* run;
};
dwf_status op_hop(dwf_handle* h, void* out, const void* in, int out_parity, int dagger,
                  dwf_prec link, dwf_prec pin, dwf_prec pout, int nrhs, double scale,
                  const void* xmoo, double* partial, cudaStream_t s);
dwf_status op_local(dwf_handle* h, LocalOp op, void* out, const void* in, const void* in2,
                    int parity, int dagger, dwf_prec pin, dwf_prec pin2, dwf_prec pout, int nrhs,
                    double scale, double* partial, cudaStream_t s);
dwf_status op_dslash_eo(dwf_handle* h, void* out, const void* in, int p, int dagger,
                        dwf_prec prec, int nrhs, void* tmp, cudaStream_t s);
dwf_status op_mpc(dwf_handle* h, void* out, const void* in, int dagger, dwf_prec pv, dwf_prec po,
                  int nrhs, void* tmpA, void* tmpB, double* partial, const CgFuse* cg,
                  cudaStream_t s);
dwf_status op_apply_d(dwf_handle* h, void* out, const void* in, int dagger, dwf_prec prec,
                      int nrhs, void* tmp, cudaStream_t s);
dwf_status op_mpc_pre(dwf_handle* h, void* out, const void* p, const void* t1, dwf_prec pv,
                      dwf_prec po, int nrhs, void* tmpA, void* tmpB, double* partial,
                      cudaStream_t s);
size_t cb_elems(const dwf_handle* h, int parity, int nrhs);
int tile_for(dwf_handle* h, int nrhs);

// ------------------------------------------------------ domain / solver
dwf_status create(dwf_handle** out, const dwf_params* p, const dwf_box* boxes, int nbox,
                  int nrhs_max);
dwf_status destroy(dwf_handle* h);
dwf_status create_cut(dwf_handle** out, const dwf_params* p, const dwf_box* cut, int ncut, int nrhs_max);
dwf_status set_gauge(dwf_handle* h, const double* U, cudaStream_t s);
dwf_status pack(dwf_handle* h, void* dst, const double* src, int nrhs, dwf_prec prec,
                cudaStream_t s);
dwf_status unpack(dwf_handle* h, double* dst, const void* src, int nrhs, dwf_prec prec,
                  cudaStream_t s);
void free_solver_ws(dwf_handle* h);
void free_nn_ws(dwf_handle* h);
void free_gcr_ws(dwf_handle* h);
dwf_status gcr_solve(dwf_handle* h, double* x, const double* b, int nrhs, dwf_nn* K, dwf_mg* mg,
                     const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t user);
dwf_status cgne_solve(dwf_handle* h, double* x, const double* b, int nrhs,
                      const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t user);

}  // namespace dwf
