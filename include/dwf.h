/*
 * dwf.h -- C ABI of the GB300 (sm_103a) domain wall fermion library.
 *
 * The library applies the 5D domain wall operator D (Shamir and Moebius),
 * its even-odd (red-black) blocks and Schur operator, and the Dirichlet
 * block operator D_Omega, and solves D x = b with them on one GPU.  The paper
 * (Boyle, Bollweg, Kelly, Yamaguchi, "Algorithms for Domain Wall Fermions",
 * LATTICE2021) states the problem: Sec. 1 and Sec. 2.3 put the Krylov solves
 * with D and with the local Dirichlet operator at the centre of HMC; Sec. 2.1
 * defines D_Omega as the block of D that connects Omega with itself, and
 * Sec. 2.4 realises it by zeroing the gauge links that cross the domain
 * boundary.  The paper never writes D itself; the conventions used are:
 *
 *   Dh psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)
 *   D_W       = (4 - M5) - Dh / 2
 *   S5 psi_s  = P_- psi_{s+1} + P_+ psi_{s-1},  psi_{Ls} = -mf psi_0, psi_{-1} = -mf psi_{Ls-1}
 *   D         = D_W (b5 + c5 S5) + (1 - S5)          (Shamir: b5 = 1, c5 = 0)
 *   M_ee = M_oo = d + e S5,  d = b5 (4 - M5) + 1,  e = c5 (4 - M5) - 1
 *   M_eo, M_oe  = -Dh (b5 + c5 S5) / 2 between the 4D checkerboards
 *   M_pc        = M_oo - M_oe M_ee^-1 M_eo           (odd checkerboard)
 *
 * with the chiral gamma basis: g_k = [[0, -i s_k], [i s_k, 0]] (k = 1..3,
 * directions x, y, z), g_4 = [[0, 1], [1, 0]] (t), g_5 = diag(1, 1, -1, -1),
 * P_+ = spins {0, 1}, P_- = spins {2, 3}.  4D parity is (x + y + z + t) mod 2.
 *
 * Entry points, by group: handles and layouts (dwf_create, dwf_create_cut
 * ... dwf_unpack); operators (dwf_dslash_eo, dwf_hop, dwf_mooee,
 * dwf_mooee_inv, dwf_mpc, dwf_apply_d, dwf_dirichlet_block); solvers
 * (dwf_cgne_solve, dwf_multishift_solve, dwf_rational_apply, dwf_gcr_solve
 * with the learned preconditioner dwf_nn_* or the multigrid dwf_mg_*); the
 * DD-HMC boundary operator and forces of Sec. 2.1 and 2.3
 * (dwf_boundary_project, dwf_boundary_r, dwf_boundary_rinv, dwf_force,
 * dwf_boundary_force, dwf_boundary_ratio_force) and the one-flavour
 * DD-RHMC term of Sec. 2.3.1 (dwf_one_flavour_action, _force, _heatbath);
 * rational approximation and multigrid set-up (dwf_zolotarev_inv_sqrt,
 * dwf_rational_power, dwf_chebyshev_filter); kernel tuning (dwf_autotune,
 * dwf_set_tile, ...).
 *
 * ------------------------------------------------------------------------
 * DOMAINS.  A handle is bound to a domain: either the whole periodic
 * lattice (nbox = 0) or a list of boxes, each box an independent Dirichlet
 * block (every link leaving the box is cut, Sec. 2.4).  Boxes may overlap in
 * the lattice: each has its own field storage, so the handle's operator is
 * the direct sum of the boxes' D_Omega.  A box is (origin[4], extent[4]) in
 * (x, y, z, t) order, 1 <= extent[mu] <= L[mu], coordinates taken modulo L
 * (boxes may wrap).  In a direction where extent == L the box is periodic.
 *
 * SITE ORDER.  Sites of box b are enumerated in box-local lexicographic
 * order l = l0 + e0 (l1 + e1 (l2 + e2 l3)), global coordinate
 * x_mu = (origin_mu + l_mu) mod L_mu.  The parity-p site list of a domain is
 * the concatenation over boxes b = 0..nbox-1 of the sites of box b whose
 * global parity is p, in that order.  For the whole lattice (Lx even) the
 * parity-p index of site lex is lex / 2.
 *
 * FIELD LAYOUTS (all device memory, owned by the caller):
 *   checkerboard field of parity p ("cb field"):
 *       [i < nsites(p)][c < 12][r < nrhs][s < Ls][re, im]
 *     c = spin * 3 + colour; element type double (DWF_FP64), float
 *     (DWF_FP32) or bfloat16 (DWF_BF16).  nrhs right-hand sides and the
 *     fifth dimension are the innermost axes ("lanes" l = r * Ls + s).
 *   full field: [cb field of parity 0][cb field of parity 1].
 *   canonical field (dwf_pack / dwf_unpack only, complex128):
 *       [box][r][box-local site l][s][spin][colour][re, im]
 *   canonical gauge field (dwf_set_gauge, complex128, whole lattice):
 *       [site lex][mu][a][b][re, im],  lex = x + Lx (y + Ly (z + Lz t)),
 *       U_mu(x) transports from x + mu to x.
 *
 * STREAMS.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 * default stream.  Operator calls are asynchronous on that stream and
 * allocate nothing.  Solves synchronise the stream and fill their stats.
 *
 * ERRORS.  Every call returns a dwf_status; dwf_last_error() returns a
 * thread-local message for the last failure on the calling thread.  A
 * failed argument check leaves the handle unchanged.  A handle belongs to
 * the device that was current when it was created: calls that take it
 * return DWF_ERR_ARG while another device is current.  Device kernels never
 * trap: a bounded wait that runs out sets a device error word, reported as
 * DWF_ERR_DEVICE by dwf_check_device() and by the solves.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DWF_OK = 0,
    DWF_ERR_ARG = 1,            /* invalid argument (nothing was launched)  */
    DWF_ERR_CUDA = 2,           /* a CUDA runtime call failed               */
    DWF_ERR_NOT_CONVERGED = 3,  /* solve hit maxiter; x = last iterate      */
    DWF_ERR_TIMEOUT = 4,        /* solve hit max_seconds; x = last iterate  */
    DWF_ERR_NAN = 5,            /* NaN/Inf met in a solve                   */
    DWF_ERR_UNSUPPORTED = 6,    /* valid but not implemented combination    */
    DWF_ERR_DEVICE = 7          /* a device-side bounded wait ran out       */
} dwf_status;

typedef enum { DWF_FP64 = 0, DWF_FP32 = 1, DWF_BF16 = 2 } dwf_prec;

/* Lattice and action.  dims = (Lx, Ly, Lz, Lt), Lx even; Shamir: b5 = 1,
 * c5 = 0; Moebius: b5, c5 free (Sec. 2.3 uses both kinds of action). */
typedef struct {
    int dims[4];
    int Ls;
    double M5, mf, b5, c5;
} dwf_params;

typedef struct {
    int origin[4];
    int extent[4];
} dwf_box;

/* A rational function in partial fractions,
 *   r(x) = a0 + sum_{i<n} residues[i] / (x + shifts[i]),
 * host arrays of n values (shifts >= 0), e.g. from dwf_rational_power. */
typedef struct {
    double a0;
    const double* shifts;
    const double* residues;
    int n;
} dwf_rational;

typedef struct dwf_handle dwf_handle;
typedef struct dwf_nn dwf_nn;
typedef struct dwf_mg dwf_mg;

/* ------------------------------------------------------------- set-up */

/* Create a handle for the whole lattice (boxes = NULL, nbox = 0) or for the
 * Dirichlet blocks D_Omega of `nbox` boxes (Sec. 2.1, Sec. 2.4).  Builds the
 * site lists, neighbour tables and tile tables on the host and allocates all
 * device workspace for up to `nrhs_max` right-hand sides, on the current
 * CUDA device.  Errors: DWF_ERR_ARG (Lx odd, Ls < 1, extents out of range,
 * nrhs_max < 1 or Ls * nrhs_max > 256), DWF_ERR_CUDA (allocation). */
dwf_status dwf_create(dwf_handle** h, const dwf_params* p, const dwf_box* boxes,
                      int nbox, int nrhs_max);
dwf_status dwf_destroy(dwf_handle* h);

/* A whole-lattice handle of D_dirichlet (Sec. 2.3.1, eq. ddrhmc: det D /
 * det D_dirichlet with D_dirichlet = D_Omega (+) D_Omega-bar): D with every
 * link U_mu(x) left out whose ends x, x + mu lie in different domains, the
 * domains being the `ncut` boxes and the rest of the lattice (Sec. 2.4's
 * Dirichlet wrapper of the gauge field).  Site order, layouts and every call
 * are those of a whole-lattice handle (dwf_create with boxes = NULL); only the
 * link tables built by dwf_set_gauge differ (the left-out links are zero), so
 * the same field serves D and D_dirichlet.  Errors as dwf_create, and
 * DWF_ERR_ARG if ncut < 1, an extent is out of range or two boxes overlap. */
dwf_status dwf_create_cut(dwf_handle** h, const dwf_params* p, const dwf_box* cut, int ncut,
                          int nrhs_max);

/* Number of sites of the handle's domain with parity `parity`. */
dwf_status dwf_domain_sites(const dwf_handle* h, int parity, int64_t* nsites);
/* Offset and count of box `box`'s parity-`parity` sites in the cb field. */
dwf_status dwf_box_sites(const dwf_handle* h, int box, int parity,
                         int64_t* offset, int64_t* count);

/* Load the gauge field (device pointer, canonical complex128 layout of the
 * whole lattice, read during the call only).  Builds the FP64/FP32/BF16
 * per-parity link tables (forward U_mu(x) and backward U_mu(x-mu)^+ per
 * site, zero for links cut by the domain); ends with a stream sync. */
dwf_status dwf_set_gauge(dwf_handle* h, const double* U, void* stream);

/* canonical complex128 <-> full field of precision `prec` (layout kernels). */
dwf_status dwf_pack(dwf_handle* h, void* dst, const double* src, int nrhs,
                    dwf_prec prec, void* stream);
dwf_status dwf_unpack(dwf_handle* h, double* dst, const void* src, int nrhs,
                      dwf_prec prec, void* stream);

/* ---------------------------------------------------------- operators
 * `in` and `out` are device cb (or full) fields of precision `prec` with
 * `nrhs` <= nrhs_max right-hand sides; they must not alias.  For DWF_BF16
 * the arithmetic is FP32 on BF16 operands (links and spinors).          */

/* out = M_{p,1-p} in  (off-diagonal block of D, the hop with the
 * (b5 + c5 S5) factor folded in), p = out_parity; dagger: out =
 * (M_{1-p,p})^+ in.  `in` has parity 1 - p. */
dwf_status dwf_dslash_eo(dwf_handle* h, void* out, const void* in, int out_parity,
                         int dagger, dwf_prec prec, int nrhs, void* stream);

/* out = Dh_{p,1-p} in: the bare Wilson hop of D_W = (4 - M5) - Dh/2 on every
 * lane (spin projection, SU(3) transport of two colour vectors, rebuild),
 * links of precision `prec`; dagger swaps the projectors (1 -+ g_mu).  This
 * single kernel is the one every operator above is built around. */
dwf_status dwf_hop(dwf_handle* h, void* out, const void* in, int out_parity,
                   int dagger, dwf_prec prec, int nrhs, void* stream);

/* out = M_ee in (= M_oo in; either parity, `parity` selects the site count);
 * dagger: M_ee^+ in. */
dwf_status dwf_mooee(dwf_handle* h, void* out, const void* in, int parity,
                     int dagger, dwf_prec prec, int nrhs, void* stream);

/* out = M_ee^-1 in (closed form per chirality); dagger: (M_ee^+)^-1 in. */
dwf_status dwf_mooee_inv(dwf_handle* h, void* out, const void* in, int parity,
                         int dagger, dwf_prec prec, int nrhs, void* stream);

/* out = M_pc in on the odd checkerboard; dagger: M_pc^+ in. */
dwf_status dwf_mpc(dwf_handle* h, void* out, const void* in, int dagger,
                   dwf_prec prec, int nrhs, void* stream);

/* Same result as dwf_mpc, for callers that may not allocate device memory
 * where they apply the operator (a framework whose pool owns all device
 * memory, a fixed-footprint embedding).
 * The paper has no counterpart: it is a deployment convenience.  The two
 * checkerboard temporaries come from a static device array of 2 x 32 MiB
 * reserved on every GPU that loads the library (held until exit); requests
 * needing more than 32 MiB per temporary fail with DWF_ERR_ARG, as do handles
 * whose tile table for this nrhs was never built.  The call allocates
 * nothing.  All calls on a device share the array (it keeps the last call's
 * contents; nothing in it needs to start at zero), so calls that overlap on
 * the GPU race: serialise them.  The first call on a device looks up the
 * array's address (cudaGetSymbolAddress) with that device current; make it
 * before any stream capture.  DWF_ERR_ARG if the current device is not the
 * one the handle was created on (as for every call taking a handle). */
dwf_status dwf_mpc_noalloc(dwf_handle* h, void* out, const void* in, int dagger,
                           dwf_prec prec, int nrhs, void* stream);

/* out = D in (full fields, both parities) for a whole-lattice handle, or
 * D_Omega in for a box handle; dagger: the adjoint. */
dwf_status dwf_apply_d(dwf_handle* h, void* out, const void* in, int dagger,
                       dwf_prec prec, int nrhs, void* stream);

/* The Dirichlet block operator D_Omega (Sec. 2.1: the part of D connecting
 * Omega with itself; Sec. 2.4: D with the links crossing the domain
 * boundary set to zero) on a box handle.  Same as dwf_apply_d but fails with
 * DWF_ERR_ARG on a whole-lattice handle. */
dwf_status dwf_dirichlet_block(dwf_handle* h, void* out, const void* in, int dagger,
                               dwf_prec prec, int nrhs, void* stream);

/* ------------------------------------------------------------- solves */

typedef struct {
    double tol;          /* target |b - D x| / |b| per system (e.g. 1e-10)      */
    int maxiter;         /* cap on inner iterations                              */
    double delta;        /* reliable-update trigger (mixed precision): an FP64
                            update when |r| drops below delta times its value at
                            the last update; <= 0 selects 0.01 for the FP32
                            operator, 0.1 for BF16 (rounding ~1e-2)            */
    int restart;         /* GCR restart length                                   */
    int use_x0;          /* 1: x holds the initial guess                         */
    dwf_prec inner_prec; /* DWF_FP64: plain FP64 CG; FP32/BF16: mixed precision  */
    double max_seconds;  /* wall-clock cap (0 = none)                            */
    int check_every;     /* iterations per captured CUDA graph (0 = default 8)   */
    double* record_x;    /* CGNE, FP64 inner only: device buffer of record_max
                            odd cb FP64 fields; the iterate x_o is copied into it
                            every record_every iterations (a multiple of
                            check_every), NULL = no recording                   */
    int record_every;
    int record_max;
} dwf_solver_params;

typedef struct {
    int iters;             /* inner iterations                               */
    int reliable_updates;  /* FP64 residual recomputations                   */
    int op_applies;        /* M_pc or M_pc^+ applications (any precision)    */
    int status;            /* dwf_status of this system                      */
    double true_resid;     /* |b - D x| / |b| recomputed in FP64 at the end  */
    double seconds;        /* wall time of the whole solve                   */
    int recorded;          /* iterates written to record_x                   */
} dwf_solver_stats;

/* Solve D x = b (D_Omega x = b on a box handle) for every box and every
 * right-hand side at once by even-odd preconditioned CGNE on
 * M_pc^+ M_pc x_o = M_pc^+ b'_o, b'_o = b_o - M_oe M_ee^-1 b_e, then
 * x_e = M_ee^-1 (b_e - M_eo x_o).  x, b: device full fields, FP64, nrhs
 * right-hand sides.  inner_prec FP64 runs plain FP64 CG; FP32/BF16 runs the
 * inner iteration with that operator and FP32 vectors, with FP64 reliable
 * updates of the residual, FP64 solution accumulation and FP64 global
 * reductions.  stats: array of nbox_or_1 * nrhs entries (box-major).
 * Returns DWF_OK when every system reached tol. */
dwf_status dwf_cgne_solve(dwf_handle* h, double* x, const double* b, int nrhs,
                          const dwf_solver_params* sp, dwf_solver_stats* stats,
                          void* stream);

/* Autotuner: time the hop kernel for nrhs right-hand sides in precision
 * `prec` over candidate tile sizes (sites per CTA tile: 8..128) and keep the
 * fastest for every later call on this handle with that nrhs (all kernels of
 * an operator chain share one tile table).  On a whole-lattice handle it then
 * times the chosen configuration with the lexicographic and the 8 x 8 blocked
 * tile order (dwf_set_tile_order) and keeps the faster for the handle.
 * Synchronous; uses the handle's scratch fields, so it must not overlap other
 * calls on the handle.  tile_sites (nullable) receives the choice. */
dwf_status dwf_autotune(dwf_handle* h, int nrhs, dwf_prec prec, int* tile_sites);

/* Persisted autotuning.  dwf_autotune_save writes every choice dwf_autotune
 * made on this handle to the text file `path`, one line per key
 *   <device name>/<SMs>|<Lx>,<Ly>,<Lz>,<Lt>|<Ls>|<boxes or "whole">|p<prec>|n<nrhs>
 * followed by tile, lanes, tensor-core kernel, chunk, fusion and the handle's tile
 * order (order, bz, bt; lines without them load as lexicographic); lines of other keys
 * already in the file are kept.  dwf_autotune_load looks up this handle's key
 * for (nrhs, prec) and, if present (*found = 1), applies it as dwf_set_tile &
 * co. would (building the tile table); a missing file or key leaves the
 * handle unchanged with *found = 0.  DWF_ERR_ARG on I/O failures or an entry
 * out of range. */
dwf_status dwf_autotune_save(const dwf_handle* h, const char* path);
dwf_status dwf_autotune_load(dwf_handle* h, const char* path, int nrhs, dwf_prec prec, int* found);

/* Manual counterpart of dwf_autotune: sites per tile (kMinTile = 4 .. 256,
 * limited by the FP64 hop's shared memory) and lanes per thread of the FP32
 * hop (1 or 2) for every later call with this nrhs.  Builds the tile table
 * (allocates); DWF_ERR_ARG on values out of range. */
dwf_status dwf_set_tile(dwf_handle* h, int nrhs, int tile_sites, int lanes_per_thread);

/* Kernel of the hop with the BF16 operator (BF16 links; operands BF16 or
 * FP32) for every later call with this nrhs: 0 = FP32 SIMT arithmetic,
 * 1 = tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation):
 * per site and mu the colour contraction U h of the +mu and -mu hops for
 * 8 lanes x 2 spins is one 16 x 16 x 8 MMA, the lower spins a second one.
 * The projected half spinor is rounded to BF16 (relative ~4e-3, within the
 * BF16 operator's tolerance).  Sec. 2.1 (the Dirac operator of the solves).
 * dwf_autotune(prec = DWF_BF16) picks between the two.  DWF_ERR_ARG on
 * values out of range. */
dwf_status dwf_set_hop_kernel(dwf_handle* h, int nrhs, int kernel);

/* Where a site's Ls * nrhs lanes fit the threads of one warp (N5 / lanes per
 * thread dividing 32), the site-local factors of the Schur operator can run
 * in the epilogues of the hops instead of separate passes: the
 * (b5 + c5 S5)(d + e S5)^-1 between the two hops of M_pc and M_pc^+ (its
 * closed form as decayed prefix sums over the fifth dimension, computed with
 * warp shuffles) and, inside CGNE, the tail M_oo^+ t - (1/4)(b5 + c5 S5^+)(.)
 * with the CG update.  fuse = 1 selects that form for every later call with
 * this nrhs, 0 the separate passes (the default); dwf_autotune times both.
 * Same results to rounding.  DWF_ERR_ARG unless fuse is 0 or 1. */
dwf_status dwf_set_fusion(dwf_handle* h, int nrhs, int fuse);
dwf_status dwf_get_fusion(const dwf_handle* h, int nrhs, int* fuse);

/* Tile order of the hop for every later call with this nrhs: each CTA of
 * the persistent grid takes `chunk` consecutive tiles (neighbouring lattice
 * rows, whose y-neighbour spinors it then re-reads from L1) before striding
 * by the grid; 1 = plain striding.  Larger chunks trade L1 reuse against the
 * load balance of the last round.  dwf_autotune picks 1 or 8.  Same results.
 * DWF_ERR_ARG unless 1 <= chunk <= 64. */
dwf_status dwf_set_hop_chunk(dwf_handle* h, int nrhs, int chunk);

/* Order in which every kernel on this handle walks the tiles of a box:
 * order 0 lexicographic in the site order (the default); order 1 blocked in
 * (z, t) -- by t / bt, z / bz, then t mod bt, z mod bz, y, x of a tile's first
 * site -- so that the two uses of a z or t neighbour spinor (as the +mu
 * neighbour of one plane and the -mu neighbour of the plane two steps on)
 * are a block's planes apart rather than a whole time slice, for L2 reuse.
 * Existing tile tables are rewritten in place (same tiles, so captured
 * graphs stay valid); the call waits for the device and must not overlap
 * other calls on the handle.  Same results up to the summation order of
 * per-tile partial norms.  DWF_ERR_ARG unless order is 0 or 1 and bz, bt >= 1. */
dwf_status dwf_set_tile_order(dwf_handle* h, int order, int bz, int bt);
/* The handle's tile order (any output may be NULL). */
dwf_status dwf_get_tile_order(const dwf_handle* h, int* order, int* bz, int* bt);

/* The kernel configuration later calls with this nrhs use (set by
 * dwf_autotune or the dwf_set_* calls; defaults 32 sites, 2 lanes, chunk 1,
 * SIMT): any output pointer may be NULL.  DWF_ERR_ARG on a bad nrhs. */
dwf_status dwf_get_tuning(const dwf_handle* h, int nrhs, int* tile_sites, int* lanes_per_thread,
                          int* chunk, int* tensor_cores);

/* The debug build (libdwf_debug.so, compiled with -DDWF_DEBUG): every entry
 * point checks, on the host and before launching anything, that each caller
 * buffer it reads or writes lies inside one device allocation of the current
 * context (the allocation range the CUDA driver reports for the pointer, so with a
 * caching allocator only overruns past its segment are seen), and the handle's
 * neighbour and link tables are range-checked when built; a failure returns
 * DWF_ERR_ARG naming the buffer.  *on = 1 in the debug build, 0 otherwise. */
dwf_status dwf_debug_build(int* on);
/* Debug build: DWF_OK if [p, p + bytes) lies inside one device allocation,
 * DWF_ERR_ARG otherwise (or for host memory, NULL or bytes = 0).  The release
 * build returns DWF_ERR_UNSUPPORTED. */
dwf_status dwf_check_range(const void* p, size_t bytes);

/* Copy `bytes` from src to dst, each device memory or page-locked host memory
 * (cudaHostAlloc / cudaHostRegister, e.g. a pinned PyTorch tensor), with the
 * GPU's own 16-byte loads and stores (a grid-stride kernel) instead of a copy
 * engine: the host <-> device transfers of a solve's source and solution where
 * the CPU-GPU link gives the SMs coherent access to host memory (NVLink-C2C).
 * Asynchronous on `stream`.  DWF_ERR_ARG, before anything is launched, for
 * NULL or pageable (unregistered) pointers, pointers not 16-byte aligned or a
 * size that is not a multiple of 16. */
dwf_status dwf_copy(void* dst, const void* src, size_t bytes, void* stream);

/* Number of kernels the library has launched in this process so far (a
 * captured CUDA graph counts its kernels on every replay). */
dwf_status dwf_launch_count(uint64_t* n);

/* Number of device memory allocations (cudaMalloc) the library has made in
 * this process so far, over all handles and devices: a caller can check that
 * a sequence of calls allocated nothing (the operator calls, once their tile
 * table exists, and dwf_mpc_noalloc always). */
dwf_status dwf_alloc_count(uint64_t* n);

/* Multi-shift CG: for every shift sigma_s >= 0 solve
 * (M_pc^+ M_pc + sigma_s) x_s = b on the odd checkerboard of every box and
 * right-hand side, all shifts from one Krylov space (CG on the smallest
 * shift, the shifted systems by the published collinear-residual
 * recurrences).  These are the rational functions of the normal operators of
 * D and D_Omega in the DD-RHMC action (Sec. 2.3.1): sum_s a_s x_s.
 * x: device, nshift odd cb FP64 fields back to back, in the order of `shifts`
 *    (written; the initial contents are ignored).
 * b: device odd cb FP64 field (nrhs right-hand sides per box).
 * shifts: host array of nshift finite values >= 0, any order.
 * sp: tol (per shift and system, relative to |b|), maxiter, max_seconds and
 *     inner_prec = DWF_FP64 (FP64 operator) or DWF_FP32 (FP32 operator with
 *     FP64 vectors and scalars to 1e-6, then, for tol < 1e-6, rounds of
 *     defect correction per shift: the FP64 residual b - (A + sigma_s) x_s,
 *     a single-shift FP32 solve of it to 1e-6, x_s += correction;
 *     stats.reliable_updates counts the rounds); the other fields are
 *     ignored.
 * stats: host [nshift][nbox * nrhs]; true_resid = |b - (A + sigma_s) x_s| / |b|
 *     recomputed with the FP64 operator.
 * Allocates its workspace for the call.  Returns the first non-OK status
 * (DWF_ERR_NOT_CONVERGED, DWF_ERR_TIMEOUT, DWF_ERR_NAN) with x the last
 * iterate; DWF_ERR_ARG on bad arguments. */
dwf_status dwf_multishift_solve(dwf_handle* h, double* x, const double* b, const double* shifts,
                                int nshift, int nrhs, const dwf_solver_params* sp,
                                dwf_solver_stats* stats, void* stream);

/* Luescher's projector of Sec. 2.1 onto the spinor components of Omega on
 * which the hops from Omega into Omega-bar act (the row space of the block
 * D_partialbar of D): out = P in on the sites of the box `omega`, zero
 * elsewhere.  Per site P is the projector onto the span of
 * (b5 + c5 S5^+) [(1 +- gamma_mu) spinors x all s] over the neighbours
 * x +- mu outside Omega, colour-blind (built on the host in FP64 per
 * pattern of outside neighbours).  h: a whole-lattice handle; in, out:
 * distinct device full FP64 fields, nrhs right-hand sides.
 * DWF_ERR_UNSUPPORTED if a site outside Omega touches two sites of Omega
 * (then P is not site-local: use a band of width >= 2). */
dwf_status dwf_boundary_project(dwf_handle* h, const dwf_box* omega, double* out, const double* in,
                                int nrhs, void* stream);

/* R^-1 = P - P D^-1 D_partialbar (Sec. 2.1), the inverse of the boundary
 * operator R = P - P D_Omega^-1 D_partial D_Omega-bar^-1 D_partialbar on the
 * range of P, which carries the DD-HMC pseudofermion of det chi = det R:
 * out = u - P D^-1 (D u restricted to Omega-bar), u = P in.  D^-1 by
 * dwf_cgne_solve with `sp` (stats: nrhs entries of that solve).  Same
 * handle, field and Omega rules as dwf_boundary_project; allocates three
 * full FP64 fields for the call. */
dwf_status dwf_boundary_rinv(dwf_handle* h, const dwf_box* omega, double* out, const double* in,
                             int nrhs, const dwf_solver_params* sp, dwf_solver_stats* stats,
                             void* stream);

/* Link force of the bilinear sum_r Re <X_r, D Y_r>: the insertion of
 * delta D between two solved fields that the DD-HMC forces of Sec. 2.3 are
 * built from (the variation of R^-1 = P - P D^-1 D_partialbar and of the
 * actions built on it).  For every link U_mu(x), out[lex][mu] (a 3 x 3
 * complex matrix, canonical gauge layout) is the traceless anti-Hermitian F
 * with  d/d eps Re <X, D(exp(i eps H) U) Y> |_0 = Re tr[i H F]  for every
 * traceless Hermitian H:
 *   F = -1/2 TA(U_mu(x) M),  M = sum_lanes Z(x+mu) ((1 - g_mu) X(x))^+
 *                                  + [Z(x) ((1 + g_mu) X(x+mu))^+]^+,
 * Z = (b5 + c5 S5) Y, TA(A) = (A - A^+)/2 - tr(A - A^+)/6.  The adjoint
 * bilinear Re <X, D^+ Y> has the force of (Y, X).  X, Y: device full fields
 * of precision `prec` (FP64: FP64 arithmetic; FP32: FP32 links and
 * arithmetic), nrhs right-hand sides summed.  `active` (nullable): only links
 * with both ends in that box get a force, the others 0 (the links the DD-HMC
 * holds fixed).  accumulate: out += F instead of out = F.  h: a whole-lattice
 * handle; fields that vanish outside a box give that box's Dirichlet force.
 * Uses the handle's scratch fields; allocates nothing. */
dwf_status dwf_force(dwf_handle* h, double* out, const void* X, const void* Y, dwf_prec prec, int nrhs,
                     const dwf_box* active, int accumulate, void* stream);

/* The boundary operator itself (Sec. 2.1), the map of the pseudofermion
 * heat bath phi = R eta:
 *   R = P - P D_Omega^-1 D_partial D_Omega-bar^-1 D_partialbar   (on the range of P),
 * out = u - P D_Omega^-1 (D b on Omega), b = D_Omega-bar^-1 (D u on Omega-bar),
 * u = P in.  The two Dirichlet solves (on the band Omega-bar, which is not a
 * box, and on Omega) run as CGNR on P_S D P_S to sp->tol (maxiter
 * sp->maxiter): in FP64 if sp->inner_prec is DWF_FP64, else FP32 CGNR rounds
 * with FP64 defect correction; stats: 2 * nrhs entries (the Omega-bar solve,
 * then the Omega solve).  Same handle, field and Omega
 * rules as dwf_boundary_project; allocates ten full FP64 fields for the
 * call.  DWF_ERR_NOT_CONVERGED if a solve misses 2 * tol. */
dwf_status dwf_boundary_r(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                          const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream);

/* Link force of the DD-HMC boundary pseudofermion action S = |R^-1 phi|^2
 * (Sec. 2.1, 2.3; R^-1 as in dwf_boundary_rinv), summed over the nrhs
 * right-hand sides: out[lex][mu] (canonical gauge layout, 3 x 3 complex,
 * traceless anti-Hermitian) with d/d eps S(exp(i eps H) U) |_0 = Re tr[i H F]
 * for every traceless Hermitian H.  With u = P phi, y = D^-1 (D u on
 * Omega-bar), chi = R^-1 phi and zeta = D^-+ chi:
 *     F = 2 F(zeta, y) - 2 F(zeta on Omega-bar, u)   (F(X, Y) as in dwf_force).
 * D^-+ comes from D^-1 by the gamma_5 R_5 Hermiticity of D (b5 + c5 S5)^-1.
 * Two solves with `sp`; stats: 2 * nrhs entries (the D^-1 v solve, then the
 * adjoint one).  `active` and `accumulate` as in dwf_force.  Same handle,
 * field and Omega rules as dwf_boundary_project; allocates four full FP64
 * fields for the call. */
dwf_status dwf_boundary_force(dwf_handle* h, const dwf_box* omega, double* out, const double* phi, int nrhs,
                              const dwf_box* active, int accumulate, const dwf_solver_params* sp,
                              dwf_solver_stats* stats, void* stream);

/* Link force of the boundary Hasenbusch ratio (Sec. 2.3) between the light
 * boundary operator R (handle h_light) and its Pauli-Villars counterpart
 * R_pv (handle h_pv: same lattice, Ls and gauge field, heavier mass):
 *   S = |R^-1 R_pv phi|^2,  d/d eps S(exp(i eps H) U) |_0 = Re tr[i H F],
 *   F = 2 F(zeta, y) - 2 F(zeta on Omega-bar, u) + 2 F_pv(eta, d - b) + 2 F_pv(kappa, b - u_pv),
 * with u_pv = P_pv phi, b = D_Ob^-1 (D u_pv on Omega-bar), d = D_O^-1 (D b on
 * Omega) (PV; R_pv phi = u_pv - P_pv d), u, y, chi = R^-1 R_pv phi as in
 * dwf_boundary_force (light), zeta = D^-+ chi, xi = R^-+ chi = chi - (D^+
 * (zeta on Omega-bar)) on Omega, eta = D_O^-+ P_pv xi and kappa = D_Ob^-+
 * (D^+ eta on Omega-bar) (PV): the four PV local solves and two light solves
 * the paper counts.  Light solves: dwf_cgne_solve with `sp`; PV Dirichlet
 * solves: CGNR to sp->tol as in dwf_boundary_r.  stats: 6 * nrhs entries in the order b, d,
 * y, the adjoint light solve, eta, kappa.  `active` and `accumulate` as in
 * dwf_force (with the boundary links inactive the crossing terms vanish, as
 * in the paper).  Same field and Omega rules as dwf_boundary_project;
 * allocates eighteen full FP64 fields for the call. */
dwf_status dwf_boundary_ratio_force(dwf_handle* h_light, dwf_handle* h_pv, const dwf_box* omega, double* out,
                                    const double* phi, int nrhs, const dwf_box* active, int accumulate,
                                    const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream);

/* Zolotarev's optimal relative rational approximation of 1/sqrt(x) on
 * [lo, hi], type (n - 1, n), in partial fractions (host only, no GPU):
 *   1/sqrt(x) ~ sum_{j<n} residues[j] / (x + shifts[j]),
 * with relative error |1 - sqrt(x) r(x)| <= *delta, equioscillating.  The
 * (D^+ D)^(-1/2) factor of the one-flavour DD-RHMC term of Sec. 2.3.1 is
 * dwf_rational_apply with these coefficients (lo, hi bracketing the spectrum
 * of M_pc^+ M_pc).  On y = x/lo, c_l = sn^2/cn^2(l K'/(2n) | 1 - lo/hi),
 * poles the odd c_l, zeros the even ones, the scale centring the error.
 * shifts, residues: caller arrays of n doubles; delta may be NULL.
 * DWF_ERR_ARG unless 1 <= n <= 64 and 0 < lo < hi. */
dwf_status dwf_zolotarev_inv_sqrt(int n, double lo, double hi, double* shifts, double* residues, double* delta);

/* Best relative rational approximation of a fractional power, type (n, n),
 * in partial fractions (host only, no GPU):
 *   x^alpha ~ a0 + sum_{i<n} residues[i] / (x + shifts[i])   on [lo, hi],
 * minimising max |r(x) / x^alpha - 1| =: *delta; the error equioscillates at
 * 2n + 2 points (Chebyshev's characterisation of the unique best fit).
 * These are the RHMC coefficients of the one-flavour DD-RHMC term of
 * Sec. 2.3.1: alpha = 1/4 for (D_dir^+ D_dir)^(1/4), -1/2 for (D^+ D)^(-1/2),
 * and -1/4, 1/4 for the heat bath (lo, hi bracketing the spectrum of
 * M_pc^+ M_pc).  Shifts are > 0; residues > 0 for alpha < 0, < 0 for
 * alpha > 0.  The Remez algorithm (Newton on the equioscillation equations,
 * exchange of the reference points), started from Zolotarev's closed form at
 * alpha = -1/2 and continued in alpha; alpha > 0 from the reciprocal of the
 * fit of x^-alpha.  shifts, residues: caller arrays of n doubles; delta may
 * be NULL.  DWF_ERR_ARG unless -1 < alpha < 1, alpha != 0, 1 <= n <= 48 and
 * 0 < lo < hi <= 1e14 lo; DWF_ERR_NOT_CONVERGED if the iteration breaks down
 * (an n whose error would fall below rounding). */
dwf_status dwf_rational_power(double alpha, int n, double lo, double hi, double* a0, double* shifts,
                              double* residues, double* delta);

/* Rational function of the normal Schur operator in partial fractions,
 *   out = a0 in + sum_i residues[i] (M_pc^+ M_pc + shifts[i])^-1 in,
 * the form the DD-RHMC action of Sec. 2.3.1 takes for the powers of the
 * normal operators of D (whole-lattice handle) and of D_Omega (box handle),
 * e.g. the (D_dir^+ D_dir)^(1/4) and (D^+ D)^(-1/2) factors with
 * coefficients from dwf_rational_power.  One dwf_multishift_solve (same sp, stats
 * [n][nbox * nrhs]) and n + 1 axpby passes.  in, out: distinct odd cb FP64
 * fields; shifts, residues: host arrays of n values (shifts >= 0).  Returns
 * the multi-shift status (out is formed from the last iterates on
 * DWF_ERR_NOT_CONVERGED); allocates n odd cb FP64 fields for the call. */
dwf_status dwf_rational_apply(dwf_handle* h, double* out, const double* in, double a0, const double* shifts,
                              const double* residues, int n, int nrhs, const dwf_solver_params* sp,
                              dwf_solver_stats* stats, void* stream);

/* The one-flavour DD-RHMC boundary term of Sec. 2.3.1,
 *   S = phi^+ r1(A_d) r2(A) r1(A_d) phi,  r1 ~ x^(1/4), r2 ~ x^(-1/2)
 * (the paper's (D_dir^+ D_dir)^(1/4) (D^+ D)^(-1/2) (D_dir^+ D_dir)^(1/4) on
 * the even-odd preconditioned operators: the site-local M_ee is common to D
 * and D_dirichlet, so the Schur operators carry det D / det D_dirichlet),
 * A = M_pc^+ M_pc of D on handle h (whole lattice), A_d that of D_dirichlet
 * on handle hd (dwf_create_cut; same lattice, action and gauge field).
 * phi: device odd cb FP64 field, nrhs pseudofermions.  Multi-shift solves
 * with `sp` (FP64 or FP32 operator as in dwf_multishift_solve).
 *
 * dwf_one_flavour_action: S[r] per right-hand side (host array of nrhs);
 *   stats: [r1->n][nrhs] (w = r1(A_d) phi) then [r2->n][nrhs] (r2(A) w).
 * dwf_one_flavour_force: the link force of S summed over right-hand sides,
 *   out[lex][mu] (canonical gauge layout, traceless anti-Hermitian) with
 *   d/d eps S(exp(i eps H) U) |_0 = Re tr[i H F], from
 *     F = 2 sum_i rho2_i F_M(M x_i, x_i) + 2 sum_j rho1_j (F_Md(M_d z_j, y_j) + F_Md(M_d y_j, z_j)),
 *   x_i = (A + s2_i)^-1 w, z_j = (A_d + s1_j)^-1 phi, y_j = (A_d + s1_j)^-1 r2(A) w,
 *   F_M(X_o, Y_o) the force of -Re <X_o, M_pc Y_o> (one dwf_force insertion
 *   of the fields completed on the even sites by M_ee^-1 M_eo and its
 *   adjoint); stats: the two above then [r1->n][nrhs] (y); `active` and
 *   `accumulate` as in dwf_force.
 * dwf_one_flavour_heatbath: phi = q1(A_d) q2(A) eta with q1 ~ x^(-1/4) and
 *   q2 ~ x^(1/4), so that S(phi) = |eta|^2 up to the approximations (eta:
 *   Gaussian noise, device odd cb FP64, distinct from phi); stats: [q2->n][nrhs]
 *   then [q1->n][nrhs].
 * Each call allocates its pole fields (n1 + n2, resp. 2 n1 + n2 + 7 odd cb
 * FP64 fields for the force) for the call and returns the first non-OK
 * status of its solves.  DWF_ERR_ARG on handles that do not form such a
 * pair, a rational function with n < 1 or a negative shift, or null arrays. */
dwf_status dwf_one_flavour_action(dwf_handle* h, dwf_handle* hd, const double* phi, int nrhs,
                                  const dwf_rational* r1, const dwf_rational* r2, const dwf_solver_params* sp,
                                  double* S, dwf_solver_stats* stats, void* stream);
dwf_status dwf_one_flavour_force(dwf_handle* h, dwf_handle* hd, double* out, const double* phi, int nrhs,
                                 const dwf_rational* r1, const dwf_rational* r2, const dwf_box* active,
                                 int accumulate, const dwf_solver_params* sp, dwf_solver_stats* stats,
                                 void* stream);
dwf_status dwf_one_flavour_heatbath(dwf_handle* h, dwf_handle* hd, double* phi, const double* eta, int nrhs,
                                    const dwf_rational* q1, const dwf_rational* q2, const dwf_solver_params* sp,
                                    dwf_solver_stats* stats, void* stream);

/* Chebyshev filter of the normal Schur operator: the recursively built
 * filter functions of Sec. 4 for a fast multigrid set-up of the local
 * solves.  out = T_order(z(A)) in with A = M_pc^+ M_pc (on a box handle each
 * box's Dirichlet operator D_Omega) and z(lam) = (hi + lo - 2 lam)/(hi - lo):
 * modes of A in [lo, hi] keep |factor| <= 1, modes below lo grow like
 * cosh(order arccosh z).  Three-term recurrence, `order` applications of A.
 * in, out: distinct odd cb fields of precision `prec` (FP64 or FP32, which is
 * also the operator's), nrhs right-hand sides.  Errors: DWF_ERR_ARG for
 * order < 0, hi <= lo or another precision.  Allocates three cb fields for
 * the call and ends with a stream sync. */
dwf_status dwf_chebyshev_filter(dwf_handle* h, void* out, const void* in, int order, double lo, double hi,
                                dwf_prec prec, int nrhs, void* stream);

/* Flexible GCR(restart) with the right preconditioner K (NULL = none) on the
 * normal equations M_pc^+ M_pc x_o = M_pc^+ b'_o (restarted GCR on M_pc
 * itself stalls for Moebius DWF, whose Schur operator has the origin in its
 * field of values); same b'_o / x_e / true-residual treatment as
 * dwf_cgne_solve, stopping on |b - D x| / |b| <= tol.  If the true residual
 * stops decreasing for two restarts (a poor K), the solve falls back to
 * mixed-precision CGNE from the current x; stats.recorded = -1 marks that. 
 * Inner vectors and operator FP32, solution and restarted residual FP64,
 * FP64 inner products.  Each new direction is orthogonalised by classical
 * Gram-Schmidt, repeated once where the first pass shrank its norm by more
 * than 1/sqrt(2) in any active system.  reliable_updates in stats counts
 * restarts. */
dwf_status dwf_gcr_solve(dwf_handle* h, double* x, const double* b, int nrhs, dwf_nn* K,
                         const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream);

/* ------------------------------------------------ multigrid (Sec. 4)
 * Two-level aggregation multigrid for A = M_pc^+ M_pc of a handle (each
 * Dirichlet box on a box handle: the local systems of Sec. 4), set up from
 * near-null vectors the caller filters with dwf_chebyshev_filter (the
 * recursively built filter functions Sec. 4 proposes for the set-up); the
 * paper describes no more of the method, so the rest is the standard
 * construction: aggregates are 4D blocks (extents `block`, dividing every
 * box's extents) of the odd sites of each box with all their Ls and
 * spin-colour components; the prolongator P holds the vectors restricted to
 * each block and orthonormalised there by Gram-Schmidt in vector order
 * (classical, twice; P^+ P = 1); the coarse operator A_c = P^+ A P (Galerkin) is dense,
 * built by nblocks applications of A with nvec lanes and inverted once on the
 * device by pivoted Gauss-Jordan in FP64 (at most 4096 coarse unknowns =
 * blocks x nvec).  The preconditioner
 * is the V(1,1) cycle z = S r; z += P A_c^-1 P^+ (r - A z); z += S (r - A z)
 * with a smoother S: none, the Chebyshev iteration for A z = r on [lo, hi]
 * (steps - 1 applications of A), or the learned network K.  FP32 fields and
 * operator, FP64 coarse algebra. */

/* Block tables and workspace for nvec vectors (1 <= nvec <= nrhs_max of h);
 * the handle must outlive the preconditioner.  DWF_ERR_ARG if a block extent
 * does not divide a box extent or the coarse space is too large. */
dwf_status dwf_mg_create(dwf_mg** mg, dwf_handle* h, const int block[4], int nvec);
dwf_status dwf_mg_destroy(dwf_mg* mg);
/* Build P and A_c^-1 from V: an odd cb FP32 field with nvec lanes
 * ([site][12][k][s], the layout of nvec right-hand sides), read during the
 * call.  Synchronous.  DWF_ERR_ARG if the vectors are linearly dependent on a
 * block or A_c is singular. */
dwf_status dwf_mg_setup(dwf_mg* mg, const float* V, void* stream);
/* Smoother of the V-cycle: kind 0 none, 1 Chebyshev iteration (steps >= 1,
 * 0 < lo < hi bracketing the part of the spectrum to damp), 2 the network K
 * (whole-lattice handles). */
dwf_status dwf_mg_set_smoother(dwf_mg* mg, int kind, int steps, double lo, double hi, dwf_nn* K);
/* z = M^-1 r (V(1,1) cycle): odd cb FP32 fields, one right-hand side,
 * distinct.  Asynchronous on `stream`; allocates nothing. */
dwf_status dwf_mg_apply(dwf_mg* mg, float* z, const float* r, void* stream);
/* c = P^+ f (device, nblocks x nvec complex FP64, block-major) and f = P c
 * for one right-hand side: the transfer operators, for tests and users. */
dwf_status dwf_mg_restrict(dwf_mg* mg, double* c, const float* f, void* stream);
dwf_status dwf_mg_prolong(dwf_mg* mg, float* f, const double* c, void* stream);
/* Number of blocks and of coarse unknowns (blocks x nvec); either pointer
 * may be NULL. */
dwf_status dwf_mg_info(const dwf_mg* mg, int* nblocks, int* ncoarse);
/* Copy (device to device, on `stream`) what = 0: the orthonormal basis (an
 * nvec-lane odd cb FP32 field), what = 1: A_c (row-major complex FP64, rows
 * and columns (block, k), k fastest) into the caller's buffer dst. */
dwf_status dwf_mg_copy(const dwf_mg* mg, int what, void* dst, void* stream);
/* The handle a set-up preconditioner belongs to. */
dwf_status dwf_mg_handle(const dwf_mg* mg, dwf_handle** h);
/* dwf_gcr_solve (one right-hand side) with the multigrid preconditioner:
 * flexible GCR on A x_o = M_pc^+ b'_o with z_j = M^-1 r_j, same residual
 * rules, stats and fallback. */
dwf_status dwf_gcr_solve_mg(dwf_handle* h, double* x, const double* b, dwf_mg* mg,
                            const dwf_solver_params* sp, dwf_solver_stats* stats, void* stream);

/* ------------------------------------------------ learned preconditioner
 * K: two linear gauge-covariant parallel-transport layers (1 -> 16 -> 1
 * channels).  Transports T_0 = 1, T_{1+mu} f(x) = U_mu(x) f(x+mu),
 * T_{5+mu} f(x) = U_mu(x-mu)^+ f(x-mu), T_9 / T_10 = shift s+1 / s-1 with
 * zero outside [0, Ls); layer: out^a = sum_{b,d} W[d][a][b] T_d in^b with
 * complex 4x4 spin matrices W (gauge covariant: they commute with colour).
 * K maps an odd cb field (embedded with zeros on even sites) to the odd
 * part of the output.  Weights: W1[d][a][0][so][si] (11 x 16 x 16 complex)
 * then W2[d][0][b][so][si], complex128 interleaved; applied in BF16,
 * trained in FP32 with Adam (beta 0.9 / 0.999).  Created as the identity. */
dwf_status dwf_nn_create(dwf_nn** K, int channels);
dwf_status dwf_nn_destroy(dwf_nn* K);
dwf_status dwf_nn_set_weights(dwf_nn* K, const double* w, size_t n_complex);
dwf_status dwf_nn_get_weights(const dwf_nn* K, double* w, size_t n_complex);
/* Write K's weights to the file `path` ("DWFNN001", int32 channels, int32 0,
 * int64 n, then n complex128 in dwf_nn_set_weights order, this host's byte
 * order) / read them back into K (same channel count).  DWF_ERR_ARG on an I/O
 * failure or a file of another network. */
dwf_status dwf_nn_save(const dwf_nn* K, const char* path);
dwf_status dwf_nn_load(dwf_nn* K, const char* path);
/* out = K in, odd cb FP32 fields with nrhs lanes (host workspace grows on
 * first use per handle and nrhs).  The two layers are linear, so this call
 * applies their product W2 W1 (formed in FP64 from the BF16 weights, stored
 * FP32) to the transported input, only on the directions that are nonzero on
 * each checkerboard (the link transports on even sites, the identity and the
 * s-shifts on odd sites); the training step runs the two layers through the
 * channels.  Both give the same K up to FP32 rounding. */
dwf_status dwf_nn_apply(dwf_nn* K, dwf_handle* h, float* out, const float* in, int nrhs,
                        void* stream);
/* One Adam step on nrhs (r, e) pairs (odd cb FP32, one pair per lane,
 * r = M_pc^+ M_pc e) of the loss  loss_kind 0: mean_k |K r_k - e_k|^2 / |e_k|^2;
 * loss_kind 1: the energy-norm error mean_k <d_k, A d_k> / <e_k, r_k>,
 * d_k = K r_k - e_k, A = M_pc^+ M_pc; loss_kind 2: the A^2-norm error
 * mean_k |A d_k|^2 / |r_k|^2 = |A K r_k - r_k|^2 / |r_k|^2.  *loss receives the loss before the
 * step.  Whole-lattice handles only. */
dwf_status dwf_nn_train_step(dwf_nn* K, dwf_handle* h, const float* r, const float* e, int nrhs,
                             int loss_kind, double lr, double* loss, void* stream);
/* One training pair of K from an FP64 solve of D x = b (nrhs = 1): with the
 * solution x* and a recorded iterate x_k (odd cb FP64 fields),
 *   e = (x* - x_k) / |x* - x_k|,   r = M_pc^+ M_pc e   (FP64 operator),
 * written as odd cb FP32 fields (r, e); *norm (host) receives |x* - x_k|,
 * and when it is 0 nothing is written.  The pair satisfies the normal
 * equations M_pc^+ M_pc e = r that flexible GCR is preconditioned for.
 * Whole-lattice handles; uses the handle's scratch fields, allocates three
 * odd cb FP64 fields for the call and synchronises the stream. */
dwf_status dwf_nn_make_pair(dwf_handle* h, const double* x_star, const double* x_k, float* r, float* e,
                            double* norm, void* stream);
/* Gradient of the last train step on handle h, layout of the weights. */
dwf_status dwf_nn_last_grad(dwf_handle* h, double* g, size_t n_complex);

/* Device error word (bounded waits that ran out); DWF_ERR_DEVICE if set. */
dwf_status dwf_check_device(dwf_handle* h);

/* Thread-local description of the last failure. */
const char* dwf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DWF_H */
