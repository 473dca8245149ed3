// Even-odd preconditioned CGNE for D x = b (or D_Omega x = b), all boxes and
// right-hand sides at once.
//
// Sec. 2.3 of the paper: the two-flavour determinants are simulated with
// red-black preconditioned solves, and the solves with D and with the
// Dirichlet operator dominate the cost.  The solve here:
//
//   b'_o = b_o - M_oe M_ee^-1 b_e
//   CG on M_pc^+ M_pc x_o = M_pc^+ b'_o
//   x_e  = M_ee^-1 (b_e - M_eo x_o)
//
// and it stops per system when |b'_o - M_pc x_o| / |b| <= tol; that is the
// full residual |b - D x| / |b| exactly (the even rows are solved exactly),
// and the final stats recompute |b - D x| with the FP64 operator.
//
// Mixed precision (reliable updates, Sleijpen & van der Vorst 1996): the
// inner iteration runs with the FP32 or BF16 operator and FP32 vectors; the
// solution increment accumulates in FP32 and is flushed into the FP64
// solution whenever the iterated residual has dropped by `delta` since the
// last flush (or reaches the stopping target); there the residual is
// recomputed in FP64 from the FP64 solution, which is also the true-residual
// test.  The search direction is kept across the update.
//
// Every inner reduction is the deterministic two-stage FP64 sum; all scalar
// recurrences (alpha, beta, the trigger tests) run on the device, and
// `check_every` iterations are replayed as one CUDA graph between host polls.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {



// per-system scalar slots (doubles) and flags (ints)
enum { S_RR, S_PAP, S_ALPHA, S_BETA, S_MAXR, S_TARGET, S_BN2, S_TR2, S_TMP, S_NDBL };
enum { F_RUN, F_ACTIVE, F_NEED, F_ITERS, F_BAD, S_NINT };

struct SysView {
    double* d;   // [S_NDBL][nsys]
    int* f;      // [S_NINT][nsys]
    int nsys;
    __host__ __device__ double* dbl(int k) const { return d + (size_t)k * nsys; }
    __host__ __device__ int* flg(int k) const { return f + (size_t)k * nsys; }
};

// alpha = <r, r> / <p, A p> for system i
__device__ void alpha_step(SysView v, int i) {
    double a = 0.0;
    // a system whose last iteration asked for an FP64 update is frozen here,
    // after its search direction has been updated
    if (v.flg(F_NEED)[i]) v.flg(F_RUN)[i] = 0;
    if (v.flg(F_RUN)[i]) {
        const double pap = v.dbl(S_PAP)[i];
        if (pap > 0.0 && isfinite(pap)) a = v.dbl(S_RR)[i] / pap;
        else { v.flg(F_RUN)[i] = 0; v.flg(F_NEED)[i] = 1; v.flg(F_BAD)[i] = 1; }
    }
    v.dbl(S_ALPHA)[i] = a;
}

// after r -= alpha A p: beta, iteration count, reliable-update trigger
__device__ void beta_step(SysView v, int i, double delta) {
    if (!v.flg(F_RUN)[i]) { v.dbl(S_BETA)[i] = 0.0; return; }
    const double rrn = v.dbl(S_TMP)[i];
    const double rr = v.dbl(S_RR)[i];
    v.flg(F_ITERS)[i] += 1;
    if (!isfinite(rrn)) {
        v.flg(F_RUN)[i] = 0; v.flg(F_NEED)[i] = 1; v.flg(F_BAD)[i] = 1;
        v.dbl(S_BETA)[i] = 0.0;
        return;
    }
    v.dbl(S_BETA)[i] = rrn / rr;
    v.dbl(S_RR)[i] = rrn;
    const double nr = sqrt(rrn);
    // FP64 update when the residual has dropped by delta, reached the target,
    // or grown far beyond its value at the last update (a diverging
    // low-precision recurrence)
    if (nr <= v.dbl(S_TARGET)[i] || (delta > 0.0 && nr <= delta * v.dbl(S_MAXR)[i]) ||
        nr > 1e3 * v.dbl(S_MAXR)[i])
        v.flg(F_NEED)[i] = 1;   // frozen by the next alpha step until the FP64 update
}

// One block per system: the deterministic sum of its tiles' partials, then
// the CG scalar step of that system -- STEP 0: <p, A p> and alpha, STEP 1:
// |r|^2 and beta.
template <int STEP>
__global__ void __launch_bounds__(1024) k_reduce_step(const double* __restrict__ partial,
                                                      const int* __restrict__ box_tb, int nrhs,
                                                      SysView v, double delta) {
    __shared__ double sh[32];
    const int sys = blockIdx.x;
    const int box = sys / nrhs, r = sys % nrhs;
    const int t0 = box_tb[box], t1 = box_tb[box + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fixed association: thread-strided sums, then warp and block shuffle trees
    double acc = 0.0;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) acc += partial[(size_t)t * nrhs + r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (warp != 0) return;
    acc = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane != 0) return;
    if (STEP == 0) {
        v.dbl(S_PAP)[sys] = acc;
        alpha_step(v, sys);
    } else {
        v.dbl(S_TMP)[sys] = acc;
        beta_step(v, sys, delta);
    }
}

__global__ void k_add2(double* out, const double* a, const double* b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i];
}

static dwf_status ws_alloc(void** p, size_t bytes) {
    *p = nullptr;
    DWF_CUDA(dev_malloc(p, bytes ? bytes : 16));
    return DWF_OK;
}

void free_solver_ws(dwf_handle* h) {
    for (auto& kv : h->ws) {
        SolverWS& w = kv.second;
        void* ptrs[] = {w.x64, w.bp64, w.t64a, w.t64b, w.t64c, w.t64d, w.full64a, w.x_lo, w.r,
                        w.p, w.t, w.tmp1, w.tmp2, w.tmp3, w.part, w.sys};
        for (void* q : ptrs) cudaFree(q);
        if (w.h_sys) cudaFreeHost(w.h_sys);
        if (w.graph_exec) cudaGraphExecDestroy(w.graph_exec);
        if (w.graph) cudaGraphDestroy(w.graph);
        if (w.graph_stream) cudaStreamDestroy(w.graph_stream);
    }
    h->ws.clear();
}

static dwf_status get_ws(dwf_handle* h, dwf_prec inner, int nrhs, SolverWS** out) {
    const int key = inner * 64 + nrhs;
    SolverWS& w = h->ws[key];
    *out = &w;
    if (w.ready) return DWF_OK;
    w.nrhs = nrhs;
    w.prec = inner;
    const size_t no = cb_elems(h, 1, nrhs), ne = cb_elems(h, 0, nrhs);
    const size_t nm = no > ne ? no : ne;
    w.field_elems = no;
    const dwf_prec pv = inner == DWF_FP64 ? DWF_FP64 : DWF_FP32;
    const size_t sv = prec_size(pv) * 2, so = prec_size(inner) * 2;
    DWF_TRY(ws_alloc((void**)&w.x64, no * 16));
    DWF_TRY(ws_alloc((void**)&w.bp64, no * 16));
    DWF_TRY(ws_alloc((void**)&w.t64a, nm * 16));
    DWF_TRY(ws_alloc((void**)&w.t64b, nm * 16));
    DWF_TRY(ws_alloc((void**)&w.t64c, nm * 16));
    DWF_TRY(ws_alloc((void**)&w.t64d, nm * 16));
    DWF_TRY(ws_alloc((void**)&w.full64a, (no + ne) * 16));
    DWF_TRY(ws_alloc(&w.x_lo, no * sv));
    DWF_TRY(ws_alloc(&w.r, no * sv));
    DWF_TRY(ws_alloc(&w.p, no * sv));
    DWF_TRY(ws_alloc(&w.t, no * sv));
    DWF_TRY(ws_alloc(&w.tmp1, nm * so));
    DWF_TRY(ws_alloc(&w.tmp2, nm * so));
    DWF_TRY(ws_alloc(&w.tmp3, no * so));   // t1 = (b5 + c5 S5) p, carried between iterations
    // partials for any tile size the autotuner may pick (>= kMinTile sites)
    const int64_t nsmax = h->nsite[0] > h->nsite[1] ? h->nsite[0] : h->nsite[1];
    const size_t ntmax = (size_t)(nsmax / kMinTile + h->nbox + 1);
    DWF_TRY(ws_alloc((void**)&w.part, ntmax * nrhs * sizeof(double)));
    w.nsys = h->nbox * nrhs;
    const size_t sys_bytes = (size_t)w.nsys * (S_NDBL * sizeof(double) + S_NINT * sizeof(int));
    DWF_TRY(ws_alloc((void**)&w.sys, sys_bytes));
    DWF_CUDA(cudaHostAlloc((void**)&w.h_sys, sys_bytes, cudaHostAllocDefault));
    DWF_CUDA(cudaStreamCreateWithFlags(&w.graph_stream, cudaStreamNonBlocking));
    w.ready = true;
    return DWF_OK;
}

// |f|^2 per system of a cb field of parity p into dst[nsys]
static dwf_status norm2_sys(dwf_handle* h, SolverWS& w, int parity, const void* f, dwf_prec pf,
                            double* dst, cudaStream_t s) {
    const int T = tile_for(h, w.nrhs);
    DWF_TRY(launch_dot_partial(h, parity, f, f, pf, pf, w.nrhs, w.part, T, s));
    return launch_reduce_sys(h, parity, w.part, w.nrhs, dst, T, s);
}

// res = b'_o - M_pc x64 (FP64) and its |.|^2 per system into S_TR2
static dwf_status true_residual(dwf_handle* h, SolverWS& w, SysView v, cudaStream_t s) {
    const int nrhs = w.nrhs;
    DWF_TRY(op_mpc(h, w.t64c, w.x64, 0, DWF_FP64, DWF_FP64, nrhs, w.t64a, w.t64b, nullptr, nullptr, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, w.bp64, DWF_FP64, nullptr, -1.0, w.t64c,
                         DWF_FP64, nullptr, tile_for(h, nrhs), s));
    return norm2_sys(h, w, 1, w.t64c, DWF_FP64, v.dbl(S_TR2), s);
}

// one CG iteration on the inner vectors (captured into the graph)
static dwf_status cg_iteration(dwf_handle* h, SolverWS& w, SysView v, dwf_prec pv, dwf_prec po,
                               double delta, cudaStream_t s) {
    const int nrhs = w.nrhs;
    // t = M_pc p from t1 = (b5 + c5 S5) p, |t|^2 = <p, A p>
    DWF_TRY(op_mpc_pre(h, w.t, w.p, w.tmp3, pv, po, nrhs, w.tmp1, w.tmp2, w.part, s));
    const TileSet* ts = nullptr;
    DWF_TRY(get_tiles(h, tile_for(h, nrhs), &ts));
    const int* box_tb = ts->d_box_tile_begin[1];
    k_reduce_step<0><<<v.nsys, 1024, 0, s>>>(w.part, box_tb, nrhs, v, delta);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    // A p = M_pc^+ t fused with x += alpha p, r -= alpha A p, |r|^2
    void* xv = (pv == DWF_FP64) ? (void*)w.x64 : w.x_lo;
    CgFuse cg{xv, w.r, w.p, v.dbl(S_ALPHA), v.flg(F_RUN)};
    DWF_TRY(op_mpc(h, nullptr, w.t, 1, pv, po, nrhs, w.tmp1, w.tmp2, w.part, &cg, s));
    k_reduce_step<1><<<v.nsys, 1024, 0, s>>>(w.part, box_tb, nrhs, v, delta);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    // p = r + beta p fused with the next iteration's t1 = (b5 + c5 S5) p
    LocalCall c{};
    c.op = L_PB;
    c.out = w.tmp3;
    c.in = w.p;
    c.in2 = w.r;
    c.parity = 1;
    c.prec_in = pv;
    c.prec_in2 = pv;
    c.prec_out = po;
    c.nrhs = nrhs;
    c.scale = 1.0;
    c.cg_p = w.p;
    c.alpha = v.dbl(S_BETA);
    c.run = v.flg(F_RUN);
    c.T = tile_for(h, nrhs);
    return launch_local(h, c, s);
}

dwf_status cgne_solve(dwf_handle* h, double* x, const double* b, int nrhs,
                      const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t user) {
    auto t_start = std::chrono::steady_clock::now();
    if (!h->have_gauge) {
        set_error("dwf_cgne_solve: no gauge field loaded");
        return DWF_ERR_ARG;
    }
    if (sp == nullptr || x == nullptr || b == nullptr || nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("dwf_cgne_solve: bad arguments");
        return DWF_ERR_ARG;
    }
    if (!(sp->tol > 0.0) || sp->maxiter < 1) {
        set_error("dwf_cgne_solve: tol must be > 0 and maxiter >= 1");
        return DWF_ERR_ARG;
    }
    const dwf_prec po = sp->inner_prec;
    const dwf_prec pv = po == DWF_FP64 ? DWF_FP64 : DWF_FP32;
    SolverWS* wp = nullptr;
    DWF_TRY(get_ws(h, po, nrhs, &wp));
    SolverWS& w = *wp;
    cudaStream_t s = w.graph_stream;
    DWF_CUDA(cudaStreamSynchronize(user));
    SysView v{w.sys, (int*)(w.sys + (size_t)S_NDBL * w.nsys), w.nsys};
    const int nsys = w.nsys;
    const size_t sys_bytes = (size_t)nsys * (S_NDBL * sizeof(double) + S_NINT * sizeof(int));
    double* hd = w.h_sys;
    int* hf = (int*)(w.h_sys + (size_t)S_NDBL * nsys);
    auto HD = [&](int k, int i) -> double& { return hd[(size_t)k * nsys + i]; };
    auto HF = [&](int k, int i) -> int& { return hf[(size_t)k * nsys + i]; };
    const size_t ne = cb_elems(h, 0, nrhs), no = cb_elems(h, 1, nrhs);
    const double* be = b;
    const double* bo = b + 2 * ne;
    double* xe = x;
    double* xo = x + 2 * ne;
    // default threshold: FP32 keeps the recursive residual accurate over two
    // decades (6 FP64 updates instead of 11 on a 16^4 x 12 Moebius solve, same
    // iteration count); BF16 rounding allows one
    const double delta = (po == DWF_FP64) ? 0.0
                         : (sp->delta > 0 ? sp->delta : (po == DWF_BF16 ? 0.1 : 0.01));
    const int K = sp->check_every > 0 ? sp->check_every : 8;

    DWF_CUDA(cudaMemsetAsync(w.sys, 0, sys_bytes, s));
    // |b|^2 per system (both parities)
    DWF_TRY(norm2_sys(h, w, 0, be, DWF_FP64, v.dbl(S_TMP), s));
    DWF_TRY(norm2_sys(h, w, 1, bo, DWF_FP64, v.dbl(S_BN2), s));
    k_add2<<<(nsys + 127) / 128, 128, 0, s>>>(v.dbl(S_BN2), v.dbl(S_BN2), v.dbl(S_TMP), nsys);
    note_launch();
    // b'_o = b_o - M_oe M_ee^-1 b_e
    DWF_TRY(op_local(h, L_MINV, w.t64a, be, nullptr, 0, 0, DWF_FP64, DWF_FP64, DWF_FP64, nrhs, 1.0, nullptr, s));
    DWF_TRY(op_dslash_eo(h, w.t64b, w.t64a, 1, 0, DWF_FP64, nrhs, w.t64d, s));
    DWF_CUDA(cudaMemcpyAsync(w.bp64, bo, no * 16, cudaMemcpyDeviceToDevice, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, -1.0, w.t64b, DWF_FP64, nullptr, 1.0, w.bp64, DWF_FP64, nullptr, tile_for(h, nrhs), s));
    // initial guess
    if (sp->use_x0) DWF_CUDA(cudaMemcpyAsync(w.x64, xo, no * 16, cudaMemcpyDeviceToDevice, s));
    else DWF_CUDA(cudaMemsetAsync(w.x64, 0, no * 16, s));
    const size_t sv = prec_size(pv) * 2;
    DWF_CUDA(cudaMemsetAsync(w.x_lo, 0, no * sv, s));

    const bool trace = getenv("DWF_SOLVER_TRACE") != nullptr;
    // host-side per-system bookkeeping
    std::vector<int> active(nsys, 1), status(nsys, DWF_ERR_NOT_CONVERGED), reliable(nsys, 0);
    std::vector<double> bnorm(nsys), tres(nsys, 1.0), target(nsys);

    // residual restart: res = b' - M_pc x64 ; r = M_pc^+ res ; returns via host mirror
    auto restart = [&](bool first) -> dwf_status {
        if (pv != DWF_FP64) {
            // flush the FP32 increment into the FP64 solution
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, w.x_lo, pv, nullptr, 1.0, w.x64, DWF_FP64, nullptr, tile_for(h, nrhs), s));
            DWF_CUDA(cudaMemsetAsync(w.x_lo, 0, no * sv, s));
        }
        DWF_TRY(true_residual(h, w, v, s));
        if (pv == DWF_FP64) {
            DWF_TRY(op_mpc(h, w.t64d, w.t64c, 1, DWF_FP64, DWF_FP64, nrhs, w.t64a, w.t64b, nullptr, nullptr, s));
            DWF_CUDA(cudaMemcpyAsync(w.r, w.t64d, no * 16, cudaMemcpyDeviceToDevice, s));
        } else {
            // r = M_pc^+ res with the FP32 operator: res = b' - M_pc x is exact to
            // FP64 (it alone decides convergence), and r only restarts the FP32
            // recursion, whose own rounding is of the same size -- half of the
            // update's FP64 hops saved.  FP64-sized scratch holds the FP32 fields.
            DWF_TRY(launch_convert(w.t64d, DWF_FP32, w.t64c, DWF_FP64, no, s));
            DWF_TRY(op_mpc(h, w.r, w.t64d, 1, DWF_FP32, DWF_FP32, nrhs, w.t64a, w.t64b, nullptr, nullptr, s));
        }
        DWF_TRY(norm2_sys(h, w, 1, w.r, pv, v.dbl(S_TMP), s));
        // the search direction is kept across an update (Sleijpen & van der
        // Vorst), except with the BF16 operator, whose ~1e-2 rounding breaks
        // conjugacy: there the inner CG restarts from the new residual
        if (first || po == DWF_BF16)
            DWF_CUDA(cudaMemcpyAsync(w.p, w.r, no * sv, cudaMemcpyDeviceToDevice, s));
        // t1 = (b5 + c5 S5) p for the next iteration's M_pc
        DWF_TRY(op_local(h, L_B, w.tmp3, w.p, nullptr, 1, 0, pv, pv, po, nrhs, 1.0, nullptr, s));
        DWF_CUDA(cudaMemcpyAsync(hd, w.sys, sys_bytes, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nsys; ++i) {
            if (first) bnorm[i] = std::sqrt(HD(S_BN2, i));
            const double bn = bnorm[i] > 0 ? bnorm[i] : 1.0;
            const double tr = std::sqrt(HD(S_TR2, i)) / bn;
            const double rn = std::sqrt(HD(S_TMP, i));
            if (trace && active[i])
                fprintf(stderr, "[dwf cg] sys %d iters %d true_resid %.3e |r| %.3e target %.3e%s\n", i,
                        HF(F_ITERS, i), tr, rn, HD(S_TARGET, i), HF(F_BAD, i) ? " BAD" : "");
            if (HF(F_BAD, i)) { status[i] = DWF_ERR_NAN; active[i] = 0; }
            if (!active[i]) { HF(F_RUN, i) = 0; HF(F_ACTIVE, i) = 0; continue; }
            tres[i] = tr;
            if (!(tr == tr) || !std::isfinite(rn)) { status[i] = DWF_ERR_NAN; active[i] = 0; HF(F_RUN, i) = 0; continue; }
            if (tr <= 0.9 * sp->tol) {
                status[i] = DWF_OK;
                active[i] = 0;
                HF(F_RUN, i) = 0;
                HF(F_ACTIVE, i) = 0;
                continue;
            }
            // target for the iterated normal residual, tightened by the
            // observed ratio of normal to true residual
            const double ratio = (HD(S_TR2, i) > 0) ? rn / std::sqrt(HD(S_TR2, i)) : 1.0;
            double tg = 0.5 * sp->tol * bn * ratio;
            if (!first && target[i] > 0) tg = std::min(tg, target[i]);
            target[i] = tg;
            HD(S_TARGET, i) = tg;
            HD(S_RR, i) = HD(S_TMP, i);
            HD(S_MAXR, i) = rn;
            HF(F_RUN, i) = 1;
            HF(F_ACTIVE, i) = 1;
            HF(F_NEED, i) = 0;
        }
        DWF_CUDA(cudaMemcpyAsync(w.sys, hd, sys_bytes, cudaMemcpyHostToDevice, s));
        return DWF_OK;
    };

    DWF_TRY(restart(true));

    // capture K iterations once per workspace
    // (delta is a kernel argument of the captured beta step: a new delta re-captures)
    if (w.graph_exec == nullptr || w.graph_iters != K || w.graph_T != tile_for(h, nrhs) ||
        w.graph_delta != delta) {
        if (w.graph_exec) { cudaGraphExecDestroy(w.graph_exec); w.graph_exec = nullptr; }
        if (w.graph) { cudaGraphDestroy(w.graph); w.graph = nullptr; }
        DWF_CUDA(cudaStreamSynchronize(s));
        DWF_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        capture_begin();
        dwf_status st = DWF_OK;
        for (int k = 0; k < K && st == DWF_OK; ++k) st = cg_iteration(h, w, v, pv, po, delta, s);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        w.graph_kernels = capture_end();
        if (st != DWF_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (ce != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(ce)); return DWF_ERR_CUDA; }
        w.graph = g;
        DWF_CUDA(cudaGraphInstantiate(&w.graph_exec, g, 0));
        w.graph_iters = K;
        w.graph_T = tile_for(h, nrhs);
        w.graph_delta = delta;
    }

    dwf_status result = DWF_OK;
    bool timed_out = false;
    // iterate recording (training data for the learned preconditioner)
    const bool rec = sp->record_x != nullptr && pv == DWF_FP64 && sp->record_max > 0;
    const int rec_batches = sp->record_every > K ? (sp->record_every + K - 1) / K : 1;
    int recorded = 0, batch_no = 0;
    for (;;) {
        bool any = false;
        for (int i = 0; i < nsys; ++i) any |= active[i] != 0;
        if (!any) break;
        DWF_CUDA(cudaGraphLaunch(w.graph_exec, s));
        note_graph_launch(w.graph_kernels);
        ++batch_no;
        if (rec && recorded < sp->record_max && batch_no % rec_batches == 0) {
            DWF_CUDA(cudaMemcpyAsync(sp->record_x + (size_t)recorded * no * 2, w.x64, no * 16,
                                     cudaMemcpyDeviceToDevice, s));
            ++recorded;
        }
        DWF_CUDA(cudaMemcpyAsync(hd, w.sys, sys_bytes, cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        bool need = false, capped = false;
        for (int i = 0; i < nsys; ++i) {
            if (!active[i]) continue;
            if (HF(F_NEED, i)) need = true;
            if (HF(F_ITERS, i) >= sp->maxiter) capped = true;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (sp->max_seconds > 0 && el > sp->max_seconds) { timed_out = true; need = true; }
        if (capped) need = true;
        if (need) {
            int rel = 0;
            for (int i = 0; i < nsys; ++i) if (active[i]) { reliable[i]++; rel++; }
            DWF_TRY(restart(false));
            if (timed_out || capped) {
                for (int i = 0; i < nsys; ++i)
                    if (active[i] && (timed_out || HF(F_ITERS, i) >= sp->maxiter)) {
                        status[i] = timed_out ? DWF_ERR_TIMEOUT : DWF_ERR_NOT_CONVERGED;
                        active[i] = 0;
                    }
                if (timed_out) break;
                DWF_CUDA(cudaStreamSynchronize(s));
                // freeze the stopped systems on the device too
                for (int i = 0; i < nsys; ++i) if (!active[i]) HF(F_RUN, i) = 0;
                DWF_CUDA(cudaMemcpyAsync(w.sys, hd, sys_bytes, cudaMemcpyHostToDevice, s));
            }
        }
    }
    // final: x_o, x_e and the FP64 residual of the full system
    if (pv != DWF_FP64) {
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, w.x_lo, pv, nullptr, 1.0, w.x64, DWF_FP64, nullptr, tile_for(h, nrhs), s));
        DWF_CUDA(cudaMemsetAsync(w.x_lo, 0, no * sv, s));
    }
    DWF_CUDA(cudaMemcpyAsync(xo, w.x64, no * 16, cudaMemcpyDeviceToDevice, s));
    DWF_TRY(op_dslash_eo(h, w.t64a, xo, 0, 0, DWF_FP64, nrhs, w.t64d, s));
    DWF_TRY(launch_axpby(h, 0, nrhs, nullptr, 1.0, be, DWF_FP64, nullptr, -1.0, w.t64a, DWF_FP64, nullptr, tile_for(h, nrhs), s));
    DWF_TRY(op_local(h, L_MINV, xe, w.t64a, nullptr, 0, 0, DWF_FP64, DWF_FP64, DWF_FP64, nrhs, 1.0, nullptr, s));
    DWF_TRY(op_apply_d(h, w.full64a, x, 0, DWF_FP64, nrhs, w.t64d, s));
    DWF_TRY(launch_axpby(h, 0, nrhs, nullptr, 1.0, be, DWF_FP64, nullptr, -1.0, w.full64a, DWF_FP64, nullptr, tile_for(h, nrhs), s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, bo, DWF_FP64, nullptr, -1.0, w.full64a + 2 * ne, DWF_FP64, nullptr, tile_for(h, nrhs), s));
    DWF_TRY(norm2_sys(h, w, 0, w.full64a, DWF_FP64, v.dbl(S_TMP), s));
    DWF_TRY(norm2_sys(h, w, 1, w.full64a + 2 * ne, DWF_FP64, v.dbl(S_TR2), s));
    k_add2<<<(nsys + 127) / 128, 128, 0, s>>>(v.dbl(S_TR2), v.dbl(S_TR2), v.dbl(S_TMP), nsys);
    note_launch();
    DWF_CUDA(cudaMemcpyAsync(hd, w.sys, sys_bytes, cudaMemcpyDeviceToHost, s));
    DWF_CUDA(cudaStreamSynchronize(s));
    int herr = 0;
    DWF_CUDA(cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    for (int i = 0; i < nsys; ++i) {
        const double bn = bnorm[i] > 0 ? bnorm[i] : 1.0;
        const double tr = std::sqrt(HD(S_TR2, i)) / bn;
        if (status[i] == DWF_OK && !(tr <= sp->tol)) status[i] = DWF_ERR_NOT_CONVERGED;
        if (stats) {
            stats[i].iters = HF(F_ITERS, i);
            stats[i].reliable_updates = reliable[i];
            stats[i].op_applies = 2 * HF(F_ITERS, i) + 2 * (reliable[i] + 1);
            stats[i].status = status[i];
            stats[i].true_resid = tr;
            stats[i].seconds = secs;
            stats[i].recorded = recorded;
        }
        if (status[i] != DWF_OK && result == DWF_OK) result = (dwf_status)status[i];
    }
    if (herr) {
        set_error("device error word 0x%x", herr);
        return DWF_ERR_DEVICE;
    }
    if (result != DWF_OK) set_error("dwf_cgne_solve: %d system(s) did not reach tol", nsys);
    return result;
}

}  // namespace dwf
