// Multi-shift CG on the normal Schur operator A = M_pc^+ M_pc.
//
// The DD-RHMC boundary action (Sec. 2.3.1) needs rational functions of the
// normal operators of D and D_Omega, sum_s a_s (A + sigma_s)^-1 b.  All the
// shifted systems share the Krylov space of A, so one CG on the smallest shift
// gives every solution with the published multi-shift recurrences (Jegerlehner,
// hep-lat/9612014): the shifted residuals stay collinear with the base one,
// r^(s) = zeta^(s) r, and only scalars per (shift, system) differ.
//
// GB300 layout of the work: one application of A per iteration (the FP64 or
// FP32 operator kernels of the solver, every box and right-hand side at
// once), deterministic FP64 reductions per system, the scalar recurrences on
// the host (a few doubles per (shift, system)), and per shift two
// per-system axpby launches (x_s += a p_s, p_s = zeta r + b p_s) on FP64
// vectors; shifts whose systems have all converged are no longer updated.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

namespace {

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

dwf_status dev_alloc(DevBuf& b, size_t bytes) {
    DWF_CUDA(dev_malloc(&b.p, bytes ? bytes : 16));
    return DWF_OK;
}

// per-system Re<a, b> (a == b: |a|^2) of odd cb fields, to the host
dwf_status sys_dot(dwf_handle* h, const void* a, const void* b, dwf_prec p, int nrhs, double* part,
                   double* d_out, std::vector<double>& out, cudaStream_t s) {
    const int T = tile_for(h, nrhs);
    DWF_TRY(launch_dot_partial(h, 1, a, b, p, p, nrhs, part, T, s));
    DWF_TRY(launch_reduce_sys(h, 1, part, nrhs, d_out, T, s));
    DWF_CUDA(cudaMemcpyAsync(out.data(), d_out, out.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    DWF_CUDA(cudaStreamSynchronize(s));
    return DWF_OK;
}

}  // namespace

// One multi-shift CG with the operator of sp->inner_prec to sp->tol on the
// recursive residuals; stats get the FP64 true residuals.
static dwf_status multishift_core(dwf_handle* h, double* x, const double* b, const double* shifts,
                                  int nshift, int nrhs, const dwf_solver_params* sp,
                                  dwf_solver_stats* stats, cudaStream_t user, bool report) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!h->have_gauge) {
        set_error("dwf_multishift_solve: no gauge field loaded");
        return DWF_ERR_ARG;
    }
    if (x == nullptr || b == nullptr || shifts == nullptr || sp == nullptr || stats == nullptr ||
        nshift < 1 || nrhs < 1 || nrhs > h->nrhs_max || !(sp->tol > 0.0) || sp->maxiter < 1 ||
        (sp->inner_prec != DWF_FP64 && sp->inner_prec != DWF_FP32)) {
        set_error("dwf_multishift_solve: bad arguments (nshift >= 1, 1 <= nrhs <= nrhs_max, "
                  "tol > 0, maxiter >= 1, inner precision FP64 or FP32)");
        return DWF_ERR_ARG;
    }
    for (int i = 0; i < nshift; ++i)
        if (!(shifts[i] >= 0.0) || !std::isfinite(shifts[i])) {
            set_error("dwf_multishift_solve: shifts must be finite and >= 0");
            return DWF_ERR_ARG;
        }
    DWF_CUDA(cudaStreamSynchronize(user));
    cudaStream_t s = user;
    const int nsys = h->nbox * nrhs;
    const size_t no = cb_elems(h, 1, nrhs);   // complex elements of one odd field
    const size_t f64 = no * 16;
    const dwf_prec po = sp->inner_prec;
    const int T = tile_for(h, nrhs);

    // shifts in ascending order: the base system is the smallest
    std::vector<int> ord(nshift);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int i, int j) { return shifts[i] < shifts[j]; });
    const double sig0 = shifts[ord[0]];

    // workspace: r, p (base), Ap, t, and p_s for the other shifts (FP64);
    // FP32 operator copies when the operator runs in FP32
    DevBuf r, p, Ap, t, tA, tB, ps, part, dsc, p32, t32, a32;
    DWF_TRY(dev_alloc(r, f64));
    DWF_TRY(dev_alloc(p, f64));
    DWF_TRY(dev_alloc(Ap, f64));
    DWF_TRY(dev_alloc(t, f64));
    DWF_TRY(dev_alloc(tA, f64));
    DWF_TRY(dev_alloc(tB, f64));
    DWF_TRY(dev_alloc(ps, f64 * (size_t)std::max(nshift - 1, 1)));
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, T, &tsp));
    const TileSet& ts = *tsp;
    DWF_TRY(dev_alloc(part, (size_t)ts.ntiles[1] * nrhs * sizeof(double)));
    // device scalars: [4][nshift][nsys] (x coefficient, zeta, beta_s, unused) + [3][nsys]
    DWF_TRY(dev_alloc(dsc, ((size_t)4 * nshift + 3) * nsys * sizeof(double)));
    if (po == DWF_FP32) {
        DWF_TRY(dev_alloc(p32, no * 8));
        DWF_TRY(dev_alloc(t32, no * 8));
        DWF_TRY(dev_alloc(a32, no * 8));
    }
    double* dR = static_cast<double*>(r.p);
    double* dP = static_cast<double*>(p.p);
    double* dAp = static_cast<double*>(Ap.p);
    double* dT = static_cast<double*>(t.p);
    double* dS = static_cast<double*>(dsc.p);
    double* dPart = static_cast<double*>(part.p);
    auto xs = [&](int k) { return x + (size_t)ord[k] * no * 2; };            // k: sorted index
    auto pk = [&](int k) { return k == 0 ? dP : static_cast<double*>(ps.p) + (size_t)(k - 1) * no * 2; };
    double* d_sys = dS + (size_t)4 * nshift * nsys;                            // [3][nsys]
    std::vector<double> h_sc((size_t)4 * nshift * nsys, 0.0);
    auto hs = [&](int q, int k, int i) -> double& { return h_sc[((size_t)q * nshift + k) * nsys + i]; };
    auto ds = [&](int q, int k) { return dS + ((size_t)q * nshift + k) * nsys; };

    // A p with the chosen operator, plus sigma0 p
    auto apply_A = [&](double* out, const double* in, double sig) -> dwf_status {
        if (po == DWF_FP64) {
            DWF_TRY(op_mpc(h, dT, in, 0, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
            DWF_TRY(op_mpc(h, out, dT, 1, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
        } else {
            DWF_TRY(launch_convert(p32.p, DWF_FP32, in, DWF_FP64, no, s));
            DWF_TRY(op_mpc(h, t32.p, p32.p, 0, DWF_FP32, DWF_FP32, nrhs, tA.p, tB.p, nullptr, nullptr, s));
            DWF_TRY(op_mpc(h, a32.p, t32.p, 1, DWF_FP32, DWF_FP32, nrhs, tA.p, tB.p, nullptr, nullptr, s));
            DWF_TRY(launch_convert(out, DWF_FP64, a32.p, DWF_FP32, no, s));
        }
        if (sig != 0.0)
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, sig, in, DWF_FP64, nullptr, 1.0, out, DWF_FP64,
                                 nullptr, T, s));
        return DWF_OK;
    };

    // start: x_s = 0, r = p = p_s = b
    std::vector<double> bn2(nsys), rr(nsys), pap(nsys), rr_new(nsys);
    DWF_TRY(sys_dot(h, b, b, DWF_FP64, nrhs, dPart, d_sys, bn2, s));
    for (int k = 0; k < nshift; ++k) {
        DWF_CUDA(cudaMemsetAsync(xs(k), 0, f64, s));
        DWF_CUDA(cudaMemcpyAsync(pk(k), b, f64, cudaMemcpyDeviceToDevice, s));
    }
    DWF_CUDA(cudaMemcpyAsync(dR, b, f64, cudaMemcpyDeviceToDevice, s));
    rr = bn2;
    std::vector<double> zeta((size_t)nshift * nsys, 1.0), zeta_prev(zeta), zeta_new(zeta);
    std::vector<double> alpha_prev(nsys, 1.0), beta_prev(nsys, 0.0);
    std::vector<char> act((size_t)nshift * nsys, 1);
    std::vector<int> its((size_t)nshift * nsys, 0);
    for (int i = 0; i < nsys; ++i)
        if (bn2[i] == 0.0)
            for (int k = 0; k < nshift; ++k) act[(size_t)k * nsys + i] = 0;   // x = 0 solves it
    auto any_active = [&] { return std::any_of(act.begin(), act.end(), [](char c) { return c != 0; }); };
    int iter = 0;
    dwf_status result = DWF_OK;
    while (any_active()) {
        if (iter >= sp->maxiter) { result = DWF_ERR_NOT_CONVERGED; break; }
        if (sp->max_seconds > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > sp->max_seconds) {
            result = DWF_ERR_TIMEOUT;
            break;
        }
        DWF_TRY(apply_A(dAp, dP, sig0));
        DWF_TRY(sys_dot(h, dP, dAp, DWF_FP64, nrhs, dPart, d_sys, pap, s));
        std::vector<double> alpha(nsys, 0.0);
        for (int i = 0; i < nsys; ++i) {
            if (!act[i]) continue;   // the base is the last to converge
            if (!(pap[i] > 0.0) || !std::isfinite(pap[i])) {
                set_error("dwf_multishift_solve: <p, A p> = %g (operator not positive?)", pap[i]);
                return DWF_ERR_NAN;
            }
            alpha[i] = rr[i] / pap[i];
        }
        // x_s += alpha_s p_s with alpha_s = alpha zeta_new / zeta
        for (int k = 0; k < nshift; ++k) {
            const double dk = shifts[ord[k]] - sig0;
            for (int i = 0; i < nsys; ++i) {
                const size_t ki = (size_t)k * nsys + i;
                if (!act[ki]) { hs(0, k, i) = 0.0; zeta_new[ki] = zeta[ki]; continue; }
                if (k == 0) {
                    zeta_new[ki] = 1.0;
                } else {
                    const double den = alpha[i] * beta_prev[i] * (zeta_prev[ki] - zeta[ki]) +
                                       zeta_prev[ki] * alpha_prev[i] * (1.0 + dk * alpha[i]);
                    zeta_new[ki] = zeta[ki] * zeta_prev[ki] * alpha_prev[i] / den;
                }
                hs(0, k, i) = alpha[i] * zeta_new[ki] / zeta[ki];
            }
        }
        for (int i = 0; i < nsys; ++i) hs(3, 0, i) = -alpha[i];
        DWF_CUDA(cudaMemcpyAsync(dS, h_sc.data(), h_sc.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        // shifts whose every system has converged are left alone (their updates
        // would be x += 0 p, p = 0 r + 1 p: whole fields streamed for nothing)
        auto shift_active = [&](int k) {
            for (int i = 0; i < nsys; ++i)
                if (act[(size_t)k * nsys + i]) return true;
            return false;
        };
        for (int k = 0; k < nshift; ++k)
            if (shift_active(k))
                DWF_TRY(launch_axpby(h, 1, nrhs, ds(0, k), 0.0, pk(k), DWF_FP64, nullptr, 1.0, xs(k),
                                     DWF_FP64, nullptr, T, s));
        // r -= alpha A p
        DWF_TRY(launch_axpby(h, 1, nrhs, ds(3, 0), 0.0, dAp, DWF_FP64, nullptr, 1.0, dR, DWF_FP64,
                             nullptr, T, s));
        DWF_TRY(sys_dot(h, dR, dR, DWF_FP64, nrhs, dPart, d_sys, rr_new, s));
        ++iter;
        // p_s = zeta_new r + beta_s p_s, beta_s = beta (zeta_new / zeta)^2
        std::vector<double> beta(nsys, 0.0);
        for (int i = 0; i < nsys; ++i) beta[i] = rr[i] > 0.0 ? rr_new[i] / rr[i] : 0.0;
        for (int k = 0; k < nshift; ++k)
            for (int i = 0; i < nsys; ++i) {
                const size_t ki = (size_t)k * nsys + i;
                if (!act[ki]) { hs(1, k, i) = 0.0; hs(2, k, i) = 1.0; continue; }
                const double q = zeta_new[ki] / zeta[ki];
                hs(1, k, i) = zeta_new[ki];
                hs(2, k, i) = beta[i] * q * q;
            }
        DWF_CUDA(cudaMemcpyAsync(dS, h_sc.data(), h_sc.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        for (int k = 0; k < nshift; ++k)
            if (shift_active(k))
                DWF_TRY(launch_axpby(h, 1, nrhs, ds(1, k), 0.0, dR, DWF_FP64, ds(2, k), 0.0, pk(k),
                                     DWF_FP64, nullptr, T, s));
        // convergence of every (shift, system): |r^(s)| = |zeta_new| |r|; a system
        // whose base shift converged stops all its shifts (they are better
        // conditioned and have converged already in exact arithmetic)
        for (int k = 0; k < nshift; ++k)
            for (int i = 0; i < nsys; ++i) {
                const size_t ki = (size_t)k * nsys + i;
                if (!act[ki]) continue;
                its[ki] = iter;
                if (!std::isfinite(rr_new[i])) { result = DWF_ERR_NAN; act[ki] = 0; continue; }
                if (std::fabs(zeta_new[ki]) * std::sqrt(rr_new[i]) <= sp->tol * std::sqrt(bn2[i]))
                    act[ki] = 0;
            }
        for (int i = 0; i < nsys; ++i)
            if (!act[i])
                for (int k = 1; k < nshift; ++k) act[(size_t)k * nsys + i] = 0;
        zeta_prev = zeta;
        zeta = zeta_new;
        for (int i = 0; i < nsys; ++i) {
            alpha_prev[i] = alpha[i] != 0.0 ? alpha[i] : alpha_prev[i];
            beta_prev[i] = beta[i];
        }
        rr = rr_new;
    }
    // true residual of every shift in FP64: |b - (A + sigma_s) x_s| / |b|
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < nshift; ++k) {
        std::vector<double> res2(nsys);
        DWF_TRY(op_mpc(h, dT, xs(k), 0, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
        DWF_TRY(op_mpc(h, dAp, dT, 1, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
        if (shifts[ord[k]] != 0.0)
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, shifts[ord[k]], xs(k), DWF_FP64, nullptr, 1.0,
                                 dAp, DWF_FP64, nullptr, T, s));
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, b, DWF_FP64, nullptr, -1.0, dAp, DWF_FP64,
                             nullptr, T, s));
        DWF_TRY(sys_dot(h, dAp, dAp, DWF_FP64, nrhs, dPart, d_sys, res2, s));
        for (int i = 0; i < nsys; ++i) {
            dwf_solver_stats& st = stats[(size_t)ord[k] * nsys + i];
            const double tr = bn2[i] > 0.0 ? std::sqrt(res2[i] / bn2[i]) : 0.0;
            st.iters = its[(size_t)k * nsys + i];
            st.reliable_updates = 0;
            st.op_applies = 2 * iter;
            st.true_resid = tr;
            st.seconds = secs;
            st.recorded = 0;
            st.status = !std::isfinite(tr) ? DWF_ERR_NAN
                        : tr <= 2.0 * sp->tol ? DWF_OK
                        : (result == DWF_OK ? DWF_ERR_NOT_CONVERGED : result);
        }
    }
    DWF_CUDA(cudaStreamSynchronize(s));
    if (!report) return result;
    for (int k = 0; k < nshift; ++k)
        for (int i = 0; i < nsys; ++i)
            if (stats[(size_t)ord[k] * nsys + i].status != DWF_OK) {
                const dwf_status st = (dwf_status)stats[(size_t)ord[k] * nsys + i].status;
                set_error("dwf_multishift_solve: shift %d system %d: true residual %.3e (tol %.1e)",
                          ord[k], i, stats[(size_t)ord[k] * nsys + i].true_resid, sp->tol);
                return st;
            }
    return DWF_OK;
}

// FP64 operator: one multi-shift CG.  FP32 operator: the multi-shift CG to
// the FP32 operator's reach (1e-6), then defect correction for every shift
// still above tol: r_s = b - (A + sigma_s) x_s in FP64 (done by the core's
// true-residual step), (A + sigma_s) e_s = r_s solved with the FP32 operator
// to 1e-6 relative, x_s += e_s; each round gains ~six digits.
dwf_status multishift_solve(dwf_handle* h, double* x, const double* b, const double* shifts,
                            int nshift, int nrhs, const dwf_solver_params* sp,
                            dwf_solver_stats* stats, cudaStream_t s) {
    if (sp == nullptr || sp->inner_prec != DWF_FP32 || !(sp->tol < 1e-6) || x == nullptr ||
        b == nullptr || shifts == nullptr || stats == nullptr || nshift < 1 || nrhs < 1 ||
        nrhs > h->nrhs_max)
        return multishift_core(h, x, b, shifts, nshift, nrhs, sp, stats, s, true);
    const auto t0 = std::chrono::steady_clock::now();
    const int nsys = h->nbox * nrhs;
    const size_t no = cb_elems(h, 1, nrhs);
    const int T = tile_for(h, nrhs);
    dwf_solver_params sp1 = *sp;
    sp1.tol = 1e-6;
    dwf_status st = multishift_core(h, x, b, shifts, nshift, nrhs, &sp1, stats, s, false);
    if (st != DWF_OK && st != DWF_ERR_NOT_CONVERGED) return st;
    DevBuf r, e, t, tA, tB;
    DWF_TRY(dev_alloc(r, no * 16));
    DWF_TRY(dev_alloc(e, no * 16));
    DWF_TRY(dev_alloc(t, no * 16));
    DWF_TRY(dev_alloc(tA, no * 16));
    DWF_TRY(dev_alloc(tB, no * 16));
    std::vector<dwf_solver_stats> st1(nsys);
    std::vector<int> corr(nshift, 0);
    for (int round = 0; round < 4; ++round) {
        bool all = true;
        for (int k = 0; k < nshift; ++k) {
            bool ok = true;
            for (int i = 0; i < nsys; ++i) ok &= stats[(size_t)k * nsys + i].true_resid <= sp->tol;
            if (ok) continue;
            all = false;
            // r = b - (A + sigma_k) x_k
            double* xk = x + (size_t)k * no * 2;
            double* dr = static_cast<double*>(r.p);
            DWF_TRY(op_mpc(h, t.p, xk, 0, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
            DWF_TRY(op_mpc(h, dr, t.p, 1, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
            if (shifts[k] != 0.0)
                DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, shifts[k], xk, DWF_FP64, nullptr, 1.0, dr,
                                     DWF_FP64, nullptr, T, s));
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, b, DWF_FP64, nullptr, -1.0, dr, DWF_FP64,
                                 nullptr, T, s));
            // (A + sigma_k) e = r in FP32, x_k += e
            st = multishift_core(h, static_cast<double*>(e.p), dr, &shifts[k], 1, nrhs, &sp1,
                                 st1.data(), s, false);
            if (st != DWF_OK && st != DWF_ERR_NOT_CONVERGED) return st;
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, e.p, DWF_FP64, nullptr, 1.0, xk, DWF_FP64,
                                 nullptr, T, s));
            ++corr[k];
            // the new true residual relative to |b|: recompute through the core's
            // FP64 check with a zero-iteration solve is wasteful; do it here
            DWF_TRY(op_mpc(h, t.p, xk, 0, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
            DWF_TRY(op_mpc(h, dr, t.p, 1, DWF_FP64, DWF_FP64, nrhs, tA.p, tB.p, nullptr, nullptr, s));
            if (shifts[k] != 0.0)
                DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, shifts[k], xk, DWF_FP64, nullptr, 1.0, dr,
                                     DWF_FP64, nullptr, T, s));
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 1.0, b, DWF_FP64, nullptr, -1.0, dr, DWF_FP64,
                                 nullptr, T, s));
            std::vector<double> rn(nsys), bn(nsys);
            DevBuf part, d2;
            const TileSet* tsp = nullptr;
            DWF_TRY(get_tiles(h, T, &tsp));
            DWF_TRY(dev_alloc(part, (size_t)tsp->ntiles[1] * nrhs * sizeof(double)));
            DWF_TRY(dev_alloc(d2, (size_t)nsys * sizeof(double)));
            DWF_TRY(sys_dot(h, dr, dr, DWF_FP64, nrhs, static_cast<double*>(part.p),
                            static_cast<double*>(d2.p), rn, s));
            DWF_TRY(sys_dot(h, b, b, DWF_FP64, nrhs, static_cast<double*>(part.p),
                            static_cast<double*>(d2.p), bn, s));
            for (int i = 0; i < nsys; ++i) {
                dwf_solver_stats& sk = stats[(size_t)k * nsys + i];
                sk.true_resid = bn[i] > 0 ? std::sqrt(rn[i] / bn[i]) : 0.0;
                sk.iters += st1[i].iters;
                sk.op_applies += st1[i].op_applies + 4;
                sk.reliable_updates = corr[k];
            }
        }
        if (all) break;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    dwf_status res = DWF_OK;
    for (int k = 0; k < nshift; ++k)
        for (int i = 0; i < nsys; ++i) {
            dwf_solver_stats& sk = stats[(size_t)k * nsys + i];
            sk.seconds = secs;
            sk.status = !std::isfinite(sk.true_resid) ? DWF_ERR_NAN
                        : sk.true_resid <= sp->tol ? DWF_OK : DWF_ERR_NOT_CONVERGED;
            if (sk.status != DWF_OK && res == DWF_OK) {
                res = (dwf_status)sk.status;
                set_error("dwf_multishift_solve: shift %d system %d: true residual %.3e (tol %.1e)", k,
                          i, sk.true_resid, sp->tol);
            }
        }
    return res;
}

// r(A) b = a0 b + sum_i residues_i (A + shifts_i)^-1 b, A = M_pc^+ M_pc (each
// box's on a box handle): a rational function in partial fractions, the form
// the DD-RHMC action takes for the powers of the normal operators of D and
// D_Omega (Sec. 2.3.1), from one multi-shift solve.
dwf_status rational_apply(dwf_handle* h, double* out, const double* in, double a0, const double* shifts,
                          const double* residues, int n, int nrhs, const dwf_solver_params* sp,
                          dwf_solver_stats* stats, cudaStream_t s) {
    if (out == nullptr || in == nullptr || out == in || residues == nullptr || n < 1 || nrhs < 1 ||
        nrhs > h->nrhs_max) {
        set_error("rational: bad arguments (distinct fields, n >= 1, 1 <= nrhs <= nrhs_max)");
        return DWF_ERR_ARG;
    }
    const size_t no = cb_elems(h, 1, nrhs);
    const int T = tile_for(h, nrhs);
    DevBuf x;
    DWF_TRY(dev_alloc(x, (size_t)n * no * 16));
    double* xs = static_cast<double*>(x.p);
    const dwf_status st = multishift_solve(h, xs, in, shifts, n, nrhs, sp, stats, s);
    if (st != DWF_OK && st != DWF_ERR_NOT_CONVERGED) return st;
    DWF_CUDA(cudaMemsetAsync(out, 0, no * 16, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, a0, in, DWF_FP64, nullptr, 1.0, out, DWF_FP64, nullptr, T, s));
    for (int i = 0; i < n; ++i)
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, residues[i], xs + (size_t)i * no * 2, DWF_FP64, nullptr, 1.0,
                             out, DWF_FP64, nullptr, T, s));
    DWF_CUDA(cudaStreamSynchronize(s));
    return st;
}

// ------------------------------------------------------------------------
// Zolotarev's optimal relative approximation of 1/sqrt(x) on [lo, hi] in
// partial fractions (host only).  On y = x / lo in [1, b] with m' = 1 - 1/b,
// K' = K(m'), c_l = sn^2 / cn^2 (l K' / (2n) | m') for l = 1 .. 2n-1,
//     r(y) = d0 prod_{i<n} (y + c_{2i}) / prod_{j<=n} (y + c_{2j-1}),
// d0 centring the relative error so that it equioscillates (found on a dense
// geometric grid).  Jacobi sn, cn and K by the arithmetic-geometric-mean
// (descending Landen) sequence, with the complementary parameter passed
// exactly (m1 = 1/b) so nothing cancels as m' -> 1.
void jacobi_sn_cn(double u, double m, double m1, double* sn, double* cn, double* K) {
    double a[64], c[64];
    a[0] = 1.0;
    c[0] = std::sqrt(m);
    double b = std::sqrt(m1);
    int N = 0;
    while (std::fabs(c[N]) > 1e-17 * a[N] && N < 60) {
        const double an = 0.5 * (a[N] + b), bn = std::sqrt(a[N] * b);
        c[N + 1] = 0.5 * (a[N] - b);
        a[N + 1] = an;
        b = bn;
        ++N;
    }
    double phi = std::ldexp(1.0, N) * a[N] * u;
    for (int k = N; k >= 1; --k) phi = 0.5 * (phi + std::asin(c[k] / a[k] * std::sin(phi)));
    if (sn) *sn = std::sin(phi);
    if (cn) *cn = std::cos(phi);
    if (K) *K = 3.14159265358979323846 / (2.0 * a[N]);
}

dwf_status zolotarev_inv_sqrt(int n, double lo, double hi, double* shifts, double* residues, double* delta) {
    if (n < 1 || n > 64 || !(lo > 0.0) || !(hi > lo) || shifts == nullptr || residues == nullptr) {
        set_error("zolotarev: need 1 <= n <= 64, 0 < lo < hi and output arrays");
        return DWF_ERR_ARG;
    }
    const double b = hi / lo, m1 = 1.0 / b, m = 1.0 - m1;
    double Kp = 0.0;
    jacobi_sn_cn(0.0, m, m1, nullptr, nullptr, &Kp);
    std::vector<double> c(2 * n);   // c[l], l = 1 .. 2n - 1
    for (int l = 1; l < 2 * n; ++l) {
        double sn = 0.0, cn = 1.0;
        jacobi_sn_cn(l * Kp / (2.0 * n), m, m1, &sn, &cn, nullptr);
        c[l] = sn * sn / (cn * cn);
    }
    // d0: centre sqrt(y) r(y) between its extremes on [1, b]
    const int G = 200001;
    double emax = -1e300, emin = 1e300;
    for (int g = 0; g < G; ++g) {
        const double y = std::exp(std::log(b) * g / (G - 1));
        double v = std::sqrt(y);
        for (int i = 1; i < n; ++i) v *= y + c[2 * i];
        for (int j = 1; j <= n; ++j) v /= y + c[2 * j - 1];
        emax = std::max(emax, v);
        emin = std::min(emin, v);
    }
    const double d0 = 2.0 / (emax + emin);
    if (delta) *delta = (emax - emin) / (emax + emin);
    for (int j = 1; j <= n; ++j) {
        const double p = c[2 * j - 1];
        double R = 1.0;
        for (int i = 1; i < n; ++i) R *= c[2 * i] - p;
        for (int k = 1; k <= n; ++k)
            if (k != j) R /= c[2 * k - 1] - p;
        shifts[j - 1] = lo * p;
        residues[j - 1] = d0 * std::sqrt(lo) * R;
    }
    return DWF_OK;
}

}  // namespace dwf
