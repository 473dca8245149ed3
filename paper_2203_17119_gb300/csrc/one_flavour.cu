// The one-flavour DD-RHMC boundary term of Sec. 2.3.1 (eq. ddrhmc): the
// boundary determinant det D / det D_dirichlet simulated with one RHMC
// pseudofermion phi on the odd checkerboard,
//
//     S = phi^+ r1(A_d) r2(A) r1(A_d) phi,   r1 ~ x^(1/4), r2 ~ x^(-1/2),
//
// A = M_pc^+ M_pc of D (handle h) and A_d that of D_dirichlet (handle hd, the
// whole-lattice handle of D with the links between domains left out,
// dwf_create_cut).  The even-even blocks of D and D_dirichlet are the same
// site-local M_ee, so det D / det D_dirichlet = det M_pc / det M_pc,d and the
// Schur operators carry the whole ratio.
//
// With w = r1(A_d) phi, v = r2(A) w and, per pole,
//     z_j = (A_d + s1_j)^-1 phi,  y_j = (A_d + s1_j)^-1 v,  x_i = (A + s2_i)^-1 w,
// the variation of S is (A, A_d Hermitian, dA = dM^+ M + M^+ dM)
//     dS = -2 sum_i rho2_i Re <M x_i, dM x_i>
//          -2 sum_j rho1_j (Re <M_d z_j, dM_d y_j> + Re <M_d y_j, dM_d z_j>),
// and a Schur bilinear Re <X_o, dM_pc Y_o> is minus the full-operator bilinear
// Re <X, dD Y> of X = (V_e, X_o), Y = (W_e, Y_o) with W_e = M_ee^-1 M_eo Y_o
// and V_e = (M_ee^+)^-1 (M_oe)^+ X_o (the hops are the only link-dependent
// blocks; the cross terms of the two pieces vanish because dD only couples
// opposite parities) -- one call of the force insertion per bilinear.  On hd
// the left-out links get no force (their table entries are zero, and so is
// -1/2 TA(U M) there).
//
// GB300 layout of the work: three multi-shift solves (every pole of r1 or r2
// from one Krylov space each), then per pole one M_pc and per bilinear two
// off-diagonal hops, two site-local M_ee^-1 and one force launch on FP64 fields.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dwf_internal.cuh"

namespace dwf {

namespace {

struct Buf {
    void* p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    double* d() const { return static_cast<double*>(p); }
};

dwf_status alloc(Buf& b, size_t bytes) {
    DWF_CUDA(dev_malloc(&b.p, bytes ? bytes : 16));
    return DWF_OK;
}

dwf_status check_rational(const dwf_rational* r, const char* which) {
    if (r == nullptr || r->n < 1 || r->shifts == nullptr || r->residues == nullptr || !std::isfinite(r->a0)) {
        set_error("one-flavour: rational function %s needs n >= 1, shifts, residues and a finite a0", which);
        return DWF_ERR_ARG;
    }
    for (int i = 0; i < r->n; ++i)
        if (!(r->shifts[i] >= 0.0) || !std::isfinite(r->shifts[i]) || !std::isfinite(r->residues[i])) {
            set_error("one-flavour: rational function %s: shifts must be finite and >= 0, residues finite", which);
            return DWF_ERR_ARG;
        }
    return DWF_OK;
}

// h and hd: two whole-lattice handles of the same lattice and action on the
// current device, hd cut into domains, h not.
dwf_status check_pair(const dwf_handle* h, const dwf_handle* hd, int nrhs) {
    if (h == nullptr || hd == nullptr || h == hd) {
        set_error("one-flavour: need two distinct handles (D and D_dirichlet)");
        return DWF_ERR_ARG;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (h->device != dev || hd->device != dev) {
        set_error("one-flavour: the handles belong to another device");
        return DWF_ERR_ARG;
    }
    const dwf_params &a = h->p, &b = hd->p;
    bool same = a.Ls == b.Ls && a.M5 == b.M5 && a.mf == b.mf && a.b5 == b.b5 && a.c5 == b.c5;
    for (int mu = 0; mu < 4; ++mu) same = same && a.dims[mu] == b.dims[mu];
    if (!same || h->dirichlet || hd->dirichlet || !h->cut.empty() || hd->cut.empty()) {
        set_error("one-flavour: h must be a whole-lattice handle of D and hd the dwf_create_cut handle of the "
                  "same lattice and action");
        return DWF_ERR_ARG;
    }
    if (!h->have_gauge || !hd->have_gauge) {
        set_error("one-flavour: no gauge field loaded (dwf_set_gauge on both handles)");
        return DWF_ERR_ARG;
    }
    if (nrhs < 1 || nrhs > h->nrhs_max || nrhs > hd->nrhs_max) {
        set_error("one-flavour: nrhs = %d outside [1, nrhs_max of both handles]", nrhs);
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

// out = a0 in + sum_i rho_i xs_i (odd cb FP64 fields, xs back to back)
dwf_status combine(dwf_handle* h, double* out, const double* in, const dwf_rational& r, const double* xs,
                   int nrhs, cudaStream_t s) {
    const size_t no = cb_elems(h, 1, nrhs);
    const int T = tile_for(h, nrhs);
    DWF_CUDA(cudaMemsetAsync(out, 0, no * 16, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, r.a0, in, DWF_FP64, nullptr, 1.0, out, DWF_FP64, nullptr, T, s));
    for (int i = 0; i < r.n; ++i)
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, r.residues[i], xs + i * no * 2, DWF_FP64, nullptr, 1.0, out,
                             DWF_FP64, nullptr, T, s));
    return DWF_OK;
}

// out (+)= coef F(X, Y), X = (V_e, coef-free X_o), Y = (W_e, Y_o): the link
// force of -coef Re <X_o, M_pc Y_o>.  X, Y: full FP64 work fields; te: an even
// cb FP64 work field.
dwf_status schur_force(dwf_handle* h, double* out, const double* Xo, const double* Yo, double coef, int nrhs,
                       const dwf_box* active, int accumulate, double* X, double* Y, double* te,
                       cudaStream_t s) {
    const size_t ne = cb_elems(h, 0, nrhs), no = cb_elems(h, 1, nrhs);
    const int T = tile_for(h, nrhs);
    double* Xe = X;
    double* Xodd = X + 2 * ne;
    double* Ye = Y;
    double* Yodd = Y + 2 * ne;
    DWF_CUDA(cudaMemsetAsync(Xodd, 0, no * 16, s));
    DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, coef, Xo, DWF_FP64, nullptr, 0.0, Xodd, DWF_FP64, nullptr, T, s));
    DWF_TRY(op_dslash_eo(h, te, Xodd, 0, 1, DWF_FP64, nrhs, h->d_tmp, s));
    DWF_TRY(op_local(h, L_MINV, Xe, te, nullptr, 0, 1, DWF_FP64, DWF_FP64, DWF_FP64, nrhs, 1.0, nullptr, s));
    DWF_CUDA(cudaMemcpyAsync(Yodd, Yo, no * 16, cudaMemcpyDeviceToDevice, s));
    DWF_TRY(op_dslash_eo(h, te, Yo, 0, 0, DWF_FP64, nrhs, h->d_tmp, s));
    DWF_TRY(op_local(h, L_MINV, Ye, te, nullptr, 0, 0, DWF_FP64, DWF_FP64, DWF_FP64, nrhs, 1.0, nullptr, s));
    return force_bilinear(h, out, X, Y, DWF_FP64, nrhs, active, accumulate, s);
}

// per-rhs Re <a, b> of odd cb FP64 fields (whole lattice: one system per rhs)
dwf_status rhs_dot(dwf_handle* h, const double* a, const double* b, int nrhs, double* out, cudaStream_t s) {
    const int T = tile_for(h, nrhs);
    const TileSet* ts = nullptr;
    DWF_TRY(get_tiles(h, T, &ts));
    Buf part, red;
    DWF_TRY(alloc(part, (size_t)ts->ntiles[1] * nrhs * sizeof(double)));
    DWF_TRY(alloc(red, (size_t)nrhs * sizeof(double)));
    DWF_TRY(launch_dot_partial(h, 1, a, b, DWF_FP64, DWF_FP64, nrhs, part.d(), T, s));
    DWF_TRY(launch_reduce_sys(h, 1, part.d(), nrhs, red.d(), T, s));
    DWF_CUDA(cudaMemcpyAsync(out, red.d(), nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    DWF_CUDA(cudaStreamSynchronize(s));
    return DWF_OK;
}

// w = r1(A_d) phi, v = r2(A) w with the pole solutions kept (zs: n1 fields,
// xs: n2 fields); stats: [n1 * nrhs] then [n2 * nrhs].
dwf_status action_pieces(dwf_handle* h, dwf_handle* hd, const double* phi, int nrhs, const dwf_rational& r1,
                         const dwf_rational& r2, const dwf_solver_params* sp, dwf_solver_stats* stats,
                         double* zs, double* xs, double* w, double* v, cudaStream_t s) {
    dwf_status st = multishift_solve(hd, zs, phi, r1.shifts, r1.n, nrhs, sp, stats, s);
    if (st != DWF_OK) return st;
    DWF_TRY(combine(hd, w, phi, r1, zs, nrhs, s));
    st = multishift_solve(h, xs, w, r2.shifts, r2.n, nrhs, sp, stats + (size_t)r1.n * nrhs, s);
    if (st != DWF_OK) return st;
    return combine(h, v, w, r2, xs, nrhs, s);
}

}  // namespace

dwf_status one_flavour_action(dwf_handle* h, dwf_handle* hd, const double* phi, int nrhs, const dwf_rational* r1,
                              const dwf_rational* r2, const dwf_solver_params* sp, double* S,
                              dwf_solver_stats* stats, cudaStream_t s) {
    DWF_TRY(check_pair(h, hd, nrhs));
    DWF_TRY(check_rational(r1, "r1"));
    DWF_TRY(check_rational(r2, "r2"));
    if (phi == nullptr || S == nullptr || sp == nullptr || stats == nullptr) {
        set_error("one-flavour action: null field, output, solver parameters or stats");
        return DWF_ERR_ARG;
    }
    const size_t no = cb_elems(h, 1, nrhs), f = no * 16;
    Buf zs, xs, w, v;
    DWF_TRY(alloc(zs, f * r1->n));
    DWF_TRY(alloc(xs, f * r2->n));
    DWF_TRY(alloc(w, f));
    DWF_TRY(alloc(v, f));
    const dwf_status st = action_pieces(h, hd, phi, nrhs, *r1, *r2, sp, stats, zs.d(), xs.d(), w.d(), v.d(), s);
    if (st != DWF_OK) {
        cudaStreamSynchronize(s);
        return st;
    }
    return rhs_dot(h, w.d(), v.d(), nrhs, S, s);
}

dwf_status one_flavour_force(dwf_handle* h, dwf_handle* hd, double* out, const double* phi, int nrhs,
                             const dwf_rational* r1, const dwf_rational* r2, const dwf_box* active, int accumulate,
                             const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t s) {
    DWF_TRY(check_pair(h, hd, nrhs));
    DWF_TRY(check_rational(r1, "r1"));
    DWF_TRY(check_rational(r2, "r2"));
    if (out == nullptr || phi == nullptr || sp == nullptr || stats == nullptr) {
        set_error("one-flavour force: null output, field, solver parameters or stats");
        return DWF_ERR_ARG;
    }
    const size_t no = cb_elems(h, 1, nrhs), f = no * 16;
    Buf zs, ys, xs, w, v, m, X, Y, te;
    DWF_TRY(alloc(zs, f * r1->n));
    DWF_TRY(alloc(ys, f * r1->n));
    DWF_TRY(alloc(xs, f * r2->n));
    DWF_TRY(alloc(w, f));
    DWF_TRY(alloc(v, f));
    DWF_TRY(alloc(m, f));
    DWF_TRY(alloc(X, 2 * f));
    DWF_TRY(alloc(Y, 2 * f));
    DWF_TRY(alloc(te, f));
    auto run = [&]() -> dwf_status {
        dwf_status st = action_pieces(h, hd, phi, nrhs, *r1, *r2, sp, stats, zs.d(), xs.d(), w.d(), v.d(), s);
        if (st != DWF_OK) return st;
        st = multishift_solve(hd, ys.d(), v.d(), r1->shifts, r1->n, nrhs, sp,
                              stats + (size_t)(r1->n + r2->n) * nrhs, s);
        if (st != DWF_OK) return st;
        int acc = accumulate;
        // the r2 poles: 2 rho2_i F(M x_i, x_i) on D
        for (int i = 0; i < r2->n; ++i) {
            const double* x = xs.d() + i * no * 2;
            DWF_TRY(op_mpc(h, m.d(), x, 0, DWF_FP64, DWF_FP64, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
            DWF_TRY(schur_force(h, out, m.d(), x, 2.0 * r2->residues[i], nrhs, active, acc, X.d(), Y.d(), te.d(),
                                s));
            acc = 1;
        }
        // the r1 poles: 2 rho1_j (F(M_d z_j, y_j) + F(M_d y_j, z_j)) on D_dirichlet
        for (int j = 0; j < r1->n; ++j) {
            const double* z = zs.d() + j * no * 2;
            const double* y = ys.d() + j * no * 2;
            const double c = 2.0 * r1->residues[j];
            DWF_TRY(op_mpc(hd, m.d(), z, 0, DWF_FP64, DWF_FP64, nrhs, hd->d_tmp, hd->d_tmp2, nullptr, nullptr, s));
            DWF_TRY(schur_force(hd, out, m.d(), y, c, nrhs, active, acc, X.d(), Y.d(), te.d(), s));
            DWF_TRY(op_mpc(hd, m.d(), y, 0, DWF_FP64, DWF_FP64, nrhs, hd->d_tmp, hd->d_tmp2, nullptr, nullptr, s));
            DWF_TRY(schur_force(hd, out, m.d(), z, c, nrhs, active, 1, X.d(), Y.d(), te.d(), s));
        }
        return DWF_OK;
    };
    const dwf_status st = run();
    cudaStreamSynchronize(s);
    return st;
}

dwf_status one_flavour_heatbath(dwf_handle* h, dwf_handle* hd, double* phi, const double* eta, int nrhs,
                                const dwf_rational* q1, const dwf_rational* q2, const dwf_solver_params* sp,
                                dwf_solver_stats* stats, cudaStream_t s) {
    DWF_TRY(check_pair(h, hd, nrhs));
    DWF_TRY(check_rational(q1, "q1"));
    DWF_TRY(check_rational(q2, "q2"));
    if (phi == nullptr || eta == nullptr || phi == eta || sp == nullptr || stats == nullptr) {
        set_error("one-flavour heat bath: need distinct phi and eta, solver parameters and stats");
        return DWF_ERR_ARG;
    }
    const size_t f = cb_elems(h, 1, nrhs) * 16;
    Buf t;
    DWF_TRY(alloc(t, f));
    // t = q2(A) eta ~ A^(1/4) eta, then phi = q1(A_d) t ~ A_d^(-1/4) t
    dwf_status st = rational_apply(h, t.d(), eta, q2->a0, q2->shifts, q2->residues, q2->n, nrhs, sp, stats, s);
    if (st != DWF_OK) return st;
    st = rational_apply(hd, phi, t.d(), q1->a0, q1->shifts, q1->residues, q1->n, nrhs, sp,
                        stats + (size_t)q2->n * nrhs, s);
    return st;
}

}  // namespace dwf
