// The boundary operator of Sec. 2.1 and the inverse the DD-HMC pseudofermion
// action uses:
//
//   R^-1 = P - P D^-1 D_partialbar,
//
// on the space projected by P (Luescher's projector): the spinor components of
// Omega on which D_partialbar, the hops from Omega to Omega-bar, act.  P is the
// orthogonal projector onto the row space of D_partialbar.  D_partialbar's
// column block at a site x of Omega is a sum of terms
// -1/2 (1 -+ gamma_mu) U (b5 + c5 S5) over the neighbours of x outside Omega
// ((1 - gamma_mu) for x - mu, (1 + gamma_mu) for x + mu), so its row space is
// colour-blind and, in the (spin, s) space of the site, the span of
// B^+ [range(1 -+ gamma_mu) x C^Ls] over those neighbours, B^+ = b5 + c5 S5^+.
// It depends on the site only through which neighbours leave Omega: one
// 4 Ls x 4 Ls projector per crossing pattern, built on the host in FP64
// (Gram-Schmidt of those columns), one pattern index per site.
//
// R^-1 psi: u = P psi, v = D u restricted to Omega-bar (= D_partialbar u),
// y = D^-1 v (the mixed-precision CGNE of the whole lattice), out = u - P y.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <map>
#include <vector>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

namespace {

using cd = std::complex<double>;

// Chiral-basis gamma_mu (mu = 0..3 <-> x..t), 4 x 4 row-major.
std::array<cd, 16> gamma_mu(int mu) {
    std::array<cd, 16> g{};
    const cd I(0, 1);
    // sigma_1, sigma_2, sigma_3
    const cd sig[3][4] = {{0, 1, 1, 0}, {0, -I, I, 0}, {1, 0, 0, -1}};
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            cd up, lo;
            if (mu < 3) {
                up = -I * sig[mu][r * 2 + c];
                lo = I * sig[mu][r * 2 + c];
            } else {
                up = lo = (r == c) ? 1.0 : 0.0;
            }
            g[r * 4 + (c + 2)] = up;   // upper right block
            g[(r + 2) * 4 + c] = lo;   // lower left block
        }
    return g;
}

// Projector (4 Ls x 4 Ls, row-major, index spin * Ls + s) onto the span of
// B^+ [range(1 + sgn gamma_mu) x C^Ls] over the crossings of `mask` (bit k:
// neighbour k = mu (+mu) or 4 + mu (-mu) lies outside Omega).
std::vector<cd> pattern_projector(int mask, int Ls, double b5, double c5, double mf) {
    const int n = 4 * Ls;
    // B^+ = b5 + c5 (P_+ S_+ + P_- S_-) on (spin, s): upper spins shift s+1, lower s-1
    auto Bdag = [&](const std::vector<cd>& v) {
        std::vector<cd> w(n);
        for (int sp = 0; sp < 4; ++sp)
            for (int s = 0; s < Ls; ++s) {
                cd sh;
                if (sp < 2) sh = s < Ls - 1 ? v[sp * Ls + s + 1] : -mf * v[sp * Ls + 0];
                else sh = s > 0 ? v[sp * Ls + s - 1] : -mf * v[sp * Ls + Ls - 1];
                w[sp * Ls + s] = b5 * v[sp * Ls + s] + c5 * sh;
            }
        return w;
    };
    std::vector<std::vector<cd>> Q;
    for (int k = 0; k < 8 && (int)Q.size() < n; ++k) {
        if (!(mask >> k & 1)) continue;
        const int mu = k & 3;
        const double sgn = k < 4 ? 1.0 : -1.0;   // x + mu: (1 + gamma), x - mu: (1 - gamma)
        const auto g = gamma_mu(mu);
        for (int col = 0; col < 4; ++col)
            for (int s = 0; s < Ls && (int)Q.size() < n; ++s) {   // a full basis spans everything
                std::vector<cd> v(n, 0.0);
                for (int sp = 0; sp < 4; ++sp) v[sp * Ls + s] = (sp == col ? 1.0 : 0.0) + sgn * g[sp * 4 + col];
                std::vector<cd> w = Bdag(v);
                // modified Gram-Schmidt, twice for stability
                for (int pass = 0; pass < 2; ++pass)
                    for (const auto& q : Q) {
                        cd dot = 0;
                        for (int i = 0; i < n; ++i) dot += std::conj(q[i]) * w[i];
                        for (int i = 0; i < n; ++i) w[i] -= dot * q[i];
                    }
                double nn = 0;
                for (int i = 0; i < n; ++i) nn += std::norm(w[i]);
                nn = std::sqrt(nn);
                if (nn > 1e-10 * (std::fabs(b5) + std::fabs(c5) + 1.0)) {
                    for (int i = 0; i < n; ++i) w[i] /= nn;
                    Q.push_back(w);
                }
            }
    }
    std::vector<cd> P((size_t)n * n, 0.0);
    for (const auto& q : Q)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) P[(size_t)i * n + j] += q[i] * std::conj(q[j]);
    return P;
}

// out = P_pat(site) in on Omega's sites (pat >= 0), 0 elsewhere (pat < 0);
// in / out full fields [parity block][site][12][N5] complex (FP64).
__global__ void k_boundary_project(const double2* __restrict__ in, double2* __restrict__ out,
                                   const int* __restrict__ pat, const double2* __restrict__ P,
                                   int64_t nsites, int Ls, int nrhs) {
    const int n4 = 4 * Ls, N5 = Ls * nrhs;
    const int64_t total = nsites * 3 * nrhs * n4;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(id % n4);                 // spin * Ls + s
        const int64_t rest = id / n4;
        const int r = (int)(rest % nrhs);
        const int colour = (int)((rest / nrhs) % 3);
        const int64_t site = rest / (nrhs * 3);
        const int sp = row / Ls, s = row % Ls;
        const int p = pat[site];
        double2 acc = make_double2(0.0, 0.0);
        if (p >= 0) {
            const double2* Pr = P + ((size_t)p * n4 + row) * n4;
            const double2* src = in + site * 12 * N5;
            for (int j = 0; j < n4; ++j) {
                const int sj = j / Ls, tj = j % Ls;
                const double2 a = Pr[j];
                const double2 v = src[(sj * 3 + colour) * N5 + r * Ls + tj];
                acc.x += a.x * v.x - a.y * v.y;
                acc.y += a.x * v.y + a.y * v.x;
            }
        }
        out[site * 12 * N5 + (sp * 3 + colour) * N5 + r * Ls + s] = acc;
    }
}

// zero the sites whose flag equals `drop` (flag: 1 in Omega, 0 outside)
template <class V>   // double2 or float2
__global__ void k_mask(V* __restrict__ f, const int* __restrict__ in_omega, int64_t nsites, int per_site,
                       int drop) {
    const int64_t total = nsites * per_site;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x)
        if (in_omega[id / per_site] == drop) f[id] = V{0, 0};
}

// out = a - out
__global__ void k_rsub(double2* __restrict__ out, const double2* __restrict__ a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 o = out[i], x = a[i];
        out[i] = make_double2(x.x - o.x, x.y - o.y);
    }
}

// out = gamma_5 R_5 in: spins 2, 3 negated, s -> Ls - 1 - s (full FP64 fields)
__global__ void k_gamma5_r5(const double2* __restrict__ in, double2* __restrict__ out, int64_t nsites,
                            int Ls, int nrhs) {
    const int N5 = Ls * nrhs;
    const int64_t total = nsites * 12 * N5;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(id % N5);
        const int c = (int)((id / N5) % 12);
        const int r = l / Ls, sidx = l - r * Ls;
        const double2 v = in[id - l + r * Ls + (Ls - 1 - sidx)];
        out[id] = c < 6 ? v : make_double2(-v.x, -v.y);
    }
}

// out = factor * in where the site flag differs from `drop`, 0 elsewhere
__global__ void k_scale_mask(const double2* __restrict__ in, double2* __restrict__ out,
                             const int* __restrict__ in_omega, int64_t nsites, int per_site, int drop,
                             double factor) {
    const int64_t total = nsites * per_site;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = in[id];
        out[id] = in_omega[id / per_site] == drop ? make_double2(0.0, 0.0)
                                                  : make_double2(factor * v.x, factor * v.y);
    }
}

struct BoundaryTables {
    std::vector<int> pat, in_omega;   // per full-field site (parity 0 block, then parity 1)
    std::vector<cd> P;                 // [npat][4Ls][4Ls]
    int npat = 0;
};

dwf_status build_tables(const dwf_handle* h, const dwf_box& om, BoundaryTables& tb) {
    const int* L = h->p.dims;
    for (int mu = 0; mu < 4; ++mu)
        if (om.extent[mu] < 1 || om.extent[mu] > L[mu]) {
            set_error("boundary: Omega extent out of range");
            return DWF_ERR_ARG;
        }
    auto inside = [&](const int* x) {
        for (int mu = 0; mu < 4; ++mu) {
            const int d = ((x[mu] - om.origin[mu]) % L[mu] + L[mu]) % L[mu];
            if (d >= om.extent[mu]) return false;
        }
        return true;
    };
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    std::map<int, int> masks;
    std::vector<int> site_mask;
    // full-field site order: parity 0 sites in lexicographic order, then parity 1
    for (int q = 0; q < 2; ++q)
        for (int64_t l = 0; l < V; ++l) {
            int x[4] = {(int)(l % L[0]), (int)((l / L[0]) % L[1]), (int)((l / ((int64_t)L[0] * L[1])) % L[2]),
                        (int)(l / ((int64_t)L[0] * L[1] * L[2]))};
            if (((x[0] + x[1] + x[2] + x[3]) & 1) != q) continue;
            if (!inside(x)) {
                tb.in_omega.push_back(0);
                site_mask.push_back(-1);
                continue;
            }
            int m = 0;
            for (int k = 0; k < 8; ++k) {
                int y[4] = {x[0], x[1], x[2], x[3]};
                const int mu = k & 3;
                y[mu] = (y[mu] + (k < 4 ? 1 : -1) + L[mu]) % L[mu];
                if (!inside(y)) m |= 1 << k;
            }
            tb.in_omega.push_back(1);
            site_mask.push_back(m);
            if (m && !masks.count(m)) {
                const int id = (int)masks.size();
                masks[m] = id;
            }
        }
    // P is the direct sum of the per-site projectors only when no site of
    // Omega-bar touches two sites of Omega (a convex box, band width >= 2)
    for (int64_t l = 0; l < V; ++l) {
        int x[4] = {(int)(l % L[0]), (int)((l / L[0]) % L[1]), (int)((l / ((int64_t)L[0] * L[1])) % L[2]),
                    (int)(l / ((int64_t)L[0] * L[1] * L[2]))};
        if (inside(x)) continue;
        int cnt = 0;
        for (int k = 0; k < 8; ++k) {
            int y[4] = {x[0], x[1], x[2], x[3]};
            const int mu = k & 3;
            y[mu] = (y[mu] + (k < 4 ? 1 : -1) + L[mu]) % L[mu];
            if (inside(y)) ++cnt;
        }
        if (cnt > 1) {
            set_error("boundary: a site outside Omega touches %d sites of Omega (the projector is "
                      "site-local only for a band of width >= 2 around a box)", cnt);
            return DWF_ERR_UNSUPPORTED;
        }
    }
    tb.npat = (int)masks.size();
    const int n4 = 4 * h->p.Ls;
    tb.P.assign((size_t)std::max(tb.npat, 1) * n4 * n4, 0.0);
    for (const auto& kv : masks) {
        const auto Pm = pattern_projector(kv.first, h->p.Ls, h->p.b5, h->p.c5, h->p.mf);
        std::copy(Pm.begin(), Pm.end(), tb.P.begin() + (size_t)kv.second * n4 * n4);
    }
    tb.pat.resize(site_mask.size());
    for (size_t i = 0; i < site_mask.size(); ++i)
        tb.pat[i] = site_mask[i] > 0 ? masks[site_mask[i]] : -1;
    return DWF_OK;
}

struct DevTables {
    int* pat = nullptr;
    int* in_omega = nullptr;
    double2* P = nullptr;
    ~DevTables() {
        cudaFree(pat);
        cudaFree(in_omega);
        cudaFree(P);
    }
};

dwf_status upload(const BoundaryTables& tb, DevTables& dt) {
    DWF_CUDA(dev_malloc(&dt.pat, tb.pat.size() * sizeof(int)));
    DWF_CUDA(dev_malloc(&dt.in_omega, tb.in_omega.size() * sizeof(int)));
    DWF_CUDA(dev_malloc(&dt.P, tb.P.size() * sizeof(double2)));
    DWF_CUDA(cudaMemcpy(dt.pat, tb.pat.data(), tb.pat.size() * sizeof(int), cudaMemcpyHostToDevice));
    DWF_CUDA(cudaMemcpy(dt.in_omega, tb.in_omega.data(), tb.in_omega.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
    DWF_CUDA(cudaMemcpy(dt.P, tb.P.data(), tb.P.size() * sizeof(double2), cudaMemcpyHostToDevice));
    return DWF_OK;
}

// The tables of the last Omega, kept on the handle (building them is host
// work of O(volume) plus a Gram-Schmidt per crossing pattern).
struct BoundaryCache {
    int key[8];
    BoundaryTables tb;
    DevTables dt;
};

dwf_status cached_tables(dwf_handle* h, const dwf_box& om, const BoundaryTables** tb, const DevTables** dt) {
    auto* c = static_cast<BoundaryCache*>(h->boundary_cache);
    const int key[8] = {om.origin[0], om.origin[1], om.origin[2], om.origin[3],
                        om.extent[0], om.extent[1], om.extent[2], om.extent[3]};
    if (c == nullptr || !std::equal(key, key + 8, c->key)) {
        delete c;
        h->boundary_cache = nullptr;
        c = new BoundaryCache();
        std::copy(key, key + 8, c->key);
        dwf_status st = build_tables(h, om, c->tb);
        if (st == DWF_OK) st = upload(c->tb, c->dt);
        if (st != DWF_OK) {
            delete c;
            return st;
        }
        h->boundary_cache = c;
    }
    *tb = &c->tb;
    *dt = &c->dt;
    return DWF_OK;
}

dwf_status project(const dwf_handle* h, const DevTables& dt, const double* in, double* out, int nrhs,
                   cudaStream_t s) {
    const int64_t ns = h->nsite[0] + h->nsite[1];
    const int64_t total = ns * 3 * nrhs * 4 * h->p.Ls;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    k_boundary_project<<<grid, 256, 0, s>>>(reinterpret_cast<const double2*>(in),
                                             reinterpret_cast<double2*>(out), dt.pat, dt.P, ns,
                                             h->p.Ls, nrhs);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

dwf_status check_whole(const dwf_handle* h, const void* out, const void* in, int nrhs) {
    if (h->dirichlet) {
        set_error("boundary: needs a whole-lattice handle (Omega is given separately)");
        return DWF_ERR_ARG;
    }
    if (out == nullptr || in == nullptr || out == in || nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("boundary: bad arguments (distinct device fields, 1 <= nrhs <= nrhs_max)");
        return DWF_ERR_ARG;
    }
    if (!h->have_gauge) {
        set_error("boundary: no gauge field loaded");
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// B^-+ (per parity, FP64 closed form with d = b5, e = c5) or B (site-local)
dwf_status five_b_full(dwf_handle* h, double* out, const double* in, int nrhs, bool inverse_adjoint,
                       cudaStream_t s) {
    const size_t off1 = cb_elems(h, 0, nrhs) * 2;   // doubles
    FiveD fb = h->f5[0];
    fb.d = h->p.b5;
    fb.e = h->p.c5;
    fb.a = -fb.e / fb.d;
    fb.inv_d = 1.0 / fb.d;
    double aL = 1.0;
    for (int i = 0; i < h->p.Ls; ++i) aL *= fb.a;
    fb.inv_den = 1.0 / (fb.d * (1.0 + h->p.mf * aL));
    for (int p = 0; p < 2; ++p) {
        LocalCall c{};
        c.op = inverse_adjoint ? L_MINV : L_B;
        c.in = in + (p ? off1 : 0);
        c.out = out + (p ? off1 : 0);
        c.parity = p;
        c.dagger = inverse_adjoint ? 1 : 0;
        c.prec_in = c.prec_in2 = c.prec_out = DWF_FP64;
        c.nrhs = nrhs;
        c.scale = 1.0;
        c.f5 = inverse_adjoint ? &fb : nullptr;
        DWF_TRY(launch_local(h, c, s));
    }
    return DWF_OK;
}

}  // namespace

dwf_status boundary_project(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                            cudaStream_t s) {
    DWF_TRY(check_whole(h, out, in, nrhs));
    if (omega == nullptr) { set_error("boundary: null Omega"); return DWF_ERR_ARG; }
    const BoundaryTables* tb = nullptr;
    const DevTables* dt = nullptr;
    DWF_TRY(cached_tables(h, *omega, &tb, &dt));
    return project(h, *dt, in, out, nrhs, s);
}

dwf_status boundary_rinv(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                         const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t s) {
    DWF_TRY(check_whole(h, out, in, nrhs));
    if (omega == nullptr || sp == nullptr || stats == nullptr) {
        set_error("boundary: null Omega, solver parameters or stats");
        return DWF_ERR_ARG;
    }
    const BoundaryTables* tbp = nullptr;
    const DevTables* dtp = nullptr;
    DWF_TRY(cached_tables(h, *omega, &tbp, &dtp));
    const BoundaryTables& tb = *tbp;
    const DevTables& dt = *dtp;
    const int64_t ns = h->nsite[0] + h->nsite[1];
    const size_t elems = (size_t)ns * 12 * h->p.Ls * nrhs;   // complex
    if (tb.npat == 0) {   // no hop leaves Omega: P = 0 and R^-1 = 0
        for (int r = 0; r < nrhs; ++r) stats[r] = dwf_solver_stats{};
        DWF_CUDA(cudaMemsetAsync(out, 0, elems * 16, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        return DWF_OK;
    }
    double* scratch = nullptr;   // u, v, y: three full FP64 fields
    DWF_CUDA(dev_malloc(&scratch, 3 * elems * 16));
    double* u = scratch;
    double* v = scratch + 2 * elems;
    double* y = scratch + 4 * elems;
    dwf_status st = DWF_OK;
    auto run = [&]() -> dwf_status {
        // u = P in ; v = D u on Omega-bar
        DWF_TRY(project(h, dt, in, u, nrhs, s));
        DWF_TRY(op_apply_d(h, v, u, 0, DWF_FP64, nrhs, h->d_tmp, s));
        const int per_site = 12 * h->p.Ls * nrhs;
        const int64_t total = ns * per_site;
        const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
        k_mask<<<grid, 256, 0, s>>>(reinterpret_cast<double2*>(v), dt.in_omega, ns, per_site, 1);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        // y = D^-1 v
        DWF_CUDA(cudaMemsetAsync(y, 0, elems * 16, s));
        const dwf_status ss = cgne_solve(h, y, v, nrhs, sp, stats, s);
        if (ss != DWF_OK) return ss;
        // out = u - P y
        DWF_TRY(project(h, dt, y, out, nrhs, s));
        const int g2 = (int)std::min<int64_t>(((int64_t)elems + 255) / 256, 152 * 16);
        k_rsub<<<g2, 256, 0, s>>>(reinterpret_cast<double2*>(out), reinterpret_cast<const double2*>(u),
                                  (int64_t)elems);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        return DWF_OK;
    };
    st = run();
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    return st;
}

}  // namespace dwf

namespace dwf {

// Force of S = |R^-1 phi|^2 (Sec. 2.1, 2.3): with u = P phi, y = D^-1 (D u on
// Omega-bar), chi = u - P y and zeta = D^-+ chi,
//     F = 2 F(zeta, y) - 2 F(zeta on Omega-bar, u),
// F(X, Y) the link force of Re <X, D Y> (force.cu).  The adjoint solve goes
// through the gamma_5 R_5 Hermiticity of D B^-1 (B = b5 + c5 S5):
// D^-+ = G B D^-1 G B^-+, G = gamma_5 R_5: one more solve with D and three
// site-local passes.
dwf_status boundary_force(dwf_handle* h, const dwf_box* omega, double* out, const double* phi, int nrhs,
                          const dwf_box* active, int accumulate, const dwf_solver_params* sp,
                          dwf_solver_stats* stats, cudaStream_t s) {
    DWF_TRY(check_whole(h, out, phi, nrhs));
    if (omega == nullptr || sp == nullptr || stats == nullptr) {
        set_error("boundary: null Omega, solver parameters or stats");
        return DWF_ERR_ARG;
    }
    const BoundaryTables* tbp = nullptr;
    const DevTables* dtp = nullptr;
    DWF_TRY(cached_tables(h, *omega, &tbp, &dtp));
    const BoundaryTables& tb = *tbp;
    const DevTables& dt = *dtp;
    const int64_t ns = h->nsite[0] + h->nsite[1];
    const size_t elems = (size_t)ns * 12 * h->p.Ls * nrhs;   // complex
    const int64_t nlinks = (int64_t)h->p.dims[0] * h->p.dims[1] * h->p.dims[2] * h->p.dims[3] * 4;
    if (tb.npat == 0) {   // no hop leaves Omega: S = 0
        for (int r = 0; r < 2 * nrhs; ++r) stats[r] = dwf_solver_stats{};
        if (!accumulate) DWF_CUDA(cudaMemsetAsync(out, 0, (size_t)nlinks * 18 * sizeof(double), s));
        DWF_CUDA(cudaStreamSynchronize(s));
        return DWF_OK;
    }
    double* scratch = nullptr;   // u, v, y, w: four full FP64 fields
    DWF_CUDA(dev_malloc(&scratch, 4 * elems * 16));
    double* u = scratch;
    double* v = scratch + 2 * elems;
    double* y = scratch + 4 * elems;
    double* w = scratch + 6 * elems;
    const int per_site = 12 * h->p.Ls * nrhs;
    const int g = grid_for((int64_t)elems);
    auto run = [&]() -> dwf_status {
        // u = P phi; v = D u on Omega-bar; y = D^-1 v
        DWF_TRY(project(h, dt, phi, u, nrhs, s));
        DWF_TRY(op_apply_d(h, v, u, 0, DWF_FP64, nrhs, h->d_tmp, s));
        k_mask<<<g, 256, 0, s>>>(reinterpret_cast<double2*>(v), dt.in_omega, ns, per_site, 1);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_CUDA(cudaMemsetAsync(y, 0, elems * 16, s));
        dwf_status st = cgne_solve(h, y, v, nrhs, sp, stats, s);
        if (st != DWF_OK) return st;
        // chi = u - P y (into v)
        DWF_TRY(project(h, dt, y, v, nrhs, s));
        k_rsub<<<g, 256, 0, s>>>(reinterpret_cast<double2*>(v), reinterpret_cast<const double2*>(u),
                                 (int64_t)elems);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        // zeta = G B D^-1 G B^-+ chi
        DWF_TRY(five_b_full(h, w, v, nrhs, true, s));
        k_gamma5_r5<<<g, 256, 0, s>>>(reinterpret_cast<const double2*>(w), reinterpret_cast<double2*>(v), ns,
                                      h->p.Ls, nrhs);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_CUDA(cudaMemsetAsync(w, 0, elems * 16, s));
        st = cgne_solve(h, w, v, nrhs, sp, stats + nrhs, s);
        if (st != DWF_OK) return st;
        DWF_TRY(five_b_full(h, v, w, nrhs, false, s));
        k_gamma5_r5<<<g, 256, 0, s>>>(reinterpret_cast<const double2*>(v), reinterpret_cast<double2*>(w), ns,
                                      h->p.Ls, nrhs);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        // v = -2 zeta on Omega-bar, w = 2 zeta; F = F(w, y) + F(v, u)
        k_scale_mask<<<g, 256, 0, s>>>(reinterpret_cast<const double2*>(w), reinterpret_cast<double2*>(v),
                                       dt.in_omega, ns, per_site, 1, -2.0);
        note_launch();
        k_scale_mask<<<g, 256, 0, s>>>(reinterpret_cast<const double2*>(w), reinterpret_cast<double2*>(w),
                                       dt.in_omega, ns, per_site, 2, 2.0);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_TRY(force_bilinear(h, out, w, y, DWF_FP64, nrhs, active, accumulate, s));
        DWF_TRY(force_bilinear(h, out, v, u, DWF_FP64, nrhs, active, 1, s));
        return DWF_OK;
    };
    const dwf_status st = run();
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    return st;
}

}  // namespace dwf

namespace dwf {
void free_boundary_cache(dwf_handle* h) {
    delete static_cast<BoundaryCache*>(h->boundary_cache);
    h->boundary_cache = nullptr;
}
}  // namespace dwf

namespace dwf {

namespace {

// per right-hand side partial sums of Re <a, b> over full fields (FP64 or
// FP32 elements, FP64 sums): grid (nblk, nrhs), block (b, r) sums the rows of
// rhs r it strides over
template <class V>
__global__ void k_dot_rhs(const V* __restrict__ a, const V* __restrict__ b, int64_t nrows, int Ls, int nrhs,
                          double* __restrict__ partial) {
    __shared__ double red[256];
    const int r = blockIdx.y;
    double acc = 0.0;
    const int64_t n = nrows * Ls;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / Ls;
        const int sidx = (int)(e - row * Ls);
        const int64_t i = (row * nrhs + r) * Ls + sidx;
        const V x = a[i], y = b[i];
        acc += (double)x.x * (double)y.x + (double)x.y * (double)y.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)r * gridDim.x + blockIdx.x] = red[0];
}

// y = a_r x + b_r y per right-hand side (scalars from a device array [2][nrhs])
template <class V>
__global__ void k_axpby_rhs(const V* __restrict__ x, V* __restrict__ y, const double* __restrict__ ab, int64_t n,
                            int Ls, int nrhs) {
    using R = decltype(V{}.x);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)((i / Ls) % nrhs);
        const R al = (R)ab[r], be = (R)ab[nrhs + r];
        const V u = x[i], v = y[i];
        y[i] = V{al * u.x + be * v.x, al * u.y + be * v.y};
    }
}

constexpr int kDotBlocks = 256;

// CGNR building blocks on P_S D P_S for fields of one precision (FP64 or FP32)
struct MaskedCG {
    dwf_handle* h;
    const int* flag;   // per full-field site: 1 in Omega, 0 outside
    int keep;          // the site set S: flag == keep
    int nrhs;
    int64_t ns, elems;
    double* part;      // [nrhs][kDotBlocks]
    double* ab;        // [2][nrhs]
    std::vector<double> hpart;
    cudaStream_t s;
    dwf_prec prec = DWF_FP64;

    size_t field_bytes() const { return (size_t)elems * (prec == DWF_FP64 ? 16 : 8); }
    void* at(void* base, int k) const { return (char*)base + (size_t)k * field_bytes(); }

    dwf_status mask(void* f) {
        if (prec == DWF_FP64)
            k_mask<<<grid_for(elems), 256, 0, s>>>(static_cast<double2*>(f), flag, ns, (int)(elems / ns), 1 - keep);
        else
            k_mask<<<grid_for(elems), 256, 0, s>>>(static_cast<float2*>(f), flag, ns, (int)(elems / ns), 1 - keep);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        return DWF_OK;
    }
    // out = P_S D(^+) P_S in (in supported on S)
    dwf_status apply(void* out, const void* in, int dagger) {
        DWF_TRY(op_apply_d(h, out, in, dagger, prec, nrhs, h->d_tmp, s));
        return mask(out);
    }
    dwf_status dot(const void* a, const void* b, std::vector<double>& out) {
        if (prec == DWF_FP64)
            k_dot_rhs<<<dim3(kDotBlocks, nrhs), 256, 0, s>>>(static_cast<const double2*>(a),
                                                             static_cast<const double2*>(b), ns * 12, h->p.Ls,
                                                             nrhs, part);
        else
            k_dot_rhs<<<dim3(kDotBlocks, nrhs), 256, 0, s>>>(static_cast<const float2*>(a),
                                                             static_cast<const float2*>(b), ns * 12, h->p.Ls,
                                                             nrhs, part);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_CUDA(cudaMemcpyAsync(hpart.data(), part, hpart.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        out.assign(nrhs, 0.0);
        for (int r = 0; r < nrhs; ++r)
            for (int k = 0; k < kDotBlocks; ++k) out[r] += hpart[(size_t)r * kDotBlocks + k];
        return DWF_OK;
    }
    dwf_status axpby(const void* x, void* y, const std::vector<double>& a, const std::vector<double>& b) {
        std::vector<double> hab(2 * nrhs);
        for (int r = 0; r < nrhs; ++r) {
            hab[r] = a[r];
            hab[nrhs + r] = b[r];
        }
        DWF_CUDA(cudaMemcpyAsync(ab, hab.data(), hab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        if (prec == DWF_FP64)
            k_axpby_rhs<<<grid_for(elems), 256, 0, s>>>(static_cast<const double2*>(x), static_cast<double2*>(y), ab,
                                                        elems, h->p.Ls, nrhs);
        else
            k_axpby_rhs<<<grid_for(elems), 256, 0, s>>>(static_cast<const float2*>(x), static_cast<float2*>(y), ab,
                                                        elems, h->p.Ls, nrhs);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        DWF_CUDA(cudaStreamSynchronize(s));   // hab is reused by the next call
        return DWF_OK;
    }
};

// x = (P_S D P_S)^-1 b (or the adjoint system) on the site set S by CGNR in
// the precision of m (one CG per right-hand side in shared launches); b
// supported on S.  work: four fields of that precision.
dwf_status masked_cgnr(MaskedCG& m, void* x, const void* b, void* work, double tol, int maxiter,
                       dwf_solver_stats* stats, bool adjoint) {
    // the operator is P_S D P_S, or its adjoint P_S D^+ P_S
    const int op = adjoint ? 1 : 0, op_adj = adjoint ? 0 : 1;
    const auto t0 = std::chrono::steady_clock::now();
    const int nrhs = m.nrhs;
    const size_t fb = m.field_bytes();
    void* r = m.at(work, 0);
    void* z = m.at(work, 1);
    void* p = m.at(work, 2);
    void* w = m.at(work, 3);
    std::vector<double> bn2, zz, zz_new, ww, rr, one(nrhs, 1.0), al(nrhs), mal(nrhs), be(nrhs);
    DWF_TRY(m.dot(b, b, bn2));
    DWF_CUDA(cudaMemsetAsync(x, 0, fb, m.s));
    DWF_CUDA(cudaMemcpyAsync(r, b, fb, cudaMemcpyDeviceToDevice, m.s));
    DWF_TRY(m.apply(z, r, op_adj));
    DWF_CUDA(cudaMemcpyAsync(p, z, fb, cudaMemcpyDeviceToDevice, m.s));
    DWF_TRY(m.dot(z, z, zz));
    std::vector<int> done(nrhs, 0), iters(nrhs, 0);
    int it = 0;
    for (; it < maxiter; ++it) {
        DWF_TRY(m.dot(r, r, rr));
        bool all = true;
        for (int k = 0; k < nrhs; ++k) {
            if (!done[k] && rr[k] <= tol * tol * bn2[k]) {
                done[k] = 1;
                iters[k] = it;
            }
            all = all && done[k];
        }
        if (all) break;
        DWF_TRY(m.apply(w, p, op));
        DWF_TRY(m.dot(w, w, ww));
        for (int k = 0; k < nrhs; ++k) {
            al[k] = (done[k] || ww[k] == 0.0) ? 0.0 : zz[k] / ww[k];
            mal[k] = -al[k];
        }
        DWF_TRY(m.axpby(p, x, al, one));    // x += alpha p
        DWF_TRY(m.axpby(w, r, mal, one));   // r -= alpha w
        DWF_TRY(m.apply(z, r, op_adj));     // z = (operator)^+ r
        DWF_TRY(m.dot(z, z, zz_new));
        for (int k = 0; k < nrhs; ++k) be[k] = (done[k] || zz[k] == 0.0) ? 0.0 : zz_new[k] / zz[k];
        DWF_TRY(m.axpby(z, p, one, be));    // p = z + beta p
        zz = zz_new;
    }
    // true residual |b - (operator) x| / |b| in the working precision
    DWF_TRY(m.apply(w, x, op));
    DWF_CUDA(cudaMemcpyAsync(r, b, fb, cudaMemcpyDeviceToDevice, m.s));
    DWF_TRY(m.axpby(w, r, std::vector<double>(nrhs, -1.0), one));
    DWF_TRY(m.dot(r, r, rr));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    dwf_status worst = DWF_OK;
    for (int k = 0; k < nrhs; ++k) {
        dwf_solver_stats st{};
        st.iters = done[k] ? iters[k] : it;
        st.op_applies = 2 * st.iters + 2;
        st.true_resid = bn2[k] > 0 ? std::sqrt(rr[k] / bn2[k]) : 0.0;
        st.seconds = secs;
        const dwf_status sk = st.true_resid <= 2 * tol ? DWF_OK : DWF_ERR_NOT_CONVERGED;
        st.status = (int)sk;
        if (sk != DWF_OK) worst = sk;
        stats[k] = st;
    }
    return worst;
}

// Dirichlet solve on the site set S: FP64 CGNR, or (inner = FP32) FP32 CGNR
// rounds to 1e-5 of the current residual with FP64 defect correction
// x += e, r = b - P_S D P_S x until |r| <= tol |b| in FP64.
// work64: four FP64 fields; work32: six FP32 fields (unused for FP64).
dwf_status masked_solve(MaskedCG& m, double* x, const double* b, double* work64, void* work32, double tol,
                        int maxiter, dwf_solver_stats* stats, bool adjoint = false, dwf_prec inner = DWF_FP64) {
    m.prec = DWF_FP64;
    if (inner == DWF_FP64) return masked_cgnr(m, x, b, work64, tol, maxiter, stats, adjoint);
    const auto t0 = std::chrono::steady_clock::now();
    const int nrhs = m.nrhs;
    const int op = adjoint ? 1 : 0;
    double* r = work64;
    double* t = work64 + 2 * m.elems;
    std::vector<double> bn2, rr, one(nrhs, 1.0), mone(nrhs, -1.0);
    std::vector<dwf_solver_stats> inner_st(nrhs);
    std::vector<int> total(nrhs, 0);
    DWF_TRY(m.dot(b, b, bn2));
    DWF_CUDA(cudaMemsetAsync(x, 0, (size_t)m.elems * 16, m.s));
    DWF_CUDA(cudaMemcpyAsync(r, b, (size_t)m.elems * 16, cudaMemcpyDeviceToDevice, m.s));
    int rounds = 0;
    for (; rounds < 30; ++rounds) {
        m.prec = DWF_FP64;
        DWF_TRY(m.dot(r, r, rr));
        bool all = true;
        for (int k = 0; k < nrhs; ++k) all = all && rr[k] <= tol * tol * bn2[k];
        if (all) break;
        // FP32 correction e with (operator) e = r to 1e-5
        m.prec = DWF_FP32;
        void* r32 = m.at(work32, 0);
        void* e32 = m.at(work32, 1);
        void* w32 = m.at(work32, 2);
        DWF_TRY(launch_convert(r32, DWF_FP32, r, DWF_FP64, (size_t)m.elems, m.s));
        const dwf_status st = masked_cgnr(m, e32, r32, w32, 1e-5, maxiter, inner_st.data(), adjoint);
        if (st != DWF_OK && st != DWF_ERR_NOT_CONVERGED) return st;
        for (int k = 0; k < nrhs; ++k) total[k] += inner_st[k].iters;
        m.prec = DWF_FP64;
        DWF_TRY(launch_convert(t, DWF_FP64, e32, DWF_FP32, (size_t)m.elems, m.s));
        DWF_TRY(m.axpby(t, x, one, one));           // x += e
        DWF_TRY(m.apply(t, x, op));                 // r = b - (operator) x
        DWF_CUDA(cudaMemcpyAsync(r, b, (size_t)m.elems * 16, cudaMemcpyDeviceToDevice, m.s));
        DWF_TRY(m.axpby(t, r, mone, one));
    }
    m.prec = DWF_FP64;
    DWF_TRY(m.dot(r, r, rr));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    dwf_status worst = DWF_OK;
    for (int k = 0; k < nrhs; ++k) {
        dwf_solver_stats st{};
        st.iters = total[k];
        st.reliable_updates = rounds;
        st.op_applies = 2 * total[k] + 2 * rounds;
        st.true_resid = bn2[k] > 0 ? std::sqrt(rr[k] / bn2[k]) : 0.0;
        st.seconds = secs;
        const dwf_status sk = st.true_resid <= 2 * tol ? DWF_OK : DWF_ERR_NOT_CONVERGED;
        st.status = (int)sk;
        if (sk != DWF_OK) worst = sk;
        stats[k] = st;
    }
    return worst;
}

}  // namespace

// R psi = P psi - P D_Omega^-1 D_partial D_Omega-bar^-1 D_partialbar P psi (Sec. 2.1): the
// boundary operator whose inverse dwf_boundary_rinv applies; the two Dirichlet
// solves (on Omega-bar, the band, and on Omega) by FP64 CGNR on P_S D P_S.
dwf_status boundary_r(dwf_handle* h, const dwf_box* omega, double* out, const double* in, int nrhs,
                      const dwf_solver_params* sp, dwf_solver_stats* stats, cudaStream_t s) {
    DWF_TRY(check_whole(h, out, in, nrhs));
    if (omega == nullptr || sp == nullptr || stats == nullptr || !(sp->tol > 0.0) || sp->maxiter < 1) {
        set_error("boundary: null Omega, solver parameters or stats, or tol <= 0 / maxiter < 1");
        return DWF_ERR_ARG;
    }
    const BoundaryTables* tbp = nullptr;
    const DevTables* dtp = nullptr;
    DWF_TRY(cached_tables(h, *omega, &tbp, &dtp));
    const DevTables& dt = *dtp;
    const int64_t ns = h->nsite[0] + h->nsite[1];
    const int64_t elems = ns * 12 * h->p.Ls * nrhs;   // complex
    if (tbp->npat == 0) {
        for (int r = 0; r < 2 * nrhs; ++r) stats[r] = dwf_solver_stats{};
        DWF_CUDA(cudaMemsetAsync(out, 0, elems * 16, s));
        DWF_CUDA(cudaStreamSynchronize(s));
        return DWF_OK;
    }
    // u, a, b, four FP64 and six FP32 solver work fields, the reduction buffers
    double* scratch = nullptr;
    const size_t fb = (size_t)elems * 16;
    DWF_CUDA(dev_malloc(&scratch, 10 * fb + ((size_t)kDotBlocks + 2) * nrhs * sizeof(double)));
    double* u = scratch;
    double* a = scratch + 2 * elems;
    double* b = scratch + 4 * elems;
    double* work = scratch + 6 * elems;
    void* work32 = scratch + 14 * elems;
    MaskedCG m{h, dt.in_omega, 0, nrhs, ns, elems, scratch + 20 * elems,
               scratch + 20 * elems + (size_t)kDotBlocks * nrhs, std::vector<double>((size_t)kDotBlocks * nrhs), s};
    const dwf_prec inner = sp->inner_prec == DWF_FP64 ? DWF_FP64 : DWF_FP32;
    auto run = [&]() -> dwf_status {
        // u = P psi; a = D u on Omega-bar; b = D_Omega-bar^-1 a
        DWF_TRY(project(h, dt, in, u, nrhs, s));
        DWF_TRY(op_apply_d(h, a, u, 0, DWF_FP64, nrhs, h->d_tmp, s));
        m.keep = 0;
        DWF_TRY(m.mask(a));
        dwf_status st = masked_solve(m, b, a, work, work32, sp->tol, sp->maxiter, stats, false, inner);
        if (st != DWF_OK) return st;
        // a = D b on Omega; b = D_Omega^-1 a
        DWF_TRY(op_apply_d(h, a, b, 0, DWF_FP64, nrhs, h->d_tmp, s));
        m.keep = 1;
        DWF_TRY(m.mask(a));
        st = masked_solve(m, b, a, work, work32, sp->tol, sp->maxiter, stats + nrhs, false, inner);
        if (st != DWF_OK) return st;
        // out = u - P b
        DWF_TRY(project(h, dt, b, out, nrhs, s));
        k_rsub<<<grid_for(elems), 256, 0, s>>>(reinterpret_cast<double2*>(out),
                                               reinterpret_cast<const double2*>(u), elems);
        note_launch();
        DWF_CUDA(cudaGetLastError());
        return DWF_OK;
    };
    const dwf_status st = run();
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    return st;
}

}  // namespace dwf

namespace dwf {

namespace {
dwf_status copy_field(double* dst, const double* src, int64_t elems, cudaStream_t s) {
    DWF_CUDA(cudaMemcpyAsync(dst, src, (size_t)elems * 16, cudaMemcpyDeviceToDevice, s));
    return DWF_OK;
}
dwf_status launch_scale_mask(const double* in, double* out, const int* flag, int64_t ns, int64_t elems, int drop,
                             double factor, cudaStream_t s) {
    k_scale_mask<<<grid_for(elems), 256, 0, s>>>(reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out),
                                                flag, ns, (int)(elems / ns), drop, factor);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}
dwf_status launch_rsub(double* out, const double* a, int64_t elems, cudaStream_t s) {
    k_rsub<<<grid_for(elems), 256, 0, s>>>(reinterpret_cast<double2*>(out), reinterpret_cast<const double2*>(a),
                                           elems);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}
dwf_status launch_mask(double* f, const int* flag, int64_t ns, int64_t elems, int drop, cudaStream_t s) {
    k_mask<<<grid_for(elems), 256, 0, s>>>(reinterpret_cast<double2*>(f), flag, ns, (int)(elems / ns), drop);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}
dwf_status launch_g5r5(const double* in, double* out, int64_t ns, int Ls, int nrhs, int64_t elems, cudaStream_t s) {
    k_gamma5_r5<<<grid_for(elems), 256, 0, s>>>(reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out),
                                                ns, Ls, nrhs);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}
}  // namespace

// Force of the boundary Hasenbusch ratio S = |R^-1 R_pv phi|^2 (Sec. 2.3),
// light operator on hl, Pauli-Villars on hp:
//   R_pv phi = u_pv - P_pv d,  u_pv = P_pv phi, b = D_Ob^-1 (D u_pv on Omega-bar), d = D_O^-1 (D b on Omega),
//   chi = R^-1 R_pv phi,  zeta = D^-+ chi,  xi = R^-+ chi = chi - (D^+ (zeta on Omega-bar)) on Omega,
//   eta = D_O^-+ P_pv xi,  kappa = D_Ob^-+ (D^+ eta on Omega-bar)   (PV),
//   F = 2 F(zeta, y) - 2 F(zeta on Omega-bar, u) + 2 F_pv(eta, d - b) + 2 F_pv(kappa, b - u_pv),
// with u, y the light R^-1 pieces: four PV local solves, two light solves.
dwf_status boundary_ratio_force(dwf_handle* hl, dwf_handle* hp, const dwf_box* omega, double* out, const double* phi,
                                int nrhs, const dwf_box* active, int accumulate, const dwf_solver_params* sp,
                                dwf_solver_stats* stats, cudaStream_t s) {
    DWF_TRY(check_whole(hl, out, phi, nrhs));
    DWF_TRY(check_whole(hp, out, phi, nrhs));
    if (omega == nullptr || sp == nullptr || stats == nullptr || !(sp->tol > 0.0) || sp->maxiter < 1) {
        set_error("boundary: null Omega, solver parameters or stats, or tol <= 0 / maxiter < 1");
        return DWF_ERR_ARG;
    }
    for (int mu = 0; mu < 4; ++mu)
        if (hl->p.dims[mu] != hp->p.dims[mu]) {
            set_error("boundary: the light and Pauli-Villars handles differ in the lattice");
            return DWF_ERR_ARG;
        }
    if (hl->p.Ls != hp->p.Ls) {
        set_error("boundary: the light and Pauli-Villars handles differ in Ls");
        return DWF_ERR_ARG;
    }
    const BoundaryTables *tl = nullptr, *tp = nullptr;
    const DevTables *dl = nullptr, *dp = nullptr;
    DWF_TRY(cached_tables(hl, *omega, &tl, &dl));
    DWF_TRY(cached_tables(hp, *omega, &tp, &dp));
    const int64_t ns = hl->nsite[0] + hl->nsite[1];
    const int64_t elems = ns * 12 * hl->p.Ls * nrhs;   // complex
    const int64_t nlinks = (int64_t)hl->p.dims[0] * hl->p.dims[1] * hl->p.dims[2] * hl->p.dims[3] * 4;
    if (tl->npat == 0) {   // no hop leaves Omega: S = 0
        for (int r = 0; r < 6 * nrhs; ++r) stats[r] = dwf_solver_stats{};
        if (!accumulate) DWF_CUDA(cudaMemsetAsync(out, 0, (size_t)nlinks * 18 * sizeof(double), s));
        DWF_CUDA(cudaStreamSynchronize(s));
        return DWF_OK;
    }
    constexpr int NF = 18;   // 15 FP64 fields, then six FP32 solver work fields
    double* scratch = nullptr;
    const size_t red = ((size_t)kDotBlocks + 2) * nrhs * sizeof(double);
    DWF_CUDA(dev_malloc(&scratch, NF * (size_t)elems * 16 + red));
    double* F[NF];
    for (int k = 0; k < NF; ++k) F[k] = scratch + 2 * elems * k;
    double *u_pv = F[0], *t1 = F[1], *b = F[2], *d = F[3], *u_l = F[4], *chi = F[5], *y = F[6], *zeta = F[7],
           *xi = F[8], *eta = F[9], *kappa = F[10], *W0 = F[11], *W1 = F[12], *W2 = F[13], *W3 = F[14];
    double* work = F[11];   // the masked solves' four FP64 work fields W0..W3
    void* work32 = F[15];
    const dwf_prec inner = sp->inner_prec == DWF_FP64 ? DWF_FP64 : DWF_FP32;
    double* part = scratch + 2 * elems * NF;
    MaskedCG m{hp, dp->in_omega, 0, nrhs, ns, elems, part, part + (size_t)kDotBlocks * nrhs,
               std::vector<double>((size_t)kDotBlocks * nrhs), s};
    const int* flag = dp->in_omega;
    const int Ls = hl->p.Ls;
    auto run = [&]() -> dwf_status {
        // R_pv phi: u_pv, b (Omega-bar solve), d (Omega solve), w = u_pv - P_pv d (in t1)
        DWF_TRY(project(hp, *dp, phi, u_pv, nrhs, s));
        DWF_TRY(op_apply_d(hp, t1, u_pv, 0, DWF_FP64, nrhs, hp->d_tmp, s));
        DWF_TRY(launch_mask(t1, flag, ns, elems, 1, s));
        dwf_status st = masked_solve(m, b, t1, work, work32, sp->tol, sp->maxiter, stats, false, inner);
        if (st != DWF_OK) return st;
        DWF_TRY(op_apply_d(hp, t1, b, 0, DWF_FP64, nrhs, hp->d_tmp, s));
        DWF_TRY(launch_mask(t1, flag, ns, elems, 0, s));
        m.keep = 1;
        st = masked_solve(m, d, t1, work, work32, sp->tol, sp->maxiter, stats + nrhs, false, inner);
        if (st != DWF_OK) return st;
        DWF_TRY(project(hp, *dp, d, t1, nrhs, s));
        DWF_TRY(launch_rsub(t1, u_pv, elems, s));                       // t1 = w
        // light R^-1 w: u_l, y = D^-1 (D u_l on Omega-bar), chi = u_l - P y
        DWF_TRY(project(hl, *dl, t1, u_l, nrhs, s));
        DWF_TRY(op_apply_d(hl, chi, u_l, 0, DWF_FP64, nrhs, hl->d_tmp, s));
        DWF_TRY(launch_mask(chi, flag, ns, elems, 1, s));
        DWF_CUDA(cudaMemsetAsync(y, 0, (size_t)elems * 16, s));
        st = cgne_solve(hl, y, chi, nrhs, sp, stats + 2 * nrhs, s);
        if (st != DWF_OK) return st;
        DWF_TRY(project(hl, *dl, y, chi, nrhs, s));
        DWF_TRY(launch_rsub(chi, u_l, elems, s));                       // chi
        // zeta = G B D^-1 G B^-+ chi (light)
        DWF_TRY(five_b_full(hl, W0, chi, nrhs, true, s));
        DWF_TRY(launch_g5r5(W0, W1, ns, Ls, nrhs, elems, s));
        DWF_CUDA(cudaMemsetAsync(W0, 0, (size_t)elems * 16, s));
        st = cgne_solve(hl, W0, W1, nrhs, sp, stats + 3 * nrhs, s);
        if (st != DWF_OK) return st;
        DWF_TRY(five_b_full(hl, W1, W0, nrhs, false, s));
        DWF_TRY(launch_g5r5(W1, zeta, ns, Ls, nrhs, elems, s));
        // xi = chi - (D^+ (zeta on Omega-bar)) on Omega
        DWF_TRY(launch_scale_mask(zeta, W0, flag, ns, elems, 1, 1.0, s));
        DWF_TRY(op_apply_d(hl, xi, W0, 1, DWF_FP64, nrhs, hl->d_tmp, s));
        DWF_TRY(launch_mask(xi, flag, ns, elems, 0, s));
        DWF_TRY(launch_rsub(xi, chi, elems, s));
        // eta = D_O^-+ P_pv xi, kappa = D_Ob^-+ (D^+ eta on Omega-bar)   (PV)
        DWF_TRY(project(hp, *dp, xi, t1, nrhs, s));
        m.keep = 1;
        st = masked_solve(m, eta, t1, work, work32, sp->tol, sp->maxiter, stats + 4 * nrhs, true, inner);
        if (st != DWF_OK) return st;
        DWF_TRY(op_apply_d(hp, t1, eta, 1, DWF_FP64, nrhs, hp->d_tmp, s));
        DWF_TRY(launch_mask(t1, flag, ns, elems, 1, s));
        m.keep = 0;
        st = masked_solve(m, kappa, t1, work, work32, sp->tol, sp->maxiter, stats + 5 * nrhs, true, inner);
        if (st != DWF_OK) return st;
        // the four insertions
        DWF_TRY(launch_scale_mask(zeta, W0, flag, ns, elems, 2, 2.0, s));     // 2 zeta
        DWF_TRY(launch_scale_mask(zeta, W1, flag, ns, elems, 1, -2.0, s));    // -2 zeta on Omega-bar
        DWF_TRY(force_bilinear(hl, out, W0, y, DWF_FP64, nrhs, active, accumulate, s));
        DWF_TRY(force_bilinear(hl, out, W1, u_l, DWF_FP64, nrhs, active, 1, s));
        DWF_TRY(copy_field(W2, b, elems, s));
        DWF_TRY(launch_rsub(W2, d, elems, s));                                  // d - b
        DWF_TRY(launch_scale_mask(eta, W3, flag, ns, elems, 2, 2.0, s));
        DWF_TRY(force_bilinear(hp, out, W3, W2, DWF_FP64, nrhs, active, 1, s));
        DWF_TRY(copy_field(W2, u_pv, elems, s));
        DWF_TRY(launch_rsub(W2, b, elems, s));                                  // b - u_pv
        DWF_TRY(launch_scale_mask(kappa, W3, flag, ns, elems, 2, 2.0, s));
        DWF_TRY(force_bilinear(hp, out, W3, W2, DWF_FP64, nrhs, active, 1, s));
        return DWF_OK;
    };
    const dwf_status st = run();
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    return st;
}

}  // namespace dwf
