// Relative minimax rational approximations of x^alpha in partial fractions
// (host only): the coefficients of the fractional powers in the one-flavour
// DD-RHMC action of Sec. 2.3.1, (D_dir^+ D_dir)^(1/4) and (D^+ D)^(-1/2), and of
// the heat bath's (D_dir^+ D_dir)^(-1/4) and (D^+ D)^(1/4).
//
//     x^alpha ~ r(x) = a0 + sum_i rho_i / (x + sigma_i),   x in [lo, hi],
//
// type (n, n), minimising max |r(x) / x^alpha - 1|.  By Chebyshev's theorem the
// best approximation is the one whose relative error equioscillates at 2n + 2
// points; the Remez algorithm finds it by alternating
//   (1) Newton's method on the 2n + 2 equations r(x_j) x_j^-alpha - 1 = (-1)^j E
//       in the unknowns a0, rho_i, log sigma_i and the level E, and
//   (2) the exchange of the reference points x_j for the extrema of the error.
// Newton needs a start close to the answer, which the method gets by
// continuation: for alpha = -1/2 Zolotarev's closed form is the best
// approximation (c_l = sn^2/cn^2(l K'/(2n + 1) | 1 - lo/hi), poles the odd c_l,
// zeros the even ones), and the solution moves smoothly with alpha, so alpha
// steps from -1/2 to -|alpha| re-solving at each step.  For alpha > 0 the
// reciprocal of the fit of x^-alpha (poles at its zeros, which interlace its
// poles on the negative axis) starts a last Remez solve for x^alpha itself.
// Everything runs on y = x / lo in [1, hi / lo]; the answer is scaled back.

#include <algorithm>
#include <cmath>
#include <vector>

#include "dwf_internal.cuh"

namespace dwf {

namespace {

struct Frac {
    double a0 = 0.0;
    std::vector<double> s, r;   // shifts sigma_i > 0 and residues rho_i
};

double frac_eval(const Frac& f, double y) {
    double v = f.a0;
    for (size_t i = 0; i < f.s.size(); ++i) v += f.r[i] / (y + f.s[i]);
    return v;
}

double rel_err(const Frac& f, double alpha, double y) { return frac_eval(f, y) * std::pow(y, -alpha) - 1.0; }

// Solve A x = b (m x m, row-major, overwritten) by Gaussian elimination with
// column scaling and partial pivoting; false if singular.
bool dense_solve(std::vector<double>& A, std::vector<double>& b, int m) {
    std::vector<double> sc(m, 0.0);
    for (int j = 0; j < m; ++j) {
        for (int i = 0; i < m; ++i) sc[j] = std::max(sc[j], std::fabs(A[i * m + j]));
        if (!(sc[j] > 0.0)) return false;
        for (int i = 0; i < m; ++i) A[i * m + j] /= sc[j];
    }
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int i = k + 1; i < m; ++i)
            if (std::fabs(A[i * m + k]) > std::fabs(A[piv * m + k])) piv = i;
        if (!(std::fabs(A[piv * m + k]) > 0.0)) return false;
        if (piv != k) {
            for (int j = 0; j < m; ++j) std::swap(A[k * m + j], A[piv * m + j]);
            std::swap(b[k], b[piv]);
        }
        for (int i = k + 1; i < m; ++i) {
            const double l = A[i * m + k] / A[k * m + k];
            if (l == 0.0) continue;
            for (int j = k; j < m; ++j) A[i * m + j] -= l * A[k * m + j];
            b[i] -= l * b[k];
        }
    }
    for (int k = m - 1; k >= 0; --k) {
        double v = b[k];
        for (int j = k + 1; j < m; ++j) v -= A[k * m + j] * b[j];
        b[k] = v / A[k * m + k];
    }
    for (int j = 0; j < m; ++j) b[j] /= sc[j];
    return true;
}

// Residual of the equioscillation equations at the reference points.
double eq_resid(const Frac& f, double alpha, double E, const std::vector<double>& xr, std::vector<double>* F) {
    double mx = 0.0;
    for (size_t j = 0; j < xr.size(); ++j) {
        const double v = rel_err(f, alpha, xr[j]) - ((j & 1) ? -E : E);
        if (F) (*F)[j] = v;
        mx = std::max(mx, std::fabs(v));
    }
    return mx;
}

// Newton's method (with backtracking on the largest residual) for a0, rho,
// log sigma and E such that the error is +-E alternately at xr; false if it
// diverges.
bool newton(Frac& f, double alpha, const std::vector<double>& xr, double& E) {
    const int n = (int)f.s.size(), m = 2 * n + 2;
    std::vector<double> F(m), A(m * m), w(m);
    for (int j = 0; j < m; ++j) w[j] = std::pow(xr[j], -alpha);
    E = 0.0;
    for (int j = 0; j < m; ++j) E += ((j & 1) ? -1.0 : 1.0) * rel_err(f, alpha, xr[j]) / m;
    double res = eq_resid(f, alpha, E, xr, &F);
    for (int it = 0; it < 60; ++it) {
        if (res <= 1e-15 + 1e-12 * std::fabs(E)) return true;
        for (int j = 0; j < m; ++j) {
            double* row = &A[j * m];
            row[0] = w[j];
            for (int i = 0; i < n; ++i) {
                const double d = 1.0 / (xr[j] + f.s[i]);
                row[1 + i] = w[j] * d;
                row[1 + n + i] = -w[j] * f.r[i] * f.s[i] * d * d;   // d/d log sigma_i
            }
            row[m - 1] = (j & 1) ? 1.0 : -1.0;
        }
        std::vector<double> dx(m);
        for (int j = 0; j < m; ++j) dx[j] = -F[j];
        if (!dense_solve(A, dx, m)) return false;
        double lam = 1.0;
        for (;;) {
            Frac g = f;
            g.a0 = f.a0 + lam * dx[0];
            for (int i = 0; i < n; ++i) {
                g.r[i] = f.r[i] + lam * dx[1 + i];
                g.s[i] = f.s[i] * std::exp(std::max(-1.0, std::min(1.0, lam * dx[1 + n + i])));
            }
            const double gE = E + lam * dx[m - 1];
            std::vector<double> gF(m);
            const double gres = eq_resid(g, alpha, gE, xr, &gF);
            if (std::isfinite(gres) && (gres < res || lam < 1e-4)) {
                f = g;
                E = gE;
                F = gF;
                res = gres;
                break;
            }
            lam *= 0.5;
        }
        if (!std::isfinite(res)) return false;
    }
    // For alpha > 0 the residues are negative and r(y) cancels at small y, so
    // the residual stalls at rounding (~1e-13) above the tolerance: accept what
    // is small against the level; the exchange step measures the real error.
    return res <= 1e-3 * std::fabs(E);
}

// The alternating extrema of the error on [1, b]: the local extrema on a grid
// in log y (and the two end points), runs of equal sign merged to their largest
// member, interior ones refined by golden-section search; then trimmed to
// 2n + 2 by dropping the smaller end.  Returns false with fewer than 2n + 2.
bool extrema(const Frac& f, double alpha, double b, int n, std::vector<double>& xr, double& emax,
             double& emin) {
    const int G = 4000 + 60 * (2 * n + 2);
    const double lb = std::log(b);
    std::vector<double> u(G), e(G);
    for (int g = 0; g < G; ++g) {
        u[g] = lb * g / (G - 1);
        e[g] = rel_err(f, alpha, std::exp(u[g]));
    }
    std::vector<int> idx{0};
    for (int g = 1; g < G - 1; ++g)
        if ((e[g] - e[g - 1]) * (e[g + 1] - e[g]) <= 0.0) idx.push_back(g);
    idx.push_back(G - 1);
    std::vector<int> pts;
    for (int g : idx) {
        if (!pts.empty() && (e[g] > 0) == (e[pts.back()] > 0)) {
            if (std::fabs(e[g]) > std::fabs(e[pts.back()])) pts.back() = g;
        } else {
            pts.push_back(g);
        }
    }
    std::vector<double> xs, es;
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    for (int g : pts) {
        double x = std::exp(u[g]);
        if (g != 0 && g != G - 1) {
            const double sg = e[g] > 0 ? -1.0 : 1.0;   // minimise sg * e
            double a = u[g - 1], c2 = u[g + 1];
            double c = c2 - gr * (c2 - a), d = a + gr * (c2 - a);
            double fc = sg * rel_err(f, alpha, std::exp(c)), fd = sg * rel_err(f, alpha, std::exp(d));
            for (int k = 0; k < 60; ++k) {
                if (fc < fd) {
                    c2 = d; d = c; fd = fc;
                    c = c2 - gr * (c2 - a);
                    fc = sg * rel_err(f, alpha, std::exp(c));
                } else {
                    a = c; c = d; fc = fd;
                    d = a + gr * (c2 - a);
                    fd = sg * rel_err(f, alpha, std::exp(d));
                }
            }
            x = std::exp(0.5 * (a + c2));
        }
        xs.push_back(x);
        es.push_back(rel_err(f, alpha, x));
    }
    while ((int)xs.size() > 2 * n + 2) {
        if (std::fabs(es.front()) < std::fabs(es.back())) {
            xs.erase(xs.begin()); es.erase(es.begin());
        } else {
            xs.pop_back(); es.pop_back();
        }
    }
    if ((int)xs.size() < 2 * n + 2) return false;
    emax = 0.0;
    emin = 1e300;
    for (double v : es) {
        emax = std::max(emax, std::fabs(v));
        emin = std::min(emin, std::fabs(v));
    }
    for (double v : e) emax = std::max(emax, std::fabs(v));
    xr = xs;
    return true;
}

// Remez iterations at fixed alpha until the extrema agree to `rtol` (or to
// the rounding floor of the error, ~1e-14 n).  False if Newton or the
// exchange breaks down; *spread = (max - min) / max of |error| at the end.
bool remez(Frac& f, double alpha, double b, std::vector<double>& xr, double rtol, double& delta,
           double& spread) {
    const int n = (int)f.s.size();
    spread = 1.0;
    for (int outer = 0; outer < 40; ++outer) {
        double E = 0.0, emax = 0.0, emin = 0.0;
        if (!newton(f, alpha, xr, E)) return false;
        if (!extrema(f, alpha, b, n, xr, emax, emin)) return false;
        delta = emax;
        spread = (emax - emin) / emax;
        if (emax - emin <= rtol * emax + 1e-14 * n) return true;
    }
    return true;
}

// Zolotarev's best type (n, n) relative approximation of y^-1/2 on [1, b].
void zolotarev_nn(int n, double b, Frac& f) {
    const double m1 = 1.0 / b, m = 1.0 - m1;
    double Kp = 0.0;
    jacobi_sn_cn(0.0, m, m1, nullptr, nullptr, &Kp);
    std::vector<double> c(2 * n + 1);
    for (int l = 1; l <= 2 * n; ++l) {
        double sn = 0.0, cn = 1.0;
        jacobi_sn_cn(l * Kp / (2.0 * n + 1.0), m, m1, &sn, &cn, nullptr);
        c[l] = sn * sn / (cn * cn);
    }
    // centre the relative error of prod (y + c_2l) / (y + c_2l-1) / sqrt(y)
    const int G = 20001;
    double vmax = -1e300, vmin = 1e300;
    for (int g = 0; g < G; ++g) {
        const double y = std::exp(std::log(b) * g / (G - 1));
        double v = std::sqrt(y);
        for (int l = 1; l <= n; ++l) v *= (y + c[2 * l]) / (y + c[2 * l - 1]);
        vmax = std::max(vmax, v);
        vmin = std::min(vmin, v);
    }
    const double D = 2.0 / (vmax + vmin);
    f.a0 = D;
    f.s.assign(n, 0.0);
    f.r.assign(n, 0.0);
    for (int j = 1; j <= n; ++j) {
        const double p = c[2 * j - 1];
        double R = D;
        for (int l = 1; l <= n; ++l) R *= c[2 * l] - p;
        for (int k = 1; k <= n; ++k)
            if (k != j) R /= c[2 * k - 1] - p;
        f.s[j - 1] = p;
        f.r[j - 1] = R;
    }
}

// 1/r for r = a0 + sum rho / (y + sigma) with a0, rho > 0: its poles are the
// zeros of r, one in each gap between consecutive sorted shifts and one
// beyond the largest (r(-t) runs from -inf to +inf, resp. to a0 > 0, there);
// residues 1 / r'(-zeta).  False if the input is not of that kind.
bool reciprocal(const Frac& f, Frac& g) {
    const int n = (int)f.s.size();
    if (!(f.a0 > 0.0)) return false;
    for (int i = 0; i < n; ++i)
        if (!(f.r[i] > 0.0) || !(f.s[i] > 0.0)) return false;
    std::vector<double> s = f.s;
    std::sort(s.begin(), s.end());
    auto rneg = [&](double t) {   // r(-t)
        double v = f.a0;
        for (int i = 0; i < n; ++i) v += f.r[i] / (f.s[i] - t);
        return v;
    };
    g.a0 = 1.0 / f.a0;
    g.s.assign(n, 0.0);
    g.r.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double a = s[i], c = (i + 1 < n) ? s[i + 1] : 2.0 * s[i];
        if (i + 1 == n)
            while (rneg(c) <= 0.0) {
                c *= 2.0;
                if (!std::isfinite(c)) return false;
            }
        // r(-t) < 0 just above s[i], > 0 just below the upper end: bisect in log t
        for (int k = 0; k < 200; ++k) {
            const double mid = std::sqrt(a * c);
            if (mid <= a || mid >= c) break;
            if (rneg(mid) < 0.0) a = mid; else c = mid;
        }
        const double z = std::sqrt(a * c);
        double dr = 0.0;   // r'(-z) = -sum rho / (sigma - z)^2
        for (int k = 0; k < n; ++k) dr -= f.r[k] / ((f.s[k] - z) * (f.s[k] - z));
        g.s[i] = z;
        g.r[i] = 1.0 / dr;
    }
    return true;
}

}  // namespace

dwf_status rational_power(double alpha, int n, double lo, double hi, double* a0, double* shifts,
                          double* residues, double* delta) {
    if (!(alpha > -1.0 && alpha < 1.0) || alpha == 0.0 || n < 1 || n > 48 || !(lo > 0.0) || !(hi > lo) ||
        !(hi / lo <= 1e14) || a0 == nullptr || shifts == nullptr || residues == nullptr) {
        set_error("rational power: need -1 < alpha < 1, alpha != 0, 1 <= n <= 48, 0 < lo < hi <= 1e14 lo "
                  "and output arrays");
        return DWF_ERR_ARG;
    }
    const double b = hi / lo;
    Frac f;
    zolotarev_nn(n, b, f);
    std::vector<double> xr;
    double emax = 0.0, emin = 0.0, dl = 0.0, spread = 1.0;
    bool ok = extrema(f, -0.5, b, n, xr, emax, emin);
    // continuation alpha = -1/2 -> -|alpha| (the closed form is polished at -1/2 too)
    const double target = -std::fabs(alpha);
    const int steps = std::max(1, (int)std::ceil(std::fabs(target + 0.5) / 0.0125));
    for (int k = 1; k <= steps && ok; ++k) {
        const double al = -0.5 + (target + 0.5) * k / steps;
        ok = remez(f, al, b, xr, k == steps ? 1e-6 : 1e-3, dl, spread);
    }
    if (ok && alpha > 0.0) {
        Frac g;
        ok = reciprocal(f, g);
        if (ok) {
            f = g;
            ok = extrema(f, alpha, b, n, xr, emax, emin) && remez(f, alpha, b, xr, 1e-6, dl, spread);
        }
    }
    // a spread of the extrema above 1% is not an equioscillating (best) fit
    ok = ok && spread < 1e-2 && std::isfinite(dl);
    if (!ok) {
        set_error("rational power: the Remez iteration failed for alpha = %g, n = %d on [%g, %g] (the error "
                  "may be below rounding: lower n)", alpha, n, lo, hi);
        return DWF_ERR_NOT_CONVERGED;
    }
    // back to x = lo y: r(x) = lo^alpha (a0 + sum rho / (x / lo + sigma))
    const double la = std::pow(lo, alpha);
    *a0 = la * f.a0;
    for (int i = 0; i < n; ++i) {
        shifts[i] = lo * f.s[i];
        residues[i] = la * lo * f.r[i];
    }
    if (delta) *delta = dl;
    return DWF_OK;
}

}  // namespace dwf
