"""Oracle: multi-shift conjugate gradient, plain FP64 numpy (test
infrastructure only).

The paper's DD-RHMC (Sec. 2.3.1, the one-flavour boundary term of the
DD-RHMC action) needs rational functions of the normal operators of D and of
the Dirichlet operator D_Omega, i.e. sum_i a_i (A + sigma_i)^-1 b for a set of
real shifts sigma_i >= 0.  All shifted systems share one Krylov space, so
one CG on the smallest shift yields every solution (the published multi-shift
CG, Jegerlehner, hep-lat/9612014): with the base CG's alpha_k, beta_k and
residual r_k, the shifted residuals are collinear, r_k^(s) = zeta_k^(s) r_k,
with

    zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1}
                 / (alpha_k beta_{k-1} (zeta_{k-1} - zeta_k)
                    + zeta_{k-1} alpha_{k-1} (1 + d_s alpha_k)),
    alpha_k^(s) = alpha_k zeta_{k+1} / zeta_k,
    beta_k^(s)  = beta_k (zeta_{k+1} / zeta_k)^2,

d_s = sigma_s - sigma_0, and x^(s) += alpha^(s) p^(s),
p^(s) = zeta_{k+1} r_{k+1} + beta^(s) p^(s).  A shift stops when its residual
zeta^(s) |r| drops to tol |b|.

Here A is any Hermitian positive operator given as a function (the tests use
M_pc^+ M_pc of the domain wall operator); vectors are arrays of any shape.
"""

from __future__ import annotations

import numpy as np


def multishift_cg(apply_A, b, shifts, tol=1e-10, maxiter=100000):
    """Solve (A + sigma_s) x_s = b for every shift (sigma_0 = min, base system).

    Returns (xs, info) with xs in the order of ``shifts`` and info a dict
    with per-shift iteration counts and the base iteration count."""
    order = np.argsort(shifts)
    sig = np.asarray(shifts, dtype=float)[order]
    n = len(sig)
    d = sig - sig[0]
    bn = np.sqrt(np.vdot(b, b).real)
    x = [np.zeros_like(b) for _ in range(n)]
    p = [b.copy() for _ in range(n)]
    r = b.copy()
    rr = np.vdot(r, r).real
    zeta = np.ones(n)
    zeta_prev = np.ones(n)
    alpha_prev, beta_prev = 1.0, 0.0
    active = np.ones(n, dtype=bool)
    iters = np.zeros(n, dtype=int)
    k = 0
    while active.any() and k < maxiter:
        Ap = apply_A(p[0]) + sig[0] * p[0]
        alpha = rr / np.vdot(p[0], Ap).real
        zeta_new = np.ones(n)
        for s in range(n):
            if not active[s]:
                continue
            if s == 0:
                zeta_new[s] = 1.0
            else:
                den = (alpha * beta_prev * (zeta_prev[s] - zeta[s])
                       + zeta_prev[s] * alpha_prev * (1.0 + d[s] * alpha))
                zeta_new[s] = zeta[s] * zeta_prev[s] * alpha_prev / den
            x[s] = x[s] + (alpha * zeta_new[s] / zeta[s]) * p[s]
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        beta = rr_new / rr
        k += 1
        for s in range(n):
            if not active[s]:
                continue
            beta_s = beta * (zeta_new[s] / zeta[s]) ** 2
            p[s] = zeta_new[s] * r + beta_s * p[s]
            iters[s] = k
            if abs(zeta_new[s]) * np.sqrt(rr_new) <= tol * bn:
                active[s] = False
        zeta_prev, zeta = zeta, zeta_new
        alpha_prev, beta_prev, rr = alpha, beta, rr_new
    xs = [None] * n
    its = [0] * n
    for i, s in enumerate(order):
        xs[s] = x[i]
        its[s] = int(iters[i])
    return xs, {"iters": its, "base_iters": k}


def rational_apply(apply_A, b, a0, shifts, residues, tol=1e-10):
    """r(A) b = a0 b + sum_i residues_i (A + shifts_i)^-1 b: a rational function
    in partial fractions (the form the DD-RHMC action of Sec. 2.3.1 uses for
    the powers of the normal operators), the shifted solves by multi-shift CG."""
    xs, _ = multishift_cg(apply_A, b, shifts, tol=tol)
    out = a0 * b
    for r, x in zip(residues, xs):
        out = out + r * x
    return out
