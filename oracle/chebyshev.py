"""Oracle: Chebyshev filter of the normal Schur operator, plain FP64 numpy
(test infrastructure only).

Sec. 4 proposes to set up the multigrid subspace of the local (D_Omega)
solves with filter functions obtained recursively from Chebyshev polynomials,
cheaper than inverse iteration.  The filter applied to a vector v is

    p_n(A) v = T_n(z(A)) v,   z(lam) = (hi + lo - 2 lam) / (hi - lo),

with A = M_pc^+ M_pc (Hermitian, positive) and [lo, hi] the part of its
spectrum to suppress: there |T_n(z)| <= 1, while below lo, z > 1 and
T_n(z) = cosh(n arccosh z) grows exponentially in n, so the low modes that
multigrid must capture dominate the result.  The three-term recurrence

    w_0 = v,  w_1 = z(A) v,  w_{k+1} = 2 z(A) w_k - w_{k-1}

gives T_n(z(A)) v with n applications of A.
"""

from __future__ import annotations


def chebyshev_filter(apply_A, v, order: int, lo: float, hi: float):
    """T_order(z(A)) v, z(lam) = (hi + lo - 2 lam) / (hi - lo)."""
    if order < 0 or not hi > lo:
        raise ValueError("order >= 0 and hi > lo")
    c0 = (hi + lo) / (hi - lo)
    c1 = -2.0 / (hi - lo)

    def z(w):
        return c0 * w + c1 * apply_A(w)

    w_prev = v.copy()
    if order == 0:
        return w_prev
    w = z(v)
    for _ in range(order - 1):
        w, w_prev = 2.0 * z(w) - w_prev, w
    return w
