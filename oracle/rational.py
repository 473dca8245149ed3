"""Oracle: Zolotarev's optimal rational approximation of 1/sqrt(x), plain
numpy / scipy (test infrastructure only).

The one-flavour DD-RHMC term of Sec. 2.3.1 needs (D^+ D)^(-1/2) (and
fractional powers of D_dir^+ D_dir) as rational functions in partial
fractions, evaluated by multi-shift CG.  For 1/sqrt(x) on [lo, hi] the
optimal relative (minimax) approximation of type (n - 1, n) is known in closed
form (Zolotarev): on y = x / lo in [1, b], b = hi / lo, with the complementary
parameter m' = 1 - 1/b and K' = K(m'),

    c_l = sn^2(l K' / (2n) | m') / cn^2(l K' / (2n) | m'),   l = 1 .. 2n - 1,
    r(y) = d0 prod_{i=1}^{n-1} (y + c_{2i}) / prod_{j=1}^{n} (y + c_{2j-1}),

the odd c the poles and the even c the zeros; d0 centres the relative error
1 - sqrt(y) r(y) so that it equioscillates between +delta and -delta.  In
partial fractions, 1/sqrt(x) ~ sum_j residue_j / (x + shift_j) with
shift_j = lo c_{2j-1} and residue_j = d0 sqrt(lo) R_j, R_j the residue of the
product form at y = -c_{2j-1}.  The elliptic functions are scipy's.
"""

from __future__ import annotations

import numpy as np
from scipy import special


def _product_form(c, n, y):
    num = np.ones_like(y)
    den = np.ones_like(y)
    for i in range(1, n):
        num = num * (y + c[2 * i - 1])
    for j in range(1, n + 1):
        den = den * (y + c[2 * j - 2])
    return num / den


def zolotarev_inv_sqrt(n: int, lo: float, hi: float, grid: int = 200001):
    """(shifts, residues, delta): 1/sqrt(x) ~ sum residues / (x + shifts) on [lo, hi]."""
    if n < 1 or not (0 < lo < hi):
        raise ValueError("n >= 1 and 0 < lo < hi")
    b = hi / lo
    mp = 1.0 - 1.0 / b
    Kp = special.ellipk(mp)
    c = []
    for l in range(1, 2 * n):
        sn, cn, _, _ = special.ellipj(l * Kp / (2 * n), mp)
        c.append(sn * sn / (cn * cn))
    y = np.geomspace(1.0, b, grid)
    e = np.sqrt(y) * _product_form(c, n, y)
    d0 = 2.0 / (e.max() + e.min())
    delta = (e.max() - e.min()) / (e.max() + e.min())
    poles = [c[2 * j - 2] for j in range(1, n + 1)]
    zeros = [c[2 * i - 1] for i in range(1, n)]
    shifts, residues = [], []
    for j, p in enumerate(poles):
        R = np.prod([z - p for z in zeros]) / np.prod([q - p for k, q in enumerate(poles) if k != j])
        shifts.append(lo * p)
        residues.append(d0 * np.sqrt(lo) * R)
    return np.array(shifts), np.array(residues), float(delta)


def partial_fraction_eval(x, shifts, residues, a0=0.0):
    x = np.asarray(x, dtype=float)
    out = np.full_like(x, a0)
    for s, r in zip(shifts, residues):
        out = out + r / (x + s)
    return out


def zolotarev_inv_sqrt_nn(n: int, lo: float, hi: float, grid: int = 200001):
    """(a0, shifts, residues, delta): the optimal relative approximation of
    1/sqrt(x) on [lo, hi] of type (n, n), 1/sqrt(x) ~ a0 + sum residues /
    (x + shifts).  Zolotarev's closed form with 2n + 1 in place of 2n: on
    y = x / lo, c_l = sn^2/cn^2(l K' / (2n + 1) | m') for l = 1 .. 2n, poles
    c_1, c_3, .., c_{2n-1}, zeros c_2, .., c_{2n}, and r(y) = D prod (y + zeros)
    / prod (y + poles) with D centring the relative error (which then
    equioscillates at 2n + 2 points)."""
    if n < 1 or not (0 < lo < hi):
        raise ValueError("n >= 1 and 0 < lo < hi")
    b = hi / lo
    mp = 1.0 - 1.0 / b
    Kp = special.ellipk(mp)
    c = []
    for l in range(1, 2 * n + 1):
        sn, cn, _, _ = special.ellipj(l * Kp / (2 * n + 1), mp)
        c.append(sn * sn / (cn * cn))
    poles = np.array(c[0::2])
    zeros = np.array(c[1::2])
    y = np.geomspace(1.0, b, grid)
    prod = np.ones_like(y)
    for z, p in zip(zeros, poles):
        prod = prod * (y + z) / (y + p)
    e = np.sqrt(y) * prod
    D = 2.0 / (e.max() + e.min())
    delta = (e.max() - e.min()) / (e.max() + e.min())
    residues = []
    for j, p in enumerate(poles):
        R = D * np.prod(zeros - p) / np.prod([q - p for k, q in enumerate(poles) if k != j])
        residues.append(R)
    # back to x = lo y: r(x) = lo^(-1/2) (D + sum R / (x / lo + p))
    s = lo ** -0.5
    return s * D, lo * poles, s * lo * np.array(residues), float(delta)
