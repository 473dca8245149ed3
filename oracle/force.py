"""Oracle: the gauge-link derivative of the fermion bilinear Re <X, D Y>,
plain FP64 numpy (test infrastructure only).

The DD-HMC forces of Sec. 2.3 (the variation of R^-1 = P - P D^-1 D_partialbar,
delta R^-1 = P D^-1 (delta D) D^-1 D_partialbar - P D^-1 delta D_partialbar,
and of the two-flavour and Hasenbusch ratio actions built from it) reduce to
insertions of delta D between two fields X and Y obtained by solves: every
term is d/d eps Re <X, D(U_eps) Y> for a variation of one link at a time.
This module states that derivative for every link.

D = D_W (b5 + c5 S5) + (1 - S5) depends on the links only through the hop of
D_W = (4 - M5) - Dh / 2, so with Z = (b5 + c5 S5) Y,

    Re <X, D Y> = const - 1/2 Re <X, Dh Z>.

For the link U_mu(x), Dh contributes X(x)^+ (1 - g_mu) U_mu(x) Z(x + mu) and
X(x + mu)^+ (1 + g_mu) U_mu(x)^+ Z(x), summed over s, spin and colour.  In
colour space those are tr[U M1] and tr[U^+ M2] with

    M1 = sum_{s, spin} Z(x + mu) ((1 - g_mu) X(x))^+,
    M2 = sum_{s, spin} Z(x) ((1 + g_mu) X(x + mu))^+.

Under U -> U + i eps H U (H Hermitian traceless: the tangent of
U -> exp(i eps H) U), Re tr[dU M1] + Re tr[dU^+ M2] = Re tr[i eps H U (M1 + M2^+)],
and only the traceless anti-Hermitian part of U (M1 + M2^+) survives the
real part.  The force of a link is therefore the traceless anti-Hermitian
3 x 3 matrix

    F_mu(x) = -1/2 TA[ U_mu(x) (M1 + M2^+) ],   TA(A) = (A - A^+)/2 - tr(A - A^+)/6,

with d/d eps Re <X, D(exp(i eps H) U) Y> at eps = 0 equal to Re tr[i H F_mu(x)].
Several right-hand sides are summed.  ``active`` (a boolean 4D mask over
links [t, z, y, x, mu]) keeps the forces of the links the DD-HMC updates and
zeroes the rest (Sec. 2.3: links in the band are held fixed).
"""

from __future__ import annotations

import numpy as np

from oracle import dwf as O


def traceless_antihermitian(A: np.ndarray) -> np.ndarray:
    """TA(A) = (A - A^+)/2 - tr(A - A^+)/6 * 1 on the last two axes."""
    ah = 0.5 * (A - np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(ah, axis1=-2, axis2=-1)
    return ah - (tr / 3.0)[..., None, None] * np.eye(3)


def force_bilinear(U: np.ndarray, X, Y, p: O.DWFParams, active=None) -> np.ndarray:
    """F[t, z, y, x, mu, a, b]: the link derivative of sum_r Re <X_r, D Y_r>.

    X, Y: one field or a list of fields (t, z, y, x, s, spin, colour)."""
    Xs = X if isinstance(X, (list, tuple)) else [X]
    Ys = Y if isinstance(Y, (list, tuple)) else [Y]
    g, _ = O.gammas()
    one = np.eye(4, dtype=np.complex128)
    F = np.zeros(U.shape, dtype=np.complex128)
    for Xr, Yr in zip(Xs, Ys):
        Z = O.five_b(Yr, p)
        for mu in range(4):
            ax = O.AXIS[mu]
            Xf = np.roll(Xr, -1, axis=ax)                       # X(x + mu)
            Zf = np.roll(Z, -1, axis=ax)                        # Z(x + mu)
            W1 = np.einsum("ij,tzyxsjb->tzyxsib", one - g[mu], Xr)
            W2 = np.einsum("ij,tzyxsjb->tzyxsib", one + g[mu], Xf)
            M1 = np.einsum("tzyxsia,tzyxsib->tzyxab", Zf, np.conj(W1))
            M2 = np.einsum("tzyxsia,tzyxsib->tzyxab", Z, np.conj(W2))
            M = M1 + np.conj(np.swapaxes(M2, -1, -2))
            F[..., mu, :, :] += -0.5 * traceless_antihermitian(U[..., mu, :, :] @ M)
    if active is not None:
        F = F * active[..., None, None]
    return F


def box_links(dims, box) -> np.ndarray:
    """Links [t, z, y, x, mu] with both ends x and x + mu inside the box."""
    m = O.box_mask(dims, box)
    out = np.zeros(m.shape + (4,), dtype=bool)
    for mu in range(4):
        out[..., mu] = m & np.roll(m, -1, axis=O.AXIS[mu])
    return out
