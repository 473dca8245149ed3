"""Oracle: dense matrices of field operators on tiny lattices (test-only).

Used for the brute-force pins (LU inverse, determinants) and for the block
algebra of Sec. 2.1: the block form of D over Omega and Omega-bar, its Schur
factorisation, eq. (schur) det D = det D_Omega det D_Omega-bar det chi, the
boundary matrix R and its inverse, and eq. (ddrhmc).
"""

from __future__ import annotations

import numpy as np


def dense_matrix(apply, shape) -> np.ndarray:
    """Matrix of the linear map ``apply`` on complex arrays of ``shape``,
    built column by column from unit vectors (flattened C order)."""
    n = int(np.prod(shape))
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = apply(e.reshape(shape)).reshape(-1)
        e[j] = 0.0
    return M


def site_mask_to_dofs(mask4d: np.ndarray, inner: int) -> np.ndarray:
    """Indices of the flattened field components on the sites where the 4D
    boolean mask holds (``inner`` = components per 4D site, Ls * 12)."""
    sites = np.flatnonzero(mask4d.reshape(-1))
    return (sites[:, None] * inner + np.arange(inner)[None, :]).reshape(-1)


def blocks(D: np.ndarray, omega: np.ndarray, omegabar: np.ndarray):
    """Block form of Sec. 2.1: (D_Omega, D_partial, D_partialbar,
    D_Omegabar) where D_partial connects Omega-bar (columns) to Omega (rows)
    and D_partialbar connects Omega (columns) to Omega-bar (rows)."""
    return (D[np.ix_(omega, omega)], D[np.ix_(omega, omegabar)],
            D[np.ix_(omegabar, omega)], D[np.ix_(omegabar, omegabar)])


def chi_matrix(D_O, D_d, D_db, D_Ob) -> np.ndarray:
    """chi = 1 - D_Omega^-1 D_partial D_Omegabar^-1 D_partialbar."""
    n = D_O.shape[0]
    return np.eye(n) - np.linalg.solve(D_O, D_d @ np.linalg.solve(D_Ob, D_db))


def rowspace_projector(A: np.ndarray, rtol: float = 1e-10):
    """Orthonormal basis V of the row space of A and the projector V V^+:
    the components on which A acts non-trivially (A P = A)."""
    _, s, vh = np.linalg.svd(A, full_matrices=True)
    k = int(np.sum(s > rtol * s[0])) if s.size else 0
    V = np.conj(vh[:k]).T
    return V, V @ np.conj(V).T


def logdet(M: np.ndarray) -> complex:
    """log det M (complex), from LU via slogdet."""
    sign, ld = np.linalg.slogdet(M)
    return np.log(sign) + ld
