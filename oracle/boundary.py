"""Oracle: matrix-free boundary operator of Sec. 2.1 for lattices too large for
dense matrices (test infrastructure only).

P, the orthogonal projector onto the row space of D_partialbar, acts site by
site on Omega: at a site x the row space is colour-blind and spanned, in the
(spin, s) space, by B^+ [range(1 -+ g_mu) x C^Ls] over the neighbours outside
Omega ((1 - g_mu) for x - mu, (1 + g_mu) for x + mu), B^+ = b5 + c5 S5^+.
Here that span is orthonormalised by an SVD of the stacked columns (this is
exact only when no site of Omega-bar touches two sites of Omega, the case of
a box with a band of width >= 2).  R^-1 = P - P D^-1 D_partialbar uses the
oracle's CGNE; the force of |R^-1 phi|^2 needs zeta = D^-+ chi, solved here by
plain CG on D D^+ (D D^+ zeta = D chi), and the insertions of oracle.force.
"""

from __future__ import annotations

import numpy as np

from oracle import dwf as O
from oracle.force import force_bilinear


def _site_projector(pattern, Ls, p: O.DWFParams):
    """4 Ls x 4 Ls projector (index spin * Ls + s) for one crossing pattern:
    pattern = tuple of (mu, sign), sign +1 for x + mu outside, -1 for x - mu."""
    g, _ = O.gammas()
    one = np.eye(4)
    cols = []
    for mu, sgn in pattern:
        Pm = one + sgn * g[mu]                  # (1 + g) for x + mu, (1 - g) for x - mu
        for col in range(4):
            for s in range(Ls):
                v = np.zeros((Ls, 4, 3), dtype=np.complex128)
                v[s, :, 0] = Pm[:, col]
                w = O.five_b(v[None, None, None, None], p, dagger=True)[0, 0, 0, 0]
                cols.append(w[:, :, 0].T.reshape(-1))     # (spin, s) order
    A = np.array(cols).T
    u, sv, _ = np.linalg.svd(A, full_matrices=False)
    k = int(np.sum(sv > 1e-10 * sv[0]))
    Q = u[:, :k]
    return Q @ np.conj(Q.T)


def project(phi, box, p: O.DWFParams):
    """P phi (zero outside Omega)."""
    dims = O.lattice_dims(phi)
    Ls = phi.shape[4]
    inside = O.box_mask(dims, box)
    out = np.zeros_like(phi)
    cache = {}
    Lt, Lz, Ly, Lx = inside.shape
    for t in range(Lt):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    if not inside[t, z, y, x]:
                        continue
                    c = [x, y, z, t]
                    pat = []
                    for mu in range(4):
                        for sgn in (1, -1):
                            n = list(c)
                            n[mu] = (n[mu] + sgn) % dims[mu]
                            if not inside[n[3], n[2], n[1], n[0]]:
                                pat.append((mu, sgn))
                    if not pat:
                        continue
                    key = tuple(pat)
                    if key not in cache:
                        cache[key] = _site_projector(key, Ls, p)
                    Pm = cache[key]
                    v = phi[t, z, y, x]                          # (Ls, 4, 3)
                    vs = v.transpose(1, 0, 2).reshape(4 * Ls, 3)  # (spin, s) x colour
                    out[t, z, y, x] = (Pm @ vs).reshape(4, Ls, 3).transpose(1, 0, 2)
    return out


def _cg_hpd(apply_A, b, tol, maxiter=200000):
    x = np.zeros_like(b)
    r = b.copy()
    p_ = r.copy()
    rr = np.vdot(r, r).real
    bn = np.sqrt(np.vdot(b, b).real)
    for _ in range(maxiter):
        if np.sqrt(rr) <= tol * bn:
            break
        Ap = apply_A(p_)
        a = rr / np.vdot(p_, Ap).real
        x = x + a * p_
        r = r - a * Ap
        rr, rr_old = np.vdot(r, r).real, rr
        p_ = r + (rr / rr_old) * p_
    return x


def rinv_pieces(U, phi, p: O.DWFParams, box, tol=1e-12):
    """u = P phi, y = D^-1 (D u on Omega-bar), chi = R^-1 phi, zeta = D^-+ chi."""
    dims = O.lattice_dims(U)
    outside = ~O.box_mask(dims, box)
    u = project(phi, box, p)
    v = O.restrict(O.apply_D(U, u, p), outside)
    y, _ = O.cgne(U, v, p, tol=tol)
    chi = u - project(y, box, p)
    zeta = _cg_hpd(lambda f: O.apply_D(U, O.apply_D(U, f, p, True), p), O.apply_D(U, chi, p), tol)
    return u, y, chi, zeta, outside


def rinv(U, phi, p: O.DWFParams, box, tol=1e-12):
    """R^-1 phi = P phi - P D^-1 (D P phi on Omega-bar)."""
    return rinv_pieces(U, phi, p, box, tol)[2]


def boundary_action_force(U, phi, p: O.DWFParams, box, tol=1e-12, active=None):
    """Link force of |R^-1 phi|^2: 2 F(zeta, y) - 2 F(zeta on Omega-bar, u)."""
    u, y, chi, zeta, outside = rinv_pieces(U, phi, p, box, tol)
    return (2.0 * force_bilinear(U, zeta, y, p, active)
            - 2.0 * force_bilinear(U, O.restrict(zeta, outside), u, p, active))
