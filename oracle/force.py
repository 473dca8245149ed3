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


# ------------------------------------------------------------------
# Force of the DD-HMC boundary pseudofermion action (Sec. 2.1, 2.3)
#
#   S = |R^-1 phi|^2,   R^-1 = P - P D^-1 D_partialbar,
#
# with P the projector onto the row space of D_partialbar (independent of the
# links: the row space of (1 -+ g_mu) U B is that of (1 -+ g_mu) B for unitary
# U).  With u = P phi, v = D u restricted to Omega-bar, y = D^-1 v and
# chi = R^-1 phi = u - P y (in the range of P):
#
#   dS = -2 Re <chi, dy>,  dy = -D^-1 dD y + D^-1 (dD u restricted to Omega-bar),
#
# so with zeta = D^-+ chi the force is 2 F(zeta, y) - 2 F(zeta on Omega-bar, u),
# two insertions of dD between solved fields (F = force_bilinear).
# Dense linear algebra: tiny lattices only.

def _dense_D(U, shape, p):
    from oracle import dense as Dn
    return Dn.dense_matrix(lambda f: O.apply_D(U, f, p), shape)


def boundary_pieces_dense(U, phi, p: O.DWFParams, box, D=None):
    """(u, y, chi, zeta, P, masks) of the boundary action for the box Omega
    (D: the dense operator of U, if already built)."""
    from oracle import dense as Dn
    dims = O.lattice_dims(U)
    Ls = phi.shape[4]
    shape = phi.shape
    if D is None:
        D = _dense_D(U, shape, p)
    ids = O.box_id_field(dims, [box])
    om = Dn.site_mask_to_dofs(ids == 0, Ls * 12)
    ob = Dn.site_mask_to_dofs(ids < 0, Ls * 12)
    _, P_O = Dn.rowspace_projector(D[np.ix_(ob, om)])
    n = D.shape[0]
    P = np.zeros((n, n), dtype=np.complex128)
    P[np.ix_(om, om)] = P_O
    u = P @ phi.reshape(-1)
    v = np.zeros(n, dtype=np.complex128)
    v[ob] = (D @ u)[ob]
    y = np.linalg.solve(D, v)
    chi = u - P @ y
    zeta = np.linalg.solve(np.conj(D.T), chi)
    return {"u": u.reshape(shape), "y": y.reshape(shape), "chi": chi.reshape(shape),
            "zeta": zeta.reshape(shape), "P": P, "omega_bar": ids < 0}


def boundary_action_dense(U, phi, p: O.DWFParams, box, D=None) -> float:
    """S = |R^-1 phi|^2 with dense P and D^-1."""
    pc = boundary_pieces_dense(U, phi, p, box, D)
    return float(np.vdot(pc["chi"], pc["chi"]).real)


def boundary_action_force_dense(U, phi, p: O.DWFParams, box, active=None) -> np.ndarray:
    """Link force of S = |R^-1 phi|^2: d/d eps S(exp(i eps H) U) = Re tr[i H F]."""
    pc = boundary_pieces_dense(U, phi, p, box)
    zeta_b = O.restrict(pc["zeta"], pc["omega_bar"])
    return (2.0 * force_bilinear(U, pc["zeta"], pc["y"], p, active)
            - 2.0 * force_bilinear(U, zeta_b, pc["u"], p, active))


# ------------------------------------------------------------------
# Hasenbusch ratio of boundary operators (Sec. 2.3): light mass R, heavy
# (Pauli-Villars) mass R_pv,
#
#   S = phi^+ R_pv^+ R^-+ R^-1 R_pv phi = |chi|^2,  chi = R^-1 R_pv phi.
#
# R_pv = P_pv - P_pv D_O^-1 D_d D_Ob^-1 D_db (PV mass); with u_pv = P_pv phi,
# b = D_Ob^-1 (D u_pv on Omega-bar), d = D_O^-1 (D b on Omega): R_pv phi = u_pv - P_pv d.
# dS = 2 Re <chi, dR^-1 w> + 2 Re <xi, dR_pv phi>, w = R_pv phi, xi = R^-+ chi
#    = chi - (D^+ (zeta on Omega-bar)) on Omega,  zeta = D^-+ chi (light mass),
# and <xi, dR_pv phi> = <eta, dD (d - b)> + <kappa, dD (b - u_pv)> with the PV
# local adjoint solves eta = D_O^-+ P_pv xi, kappa = D_Ob^-+ (D^+ eta on Omega-bar):
# four PV local solves (b, d, eta, kappa) and two light solves (y, zeta).
def _blocks_dense(U, shape, p, box, D=None):
    from oracle import dense as Dn
    dims = O.lattice_dims(U)
    Ls = shape[4]
    if D is None:
        D = _dense_D(U, shape, p)
    ids = O.box_id_field(dims, [box])
    om = Dn.site_mask_to_dofs(ids == 0, Ls * 12)
    ob = Dn.site_mask_to_dofs(ids < 0, Ls * 12)
    _, P_O = Dn.rowspace_projector(D[np.ix_(ob, om)])
    n = D.shape[0]
    P = np.zeros((n, n), dtype=np.complex128)
    P[np.ix_(om, om)] = P_O
    return D, P, om, ob


def _dirichlet_solve(D, idx, rhs, adjoint=False):
    """x supported on idx with (D restricted to idx) x = rhs (or its adjoint)."""
    A = D[np.ix_(idx, idx)]
    if adjoint:
        A = np.conj(A.T)
    x = np.zeros_like(rhs)
    x[idx] = np.linalg.solve(A, rhs[idx])
    return x


def ratio_pieces_dense(U, phi, p_light: O.DWFParams, p_pv: O.DWFParams, box, Dl=None, Dp=None):
    shape = phi.shape
    Dl, Pl, om, ob = _blocks_dense(U, shape, p_light, box, Dl)
    Dp, Pp, _, _ = _blocks_dense(U, shape, p_pv, box, Dp)
    n = Dl.shape[0]

    def restrict(v, idx):
        out = np.zeros(n, dtype=np.complex128)
        out[idx] = v[idx]
        return out

    u_pv = Pp @ phi.reshape(-1)
    b = _dirichlet_solve(Dp, ob, restrict(Dp @ u_pv, ob))
    d = _dirichlet_solve(Dp, om, restrict(Dp @ b, om))
    w = u_pv - Pp @ d
    u_l = Pl @ w
    y = np.linalg.solve(Dl, restrict(Dl @ u_l, ob))
    chi = u_l - Pl @ y
    zeta = np.linalg.solve(np.conj(Dl.T), chi)
    xi = chi - restrict(np.conj(Dl.T) @ restrict(zeta, ob), om)
    eta = _dirichlet_solve(Dp, om, Pp @ xi, adjoint=True)
    kappa = _dirichlet_solve(Dp, ob, restrict(np.conj(Dp.T) @ eta, ob), adjoint=True)
    r = {k: v.reshape(shape) for k, v in dict(u_pv=u_pv, b=b, d=d, u_l=u_l, y=y, chi=chi, zeta=zeta,
                                               eta=eta, kappa=kappa).items()}
    r["omega_bar"] = O.box_id_field(O.lattice_dims(U), [box]) < 0
    return r


def ratio_action_dense(U, phi, p_light, p_pv, box, Dl=None, Dp=None) -> float:
    """S = |R^-1 R_pv phi|^2 with dense P, R, R_pv."""
    pc = ratio_pieces_dense(U, phi, p_light, p_pv, box, Dl, Dp)
    return float(np.vdot(pc["chi"], pc["chi"]).real)


def ratio_action_force_dense(U, phi, p_light, p_pv, box, active=None) -> np.ndarray:
    """Link force of the boundary Hasenbusch ratio action."""
    pc = ratio_pieces_dense(U, phi, p_light, p_pv, box)
    zeta_b = O.restrict(pc["zeta"], pc["omega_bar"])
    return (2.0 * force_bilinear(U, pc["zeta"], pc["y"], p_light, active)
            - 2.0 * force_bilinear(U, zeta_b, pc["u_l"], p_light, active)
            + 2.0 * force_bilinear(U, pc["eta"], pc["d"] - pc["b"], p_pv, active)
            + 2.0 * force_bilinear(U, pc["kappa"], pc["b"] - pc["u_pv"], p_pv, active))


# ------------------------------------------------------------------
# One-flavour DD-RHMC boundary term (Sec. 2.3.1): det chi = det D / det D_dir,
# D_dir = D with the links between Omega and Omega-bar cut (eq. ddrhmc).  With
# A = M_pc^+ M_pc of D and A_d that of D_dir on the odd checkerboard and two
# rational functions r1 ~ x^(1/4), r2 ~ x^(-1/2) in partial fractions
# (a0, shifts, residues),
#
#   S = <w, r2(A) w>,  w = r1(A_d) phi.
#
# With z_j = (A_d + s'_j)^-1 phi, x_i = (A + s_i)^-1 w, v = r2(A) w and
# y_j = (A_d + s'_j)^-1 v, the force is
#
#   F = -sum_i rho_i 2 F_M(M x_i, x_i) - 2 sum_j rho'_j [F_Md(M_d z_j, y_j) + F_Md(M_d y_j, z_j)],
#
# F_M(X, Y) the link derivative of Re <X, M_pc Y>: M_pc = D_oo - D_oe D_ee^-1 D_eo
# and D_ee, D_oo do not depend on the links, so
# F_M(X, Y) = -F(X_o, (D_ee^-1 D_eo Y)_e) - F((D_ee^-+ D_oe^+ X)_e, Y_o).
# The formula holds for any rational functions; dense linear algebra.
def _rational_dense(Amat, v, r):
    a0, shifts, residues = r
    n = Amat.shape[0]
    out = a0 * v
    sols = []
    for s, rho in zip(shifts, residues):
        x = np.linalg.solve(Amat + s * np.eye(n), v)
        sols.append(x)
        out = out + rho * x
    return out, sols


class _SchurDense:
    """Dense D of a gauge field, its odd/even blocks and M_pc on odd dofs."""

    def __init__(self, U, p, shape, D=None):
        from oracle import dense as Dn
        dims = O.lattice_dims(U)
        self.U, self.p, self.shape = U, p, shape
        self.D = _dense_D(U, shape, p) if D is None else D
        par = O.parity_field(dims)
        per = shape[4] * 12
        self.od = Dn.site_mask_to_dofs(par == 1, per)
        self.ev = Dn.site_mask_to_dofs(par == 0, per)
        D = self.D
        self.Dee = D[np.ix_(self.ev, self.ev)]
        self.Deo = D[np.ix_(self.ev, self.od)]
        self.Doe = D[np.ix_(self.od, self.ev)]
        self.M = D[np.ix_(self.od, self.od)] - self.Doe @ np.linalg.solve(self.Dee, self.Deo)
        self.A = np.conj(self.M.T) @ self.M

    def full(self, v_o=None, v_e=None):
        f = np.zeros(self.D.shape[0], dtype=np.complex128)
        if v_o is not None:
            f[self.od] = v_o
        if v_e is not None:
            f[self.ev] = v_e
        return f.reshape(self.shape)

    def force_M(self, X_o, Y_o):
        """Link derivative of Re <X_o, M_pc Y_o>."""
        W_e = np.linalg.solve(self.Dee, self.Deo @ Y_o)
        V_e = np.linalg.solve(np.conj(self.Dee.T), np.conj(self.Doe.T) @ X_o)
        return (-force_bilinear(self.U, self.full(v_o=X_o), self.full(v_e=W_e), self.p)
                - force_bilinear(self.U, self.full(v_e=V_e), self.full(v_o=Y_o), self.p))


def _one_flavour_pieces(U, phi, p, box, r1, r2, D=None, Dd=None):
    shape = phi.shape
    L = _SchurDense(U, p, shape, D)
    Ld = _SchurDense(O.cut_gauge(U, [box]), p, shape, Dd)
    ph = phi.reshape(-1)[L.od]
    w, zs = _rational_dense(Ld.A, ph, r1)
    v, xs = _rational_dense(L.A, w, r2)
    return L, Ld, w, v, zs, xs


def one_flavour_action_dense(U, phi, p, box, r1, r2, D=None, Dd=None) -> float:
    """S = <w, r2(A) w>, w = r1(A_d) phi (the odd sites of the full field phi);
    D, Dd: the dense D of U and of the cut field, if already built."""
    _, _, w, v, _, _ = _one_flavour_pieces(U, phi, p, box, r1, r2, D, Dd)
    return float(np.vdot(w, v).real)


def one_flavour_force_dense(U, phi, p, box, r1, r2) -> np.ndarray:
    """Link force of the one-flavour DD-RHMC term S (d/d eps S(exp(i eps H) U) = Re tr[i H F])."""
    L, Ld, w, v, zs, xs = _one_flavour_pieces(U, phi, p, box, r1, r2)
    F = np.zeros(U.shape, dtype=np.complex128)
    for rho, x in zip(r2[2], xs):
        F -= 2.0 * rho * L.force_M(L.M @ x, x)
    n = Ld.A.shape[0]
    for s, rho, z in zip(r1[1], r1[2], zs):
        y = np.linalg.solve(Ld.A + s * np.eye(n), v)
        F -= 2.0 * rho * (Ld.force_M(Ld.M @ z, y) + Ld.force_M(Ld.M @ y, z))
    return F
