"""Oracle: 5D domain wall fermion operator in plain FP64 numpy (test-only).

The paper (Sec. 1, Sec. 2.3) names the domain wall operator D, its red-black
(even-odd) preconditioned solves and the Dirichlet block operator D_Omega
(Sec. 2.1, Sec. 2.4) but never writes D out.  The definitions below are the
standard Shamir / Moebius conventions, adopted as readings:

* chiral gamma basis: gamma_k = [[0, -i s_k], [i s_k, 0]] (k = 1..3),
  gamma_4 = [[0, 1], [1, 0]], gamma_5 = g1 g2 g3 g4 = diag(1, 1, -1, -1),
  P_+- = (1 +- gamma_5)/2, direction mu = 0..3 <-> gamma_1..gamma_4 <-> x..t;
* Wilson hop  (Dh psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
                                 + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu);
* Wilson operator D_W = (4 - M5) - Dh/2;
* fifth-dimension hop S5 psi_s = P_- psi_{s+1} + P_+ psi_{s-1} with the
  walls psi_{Ls} := -m_f psi_0 and psi_{-1} := -m_f psi_{Ls-1};
* Moebius D = D_W (b5 + c5 S5) + (1 - S5); Shamir is (b5, c5) = (1, 0);
* adjoint D^+ = (b5 + c5 S5^+) D_W^+ + (1 - S5^+), where D_W^+ swaps the
  hop projectors and S5^+ psi_s = P_+ psi_{s+1} + P_- psi_{s-1};
* even-odd split by 4D parity p(x) = (x+y+z+t) mod 2:
  M_ee = M_oo = d + e S5, d = b5 (4-M5) + 1, e = c5 (4-M5) - 1,
  M_eo, M_oe = the hop part H = -Dh (b5 + c5 S5)/2 restricted to parities;
* Schur operator on the odd checkerboard M_pc = M_oo - M_oe M_ee^-1 M_eo.

Fields are full-lattice arrays psi[t, z, y, x, s, spin, colour] (complex128),
gauge fields U[t, z, y, x, mu, a, b].  Even-odd restricted fields are stored
in the same shape with zeros on the other parity.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# array axis of direction mu for arrays ordered (t, z, y, x, ...)
AXIS = (3, 2, 1, 0)


# ---------------------------------------------------------------- basics
def gammas():
    """Chiral-basis Euclidean gamma matrices: (gamma[0..3], gamma_5)."""
    sig = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
           np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
           np.array([[1, 0], [0, -1]], dtype=np.complex128)]
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    for k in range(3):
        g[k, 0:2, 2:4] = -1j * sig[k]
        g[k, 2:4, 0:2] = 1j * sig[k]
    g[3, 0:2, 2:4] = np.eye(2)
    g[3, 2:4, 0:2] = np.eye(2)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


@dataclass(frozen=True)
class DWFParams:
    """Operator parameters: Shamir is b5 = 1, c5 = 0."""
    M5: float
    mf: float
    b5: float = 1.0
    c5: float = 0.0

    @property
    def d(self) -> float:
        """Diagonal coefficient of M_ee = d + e S5."""
        return self.b5 * (4.0 - self.M5) + 1.0

    @property
    def e(self) -> float:
        """S5 coefficient of M_ee = d + e S5."""
        return self.c5 * (4.0 - self.M5) - 1.0


def lattice_dims(psi_or_U) -> tuple:
    """(Lx, Ly, Lz, Lt) of a field or gauge array."""
    Lt, Lz, Ly, Lx = psi_or_U.shape[:4]
    return (Lx, Ly, Lz, Lt)


def parity_field(dims) -> np.ndarray:
    """4D parity (x+y+z+t) mod 2 as an array (t, z, y, x)."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return (x + y + z + t) % 2


def restrict(psi: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """psi on the sites where the 4D boolean ``mask`` holds, zero elsewhere."""
    return psi * mask[..., None, None, None]


def parity_part(psi: np.ndarray, p: int) -> np.ndarray:
    """Restriction to the 4D checkerboard of parity ``p``."""
    return restrict(psi, parity_field(lattice_dims(psi)) == p)


# ------------------------------------------------------------ Wilson hop
def hop(U: np.ndarray, psi: np.ndarray, dagger: bool = False) -> np.ndarray:
    """Wilson hop Dh psi (or Dh^+ psi, projectors swapped), full 4x4 spin
    matrices, no spin projection trick."""
    g, _ = gammas()
    one = np.eye(4, dtype=np.complex128)
    sgn = 1.0 if dagger else -1.0
    out = np.zeros_like(psi)
    for mu in range(4):
        ax = AXIS[mu]
        Pf = one + sgn * g[mu]          # forward projector: (1 - gamma_mu)
        Pb = one - sgn * g[mu]          # backward projector: (1 + gamma_mu)
        Umu = U[..., mu, :, :]
        fwd = np.roll(psi, -1, axis=ax)                 # psi(x + mu)
        t = np.einsum("tzyxab,tzyxsib->tzyxsia", Umu, fwd)
        out += np.einsum("ij,tzyxsja->tzyxsia", Pf, t)
        Ub = np.roll(Umu, 1, axis=ax)                   # U_mu(x - mu)
        bwd = np.roll(psi, 1, axis=ax)                  # psi(x - mu)
        t = np.einsum("tzyxba,tzyxsib->tzyxsia", np.conj(Ub), bwd)
        out += np.einsum("ij,tzyxsja->tzyxsia", Pb, t)
    return out


def wilson(U, psi, M5: float, dagger: bool = False) -> np.ndarray:
    """D_W(-M5) psi = (4 - M5) psi - Dh psi / 2 (or its adjoint)."""
    return (4.0 - M5) * psi - 0.5 * hop(U, psi, dagger)


# ------------------------------------------------------ fifth dimension
def _shift_plus(psi, mf):
    """(S_+ psi)_s = psi_{s+1}, psi_{Ls} := -m_f psi_0."""
    return np.concatenate([psi[..., 1:, :, :], -mf * psi[..., 0:1, :, :]], axis=4)


def _shift_minus(psi, mf):
    """(S_- psi)_s = psi_{s-1}, psi_{-1} := -m_f psi_{Ls-1}."""
    return np.concatenate([-mf * psi[..., -1:, :, :], psi[..., :-1, :, :]], axis=4)


def s5(psi: np.ndarray, mf: float, dagger: bool = False) -> np.ndarray:
    """S5 psi = P_- S_+ psi + P_+ S_- psi; adjoint P_+ S_+ + P_- S_-."""
    sp, sm = _shift_plus(psi, mf), _shift_minus(psi, mf)
    out = np.empty_like(psi)
    if not dagger:
        out[..., 0:2, :] = sm[..., 0:2, :]
        out[..., 2:4, :] = sp[..., 2:4, :]
    else:
        out[..., 0:2, :] = sp[..., 0:2, :]
        out[..., 2:4, :] = sm[..., 2:4, :]
    return out


def five_b(psi, p: DWFParams, dagger: bool = False) -> np.ndarray:
    """(b5 + c5 S5) psi (or with S5^+)."""
    return p.b5 * psi + p.c5 * s5(psi, p.mf, dagger)


# ------------------------------------------------------ full operator
def apply_D(U, psi, p: DWFParams, dagger: bool = False) -> np.ndarray:
    """Moebius / Shamir domain wall operator D psi (or D^+ psi)."""
    if not dagger:
        return wilson(U, five_b(psi, p), p.M5) + psi - s5(psi, p.mf)
    return (five_b(wilson(U, psi, p.M5, True), p, True)
            + psi - s5(psi, p.mf, True))


def hop_part(U, psi, p: DWFParams, dagger: bool = False) -> np.ndarray:
    """Off-diagonal (parity-changing) part H of D: H = -Dh (b5 + c5 S5)/2;
    adjoint H^+ = -(b5 + c5 S5^+) Dh^+ / 2.  Applied to a field of parity q
    it returns M_{1-q, q} psi (or the adjoint block)."""
    if not dagger:
        return -0.5 * hop(U, five_b(psi, p))
    return -0.5 * five_b(hop(U, psi, True), p, True)


def mooee(psi, p: DWFParams, dagger: bool = False) -> np.ndarray:
    """Site-diagonal block M_ee = M_oo = d + e S5 (or d + e S5^+)."""
    return p.d * psi + p.e * s5(psi, p.mf, dagger)


def mooee_inv_matrices(Ls: int, p: DWFParams, dagger: bool = False):
    """Closed-form Ls x Ls inverses of M_ee per chirality: (upper, lower).

    With alpha = e/d and S_-^Ls = S_+^Ls = -m_f, the inverse of d + e S_- is
    (-alpha)^k c / (d (1 + m_f (-alpha)^Ls)), k = (s - t) mod Ls, c = 1 for
    t <= s and -m_f otherwise; d + e S_+ is the same with s and t swapped.
    Non-adjoint: upper spins see S_-, lower spins S_+; the adjoint swaps them.
    """
    d, e, mf = p.d, p.e, p.mf
    a = -e / d
    den = d * (1.0 + mf * a ** Ls)
    s = np.arange(Ls)[:, None]
    t = np.arange(Ls)[None, :]
    minus = np.where(t <= s, 1.0, -mf) * a ** ((s - t) % Ls) / den
    plus = np.where(t >= s, 1.0, -mf) * a ** ((t - s) % Ls) / den
    return (plus, minus) if dagger else (minus, plus)


def mooee_inv(psi, p: DWFParams, dagger: bool = False) -> np.ndarray:
    """M_ee^-1 psi (or (M_ee^+)^-1 psi) from the closed form."""
    Ls = psi.shape[4]
    up, lo = mooee_inv_matrices(Ls, p, dagger)
    out = np.empty_like(psi)
    out[..., 0:2, :] = np.einsum("st,...tia->...sia", up, psi[..., 0:2, :])
    out[..., 2:4, :] = np.einsum("st,...tia->...sia", lo, psi[..., 2:4, :])
    return out


def mpc(U, psi_o, p: DWFParams, dagger: bool = False) -> np.ndarray:
    """Schur operator on the odd checkerboard (or its adjoint):
    M_pc = M_oo - M_oe M_ee^-1 M_eo,  M_pc^+ = M_oo^+ - M_eo^+ M_ee^-+ M_oe^+.
    ``psi_o`` must vanish on even sites; the result does too."""
    t = hop_part(U, psi_o, p, dagger)              # even checkerboard
    t = mooee_inv(t, p, dagger)
    t = hop_part(U, t, p, dagger)                  # odd checkerboard
    return mooee(psi_o, p, dagger) - t


def eo_block(U, psi, p: DWFParams, out_parity: int, dagger: bool = False):
    """M_{out, 1-out} psi_{1-out} (or (M_{1-out, out})^+ psi_{1-out})."""
    src = parity_part(psi, 1 - out_parity)
    return parity_part(hop_part(U, src, p, dagger), out_parity)


# ------------------------------------------------------------ solver
def norm(v) -> float:
    return float(np.sqrt(np.vdot(v, v).real))


def schur_source(U, b, p: DWFParams) -> np.ndarray:
    """b'_o = b_o - M_oe M_ee^-1 b_e."""
    be, bo = parity_part(b, 0), parity_part(b, 1)
    return bo - parity_part(hop_part(U, mooee_inv(be, p), p), 1)


def reconstruct_even(U, b, x_o, p: DWFParams) -> np.ndarray:
    """x_e = M_ee^-1 (b_e - M_eo x_o)."""
    be = parity_part(b, 0)
    return mooee_inv(be - parity_part(hop_part(U, x_o, p), 0), p)


def cgne(U, b, p: DWFParams, tol: float = 1e-10, maxiter: int = 100000,
         x_iterates=None):
    """Even-odd preconditioned CGNE: CG on M_pc^+ M_pc x_o = M_pc^+ b'_o from
    x_o = 0, then x_e = M_ee^-1 (b_e - M_eo x_o).  Stops when the true
    residual |b - D x| / |b| = |b'_o - M_pc x_o| / |b| is <= tol.

    Returns (x, info) with info = dict(iters, true_resid).  If
    ``x_iterates`` is a list, every odd-checkerboard iterate x_o is appended.
    """
    bnorm = norm(b)
    bp = schur_source(U, b, p)
    rhs = mpc(U, bp, p, True)
    x = np.zeros_like(b)
    r = rhs.copy()
    pv = r.copy()
    rr = np.vdot(r, r).real
    rhs_norm = np.sqrt(rr)
    target = tol * rhs_norm
    it = 0
    true_res = norm(bp) / bnorm
    while it < maxiter:
        t = mpc(U, pv, p)
        pAp = np.vdot(t, t).real
        alpha = rr / pAp
        x = x + alpha * pv
        r = r - alpha * mpc(U, t, p, True)
        rr_new = np.vdot(r, r).real
        it += 1
        if x_iterates is not None:
            x_iterates.append(x.copy())
        if np.sqrt(rr_new) <= target:
            true_res = norm(bp - mpc(U, x, p)) / bnorm
            if true_res <= tol:
                break
            target *= 0.5
        pv = r + (rr_new / rr) * pv
        rr = rr_new
    xe = reconstruct_even(U, b, x, p)
    return xe + x, {"iters": it, "true_resid": true_res}


def true_residual(U, x, b, p: DWFParams) -> float:
    """|b - D x| / |b| in FP64."""
    return norm(b - apply_D(U, x, p)) / norm(b)


# ------------------------------------------------- Dirichlet blocks
def box_id_field(dims, boxes) -> np.ndarray:
    """Array (t, z, y, x) holding the index of the box containing each site
    (boxes given as (origin[4], extent[4]) in (x, y, z, t) order, periodic
    wrap allowed) and -1 for sites of the complement Omega-bar."""
    Lx, Ly, Lz, Lt = dims
    L = (Lx, Ly, Lz, Lt)
    ids = -np.ones((Lt, Lz, Ly, Lx), dtype=np.int64)
    for k, (org, ext) in enumerate(boxes):
        sel = [((np.arange(L[mu]) - org[mu]) % L[mu]) < ext[mu] for mu in range(4)]
        m = (sel[3][:, None, None, None] & sel[2][None, :, None, None]
             & sel[1][None, None, :, None] & sel[0][None, None, None, :])
        if np.any(ids[m] >= 0):
            raise ValueError("boxes overlap")
        ids[m] = k
    return ids


def band_box(dims, w: int, dirs=(0, 1, 2, 3)):
    """Interior box Omega of a cell of the size of the lattice with a
    Dirichlet band of width ``w`` (Sec. 2.2 and Sec. 2.4: a layer of sites on
    the node surface is inactive).  In each cut direction the sites with
    (x mod L) in [L - ceil(w/2), L) or [0, floor(w/2)) belong to Omega-bar."""
    org, ext = [0] * 4, list(dims)
    for mu in dirs:
        org[mu] = w // 2
        ext[mu] = dims[mu] - w
    return (tuple(org), tuple(ext))


def cut_gauge(U, boxes) -> np.ndarray:
    """Dirichlet wrapper of Sec. 2.4: zero every link U_mu(x) whose two ends
    x and x + mu lie in different blocks (Omega-bar or different boxes).  The
    edges are found by comparing the block mask with its shift by one in
    each direction."""
    ids = box_id_field(lattice_dims(U), boxes)
    Uc = U.copy()
    for mu in range(4):
        shifted = np.roll(ids, -1, axis=AXIS[mu])      # block of x + mu
        Uc[..., mu, :, :] *= (ids == shifted)[..., None, None]
    return Uc


def dirichlet_D(U, psi, p: DWFParams, boxes, dagger: bool = False):
    """D_Omega psi in mask form: sum over boxes B of P_B D P_B psi (Sec. 2.1:
    the part of D connecting Omega with itself, each box its own block)."""
    ids = box_id_field(lattice_dims(U), boxes)
    out = np.zeros_like(psi)
    for k in range(len(boxes)):
        m = ids == k
        out += restrict(apply_D(U, restrict(psi, m), p, dagger), m)
    return out


def dirichlet_D_cut(U, psi, p: DWFParams, boxes, dagger: bool = False):
    """D_Omega psi in cut-link form: P_Omega D(U_cut) P_Omega psi."""
    m = box_id_field(lattice_dims(U), boxes) >= 0
    return restrict(apply_D(cut_gauge(U, boxes), restrict(psi, m), p, dagger), m)


# ------------------------------------------ per-site (sampled) checks
def hop_site(U, psi, site, dagger: bool = False) -> np.ndarray:
    """(Dh psi) at one 4D site (x, y, z, t): array (Ls, 4, 3).  Plain loops
    over the eight neighbours, for sampled checks on large lattices."""
    g, _ = gammas()
    one = np.eye(4, dtype=np.complex128)
    sgn = 1.0 if dagger else -1.0
    L = lattice_dims(U)
    x = list(site)
    out = np.zeros(psi.shape[4:], dtype=np.complex128)
    for mu in range(4):
        xf = list(x); xf[mu] = (x[mu] + 1) % L[mu]
        xb = list(x); xb[mu] = (x[mu] - 1) % L[mu]
        Uf = U[x[3], x[2], x[1], x[0], mu]
        Ub = U[xb[3], xb[2], xb[1], xb[0], mu]
        pf = psi[xf[3], xf[2], xf[1], xf[0]]            # (Ls, 4, 3)
        pb = psi[xb[3], xb[2], xb[1], xb[0]]
        out += np.einsum("ij,ab,sjb->sia", one + sgn * g[mu], Uf, pf)
        out += np.einsum("ij,ba,sjb->sia", one - sgn * g[mu], np.conj(Ub), pb)
    return out


def eo_block_site(U, psi, p: DWFParams, site, dagger: bool = False):
    """M_{p,1-p} psi at one 4D site (off-diagonal block of D, or of D^+):
    -Dh (b5 + c5 S5) psi / 2, resp. -(b5 + c5 S5^+) Dh^+ psi / 2, evaluated
    from the nine sites involved only.  Returns (Ls, 4, 3)."""
    if dagger:
        h = hop_site(U, psi, site, True)
        return -0.5 * five_b(h[None, None, None, None], p, True)[0, 0, 0, 0]
    L = lattice_dims(U)
    x = list(site)
    g, _ = gammas()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros(psi.shape[4:], dtype=np.complex128)
    for mu in range(4):
        xf = list(x); xf[mu] = (x[mu] + 1) % L[mu]
        xb = list(x); xb[mu] = (x[mu] - 1) % L[mu]
        pf = five_b(psi[xf[3], xf[2], xf[1], xf[0]][None, None, None, None], p)[0, 0, 0, 0]
        pb = five_b(psi[xb[3], xb[2], xb[1], xb[0]][None, None, None, None], p)[0, 0, 0, 0]
        Uf = U[x[3], x[2], x[1], x[0], mu]
        Ub = U[xb[3], xb[2], xb[1], xb[0], mu]
        out += np.einsum("ij,ab,sjb->sia", one - g[mu], Uf, pf)
        out += np.einsum("ij,ba,sjb->sia", one + g[mu], np.conj(Ub), pb)
    return -0.5 * out


# ----------------------------------------- operators of one Dirichlet block
def eo_block_in(U, psi, p: DWFParams, mask, out_parity: int, dagger: bool = False):
    """Off-diagonal block of P D P (mask form of D_Omega, Sec. 2.1) from
    parity 1 - out_parity to out_parity: P M_{out,1-out} P psi (or adjoint)."""
    src = restrict(parity_part(psi, 1 - out_parity), mask)
    return restrict(parity_part(hop_part(U, src, p, dagger), out_parity), mask)


def mpc_in(U, psi_o, p: DWFParams, mask, dagger: bool = False):
    """Schur operator of the Dirichlet block P D P on the sites of ``mask``
    (M_oo - M_oe M_ee^-1 M_eo with every hop restricted to the block)."""
    H = lambda f: restrict(hop_part(U, restrict(f, mask), p, dagger), mask)
    t = mooee_inv(H(psi_o), p, dagger)
    return restrict(mooee(psi_o, p, dagger), mask) - H(t)


def box_mask(dims, box) -> np.ndarray:
    """Boolean 4D mask of one box (origin, extent), periodic wrap allowed."""
    return box_id_field(dims, [box]) == 0


class _SiteField:
    """A field given site by site: ``f[t, z, y, x]`` -> (Ls, 4, 3) array from
    ``value(site)``, site = (x, y, z, t), computed once per site.  ``shape``
    is that of the full-lattice array it stands for."""

    def __init__(self, shape, value):
        self.shape = tuple(shape)
        self._value = value
        self._memo = {}

    def __getitem__(self, key):
        t, z, y, x = (int(k) for k in key)
        site = (x, y, z, t)
        v = self._memo.get(site)
        if v is None:
            v = self._memo[site] = self._value(site)
        return v


def _one_site(op, v, *args):
    """A whole-field operator of the fifth dimension applied to one site's
    (Ls, 4, 3) values."""
    return op(v[None, None, None, None], *args)[0, 0, 0, 0]


def mpc_in_site(U, psi, p: DWFParams, site, inside, dagger: bool = False):
    """(M_pc psi)(x) of the Dirichlet block on the sites where ``inside``
    holds (the Schur operator of mpc_in: M_oo - M_oe M_ee^-1 M_eo, every hop
    restricted to the block), at one odd site x = ``site`` of the block, from
    the sites within two hops of x only.  ``psi`` is indexed psi[t, z, y, x]
    -> (Ls, 4, 3) (a full array or any object with that indexing and a
    ``shape``); it is restricted to the block's odd sites here.  ``inside``
    maps a site (x, y, z, t) to True / False.  Returns (Ls, 4, 3)."""
    L = lattice_dims(U)
    shape = tuple(L[::-1]) + tuple(psi.shape[4:])
    zero = np.zeros(psi.shape[4:], dtype=np.complex128)
    odd = lambda s: (s[0] + s[1] + s[2] + s[3]) % 2 == 1

    def src(s):
        return np.asarray(psi[s[3], s[2], s[1], s[0]]) if inside(s) and odd(s) else zero

    f = _SiteField(shape, src)

    def mid(s):   # (M_ee^-1 M_eo psi)(s) on the block's even sites, zero elsewhere
        if not inside(s) or odd(s):
            return zero
        return _one_site(mooee_inv, eo_block_site(U, f, p, s, dagger), p, dagger)

    t = _SiteField(shape, mid)
    return _one_site(mooee, f[site[3], site[2], site[1], site[0]], p, dagger) \
        - eo_block_site(U, t, p, site, dagger)
