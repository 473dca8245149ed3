"""Brute-force pins of the oracle on tiny lattices: dense LU inverse, the
determinant factorisations, the Dirichlet block operator, the block algebra
of Sec. 2.1 (Schur factorisation, eq. schur, R R^-1 = P, det chi = det R,
eq. ddrhmc) and the band geometry printed in Sec. 2.4."""

import json
import os

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import dwf as O
from paper_2203_17119_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
SHAMIR = O.DWFParams(M5=1.8, mf=0.01)
MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)


@pytest.fixture(scope="module")
def tiny():
    """2^4 x Ls=4 lattice: every +mu and -mu neighbour coincide, so both
    hop terms land on the same site (768 x 768 dense matrices)."""
    dims, Ls = (2, 2, 2, 2), 4
    rng = np.random.default_rng(1234)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    b = inputs.gaussian_source(dims, Ls, rng=rng)
    return dims, Ls, U, b


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_dense_inverse_and_cgne(tiny, prm):
    dims, Ls, U, b = tiny
    shape = b.shape
    D = Dn.dense_matrix(lambda f: O.apply_D(U, f, prm), shape)
    Dd = Dn.dense_matrix(lambda f: O.apply_D(U, f, prm, True), shape)
    assert np.allclose(Dd, D.conj().T, atol=1e-14)
    x_lu = np.linalg.solve(D, b.reshape(-1)).reshape(shape)
    x_cg, info = O.cgne(U, b, prm, tol=1e-12)
    assert info["true_resid"] <= 1e-12
    assert np.linalg.norm(x_cg - x_lu) <= 1e-10 * np.linalg.norm(x_lu)
    # the residual is the residual of the dense system
    r = b.reshape(-1) - D @ x_cg.reshape(-1)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_det_eo_factorisation(tiny, prm):
    """det D = det M_ee * det M_pc, with M_pc from the oracle's Schur
    operator on the odd sites and M_ee from its site-diagonal block."""
    dims, Ls, U, b = tiny
    shape = b.shape
    D = Dn.dense_matrix(lambda f: O.apply_D(U, f, prm), shape)
    par = O.parity_field(dims)
    inner = Ls * 12
    ev = Dn.site_mask_to_dofs(par == 0, inner)
    od = Dn.site_mask_to_dofs(par == 1, inner)
    Mpc = Dn.dense_matrix(lambda f: O.mpc(U, O.parity_part(f, 1), prm), shape)[np.ix_(od, od)]
    Mee = Dn.dense_matrix(lambda f: O.mooee(f, prm), shape)[np.ix_(ev, ev)]
    # the blocks of D themselves
    assert np.allclose(D[np.ix_(ev, ev)], Mee, atol=1e-14)
    Moe = D[np.ix_(od, ev)]
    Meo = D[np.ix_(ev, od)]
    assert np.allclose(Mpc, D[np.ix_(od, od)] - Moe @ np.linalg.solve(Mee, Meo), atol=1e-12)
    lhs = Dn.logdet(D)
    rhs = Dn.logdet(Mee) + Dn.logdet(Mpc)
    assert abs(np.exp(lhs - rhs) - 1) < 1e-10


@pytest.fixture(scope="module")
def slab():
    """4 x 2 x 2 x 2, Ls = 4, Moebius, Omega = the interior x in {1, 2} of a
    cell with a band of width 2 in the x direction (1536 x 1536)."""
    dims, Ls = (4, 2, 2, 2), 4
    rng = np.random.default_rng(99)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)
    box = O.band_box(dims, 2, dirs=(0,))
    D = Dn.dense_matrix(lambda f: O.apply_D(U, f, MOBIUS), shape)
    ids = O.box_id_field(dims, [box])
    om = Dn.site_mask_to_dofs(ids == 0, Ls * 12)
    ob = Dn.site_mask_to_dofs(ids < 0, Ls * 12)
    return dims, Ls, U, shape, box, D, om, ob


def test_band_box_geometry_paper(slab):
    with open(os.path.join(HERE, "golden", "paper_geometry.json")) as f:
        gold = json.load(f)
    org, ext = O.band_box(gold["gpu_block"], gold["band_width"], gold["cut_dirs"])
    assert list(ext) == gold["interior"]
    ids = O.box_id_field(gold["gpu_block"], [(org, ext)])
    t_active = np.flatnonzero((ids >= 0).any(axis=(1, 2, 3)))
    assert t_active.size == gold["interior"][3]
    assert 0 not in t_active and gold["gpu_block"][3] - 1 not in t_active
    # widths 1, 2, 4 on a 32 cell: inactive layers top / top+bottom / 2+2
    for w, lo, hi in ((1, 0, 31), (2, 1, 31), (4, 2, 30)):
        o, e = O.band_box((32,) * 4, w)
        assert (o[0], o[0] + e[0]) == (lo, hi)


def test_dirichlet_mask_equals_cut(slab):
    dims, Ls, U, shape, box, D, om, ob = slab
    rng = np.random.default_rng(5)
    psi = inputs.gaussian_source(dims, Ls, rng=rng)
    for dag in (False, True):
        a = O.dirichlet_D(U, psi, MOBIUS, [box], dag)
        c = O.dirichlet_D_cut(U, psi, MOBIUS, [box], dag)
        assert np.max(np.abs(a - c)) < 1e-13
    # D(U_cut) is block diagonal and its Omega block is the D_Omega block of D
    Dc = Dn.dense_matrix(lambda f: O.apply_D(O.cut_gauge(U, [box]), f, MOBIUS), shape)
    assert np.max(np.abs(Dc[np.ix_(om, ob)])) == 0
    assert np.max(np.abs(Dc[np.ix_(ob, om)])) == 0
    assert np.allclose(Dc[np.ix_(om, om)], D[np.ix_(om, om)], atol=1e-14)
    assert np.allclose(Dc[np.ix_(ob, ob)], D[np.ix_(ob, ob)], atol=1e-14)


def test_two_boxes_cut_between_them():
    """Adjacent boxes are separate Dirichlet blocks: the mask form sums
    P_B D P_B per box, which equals the cut-link form."""
    dims, Ls = (4, 4, 2, 2), 2
    rng = np.random.default_rng(8)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    psi = inputs.gaussian_source(dims, Ls, rng=rng)
    boxes = [((0, 0, 0, 0), (2, 4, 2, 2)), ((2, 1, 0, 0), (2, 2, 2, 2))]
    a = O.dirichlet_D(U, psi, MOBIUS, boxes)
    c = O.dirichlet_D_cut(U, psi, MOBIUS, boxes)
    assert np.max(np.abs(a - c)) < 1e-13


def test_schur_factorisation_and_eq_schur(slab):
    dims, Ls, U, shape, box, D, om, ob = slab
    DO, Dd, Ddb, DOb = Dn.blocks(D, om, ob)
    nO, nOb = DO.shape[0], DOb.shape[0]
    I0, I1 = np.eye(nO), np.eye(nOb)
    Z01, Z10 = np.zeros((nO, nOb)), np.zeros((nOb, nO))
    DObi_Ddb = np.linalg.solve(DOb, Ddb)
    Dd_DObi = np.linalg.solve(DOb.T, Dd.T).T
    L = np.block([[I0, Dd_DObi], [Z10, I1]])
    M = np.block([[DO - Dd @ DObi_Ddb, Z01], [Z10, DOb]])
    R = np.block([[I0, Z01], [DObi_Ddb, I1]])
    Dblk = np.block([[DO, Dd], [Ddb, DOb]])
    assert np.allclose(L @ M @ R, Dblk, atol=1e-11)
    chi = Dn.chi_matrix(DO, Dd, Ddb, DOb)
    lhs = Dn.logdet(D)
    rhs = Dn.logdet(DO) + Dn.logdet(DOb) + Dn.logdet(chi)
    assert abs(np.exp(lhs - rhs) - 1) < 1e-9


def test_boundary_R_inverse_and_det(slab):
    """R = P - P D_O^-1 D_d D_Ob^-1 D_db (on Omega) with P the projector onto
    the components D_db acts on; R^-1 = P - P D^-1 D_db-hat; R R^-1 = P and
    det chi = det R restricted to the range of P."""
    dims, Ls, U, shape, box, D, om, ob = slab
    DO, Dd, Ddb, DOb = Dn.blocks(D, om, ob)
    V, P = Dn.rowspace_projector(Ddb)
    assert np.allclose(Ddb @ P, Ddb, atol=1e-12)
    k, nO = V.shape[1], DO.shape[0]
    assert 0 < k < nO
    Y = np.linalg.solve(DO, Dd @ np.linalg.solve(DOb, Ddb))
    R = P - P @ Y
    # D^-1 restricted: the Omega rows of D^-1 times the embedded D_db
    Dinv = np.linalg.inv(np.block([[DO, Dd], [Ddb, DOb]]))
    Rinv = P - P @ (Dinv[:nO, nO:] @ Ddb)
    assert np.allclose(R @ Rinv, P, atol=1e-10)
    chi = np.eye(nO) - Y
    detR = np.linalg.det(np.conj(V).T @ R @ V)
    assert abs(detR / np.linalg.det(chi) - 1) < 1e-9


def test_eq_ddrhmc(slab):
    """det chi = det D / det D_dirichlet with D_dirichlet = D(U_cut)."""
    dims, Ls, U, shape, box, D, om, ob = slab
    DO, Dd, Ddb, DOb = Dn.blocks(D, om, ob)
    Dc = Dn.dense_matrix(lambda f: O.apply_D(O.cut_gauge(U, [box]), f, MOBIUS), shape)
    chi = Dn.chi_matrix(DO, Dd, Ddb, DOb)
    lhs = Dn.logdet(chi)
    rhs = Dn.logdet(D) - Dn.logdet(Dc)
    assert abs(np.exp(lhs - rhs) - 1) < 1e-9


@pytest.fixture(scope="module")
def wrapped_box():
    """4 x 4 x 4 x 2, Ls = 4, Moebius; Omega one box with odd extents that
    wraps in x and z and is one layer thick in t: origin (3, 1, 2, 1),
    extent (3, 3, 3, 1) (27 sites; hops leave it in every direction).  Only
    the columns of D on Omega are built (1296 of them)."""
    dims, Ls = (4, 4, 4, 2), 4
    rng = np.random.default_rng(2718)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    box = ((3, 1, 2, 1), (3, 3, 3, 1))
    shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)
    mask = O.box_mask(dims, box)
    par = O.parity_field(dims)
    inner = Ls * 12
    om_e = Dn.site_mask_to_dofs(mask & (par == 0), inner)
    om_o = Dn.site_mask_to_dofs(mask & (par == 1), inner)
    cols = np.concatenate([om_e, om_o])
    n = int(np.prod(shape))
    DO = np.empty((cols.size, cols.size), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j, c in enumerate(cols):
        e[c] = 1.0
        DO[:, j] = O.apply_D(U, e.reshape(shape), MOBIUS).reshape(-1)[cols]
        e[c] = 0.0
    ne = om_e.size
    blocks = {"ee": DO[:ne, :ne], "eo": DO[:ne, ne:], "oe": DO[ne:, :ne], "oo": DO[ne:, ne:]}
    return dims, Ls, U, shape, mask, om_e, om_o, blocks, rng


def _check_on_random_vectors(apply, shape, src, dst, want, rng, tol):
    """apply(v) = want @ v on the dofs ``dst`` and 0 on every other dof, for
    three random complex v supported on the dofs ``src`` (a linear identity
    checked on random vectors: a wrong block fails it with probability 1)."""
    n = int(np.prod(shape))
    off = np.ones(n, dtype=bool)
    off[dst] = False
    for _ in range(3):
        v = rng.standard_normal(src.size) + 1j * rng.standard_normal(src.size)
        f = np.zeros(n, dtype=np.complex128)
        f[src] = v
        got = apply(f.reshape(shape)).reshape(-1)
        assert np.max(np.abs(got[off])) == 0.0
        w = want @ v
        assert np.linalg.norm(got[dst] - w) <= tol * np.linalg.norm(w)


@pytest.mark.parametrize("dagger", [False, True])
def test_mpc_in_is_schur_complement_of_D_Omega(wrapped_box, dagger):
    """The Dirichlet-block Schur operator of the oracle (every hop restricted
    to the box) equals the Schur complement of the dense D_Omega = D[Omega,
    Omega] (Sec. 2.1) over its 4D parity split:
    S = D_oo - D_oe D_ee^-1 D_eo on the odd sites of Omega (its adjoint for
    dagger), and it puts nothing anywhere else."""
    dims, Ls, U, shape, mask, om_e, om_o, B, rng = wrapped_box
    S = B["oo"] - B["oe"] @ np.linalg.solve(B["ee"], B["eo"])
    want = S.conj().T if dagger else S
    _check_on_random_vectors(lambda f: O.mpc_in(U, f, MOBIUS, mask, dagger), shape,
                             om_o, om_o, want, rng, 1e-12)


@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_eo_block_in_is_block_of_D_Omega(wrapped_box, out_parity, dagger):
    """eo_block_in(out_parity) is the off-diagonal parity block of the dense
    D_Omega (D_eo into even, D_oe into odd); dagger gives the adjoint of the
    opposite block ((D_oe)^+ into even, (D_eo)^+ into odd).  Nothing lands
    outside Omega's sites of the output parity."""
    dims, Ls, U, shape, mask, om_e, om_o, B, rng = wrapped_box
    src = om_o if out_parity == 0 else om_e
    dst = om_e if out_parity == 0 else om_o
    if not dagger:
        want = B["eo"] if out_parity == 0 else B["oe"]
    else:
        want = (B["oe"] if out_parity == 0 else B["eo"]).conj().T
    _check_on_random_vectors(lambda f: O.eo_block_in(U, f, MOBIUS, mask, out_parity, dagger),
                             shape, src, dst, want, rng, 1e-13)
