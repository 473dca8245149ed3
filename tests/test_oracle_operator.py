"""Pins of the CPU oracle's domain wall operator against facts fixed by the
mathematics, not by the oracle's own code: gamma algebra, the free-field
momentum-space closed form, gauge covariance, adjointness, gamma5-R5
hermiticity, the closed-form M_ee^-1 against a dense inverse, and per-site
evaluation against the whole-lattice one."""

import numpy as np
import pytest

from oracle import dwf as O
from paper_2203_17119_gb300 import inputs

SHAMIR = O.DWFParams(M5=1.8, mf=0.01)
MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)


def rand_field(dims, Ls, seed):
    return inputs.gaussian_source(dims, Ls, seed=seed)


def vdot(a, b):
    return np.vdot(a, b)


# ----------------------------------------------------------------- gammas
def test_gamma_algebra():
    g, g5 = O.gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * (mu == nu) * np.eye(4))
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


# ------------------------------------------------------ free-field closed form
def _s5_matrix(Ls, mf, dagger=False):
    """S5 as a (Ls*4) x (Ls*4) matrix, index s*4 + spin, from its definition:
    (S5 psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}, walls -m_f."""
    Pp = np.diag([1, 1, 0, 0]).astype(complex)
    Pm = np.diag([0, 0, 1, 1]).astype(complex)
    if dagger:
        Pp, Pm = Pm, Pp
    S = np.zeros((4 * Ls, 4 * Ls), dtype=complex)
    for s in range(Ls):
        up, fac_u = (s + 1, 1.0) if s + 1 < Ls else (0, -mf)
        dn, fac_d = (s - 1, 1.0) if s - 1 >= 0 else (Ls - 1, -mf)
        S[4 * s:4 * s + 4, 4 * up:4 * up + 4] += fac_u * Pm
        S[4 * s:4 * s + 4, 4 * dn:4 * dn + 4] += fac_d * Pp
    return S


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_free_field_plane_wave(prm):
    dims, Ls = (4, 6, 4, 8), 6
    n = (1, 2, 3, 3)                     # distinct momenta per direction
    pmom = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
    rng = np.random.default_rng(7)
    v = rng.standard_normal((Ls, 4)) + 1j * rng.standard_normal((Ls, 4))
    c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    phase = np.exp(1j * (pmom[0] * x + pmom[1] * y + pmom[2] * z + pmom[3] * t))
    psi = phase[..., None, None, None] * np.einsum("si,a->sia", v, c)
    U = inputs.gauge_field(dims, "unit")
    g, _ = O.gammas()
    DW = (-prm.M5 + sum(1 - np.cos(pm) for pm in pmom)) * np.eye(4) \
        + 1j * sum(g[mu] * np.sin(pmom[mu]) for mu in range(4))
    S = _s5_matrix(Ls, prm.mf)
    Dp = np.kron(np.eye(Ls), DW) @ (prm.b5 * np.eye(4 * Ls) + prm.c5 * S) \
        + np.eye(4 * Ls) - S
    for dag, M in ((False, Dp), (True, Dp.conj().T)):
        got = O.apply_D(U, psi, prm, dagger=dag)
        want = phase[..., None, None, None] * np.einsum(
            "si,a->sia", (M @ v.reshape(-1)).reshape(Ls, 4), c)
        assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


# ------------------------------------------------------- gauge covariance
@pytest.mark.parametrize("dag", [False, True])
def test_gauge_covariance(dag):
    dims, Ls = (4, 4, 2, 6), 4
    rng = np.random.default_rng(11)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    psi = inputs.gaussian_source(dims, Ls, rng=rng)
    gx = inputs.haar_su3(rng, int(np.prod(dims))).reshape(dims[3], dims[2], dims[1], dims[0], 3, 3)
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = np.roll(gx, -1, axis=O.AXIS[mu])
        Ug[..., mu, :, :] = gx @ U[..., mu, :, :] @ np.conj(np.swapaxes(gfwd, -1, -2))
    rot = lambda f: np.einsum("tzyxab,tzyxsib->tzyxsia", gx, f)
    got = O.apply_D(Ug, rot(psi), MOBIUS, dag)
    want = rot(O.apply_D(U, psi, MOBIUS, dag))
    assert np.max(np.abs(got - want)) < 1e-12


# --------------------------------------------------------------- adjoints
def test_adjointness_all_pieces():
    dims, Ls = (4, 2, 4, 2), 6
    rng = np.random.default_rng(3)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    a = inputs.gaussian_source(dims, Ls, rng=rng)
    b = inputs.gaussian_source(dims, Ls, rng=rng)
    ao, bo = O.parity_part(a, 1), O.parity_part(b, 1)
    for prm in (SHAMIR, MOBIUS):
        ops = [
            lambda f, d: O.apply_D(U, f, prm, d),
            lambda f, d: O.hop_part(U, f, prm, d),
            lambda f, d: O.mooee(f, prm, d),
            lambda f, d: O.mooee_inv(f, prm, d),
            lambda f, d: O.hop(U, f, d),
            lambda f, d: O.s5(f, prm.mf, d),
        ]
        for op in ops:
            lhs = vdot(a, op(b, False))
            rhs = vdot(op(a, True), b)
            assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-12
        lhs = vdot(ao, O.mpc(U, bo, prm, False))
        rhs = vdot(O.mpc(U, ao, prm, True), bo)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _gamma5_r5(f):
    _, g5 = O.gammas()
    return np.einsum("ij,tzyxsja->tzyxsia", g5, f[..., ::-1, :, :])


def test_gamma5_r5_hermiticity():
    """Shamir: gamma5 R5 D is Hermitian.  Moebius: gamma5 R5 D (b5 + c5 S5)^-1
    is (D_W commutes with neither P_+- nor S5, so the (b5 + c5 S5) factor has
    to be divided out; (b5 + c5 S5)^-1 is taken from a dense matrix here)."""
    dims, Ls = (4, 4, 2, 2), 6
    rng = np.random.default_rng(5)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    a = inputs.gaussian_source(dims, Ls, rng=rng)
    b = inputs.gaussian_source(dims, Ls, rng=rng)
    H = lambda f: _gamma5_r5(O.apply_D(U, f, SHAMIR))
    assert abs(vdot(a, H(b)) - vdot(H(a), b)) < 1e-12 * abs(vdot(a, H(b)))
    Bm = MOBIUS.b5 * np.eye(4 * Ls) + MOBIUS.c5 * _s5_matrix(Ls, MOBIUS.mf)
    Binv = np.linalg.inv(Bm)
    binv = lambda f: np.einsum("xy,...ya->...xa", Binv,
                               f.reshape(f.shape[:4] + (4 * Ls, 3))).reshape(f.shape)
    Hm = lambda f: _gamma5_r5(O.apply_D(U, binv(f), MOBIUS))
    lhs, rhs = vdot(a, Hm(b)), vdot(Hm(a), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and without dividing out (b5 + c5 S5) the Moebius operator is not
    Hn = lambda f: _gamma5_r5(O.apply_D(U, f, MOBIUS))
    assert abs(vdot(a, Hn(b)) - vdot(Hn(a), b)) > 1e-3 * abs(vdot(a, Hn(b)))


# ------------------------------------------------------------ M_ee inverse
@pytest.mark.parametrize("Ls", [1, 2, 5, 8, 12, 16])
@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS, O.DWFParams(1.8, 0.005, 1.5, 0.5)])
def test_mooee_inv_closed_form(Ls, prm):
    for dag in (False, True):
        up, lo = O.mooee_inv_matrices(Ls, prm, dag)
        S = _s5_matrix(Ls, prm.mf, dag)
        M = prm.d * np.eye(4 * Ls) + prm.e * S
        Minv = np.linalg.inv(M)
        # spin 0 block (upper chirality) and spin 2 block (lower)
        assert np.allclose(up, Minv[0::4, 0::4], atol=1e-14, rtol=1e-13)
        assert np.allclose(lo, Minv[2::4, 2::4], atol=1e-14, rtol=1e-13)
    if Ls == 1:
        assert np.isclose(O.mooee_inv_matrices(1, prm)[0][0, 0],
                          1.0 / (prm.d - prm.e * prm.mf))


def test_mooee_inv_times_mooee():
    dims, Ls = (2, 2, 2, 2), 8
    f = rand_field(dims, Ls, 9)
    for dag in (False, True):
        g = O.mooee_inv(O.mooee(f, MOBIUS, dag), MOBIUS, dag)
        assert np.max(np.abs(g - f)) < 1e-14


# ------------------------------------------------------- per-site helpers
def test_site_evaluation_matches_lattice():
    dims, Ls = (4, 4, 4, 6), 4
    rng = np.random.default_rng(21)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    psi = inputs.gaussian_source(dims, Ls, rng=rng)
    for dag in (False, True):
        full = O.hop(U, psi, dag)
        blk = O.hop_part(U, psi, MOBIUS, dag)
        for site in [(0, 0, 0, 0), (3, 1, 2, 5), (1, 3, 3, 0)]:
            x = site
            assert np.allclose(O.hop_site(U, psi, x, dag), full[x[3], x[2], x[1], x[0]],
                               atol=1e-13)
            assert np.allclose(O.eo_block_site(U, psi, MOBIUS, x, dag),
                               blk[x[3], x[2], x[1], x[0]], atol=1e-13)


@pytest.mark.parametrize("dagger", [False, True])
def test_mpc_site_evaluation_matches_block_operator(dagger):
    """The per-site Dirichlet-block Schur operator (two hops of stencil) equals
    mpc_in on the whole lattice at odd sites inside a box that wraps and at
    its faces, and mpc itself for a box that is the whole lattice."""
    dims, Ls = (4, 4, 6, 4), 4
    rng = np.random.default_rng(23)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    psi = O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1)
    box = ((3, 0, 4, 1), (3, 4, 5, 2))
    mask = O.box_mask(dims, box)
    full = O.mpc_in(U, psi, MOBIUS, mask, dagger)
    inside = lambda s: bool(mask[s[3], s[2], s[1], s[0]])
    cand = [(x, y, z, t) for t in range(dims[3]) for z in range(dims[2]) for y in range(dims[1])
            for x in range(dims[0]) if (x + y + z + t) % 2 == 1 and inside((x, y, z, t))]
    sites = cand[::7] + [cand[-1]]          # spread over the box, faces and wrap included
    assert len(sites) >= 8
    for x in sites:
        got = O.mpc_in_site(U, psi, MOBIUS, x, inside, dagger)
        assert np.allclose(got, full[x[3], x[2], x[1], x[0]], atol=1e-12), x
    whole = O.mpc(U, psi, MOBIUS, dagger)
    for x in [(1, 0, 0, 0), (2, 3, 5, 3)]:
        got = O.mpc_in_site(U, psi, MOBIUS, x, lambda s: True, dagger)
        assert np.allclose(got, whole[x[3], x[2], x[1], x[0]], atol=1e-12), x
