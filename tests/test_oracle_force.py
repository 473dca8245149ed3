"""Pins of the link-force oracle (CPU).

D is affine in the links (U and U^+ enter linearly), so for the tangent
perturbation U -> U + i H U of any set of links the change of Re <X, D Y> is
exactly linear: f(U + i H U) - f(U) = sum over the perturbed links of
Re tr[i H F].  That fixes every term of the force independently of its own
formula (the D used is the oracle's operator, itself pinned elsewhere).
Further: F is traceless anti-Hermitian, transforms covariantly under gauge
transformations, the adjoint bilinear Re <X, D^+ Y> has the force of
(Y, X), and the active-link mask zeroes the links it leaves out."""

import numpy as np
import pytest

from oracle import dwf as O
from oracle.force import box_links, force_bilinear
from paper_2203_17119_gb300 import inputs

SHAMIR = O.DWFParams(M5=1.8, mf=0.1)
MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)
DIMS, LS = (4, 4, 2, 2), 4


def _hermitian_traceless(rng, shape=()):
    A = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    return H - (np.trace(H, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)


def _setup(seed):
    rng = np.random.default_rng(seed)
    U = inputs.gauge_field(DIMS, "haar", rng=rng)
    X = inputs.gaussian_source(DIMS, LS, rng=rng)
    Y = inputs.gaussian_source(DIMS, LS, rng=rng)
    return rng, U, X, Y


def _f(U, X, Y, prm, dagger=False):
    return float(np.real(np.vdot(X, O.apply_D(U, Y, prm, dagger))))


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_single_link_perturbations_are_exact(prm):
    rng, U, X, Y = _setup(1)
    F = force_bilinear(U, X, Y, prm)
    f0 = _f(U, X, Y, prm)
    for _ in range(6):
        t, z, y, x = (int(rng.integers(n)) for n in DIMS[::-1])
        mu = int(rng.integers(4))
        H = _hermitian_traceless(rng)
        U2 = U.copy()
        U2[t, z, y, x, mu] = U[t, z, y, x, mu] + 1j * H @ U[t, z, y, x, mu]
        want = _f(U2, X, Y, prm) - f0
        got = float(np.real(np.trace(1j * H @ F[t, z, y, x, mu])))
        assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (t, z, y, x, mu)


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_all_links_at_once(prm):
    rng, U, X, Y = _setup(2)
    F = force_bilinear(U, X, Y, prm)
    H = _hermitian_traceless(rng, U.shape[:-2])
    want = _f(U + 1j * H @ U, X, Y, prm) - _f(U, X, Y, prm)
    got = float(np.real(np.einsum("...ab,...ba->...", 1j * H, F).sum()))
    assert abs(got - want) <= 1e-10 * abs(want)


def test_traceless_antihermitian():
    _, U, X, Y = _setup(3)
    F = force_bilinear(U, X, Y, MOBIUS)
    assert np.abs(F + np.conj(np.swapaxes(F, -1, -2))).max() <= 1e-13
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() <= 1e-13
    assert np.abs(F).max() > 0.1


def test_gauge_covariance():
    rng, U, X, Y = _setup(4)
    G = inputs.gauge_field(DIMS, "haar", rng=rng)[..., 0, :, :]    # one SU(3) per site
    Ug = U.copy()
    for mu in range(4):
        Gf = np.roll(G, -1, axis=O.AXIS[mu])
        Ug[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(Gf, -1, -2))
    Xg = np.einsum("tzyxab,tzyxsib->tzyxsia", G, X)
    Yg = np.einsum("tzyxab,tzyxsib->tzyxsia", G, Y)
    F = force_bilinear(U, X, Y, MOBIUS)
    Fg = force_bilinear(Ug, Xg, Yg, MOBIUS)
    Gd = np.conj(np.swapaxes(G, -1, -2))
    want = np.einsum("tzyxab,tzyxmbc,tzyxcd->tzyxmad", G, F, Gd)
    assert np.abs(Fg - want).max() <= 1e-12 * np.abs(F).max()


def test_adjoint_bilinear_swaps_fields():
    rng, U, X, Y = _setup(5)
    F = force_bilinear(U, Y, X, MOBIUS)
    H = _hermitian_traceless(rng, U.shape[:-2])
    want = _f(U + 1j * H @ U, X, Y, MOBIUS, True) - _f(U, X, Y, MOBIUS, True)
    got = float(np.real(np.einsum("...ab,...ba->...", 1j * H, F).sum()))
    assert abs(got - want) <= 1e-10 * abs(want)


def test_rhs_sum_and_active_mask():
    rng, U, X, Y = _setup(6)
    X2 = inputs.gaussian_source(DIMS, LS, rng=rng)
    Y2 = inputs.gaussian_source(DIMS, LS, rng=rng)
    F = force_bilinear(U, [X, X2], [Y, Y2], MOBIUS)
    assert np.abs(F - force_bilinear(U, X, Y, MOBIUS) - force_bilinear(U, X2, Y2, MOBIUS)).max() <= 1e-12
    box = ((1, 0, 0, 0), (2, 4, 2, 2))
    act = box_links(DIMS, box)
    # x-links leave the box from x = 2; links in y, z, t stay inside
    assert act[..., 0].sum() == 16 and act[..., 1].sum() == 32 and act[..., 3].sum() == 32
    Fm = force_bilinear(U, [X, X2], [Y, Y2], MOBIUS, active=act)
    assert np.array_equal(Fm[act], F[act]) and np.abs(Fm[~act]).max() == 0.0


# ---------------------------------------------------------------- boundary action
from oracle.force import boundary_action_dense, boundary_action_force_dense  # noqa: E402

SLAB = (4, 2, 2, 2)


def _expm_i(H, eps):
    w, V = np.linalg.eigh(H)
    return (V * np.exp(1j * eps * w)) @ np.conj(V.T)


def _dense_after_link_change(D0, U2, prm, shape, site, mu):
    """D(U2) from D(U) when only U_mu(site) changed: only the columns of the
    link's two end sites change; they are rebuilt by applying D(U2)."""
    t, z, y, x = site
    dims = (shape[3], shape[2], shape[1], shape[0])
    fwd = [x, y, z, t]
    fwd[mu] = (fwd[mu] + 1) % dims[mu]
    D = D0.copy()
    per_site = shape[4] * 12
    for (tt, zz, yy, xx) in {(t, z, y, x), (fwd[3], fwd[2], fwd[1], fwd[0])}:
        lex = ((tt * shape[1] + zz) * shape[2] + yy) * shape[3] + xx
        for j in range(lex * per_site, (lex + 1) * per_site):
            e = np.zeros(int(np.prod(shape)), dtype=np.complex128)
            e[j] = 1.0
            D[:, j] = O.apply_D(U2, e.reshape(shape), prm).reshape(-1)
    return D


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_boundary_action_force_matches_finite_differences(prm):
    """Central differences of S(exp(i eps H) U) = |R^-1 phi|^2 (dense R^-1)
    against Re tr[i H F] at links inside, across and outside Omega."""
    rng = np.random.default_rng(31)
    U = inputs.gauge_field(SLAB, "haar", rng=rng)
    phi = inputs.gaussian_source(SLAB, 4, rng=rng)
    box = O.band_box(SLAB, 2, dirs=(0,))          # Omega: x in {1, 2}
    F = boundary_action_force_dense(U, phi, prm, box)
    from oracle import dense as Dn
    D0 = Dn.dense_matrix(lambda f: O.apply_D(U, f, prm), phi.shape)
    eps = 1e-5
    # (t, z, y, x, mu): an x-link inside Omega, x-links across both faces, a
    # link in Omega-bar, a y-link in Omega
    for (t, z, y, x, mu) in [(0, 0, 0, 1, 0), (1, 0, 1, 0, 0), (0, 1, 0, 2, 0), (1, 1, 1, 3, 1), (0, 1, 1, 2, 1)]:
        H = _hermitian_traceless(rng)
        Up, Um = U.copy(), U.copy()
        Up[t, z, y, x, mu] = _expm_i(H, eps) @ U[t, z, y, x, mu]
        Um[t, z, y, x, mu] = _expm_i(H, -eps) @ U[t, z, y, x, mu]
        Dp_ = _dense_after_link_change(D0, Up, prm, phi.shape, (t, z, y, x), mu)
        Dm_ = _dense_after_link_change(D0, Um, prm, phi.shape, (t, z, y, x), mu)
        fd = (boundary_action_dense(Up, phi, prm, box, Dp_) - boundary_action_dense(Um, phi, prm, box, Dm_)) / (2 * eps)
        got = float(np.real(np.trace(1j * H @ F[t, z, y, x, mu])))
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (t, z, y, x, mu, got, fd)


def test_adjoint_solve_through_gamma5_r5():
    """D^-+ = G B D^-1 G B^-+ with G = gamma_5 R_5 (R_5: s -> Ls - 1 - s) and
    B = b5 + c5 S5: the Moebius gamma_5 R_5 Hermiticity of D B^-1, the route
    the library takes to the adjoint solve of the boundary force."""
    from oracle import dense as Dn
    rng = np.random.default_rng(32)
    dims, Ls = (2, 2, 2, 2), 4
    U = inputs.gauge_field(dims, "haar", rng=rng)
    chi = inputs.gaussian_source(dims, Ls, rng=rng)
    shape = chi.shape
    _, g5 = O.gammas()

    def G(f):
        return np.einsum("ij,tzyxsja->tzyxsia", g5, f[..., ::-1, :, :])

    for prm in (SHAMIR, MOBIUS):
        D = Dn.dense_matrix(lambda f: O.apply_D(U, f, prm), shape)
        B = Dn.dense_matrix(lambda f: O.five_b(f, prm), shape)
        want = np.linalg.solve(np.conj(D.T), chi.reshape(-1))
        w = np.linalg.solve(np.conj(B.T), chi.reshape(-1)).reshape(shape)
        w = np.linalg.solve(D, G(w).reshape(-1)).reshape(shape)
        got = G((B @ w.reshape(-1)).reshape(shape)).reshape(-1)
        assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


from oracle.force import ratio_action_dense, ratio_action_force_dense  # noqa: E402


@pytest.mark.parametrize("light,pv", [(SHAMIR, O.DWFParams(M5=1.8, mf=1.0)),
                                      (MOBIUS, O.DWFParams(M5=1.8, mf=1.0, b5=1.5, c5=0.5))],
                         ids=["shamir", "mobius"])
def test_ratio_action_force_matches_finite_differences(light, pv):
    """Central differences of |R^-1 R_pv phi|^2 (dense R, R_pv) against the
    force assembled from four PV local solves and two light solves."""
    rng = np.random.default_rng(33)
    U = inputs.gauge_field(SLAB, "haar", rng=rng)
    phi = inputs.gaussian_source(SLAB, 4, rng=rng)
    box = O.band_box(SLAB, 2, dirs=(0,))
    F = ratio_action_force_dense(U, phi, light, pv, box)
    from oracle import dense as Dn
    Dl0 = Dn.dense_matrix(lambda f: O.apply_D(U, f, light), phi.shape)
    Dp0 = Dn.dense_matrix(lambda f: O.apply_D(U, f, pv), phi.shape)
    eps = 1e-5
    # a y-link inside Omega, an x-link across the face at x = 0 | 1, a y-link in Omega-bar
    for (t, z, y, x, mu) in [(0, 1, 1, 2, 1), (1, 0, 1, 0, 0), (1, 1, 1, 3, 1)]:
        H = _hermitian_traceless(rng)
        Up, Um = U.copy(), U.copy()
        Up[t, z, y, x, mu] = _expm_i(H, eps) @ U[t, z, y, x, mu]
        Um[t, z, y, x, mu] = _expm_i(H, -eps) @ U[t, z, y, x, mu]
        site = (t, z, y, x)
        sp = ratio_action_dense(Up, phi, light, pv, box, _dense_after_link_change(Dl0, Up, light, phi.shape, site, mu),
                                _dense_after_link_change(Dp0, Up, pv, phi.shape, site, mu))
        sm = ratio_action_dense(Um, phi, light, pv, box, _dense_after_link_change(Dl0, Um, light, phi.shape, site, mu),
                                _dense_after_link_change(Dp0, Um, pv, phi.shape, site, mu))
        fd = (sp - sm) / (2 * eps)
        got = float(np.real(np.trace(1j * H @ F[t, z, y, x, mu])))
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (t, z, y, x, mu, got, fd)


from oracle.force import one_flavour_action_dense, one_flavour_force_dense  # noqa: E402


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_one_flavour_force_matches_finite_differences(prm):
    """Central differences of S = <w, r2(A) w>, w = r1(A_d) phi (A, A_d the
    normal Schur operators of D and of D with the Omega / Omega-bar links cut)
    against the force assembled from Schur-operator insertions, at a link
    inside Omega, a cut link and a link in Omega-bar.  The rational functions
    are arbitrary partial fractions: the formula holds for any."""
    rng = np.random.default_rng(35)
    U = inputs.gauge_field(SLAB, "haar", rng=rng)
    odd = O.parity_field(SLAB) == 1
    phi = O.restrict(inputs.gaussian_source(SLAB, 4, rng=rng), odd)
    box = O.band_box(SLAB, 2, dirs=(0,))
    r1 = (0.4, [0.3, 2.0], [0.25, 1.5])
    r2 = (0.1, [0.05, 0.7, 4.0], [0.2, 0.6, 2.5])
    F = one_flavour_force_dense(U, phi, prm, box, r1, r2)
    from oracle import dense as Dn
    D0 = Dn.dense_matrix(lambda f: O.apply_D(U, f, prm), phi.shape)
    Dd0 = Dn.dense_matrix(lambda f: O.apply_D(O.cut_gauge(U, [box]), f, prm), phi.shape)
    eps = 1e-5
    # (t, z, y, x, mu): y-link inside Omega, the cut x-link from x = 0 to 1, y-link in Omega-bar
    for (t, z, y, x, mu) in [(0, 1, 1, 2, 1), (1, 0, 1, 0, 0), (1, 1, 1, 3, 1)]:
        H = _hermitian_traceless(rng)
        vals = []
        for sgn in (1, -1):
            U2 = U.copy()
            U2[t, z, y, x, mu] = _expm_i(H, sgn * eps) @ U[t, z, y, x, mu]
            D2 = _dense_after_link_change(D0, U2, prm, phi.shape, (t, z, y, x), mu)
            Dd2 = _dense_after_link_change(Dd0, O.cut_gauge(U2, [box]), prm, phi.shape, (t, z, y, x), mu)
            vals.append(one_flavour_action_dense(U2, phi, prm, box, r1, r2, D2, Dd2))
        fd = (vals[0] - vals[1]) / (2 * eps)
        got = float(np.real(np.trace(1j * H @ F[t, z, y, x, mu])))
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (t, z, y, x, mu, got, fd)
