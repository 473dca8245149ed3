"""Pins of the oracle's parallel-transport preconditioner and GCR: identity
weights give K = 1, gauge equivariance, adjoint transports, central finite
differences for the analytic gradient, the closed form of Adam's first step,
GCR against a dense LU solve, and the folded checkerboard form of K that
inference uses."""

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import dwf as O
from oracle import nn as N
from paper_2203_17119_gb300 import inputs

MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)


def rand_w(rng, C, scale=0.3):
    def c(shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale
    return c((N.NDIR, C, 1, 4, 4)), c((N.NDIR, 1, C, 4, 4)) / np.sqrt(C)


def test_identity_weights_give_identity():
    dims, Ls = (4, 2, 2, 4), 4
    rng = np.random.default_rng(1)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    r = inputs.gaussian_source(dims, Ls, rng=rng)
    W1, W2 = N.identity_weights(16)
    assert np.allclose(N.apply_K(U, r, W1, W2), O.parity_part(r, 1), atol=1e-15)


def test_folded_checkerboard_form_equals_two_layers():
    """The inference form the GPU applies: for an input on odd sites,
    R_d = T_d r vanishes on odd sites for the link directions 1..8 and on even
    sites for 0, 9, 10 (exactly), and with the layers linear K r on odd sites
    is sum_d T_d (sum_d' M[d][d'] R_d') with M = W2 W1 over each
    checkerboard's own directions."""
    dims, Ls, C = (4, 2, 4, 2), 4, 5
    rng = np.random.default_rng(8)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    r = O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1)
    W1, W2 = rand_w(rng, C)
    links, local = list(range(1, 9)), [0, 9, 10]
    for d in range(N.NDIR):
        T = N.transport(U, r, d)
        assert np.max(np.abs(O.parity_part(T, 1 if d in links else 0))) == 0.0, d
    M = np.einsum("dbot,ebti->deoi", W2[:, 0], W1[:, :, 0])
    z = np.zeros_like(r)
    for p, ds in ((0, links), (1, local)):
        R = {e: O.parity_part(N.transport(U, r, e), p) for e in ds}
        for d in ds:
            psi = sum(np.einsum("ij,tzyxsja->tzyxsia", M[d, e], R[e]) for e in ds)
            z += N.transport(U, psi, d)
    want = N.apply_K(U, r, W1, W2)
    assert np.linalg.norm(O.parity_part(z, 1) - want) <= 1e-13 * np.linalg.norm(want)


def test_transport_adjoints():
    dims, Ls = (4, 2, 4, 2), 4
    rng = np.random.default_rng(2)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    a = inputs.gaussian_source(dims, Ls, rng=rng)
    b = inputs.gaussian_source(dims, Ls, rng=rng)
    for d in range(N.NDIR):
        lhs = np.vdot(a, N.transport(U, b, d))
        rhs = np.vdot(N.transport(U, a, N.ADJ[d]), b)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs), d


def test_gauge_equivariance():
    dims, Ls, C = (2, 4, 2, 4), 4, 3
    rng = np.random.default_rng(3)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    r = inputs.gaussian_source(dims, Ls, rng=rng)
    W1, W2 = rand_w(rng, C)
    g = inputs.haar_su3(rng, int(np.prod(dims))).reshape(dims[3], dims[2], dims[1], dims[0], 3, 3)
    Ug = np.empty_like(U)
    for mu in range(4):
        gf = np.roll(g, -1, axis=O.AXIS[mu])
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gf, -1, -2))
    rot = lambda f: np.einsum("tzyxab,tzyxsib->tzyxsia", g, f)
    got = N.apply_K(Ug, rot(r), W1, W2)
    want = rot(N.apply_K(U, r, W1, W2))
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("energy", [False, True, "a2"])
def test_gradient_central_differences(energy):
    dims, Ls, C = (4, 2, 2, 2), 4, 2
    rng = np.random.default_rng(4)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    A = None
    if energy:
        A = lambda f: O.mpc(U, O.mpc(U, f, MOBIUS), MOBIUS, True)
        es = [O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1) for _ in range(2)]
        pairs = [(A(e), e) for e in es]
    else:
        pairs = [(inputs.gaussian_source(dims, Ls, rng=rng),
                  O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1)) for _ in range(2)]
    W1, W2 = rand_w(rng, C)
    kind = "a2" if energy == "a2" else None
    L, g1, g2 = N.loss_and_grad(U, pairs, W1, W2, A, kind)
    h = 1e-6
    picks = [(0, (0, 0, 0, 1, 2)), (0, (3, 1, 0, 0, 0)), (0, (9, 0, 0, 2, 3)),
             (1, (0, 0, 1, 3, 3)), (1, (6, 0, 0, 1, 0)), (1, (10, 0, 1, 2, 1))]
    for which, idx in picks:
        for part in (1.0, 1j):
            Wp = [W1.copy(), W2.copy()]
            Wm = [W1.copy(), W2.copy()]
            Wp[which][idx] += h * part
            Wm[which][idx] -= h * part
            Lp = N.loss_and_grad(U, pairs, *Wp, A, kind)[0]
            Lm = N.loss_and_grad(U, pairs, *Wm, A, kind)[0]
            fd = (Lp - Lm) / (2 * h)
            an = (g1 if which == 0 else g2)[idx]
            an = an.real if part == 1.0 else an.imag
            # the central difference (L+ - L-) / 2h carries a rounding error of
            # about eps |L| / h = 2.2e-16 |L| / 1e-6 = 2.2e-10 |L| besides its
            # O(h^2) truncation error: the absolute slack is five times that bound
            assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3) + 1e-9 * abs(L), (which, idx, part, fd, an)


def test_adam_first_step_closed_form():
    """Adam's first step moves every real parameter by lr * sign(grad)."""
    rng = np.random.default_rng(5)
    p = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    g = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    opt = N.Adam([p.shape], lr=1e-3, eps=1e-12)
    (q,) = opt.step([p], [g])
    want = p - 1e-3 * (np.sign(g.real) + 1j * np.sign(g.imag))
    assert np.allclose(q, want, atol=1e-12)


def test_gcr_stagnates_on_mpc_but_not_on_normal_equations():
    """Restarted GCR on the Moebius Schur operator stalls (its field of values
    contains the origin); on M_pc^+ M_pc it converges to the dense solution."""
    dims, Ls = (4, 4, 2, 4), 8
    rng = np.random.default_rng(14)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    b = O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1)
    A = lambda f: O.mpc(U, f, MOBIUS)
    x, it = N.gcr(U, b, MOBIUS, A, tol=1e-12, maxiter=96)
    assert np.linalg.norm(b - A(x)) > 1e-3 * np.linalg.norm(b)
    AtA = lambda f: O.mpc(U, O.mpc(U, f, MOBIUS), MOBIUS, True)
    bb = O.mpc(U, b, MOBIUS, True)
    x, it = N.gcr(U, bb, MOBIUS, AtA, tol=1e-13, maxiter=20000)
    assert np.linalg.norm(b - A(x)) <= 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("use_k", [False, True])
def test_gcr_matches_dense_solve(use_k):
    dims, Ls = (2, 2, 2, 2), 4
    rng = np.random.default_rng(6)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    b = O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1)
    par = O.parity_field(dims)
    od = Dn.site_mask_to_dofs(par == 1, Ls * 12)
    M = Dn.dense_matrix(lambda f: O.mpc(U, O.parity_part(f, 1), MOBIUS), b.shape)[np.ix_(od, od)]
    x_lu = np.linalg.solve(M, b.reshape(-1)[od])
    K = None
    if use_k:
        W1, W2 = rand_w(rng, 2, scale=0.003)
        W1[0, 0, 0] += np.eye(4) / 4.3
        W2[0, 0, 0] += np.eye(4)
        K = lambda r: N.apply_K(U, r, W1, W2)
    x, it = N.gcr(U, b, MOBIUS, lambda f: O.mpc(U, f, MOBIUS), K=K, tol=1e-12)
    assert np.linalg.norm(x.reshape(-1)[od] - x_lu) <= 1e-10 * np.linalg.norm(x_lu)
