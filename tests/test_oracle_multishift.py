"""Pins of the multi-shift CG oracle (CPU).

The oracle follows the published multi-shift recurrences; these tests pin it
to what linear algebra fixes independently of them: every returned x_s
solves (A + sigma_s) x_s = b, compared with LAPACK solves of the same dense
systems, for a random Hermitian positive matrix and for the normal Schur
operator M_pc^+ M_pc of the domain wall operator on a tiny lattice (built
column by column), plus the single-shift case, which must reproduce plain CG's
solution, and shift order independence."""

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import dwf as O
from oracle.multishift import multishift_cg
from paper_2203_17119_gb300 import inputs


def test_random_hermitian_positive_matches_lapack():
    rng = np.random.default_rng(3)
    n = 80
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = M.conj().T @ M + 0.05 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    shifts = [0.3, 0.0, 1.7, 25.0, 0.01]
    xs, info = multishift_cg(lambda v: A @ v, b, shifts, tol=1e-12)
    for s, x in zip(shifts, xs):
        ref = np.linalg.solve(A + s * np.eye(n), b)
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref), s
    # larger shifts are better conditioned: they stop no later than the base
    assert max(info["iters"]) == info["base_iters"]
    assert info["iters"][3] < info["iters"][1]


def test_dwf_normal_operator_matches_dense():
    dims, Ls = (2, 2, 2, 2), 4
    prm = O.DWFParams(M5=1.8, mf=0.1, b5=1.5, c5=0.5)
    U = inputs.gauge_field(dims, "haar", seed=11)
    odd = O.parity_field(dims) == 1
    shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)
    rng = np.random.default_rng(12)

    def A(v):
        v = O.restrict(v, odd)
        return O.mpc(U, O.mpc(U, v, prm), prm, True)

    b = O.restrict(inputs.gaussian_source(dims, Ls, rng=rng), odd)
    shifts = [0.0, 0.05, 0.5, 4.0]
    xs, info = multishift_cg(A, b, shifts, tol=1e-12)
    dofs = Dn.site_mask_to_dofs(odd, Ls * 12)
    Ad = Dn.dense_matrix(A, shape)[np.ix_(dofs, dofs)]
    for s, x in zip(shifts, xs):
        ref = np.linalg.solve(Ad + s * np.eye(len(dofs)), b.reshape(-1)[dofs])
        assert np.linalg.norm(x.reshape(-1)[dofs] - ref) <= 1e-9 * np.linalg.norm(ref), s
        # the even sites stay zero
        assert np.abs(x.reshape(-1)[np.setdiff1d(np.arange(x.size), dofs)]).max() == 0.0


def test_single_shift_is_plain_cg():
    rng = np.random.default_rng(5)
    n = 50
    M = rng.standard_normal((n, n))
    A = M.T @ M + 0.5 * np.eye(n)
    b = rng.standard_normal(n)
    (x,), info = multishift_cg(lambda v: A @ v, b, [0.0], tol=1e-13)
    # textbook CG on the same system
    y = np.zeros(n)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    for _ in range(info["base_iters"]):
        Ap = A @ p
        a = rr / (p @ Ap)
        y += a * p
        r -= a * Ap
        rr, rr_old = r @ r, rr
        p = r + (rr / rr_old) * p
    assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)


@pytest.mark.parametrize("perm", [[0, 1, 2], [2, 0, 1], [1, 2, 0]])
def test_order_of_shifts_does_not_matter(perm):
    rng = np.random.default_rng(6)
    n = 40
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = M.conj().T @ M + 0.2 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    shifts = np.array([0.1, 1.0, 3.0])
    xs, _ = multishift_cg(lambda v: A @ v, b, list(shifts[perm]), tol=1e-12)
    for s, x in zip(shifts[perm], xs):
        ref = np.linalg.solve(A + s * np.eye(n), b)
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_rational_apply_is_the_partial_fraction_function():
    """f(x) = (x + 3) / ((x + 1)(x + 2)) = 2/(x + 1) - 1/(x + 2) (+ a0) applied
    to a Hermitian positive matrix equals f on its eigenvalues."""
    from oracle.multishift import rational_apply
    rng = np.random.default_rng(9)
    n = 50
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = M.conj().T @ M / n + 0.05 * np.eye(n)
    w, V = np.linalg.eigh(A)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = rational_apply(lambda v: A @ v, b, 0.25, [1.0, 2.0], [2.0, -1.0], tol=1e-13)
    f = 0.25 + (w + 3) / ((w + 1) * (w + 2))
    want = V @ (f * (V.conj().T @ b))
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
