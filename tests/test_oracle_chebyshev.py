"""Pins of the Chebyshev filter oracle (CPU).

The recurrence must give T_n(z(A)) v: checked against the eigendecomposition
of A (numpy eigh, then the closed forms cos(n arccos z) inside [lo, hi] and
cosh(n arccosh z) below lo) for a random Hermitian positive matrix and for the
normal Schur operator M_pc^+ M_pc of the domain wall operator built column by
column; orders 0 and 1 reduce to v and z(A) v; a multiple of the identity
gives the scalar polynomial; the filter enriches the low modes (Rayleigh
quotient falls)."""

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import dwf as O
from oracle.chebyshev import chebyshev_filter
from paper_2203_17119_gb300 import inputs


def _cheb_scalar(n, z):
    z = np.asarray(z, dtype=float)
    out = np.empty_like(z)
    inside = np.abs(z) <= 1
    out[inside] = np.cos(n * np.arccos(z[inside]))
    big = z > 1
    out[big] = np.cosh(n * np.arccosh(z[big]))
    small = z < -1
    out[small] = (-1) ** n * np.cosh(n * np.arccosh(-z[small]))
    return out


@pytest.mark.parametrize("order", [0, 1, 2, 7, 24])
def test_random_hermitian_against_eigendecomposition(order):
    rng = np.random.default_rng(7)
    n = 60
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = M.conj().T @ M / n + 0.01 * np.eye(n)
    w, V = np.linalg.eigh(A)
    lo, hi = 0.2, 1.1 * w[-1]
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = chebyshev_filter(lambda x: A @ x, v, order, lo, hi)
    z = (hi + lo - 2 * w) / (hi - lo)
    want = V @ (_cheb_scalar(order, z) * (V.conj().T @ v))
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_multiple_of_identity_is_the_scalar_polynomial():
    v = np.arange(5, dtype=float) + 1.0
    for lam in (0.01, 0.5, 2.0):
        got = chebyshev_filter(lambda x: lam * x, v, 9, 0.1, 2.0)
        z = (2.0 + 0.1 - 2 * lam) / (2.0 - 0.1)
        assert np.allclose(got, _cheb_scalar(9, np.array([z]))[0] * v, rtol=1e-12)


def test_dwf_normal_operator_and_low_mode_enrichment():
    dims, Ls = (2, 2, 2, 2), 4
    prm = O.DWFParams(M5=1.8, mf=0.01)
    U = inputs.gauge_field(dims, "haar", seed=17)
    odd = O.parity_field(dims) == 1
    shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)

    def A(f):
        f = O.restrict(f, odd)
        return O.mpc(U, O.mpc(U, f, prm), prm, True)

    dofs = Dn.site_mask_to_dofs(odd, Ls * 12)
    Ad = Dn.dense_matrix(A, shape)[np.ix_(dofs, dofs)]
    w, V = np.linalg.eigh(Ad)
    lo, hi = 0.05 * w[-1], 1.05 * w[-1]
    v = O.restrict(inputs.gaussian_source(dims, Ls, seed=18), odd)
    got = chebyshev_filter(A, v, 12, lo, hi)
    z = (hi + lo - 2 * w) / (hi - lo)
    want = V @ (_cheb_scalar(12, z) * (V.conj().T @ v.reshape(-1)[dofs]))
    assert np.linalg.norm(got.reshape(-1)[dofs] - want) <= 1e-10 * np.linalg.norm(want)

    def rq(x):
        return float(np.vdot(x, A(x)).real / np.vdot(x, x).real)

    assert rq(got) < 0.2 * rq(v)


def test_bad_arguments():
    with pytest.raises(ValueError):
        chebyshev_filter(lambda x: x, np.ones(3), -1, 0.0, 1.0)
    with pytest.raises(ValueError):
        chebyshev_filter(lambda x: x, np.ones(3), 3, 1.0, 1.0)
