"""Pins of the Zolotarev approximation oracle (CPU).

What fixes it independently of its formula: the optimal relative
approximation of type (n - 1, n) equioscillates, so the relative error
1 - sqrt(x) r(x) on [lo, hi] must reach +-delta alternately at 2n + 1 points
(endpoints included); delta falls exponentially with n; the partial
fractions reproduce the product form; applied to a Hermitian positive matrix
the rational function is within delta of A^(-1/2) from eigh."""

import numpy as np
import pytest

from oracle.rational import partial_fraction_eval, zolotarev_inv_sqrt


def _extrema(err):
    """Values at the local extrema of err on its grid, endpoints included."""
    d = np.diff(err)
    idx = [0] + [i for i in range(1, len(err) - 1) if d[i - 1] * d[i] < 0] + [len(err) - 1]
    return err[idx]


@pytest.mark.parametrize("n,lo,hi", [(4, 1e-2, 10.0), (8, 1e-4, 50.0), (12, 1e-4, 1e2)])
def test_equioscillation(n, lo, hi):
    shifts, res, delta = zolotarev_inv_sqrt(n, lo, hi)
    x = np.geomspace(lo, hi, 400001)
    err = 1.0 - np.sqrt(x) * partial_fraction_eval(x, shifts, res)
    ext = _extrema(err)
    assert len(ext) == 2 * n + 1
    assert np.all(np.sign(ext[1:]) == -np.sign(ext[:-1]))
    assert np.allclose(np.abs(ext), delta, rtol=1e-3)
    assert np.abs(err).max() <= delta * (1 + 1e-6)
    assert np.all(shifts > 0)


def test_error_falls_exponentially_and_matrix_function():
    deltas = [zolotarev_inv_sqrt(n, 1e-3, 10.0)[2] for n in (4, 8, 12)]
    assert deltas[1] < deltas[0] ** 1.5 and deltas[2] < deltas[1] ** 1.2 and deltas[2] < 1e-6
    rng = np.random.default_rng(3)
    M = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    A = M.conj().T @ M / 40 + 0.01 * np.eye(40)
    w, V = np.linalg.eigh(A)
    shifts, res, delta = zolotarev_inv_sqrt(12, 0.9 * w[0], 1.1 * w[-1])
    b = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    got = sum(r * np.linalg.solve(A + s * np.eye(40), b) for s, r in zip(shifts, res))
    want = V @ ((w ** -0.5) * (V.conj().T @ b))
    assert np.linalg.norm(got - want) <= 2 * delta * np.linalg.norm(want)


def test_bad_arguments():
    with pytest.raises(ValueError):
        zolotarev_inv_sqrt(0, 1.0, 2.0)
    with pytest.raises(ValueError):
        zolotarev_inv_sqrt(4, 2.0, 1.0)


@pytest.mark.parametrize("n,lo,hi", [(3, 1e-2, 10.0), (8, 1e-4, 50.0), (12, 1e-5, 1e2)])
def test_type_nn_equioscillation(n, lo, hi):
    """Type (n, n): 2n + 2 alternating extrema of equal size (Chebyshev's
    characterisation of the best approximation), a0 > 0, positive residues
    and shifts, and a smaller error than type (n - 1, n) with the same poles
    count (one more free parameter)."""
    from oracle.rational import zolotarev_inv_sqrt_nn
    a0, shifts, res, delta = zolotarev_inv_sqrt_nn(n, lo, hi)
    x = np.geomspace(lo, hi, 400001)
    err = np.sqrt(x) * partial_fraction_eval(x, shifts, res, a0) - 1.0
    ext = _extrema(err)
    assert len(ext) == 2 * n + 2
    assert np.all(np.sign(ext[1:]) == -np.sign(ext[:-1]))
    assert np.allclose(np.abs(ext), delta, rtol=1e-3)
    assert np.abs(err).max() <= delta * (1 + 1e-6)
    assert a0 > 0 and np.all(shifts > 0) and np.all(res > 0)
    assert delta < zolotarev_inv_sqrt(n, lo, hi)[2]
