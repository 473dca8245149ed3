"""Seeded synthetic inputs: gauge fields and Gaussian sources.

This module holds no arithmetic of the domain wall operator or its solvers;
it only draws the random SU(3) link variables and pseudofermion-like sources
on which both the CPU oracle and the CUDA path are evaluated.  Every draw is
made from ``numpy.random.default_rng(seed)`` (PCG64), whose stream is the same
on every platform, in a fixed order: links first (canonical site order, then
direction), then sources.

Layouts (canonical, shared by every consumer):

* gauge field  ``U[t, z, y, x, mu, a, b]`` complex128: U_mu(x) is the
  parallel transporter from x to x + mu_hat (mu = 0..3 <-> x, y, z, t);
  flattened this is ``[site lex][mu][3][3]`` with
  lex = x + Lx*(y + Ly*(z + Lz*t)).
* 5D fermion   ``psi[t, z, y, x, s, spin, colour]`` complex128, flattened
  ``[site lex][s][spin 4][colour 3]``; a batch of ``nrhs`` sources adds a
  leading ``rhs`` axis.

Generators (the lattice set-up of the paper's DWF workloads, Sec. 2.4):

* ``haar_su3``: Gram-Schmidt on the first two rows of a complex Gaussian 3x3
  matrix (re, im ~ N(0, 1/2)); the third row is the complex conjugate of the
  cross product of the first two, which fixes det U = 1 exactly.
* ``exp_su3``: U = exp(i eps H) with H = sum_a h_a lambda_a / 2, h_a ~ N(0,1),
  lambda_a the Gell-Mann matrices, via the Hermitian eigendecomposition.
* ``gaussian_source``: complex entries with re, im ~ N(0, 1/2) (E|z|^2 = 1).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "haar_su3",
    "exp_su3",
    "gauge_field",
    "gaussian_source",
    "config_seed",
]


def config_seed(index: int) -> int:
    """Seed used for workload ``index`` of the measured configurations."""
    return 1000 + int(index)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


def _complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    z = rng.standard_normal(tuple(shape) + (2,)) * np.sqrt(0.5)
    return z[..., 0] + 1j * z[..., 1]


def haar_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """``n`` Haar-random SU(3) matrices, shape (n, 3, 3)."""
    g = _complex_normal(rng, (n, 3, 3))
    r0 = g[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=1, keepdims=True)
    r1 = g[:, 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=1)


def exp_su3(rng: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """``n`` matrices exp(i eps H), H = sum_a h_a lambda_a/2, shape (n, 3, 3)."""
    h = rng.standard_normal((n, 8))
    H = np.einsum("na,aij->nij", h, gell_mann() / 2)
    w, v = np.linalg.eigh(H)
    U = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * w), np.conj(v))
    # one polar re-unitarisation step removes the O(1e-16) drift of eigh
    u, _, vh = np.linalg.svd(U)
    U = u @ vh
    det = np.linalg.det(U)
    U = U / (det ** (1.0 / 3.0))[:, None, None]
    return U


def gauge_field(dims, kind: str = "haar", seed: int = 0, eps: float = 0.3,
                rng: np.random.Generator | None = None) -> np.ndarray:
    """Gauge field of shape (Lt, Lz, Ly, Lx, 4, 3, 3).

    ``dims`` = (Lx, Ly, Lz, Lt).  ``kind`` is ``"haar"``, ``"exp"`` (with
    ``eps``) or ``"unit"`` (free field).
    """
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    n = Lx * Ly * Lz * Lt * 4
    if rng is None:
        rng = np.random.default_rng(seed)
    if kind == "haar":
        U = haar_su3(rng, n)
    elif kind == "exp":
        U = exp_su3(rng, n, eps)
    elif kind == "unit":
        U = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return U.reshape(Lt, Lz, Ly, Lx, 4, 3, 3)


def gaussian_source(dims, Ls: int, nrhs: int | None = None, seed: int = 0,
                    rng: np.random.Generator | None = None) -> np.ndarray:
    """Gaussian complex 5D field(s), shape ([nrhs,] Lt, Lz, Ly, Lx, Ls, 4, 3)."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    if rng is None:
        rng = np.random.default_rng(seed)
    shape = (Lt, Lz, Ly, Lx, int(Ls), 4, 3)
    if nrhs is not None:
        shape = (int(nrhs),) + shape
    return _complex_normal(rng, shape)
