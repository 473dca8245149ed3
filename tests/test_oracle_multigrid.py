"""Pins of the two-level multigrid oracle (oracle/multigrid.py) against what
linear algebra fixes: block-orthonormality and span of the prolongator,
P^+ as the adjoint of P, the Galerkin operator against dense matrices, the
error propagator of the V-cycle, the exact inverse when the coarse space is
everything, and the Chebyshev smoother's residual polynomial (the scaled
Chebyshev polynomial of the first kind, textbook closed form)."""

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import dwf as O
from oracle import multigrid as MG
from paper_2203_17119_gb300 import inputs

MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)


@pytest.fixture(scope="module")
def small():
    """4 x 4 x 2 x 2 x Ls=2 Moebius lattice, Omega a 4 x 2 x 2 x 2 box that
    wraps in y (cut in y, periodic in z and t), blocks of 2 x 2 x 2 x 2 (2
    blocks, 8 odd sites each: 384 odd degrees of freedom), A = M_pc^+ M_pc of
    D_Omega."""
    dims, Ls = (4, 4, 2, 2), 2
    rng = np.random.default_rng(61)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    box = ((0, 3, 0, 0), (4, 2, 2, 2))
    mask = O.box_mask(dims, box)
    bid, nb = MG.block_index(dims, box, (2, 2, 2, 2))

    def A(f):
        return O.mpc_in(U, O.mpc_in(U, f, MOBIUS, mask), MOBIUS, mask, True)

    odd = (bid >= 0)[..., None, None, None]
    vecs = [np.where(odd, inputs.gaussian_source(dims, Ls, rng=rng), 0) for _ in range(3)]
    return dims, Ls, U, mask, bid, nb, A, vecs, rng


def test_block_index_counts(small):
    dims, Ls, U, mask, bid, nb, A, vecs, rng = small
    assert nb == 2
    counts = np.bincount(bid[bid >= 0], minlength=nb)
    assert np.all(counts == 8)            # 16 sites per block, half of them odd
    # every odd site of the box is in exactly one block, nothing else is
    odd = (O.parity_field(dims) == 1) & mask
    assert np.array_equal(bid >= 0, odd)


def test_prolongator_orthonormal_and_span(small):
    dims, Ls, U, mask, bid, nb, A, vecs, rng = small
    B = MG.block_orthonormalize(vecs, bid, nb)
    for b in range(nb):
        m = (bid == b)[..., None, None, None]
        G = np.array([[np.vdot(u * m, w * m) for w in B] for u in B])
        assert np.allclose(G, np.eye(len(B)), atol=1e-13)
        # span{B_0..B_k} = span{v_0..v_k} on the block (Gram-Schmidt order)
        for k in range(len(B)):
            Q = np.stack([(B[j] * m).reshape(-1) for j in range(k + 1)], axis=1)
            v = (vecs[k] * m).reshape(-1)
            assert np.linalg.norm(v - Q @ (Q.conj().T @ v)) <= 1e-12 * np.linalg.norm(v)
    # P^+ P = 1 and P^+ is the adjoint of P
    c = rng.standard_normal((nb, len(B))) + 1j * rng.standard_normal((nb, len(B)))
    assert np.allclose(MG.restrict(B, bid, nb, MG.prolong(B, bid, nb, c)), c, atol=1e-13)
    f = np.where((bid >= 0)[..., None, None, None], inputs.gaussian_source(dims, Ls, rng=rng), 0)
    lhs = np.vdot(c, MG.restrict(B, bid, nb, f))
    rhs = np.vdot(MG.prolong(B, bid, nb, c), f)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_galerkin_operator_against_dense(small):
    dims, Ls, U, mask, bid, nb, A, vecs, rng = small
    B = MG.block_orthonormalize(vecs, bid, nb)
    Ac = MG.coarse_operator(A, B, bid, nb)
    shape = B[0].shape
    dofs = Dn.site_mask_to_dofs(bid >= 0, Ls * 12)
    # dense P (columns (block, k), k fastest) and dense A on the odd sites of Omega
    P = np.stack([MG.prolong(B, bid, nb, np.eye(nb * len(B))[j].reshape(nb, len(B))).reshape(-1)[dofs]
                  for j in range(nb * len(B))], axis=1)
    Ad = np.empty((dofs.size, dofs.size), dtype=np.complex128)
    e = np.zeros(int(np.prod(shape)), dtype=np.complex128)
    for j, d in enumerate(dofs):
        e[d] = 1.0
        Ad[:, j] = A(e.reshape(shape)).reshape(-1)[dofs]
        e[d] = 0.0
    assert np.allclose(Ad, Ad.conj().T, atol=1e-12)
    want = P.conj().T @ Ad @ P
    assert np.linalg.norm(Ac - want) <= 1e-12 * np.linalg.norm(want)
    assert np.all(np.linalg.eigvalsh(0.5 * (Ac + Ac.conj().T)) > 0)


@pytest.mark.parametrize("smooth", ["none", "chebyshev"])
def test_vcycle_error_propagator(small, smooth):
    """1 - M^-1 A = (1 - S A)(1 - P A_c^-1 P^+ A)(1 - S A) on random vectors,
    with dense matrices for A, P and the smoother."""
    dims, Ls, U, mask, bid, nb, A, vecs, rng = small
    B = MG.block_orthonormalize(vecs, bid, nb)
    Ac = MG.coarse_operator(A, B, bid, nb)
    Ac_inv = np.linalg.inv(Ac)
    shape = B[0].shape
    dofs = Dn.site_mask_to_dofs(bid >= 0, Ls * 12)
    n = int(np.prod(shape))

    def emb(v):
        f = np.zeros(n, dtype=np.complex128)
        f[dofs] = v
        return f.reshape(shape)

    def mat(fn):
        return np.stack([fn(emb(np.eye(dofs.size)[j])).reshape(-1)[dofs] for j in range(dofs.size)], axis=1)

    Ad = mat(A)
    lam_max = float(np.max(np.linalg.eigvalsh(0.5 * (Ad + Ad.conj().T))))
    S = None
    if smooth == "chebyshev":
        S = lambda r: MG.chebyshev_smoother(A, r, 3, lam_max / 8, 1.05 * lam_max)
    M = mat(lambda r: MG.vcycle(A, B, bid, nb, Ac_inv, S, r))
    P = np.stack([MG.prolong(B, bid, nb, np.eye(nb * len(B))[j].reshape(nb, len(B))).reshape(-1)[dofs]
                  for j in range(nb * len(B))], axis=1)
    I = np.eye(dofs.size)
    C = I - P @ Ac_inv @ P.conj().T @ Ad
    Sd = mat(S) if S is not None else np.zeros_like(I)
    E = (I - Sd @ Ad) @ C @ (I - Sd @ Ad)
    assert np.linalg.norm((I - M @ Ad) - E) <= 1e-10 * np.linalg.norm(E)
    # the coarse correction is an A-orthogonal projector: C^2 = C, P^+ A C = 0
    assert np.linalg.norm(C @ C - C) <= 1e-10 * np.linalg.norm(C)
    assert np.linalg.norm(P.conj().T @ Ad @ C) <= 1e-10 * np.linalg.norm(Ad)


def test_vcycle_exact_when_coarse_space_is_everything():
    """One block holding the whole box and as many near-null vectors as the
    box has odd degrees of freedom: P is unitary and M^-1 = A^-1."""
    dims, Ls = (2, 2, 2, 2), 2
    rng = np.random.default_rng(62)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    box = ((0, 0, 0, 0), (2, 2, 2, 2))
    mask = O.box_mask(dims, box)
    bid, nb = MG.block_index(dims, box, (2, 2, 2, 2))
    A = lambda f: O.mpc_in(U, O.mpc_in(U, f, MOBIUS, mask), MOBIUS, mask, True)
    odd = (bid >= 0)[..., None, None, None]
    ndof = int(np.sum(bid >= 0)) * Ls * 12
    vecs = [np.where(odd, inputs.gaussian_source(dims, Ls, rng=rng), 0) for _ in range(ndof)]
    B = MG.block_orthonormalize(vecs, bid, nb)
    Ac_inv = np.linalg.inv(MG.coarse_operator(A, B, bid, nb))
    r = np.where(odd, inputs.gaussian_source(dims, Ls, rng=rng), 0)
    z = MG.vcycle(A, B, bid, nb, Ac_inv, None, r)
    assert np.linalg.norm(A(z) - r) <= 1e-11 * np.linalg.norm(r)


def test_chebyshev_smoother_residual_polynomial():
    """After k steps on A z = r from z = 0, r - A z = T_k((theta - A)/delta) r
    / T_k(theta/delta), theta, delta the centre and half-width of [lo, hi]:
    checked on a random Hermitian positive matrix in its eigenbasis."""
    rng = np.random.default_rng(63)
    n = 40
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, _ = np.linalg.qr(X)
    lam = np.linspace(0.05, 3.0, n)
    Am = (Q * lam) @ Q.conj().T
    A = lambda v: Am @ v
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lo, hi = 0.4, 3.1
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    for k in (1, 2, 5, 9):
        z = MG.chebyshev_smoother(A, r, k, lo, hi)
        Tk = lambda x: np.cosh(k * np.arccosh(x)) if x >= 1 else np.cos(k * np.arccos(np.clip(x, -1, 1)))
        fac = np.array([Tk((theta - l) / delta) / Tk(theta / delta) for l in lam])
        want = Q @ (fac * (Q.conj().T @ r))
        assert np.linalg.norm((r - A(z)) - want) <= 1e-12 * np.linalg.norm(r), k
