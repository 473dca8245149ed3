"""Oracle: two-level aggregation multigrid for the normal Schur operator,
plain FP64 numpy (test infrastructure only).

Sec. 4 proposes a multigrid solver for the local (D_Omega) systems of the
domain-decomposed HMC, set up with recursively built Chebyshev filter
functions instead of inverse iteration, and states that set-up plus solve
beat one red-black Krylov solve.  The paper gives the filter, not the rest;
the construction here is the standard two-level aggregation method, taken as
a reading:

* A = M_pc^+ M_pc on the odd checkerboard of the handle's domain (Hermitian,
  positive definite), the operator whose CG is the red-black solve;
* aggregates: 4D blocks of the domain's odd sites, with all of their
  fifth-dimension and spin-colour components;
* near-null vectors v_1..v_n: Chebyshev-filtered Gaussian vectors
  T_m(z(A)) v (oracle.chebyshev);
* prolongator P: the restrictions of v_1..v_n to each block, orthonormalised
  within the block by modified Gram-Schmidt in the order v_1, v_2, ...
  (P^+ P = 1); restriction P^+;
* Galerkin coarse operator A_c = P^+ A P (dense here), coarse solve exact;
* preconditioner: the V(1,1) cycle with a smoother S (a fixed linear map:
  the learned network K, a polynomial in A, or none),
      z = S r;  z += P A_c^-1 P^+ (r - A z);  z += S (r - A z),
  whose error propagator is (1 - S A)(1 - P A_c^-1 P^+ A)(1 - S A).

Coarse vectors are arrays c[block, k] (complex).  Fields are oracle layout
arrays (t, z, y, x, s, spin, colour) vanishing off the domain's odd sites.
"""

from __future__ import annotations

import numpy as np


def block_index(dims, box, block):
    """Array (t, z, y, x) with the aggregate index of every odd site of the
    box (origin, extent), -1 elsewhere.  The box is cut into blocks of
    extents ``block`` (x, y, z, t) from its origin, lexicographic in
    box-local block coordinates (x fastest); extents must divide."""
    org, ext = box
    L = dims
    nb = [ext[m] // block[m] for m in range(4)]
    if any(ext[m] % block[m] for m in range(4)):
        raise ValueError("block extents must divide the box extents")
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    coords = (x, y, z, t)
    loc = [(coords[m] - org[m]) % L[m] for m in range(4)]
    inside = np.ones(x.shape, dtype=bool)
    for m in range(4):
        inside &= loc[m] < ext[m]
    odd = (x + y + z + t) % 2 == 1
    bc = [loc[m] // block[m] for m in range(4)]
    bid = bc[0] + nb[0] * (bc[1] + nb[1] * (bc[2] + nb[2] * bc[3]))
    return np.where(inside & odd, bid, -1), int(np.prod(nb))


def block_orthonormalize(vectors, bid, nblocks):
    """Basis B[k] (list of fields): v_k restricted to each block and
    orthonormalised there against B[0..k-1] by modified Gram-Schmidt."""
    out = []
    for v in vectors:
        w = np.where((bid >= 0)[..., None, None, None], v, 0)
        for b in range(nblocks):
            m = (bid == b)[..., None, None, None]
            for u in out:
                w = w - m * np.vdot(u * m, w * m) * u
            nrm = np.linalg.norm(w * m)
            if not nrm > 0:
                raise ValueError("near-null vector vanishes on a block")
            w = np.where(m, w / nrm, w)
        out.append(w)
    return out


def restrict(B, bid, nblocks, f):
    """P^+ f: c[b, k] = <B_k on block b, f>."""
    c = np.zeros((nblocks, len(B)), dtype=np.complex128)
    for b in range(nblocks):
        m = (bid == b)[..., None, None, None]
        for k, u in enumerate(B):
            c[b, k] = np.vdot(u * m, f * m)
    return c


def prolong(B, bid, nblocks, c):
    """P c = sum_{b, k} c[b, k] (B_k on block b)."""
    f = np.zeros_like(B[0])
    for b in range(nblocks):
        m = (bid == b)[..., None, None, None]
        for k, u in enumerate(B):
            f = f + c[b, k] * (u * m)
    return f


def coarse_operator(apply_A, B, bid, nblocks):
    """Dense A_c = P^+ A P, rows and columns in (block, k) order (k fastest)."""
    n = nblocks * len(B)
    Ac = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros((nblocks, len(B)), dtype=np.complex128)
        e.reshape(-1)[j] = 1.0
        Ac[:, j] = restrict(B, bid, nblocks, apply_A(prolong(B, bid, nblocks, e))).reshape(-1)
    return Ac


def vcycle(apply_A, B, bid, nblocks, Ac_inv, smoother, r):
    """The V(1,1) cycle z = M^-1 r: pre-smoothing, exact coarse correction,
    post-smoothing (``smoother`` None: no smoothing steps)."""
    z = smoother(r) if smoother is not None else np.zeros_like(r)
    rc = restrict(B, bid, nblocks, r - apply_A(z)).reshape(-1)
    z = z + prolong(B, bid, nblocks, (Ac_inv @ rc).reshape(nblocks, len(B)))
    if smoother is not None:
        z = z + smoother(r - apply_A(z))
    return z


def chebyshev_smoother(apply_A, r, steps: int, lo: float, hi: float):
    """The Chebyshev iteration for A z = r started from z = 0 with the
    spectrum bounds [lo, hi] (the standard polynomial smoother: it damps the
    error components with eigenvalues in [lo, hi]); steps - 1 applications
    of A, after which r - A z = T_steps((theta - A)/delta) r / T_steps(theta/delta)
    with theta, delta the centre and half-width of [lo, hi].  Three-term
    recurrence of the scaled Chebyshev polynomials."""
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    d = r / theta
    z = np.zeros_like(r)
    res = r.copy()
    for k in range(steps):
        z = z + d
        if k == steps - 1:
            break
        res = res - apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * res
        rho = rho_new
    return z
