"""Pins of the matrix-free boundary-operator oracle (CPU): on the slab it must
reproduce the dense constructions (P from the SVD of the D_partialbar block,
R^-1 with a dense inverse, the boundary-action force pinned by finite
differences in test_oracle_force), and on a larger lattice P must be a
Hermitian idempotent that D_partialbar does not see the complement of."""

import numpy as np
import pytest

from oracle import boundary as B
from oracle import dense as Dn
from oracle import dwf as O
from oracle.force import boundary_action_force_dense, boundary_pieces_dense
from paper_2203_17119_gb300 import inputs

MOBIUS = O.DWFParams(M5=1.8, mf=0.1, b5=1.5, c5=0.5)
SHAMIR = O.DWFParams(M5=1.8, mf=0.1)
SLAB = (4, 2, 2, 2)


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_slab_matches_dense(prm):
    rng = np.random.default_rng(81)
    U = inputs.gauge_field(SLAB, "haar", rng=rng)
    phi = inputs.gaussian_source(SLAB, 4, rng=rng)
    box = O.band_box(SLAB, 2, dirs=(0,))
    pc = boundary_pieces_dense(U, phi, prm, box)
    Pphi = (pc["P"] @ phi.reshape(-1)).reshape(phi.shape)
    assert np.linalg.norm(B.project(phi, box, prm) - Pphi) <= 1e-12 * np.linalg.norm(Pphi)
    chi = B.rinv(U, phi, prm, box)
    assert np.linalg.norm(chi - pc["chi"]) <= 1e-9 * np.linalg.norm(pc["chi"])
    F = B.boundary_action_force(U, phi, prm, box)
    Fd = boundary_action_force_dense(U, phi, prm, box)
    assert np.linalg.norm(F - Fd) <= 1e-8 * np.linalg.norm(Fd)


def test_projector_properties_two_direction_band():
    dims, Ls = (6, 6, 2, 2), 4
    rng = np.random.default_rng(82)
    box = O.band_box(dims, 2, dirs=(0, 1))
    inside = O.box_mask(dims, box)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    a, b = (inputs.gaussian_source(dims, Ls, rng=rng) for _ in range(2))
    Pa, Pb = B.project(a, box, MOBIUS), B.project(b, box, MOBIUS)
    assert abs(np.vdot(a, Pb) - np.vdot(Pa, b)) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)
    assert np.linalg.norm(B.project(Pa, box, MOBIUS) - Pa) <= 1e-12 * np.linalg.norm(Pa)
    lhs = O.restrict(O.apply_D(U, Pa, MOBIUS), ~inside)
    rhs = O.restrict(O.apply_D(U, O.restrict(a, inside), MOBIUS), ~inside)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)
