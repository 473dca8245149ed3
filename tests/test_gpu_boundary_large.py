"""GPU parity of the boundary-action force (dwf_boundary_force) on a lattice
of several tiles: an 8 x 8 x 4 x 4 Moebius lattice cut in x and y (crossing
patterns of one and two directions) against the matrix-free oracle
(oracle.boundary, itself pinned to the dense construction).  Kept in a file
of its own that runs last: the oracle needs about a minute of CPU."""

import numpy as np
import pytest

from oracle import dwf as O
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402


def _dev(fields, dims):
    return torch.view_as_real(torch.from_numpy(LY.to_full(fields, dims, None))).cuda().contiguous()


def test_boundary_force_two_direction_band_matches_matrix_free_oracle():
    """The force of |R^-1 phi|^2 on an 8 x 8 x 4 x 4 Moebius lattice cut in x
    and y (several tiles, crossing patterns of one and two directions) against
    the matrix-free oracle (itself pinned to the dense construction)."""
    from oracle import boundary as B
    dims, Ls = (8, 8, 4, 4), 4
    prm = O.DWFParams(M5=1.8, mf=0.1, b5=1.5, c5=0.5)
    rng = np.random.default_rng(91)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    phi = inputs.gaussian_source(dims, Ls, rng=rng)
    box = O.band_box(dims, 2, dirs=(0, 1))
    want = B.boundary_action_force(U, phi, prm, box, tol=1e-13)
    h = G.Handle(dims, Ls, G.Action(prm.M5, prm.mf, prm.b5, prm.c5))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    stats = h.boundary_force(out, _dev([[phi]], dims), box, tol=1e-12)
    assert all(s["true_resid"] <= 1e-11 for s in stats)
    got = torch.view_as_complex(out.view(-1, 2).cpu()).numpy().reshape(U.shape)
    assert LY.rel_l2(got, want) <= 2e-7
