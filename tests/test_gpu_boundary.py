"""GPU parity of the boundary operator of Sec. 2.1 (dwf_boundary_project,
dwf_boundary_rinv) against the FP64 oracle.

On the 4 x 2 x 2 x 2, Ls = 4 Moebius slab (Omega: a band of width 2 cut in
x) the projector P and R^-1 = P - P D^-1 D_partialbar are compared element
by element with the dense oracle: P from the SVD of the D_partialbar block
of the dense D, D^-1 from LU.  On an 8 x 8 x 4 x 4 lattice cut in x and y, P must be a Hermitian idempotent supported on Omega that
D_partialbar does not see the complement of (D_partialbar P = D_partialbar,
through the oracle's D), and R^-1 must match u - P D^-1 (D u on Omega-bar)
with D^-1 from the oracle's CGNE.  Bad geometries are rejected."""

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import dwf as O
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)
SHAMIR = O.DWFParams(M5=1.8, mf=0.1)


def _handle(dims, Ls, prm, U, nrhs=1):
    h = G.Handle(dims, Ls, G.Action(prm.M5, prm.mf, prm.b5, prm.c5), nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    return h


def _dev(fields, dims):
    return torch.view_as_real(torch.from_numpy(LY.to_full(fields, dims, None))).cuda().contiguous()


def _host(t, dims, Ls):
    return LY.from_full(torch.view_as_complex(t.cpu()).numpy(), dims, None, Ls)


def test_slab_matches_dense_oracle():
    dims, Ls = (4, 2, 2, 2), 4
    rng = np.random.default_rng(99)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)
    box = O.band_box(dims, 2, dirs=(0,))
    D = Dn.dense_matrix(lambda f: O.apply_D(U, f, MOBIUS), shape)
    ids = O.box_id_field(dims, [box])
    om = Dn.site_mask_to_dofs(ids == 0, Ls * 12)
    ob = Dn.site_mask_to_dofs(ids < 0, Ls * 12)
    DO, Dd, Ddb, DOb = Dn.blocks(D, om, ob)
    _, P = Dn.rowspace_projector(Ddb)
    nO = DO.shape[0]
    Dinv = np.linalg.inv(np.block([[DO, Dd], [Ddb, DOb]]))
    Rinv = P - P @ (Dinv[:nO, nO:] @ Ddb)

    nrhs = 2
    psis = [inputs.gaussian_source(dims, Ls, rng=rng) for _ in range(nrhs)]
    h = _handle(dims, Ls, MOBIUS, U, nrhs)
    src = _dev([psis], dims)
    out = torch.zeros_like(src)
    h.boundary_project(out, src, box, nrhs=nrhs)
    got = _host(out, dims, Ls)[0]
    for r in range(nrhs):
        want = np.zeros(np.prod(shape), complex)
        want[om] = P @ psis[r].reshape(-1)[om]
        assert LY.rel_l2(got[r].reshape(-1), want) <= 1e-12
    stats = h.boundary_rinv(out, src, box, nrhs=nrhs, tol=1e-12)
    assert all(s["true_resid"] <= 1e-11 for s in stats)
    got = _host(out, dims, Ls)[0]
    for r in range(nrhs):
        want = np.zeros(np.prod(shape), complex)
        want[om] = Rinv @ psis[r].reshape(-1)[om]
        assert LY.rel_l2(got[r].reshape(-1), want) <= 1e-9


def _interior(dims, box):
    """Sites of Omega whose eight neighbours all lie in Omega."""
    m = O.box_mask(dims, box)
    out = m.copy()
    for ax in range(4):
        out &= np.roll(m, 1, axis=ax) & np.roll(m, -1, axis=ax)
    return out


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_two_direction_band_properties(prm):
    dims, Ls = (8, 8, 4, 4), 4
    rng = np.random.default_rng(7)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    box = O.band_box(dims, 2, dirs=(0, 1))
    inside = O.box_mask(dims, box)
    a, b = (inputs.gaussian_source(dims, Ls, rng=rng) for _ in range(2))
    h = _handle(dims, Ls, prm, U, 2)
    src = _dev([[a, b]], dims)
    out = torch.zeros_like(src)
    h.boundary_project(out, src, box, nrhs=2)
    Pa, Pb = _host(out, dims, Ls)[0]
    # supported on Omega, Hermitian, idempotent
    assert np.abs(O.restrict(Pa, ~inside)).max() == 0.0
    assert abs(np.vdot(a, Pb) - np.vdot(Pa, b)) <= 1e-12 * O.norm(a) * O.norm(b)
    src2 = _dev([[Pa, Pb]], dims)
    h.boundary_project(out, src2, box, nrhs=2)
    PPa, PPb = _host(out, dims, Ls)[0]
    assert LY.rel_l2(PPa, Pa) <= 1e-13 and LY.rel_l2(PPb, Pb) <= 1e-13
    # D_partialbar P = D_partialbar: the hops from Omega into Omega-bar see P a as a
    a_in = O.restrict(a, inside)
    lhs = O.restrict(O.apply_D(U, Pa, prm), ~inside)
    rhs = O.restrict(O.apply_D(U, a_in, prm), ~inside)
    assert LY.rel_l2(lhs, rhs) <= 1e-13
    # no hop leaves Omega from its interior sites: P vanishes there
    assert np.abs(O.restrict(Pa, _interior(dims, box))).max() == 0.0
    assert _interior(dims, box).sum() == 4 * 4 * 4 * 4

    # R^-1 a against the oracle's CGNE for D^-1
    stats = h.boundary_rinv(out, src, box, nrhs=2, tol=1e-11)
    assert all(s["true_resid"] <= 1e-10 for s in stats)
    got = _host(out, dims, Ls)[0]
    # (the first right-hand side: one oracle solve of ~130 CG iterations)
    v = O.restrict(O.apply_D(U, Pa, prm), ~inside)
    y, _ = O.cgne(U, v, prm, tol=1e-12)
    h.boundary_project(out, _dev([[y, y]], dims), box, nrhs=2)
    Py = _host(out, dims, Ls)[0][0]
    assert LY.rel_l2(got[0], Pa - Py) <= 1e-8
    assert O.norm(got[1]) > 0.0


def test_whole_lattice_omega_is_zero():
    dims, Ls = (4, 4, 4, 4), 4
    rng = np.random.default_rng(8)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    h = _handle(dims, Ls, SHAMIR, U)
    src = _dev([[inputs.gaussian_source(dims, Ls, rng=rng)]], dims)
    out = torch.ones_like(src)
    full = ((0, 0, 0, 0), dims)
    h.boundary_rinv(out, src, full)
    assert float(out.abs().max()) == 0.0
    out.fill_(1.0)
    h.boundary_project(out, src, full)
    assert float(out.abs().max()) == 0.0


def test_bad_geometry_rejected():
    dims, Ls = (4, 4, 4, 4), 4
    rng = np.random.default_rng(9)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    h = _handle(dims, Ls, SHAMIR, U)
    src = _dev([[inputs.gaussian_source(dims, Ls, rng=rng)]], dims)
    out = torch.zeros_like(src)
    # band of width 1: the site x = 3 touches x = 2 and (periodically) x = 0
    with pytest.raises(G.DWFError):
        h.boundary_project(out, src, ((0, 0, 0, 0), (3, 4, 4, 4)))
    with pytest.raises(G.DWFError):
        h.boundary_project(out, out, O.band_box(dims, 2))
    hb = G.Handle(dims, Ls, G.Action(1.8, 0.1), boxes=[O.band_box(dims, 2)])
    hb.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    with pytest.raises(G.DWFError):
        hb.boundary_project(out, src, O.band_box(dims, 2))


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_boundary_action_force_matches_oracle(prm):
    """Force of |R^-1 phi|^2 on the 4 x 2 x 2 x 2 slab against the dense
    oracle (itself pinned by finite differences of the action), both
    right-hand sides summed; then with an active box and accumulation."""
    from oracle.force import box_links, boundary_action_force_dense
    dims, Ls = (4, 2, 2, 2), 4
    rng = np.random.default_rng(41)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    phis = [inputs.gaussian_source(dims, Ls, rng=rng) for _ in range(2)]
    box = O.band_box(dims, 2, dirs=(0,))
    want = sum(boundary_action_force_dense(U, f, prm, box) for f in phis)
    h = _handle(dims, Ls, prm, U, 2)
    src = _dev([phis], dims)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    stats = h.boundary_force(out, src, box, nrhs=2, tol=1e-12)
    assert len(stats) == 4 and all(s["true_resid"] <= 1e-11 for s in stats)
    got = torch.view_as_complex(out.view(-1, 2).cpu()).numpy().reshape(U.shape)
    assert LY.rel_l2(got, want) <= 1e-9
    # active links: both ends in x in {1, 2}; accumulate onto the previous result
    act_box = ((1, 0, 0, 0), (2, 2, 2, 2))
    act = box_links(dims, act_box)
    h.boundary_force(out, src, box, nrhs=2, active=act_box, accumulate=True, tol=1e-12)
    got2 = torch.view_as_complex(out.view(-1, 2).cpu()).numpy().reshape(U.shape)
    assert LY.rel_l2(got2, want + want * act[..., None, None]) <= 1e-9


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_r_matches_dense_oracle_and_inverts_rinv(inner):
    """R = P - P D_O^-1 D_d D_Ob^-1 D_db on the slab against the dense oracle
    (Dirichlet solves by FP64 CGNR, or FP32 CGNR with FP64 defect
    correction); then R (R^-1 psi) = P psi (Sec. 2.1) with both library calls."""
    prec = G.FP64 if inner == "fp64" else G.FP32
    dims, Ls = (4, 2, 2, 2), 4
    rng = np.random.default_rng(99)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)
    box = O.band_box(dims, 2, dirs=(0,))
    D = Dn.dense_matrix(lambda f: O.apply_D(U, f, MOBIUS), shape)
    ids = O.box_id_field(dims, [box])
    om = Dn.site_mask_to_dofs(ids == 0, Ls * 12)
    ob = Dn.site_mask_to_dofs(ids < 0, Ls * 12)
    DO, Dd, Ddb, DOb = Dn.blocks(D, om, ob)
    _, P = Dn.rowspace_projector(Ddb)
    R = P - P @ np.linalg.solve(DO, Dd @ np.linalg.solve(DOb, Ddb))
    psis = [inputs.gaussian_source(dims, Ls, rng=rng) for _ in range(2)]
    h = _handle(dims, Ls, MOBIUS, U, 2)
    src = _dev([psis], dims)
    out = torch.zeros_like(src)
    stats = h.boundary_r(out, src, box, nrhs=2, tol=1e-12, inner=prec)
    assert len(stats) == 4 and all(s["true_resid"] <= 2e-12 for s in stats)
    got = _host(out, dims, Ls)[0]
    for r in range(2):
        want = np.zeros(np.prod(shape), complex)
        want[om] = R @ psis[r].reshape(-1)[om]
        assert LY.rel_l2(got[r].reshape(-1), want) <= 1e-9
    # R R^-1 = P
    rinv = torch.zeros_like(src)
    h.boundary_rinv(rinv, src, box, nrhs=2, tol=1e-12)
    h.boundary_r(out, rinv, box, nrhs=2, tol=1e-12, inner=prec)
    proj = torch.zeros_like(src)
    h.boundary_project(proj, src, box, nrhs=2)
    assert LY.rel_l2(_host(out, dims, Ls)[0][0], _host(proj, dims, Ls)[0][0]) <= 1e-9


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS], ids=["shamir", "mobius"])
def test_r_inverts_rinv_two_direction_band(prm):
    dims, Ls = (8, 8, 4, 4), 4
    rng = np.random.default_rng(71)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    box = O.band_box(dims, 2, dirs=(0, 1))
    h = _handle(dims, Ls, prm, U, 1)
    src = _dev([[inputs.gaussian_source(dims, Ls, rng=rng)]], dims)
    rinv, out, proj = torch.zeros_like(src), torch.zeros_like(src), torch.zeros_like(src)
    h.boundary_rinv(rinv, src, box, tol=1e-12)
    stats = h.boundary_r(out, rinv, box, tol=1e-11)
    assert all(s["true_resid"] <= 2e-11 for s in stats)
    h.boundary_project(proj, src, box)
    assert LY.rel_l2(_host(out, dims, Ls)[0][0], _host(proj, dims, Ls)[0][0]) <= 1e-8


@pytest.mark.parametrize("light,pv", [(SHAMIR, O.DWFParams(M5=1.8, mf=1.0)),
                                      (MOBIUS, O.DWFParams(M5=1.8, mf=1.0, b5=1.5, c5=0.5))],
                         ids=["shamir", "mobius"])
def test_ratio_force_matches_oracle(light, pv):
    """Force of |R^-1 R_pv phi|^2 on the slab against the dense oracle (itself
    pinned by finite differences), then with the boundary links inactive."""
    from oracle.force import box_links, ratio_action_force_dense
    dims, Ls = (4, 2, 2, 2), 4
    rng = np.random.default_rng(43)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    phi = inputs.gaussian_source(dims, Ls, rng=rng)
    box = O.band_box(dims, 2, dirs=(0,))
    want = ratio_action_force_dense(U, phi, light, pv, box)
    hl = _handle(dims, Ls, light, U)
    hp = _handle(dims, Ls, pv, U)
    src = _dev([[phi]], dims)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    stats = hl.boundary_ratio_force(hp, out, src, box, tol=1e-12)
    assert len(stats) == 6 and all(s["true_resid"] <= 1e-11 for s in stats)
    got = torch.view_as_complex(out.view(-1, 2).cpu()).numpy().reshape(U.shape)
    assert LY.rel_l2(got, want) <= 1e-9
    act_box = ((1, 0, 0, 0), (2, 2, 2, 2))
    act = box_links(dims, act_box)
    hl.boundary_ratio_force(hp, out, src, box, active=act_box, tol=1e-12)
    got = torch.view_as_complex(out.view(-1, 2).cpu()).numpy().reshape(U.shape)
    assert LY.rel_l2(got, want * act[..., None, None]) <= 1e-9

