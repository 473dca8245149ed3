"""GPU parity of the one-flavour DD-RHMC boundary term (Sec. 2.3.1):
D_dirichlet as the cut-link handle (dwf_create_cut) against D of the oracle's
cut gauge field; the action S = phi^+ r1(A_d) r2(A) r1(A_d) phi and its link
force (dwf_one_flavour_action / _force) against the dense oracle
(oracle.force.one_flavour_*_dense, pinned by central differences) on the
4 x 2 x 2 x 2 slab, Shamir and Moebius, two pseudofermions, with arbitrary
partial fractions, FP64 and FP32 operators, an active box with accumulation;
at 8^4 x 8 with fitted powers (dwf_rational_power): the heat bath makes
S(phi) = |eta|^2, and the force equals central differences of the GPU action
along a random direction on every link.

Tolerances: FP64 solves to 1e-12 give S and F to ~1e-10 relative (1e-9 is
asserted); the FP32 operator with FP64 defect correction to 1e-11, 1e-8;
heat bath 1e-6 (the product of four fits with delta < 1e-8 each); central
differences at eps = 1e-4 (truncation ~eps^2, solver noise ~1e-12 S / eps),
1e-5 relative."""

import numpy as np
import pytest

from oracle import dwf as O
from oracle.force import box_links, one_flavour_action_dense, one_flavour_force_dense
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

SHAMIR = O.DWFParams(M5=1.8, mf=0.1)
MOBIUS = O.DWFParams(M5=1.8, mf=0.05, b5=1.5, c5=0.5)
SLAB, LS = (4, 2, 2, 2), 4
R1 = (0.4, [0.3, 2.0], [0.25, 1.5])
R2 = (0.1, [0.05, 0.7, 4.0], [0.2, 0.6, 2.5])


def _act(prm):
    return G.Action(prm.M5, prm.mf, prm.b5, prm.c5)


def _pair(dims, Ls, prm, cut, U, nrhs):
    h = G.Handle(dims, Ls, _act(prm), nrhs_max=nrhs)
    hd = G.Handle(dims, Ls, _act(prm), nrhs_max=nrhs, cut=cut)
    Ut = torch.from_numpy(U.reshape(-1)).cuda()
    h.set_gauge(Ut)
    hd.set_gauge(Ut)
    return h, hd


def _odd_dev(fields, dims):
    return torch.view_as_real(torch.from_numpy(LY.to_cb([fields], dims, None, 1))).cuda().contiguous()


def _force_host(out, U):
    return torch.view_as_complex(out.view(-1, 2).cpu()).numpy().reshape(U.shape)


def test_cut_handle_is_d_on_the_cut_gauge_field():
    """D and M_pc of the cut handle equal those of the oracle on cut_gauge(U,
    boxes): two boxes, one wrapping, and the rest of the lattice as a third
    domain; the plain handle stays D."""
    dims, Ls, prm = (8, 4, 4, 6), 6, MOBIUS
    rng = np.random.default_rng(71)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    cut = [((1, 0, 0, 0), (3, 4, 4, 3)), ((6, 1, 0, 4), (4, 2, 4, 2))]
    h, hd = _pair(dims, Ls, prm, cut, U, 1)
    Uc = O.cut_gauge(U, cut)
    f = inputs.gaussian_source(dims, Ls, rng=rng)
    x = torch.view_as_real(torch.from_numpy(LY.to_full([[f]], dims, None))).cuda().contiguous()
    for hh, UU in ((hd, Uc), (h, U)):
        for dag in (False, True):
            y = torch.empty_like(x)
            hh.apply_d(y, x, dagger=dag)
            got = LY.from_full(torch.view_as_complex(y.cpu()).numpy(), dims, None, Ls)[0][0]
            assert LY.rel_l2(got, O.apply_D(UU, f, prm, dag)) <= 1e-13
    odd = O.parity_field(dims) == 1
    fo = O.restrict(f, odd)
    xo = _odd_dev([fo], dims)
    yo = torch.empty_like(xo)
    hd.mpc(yo, xo)
    got = LY.from_cb(torch.view_as_complex(yo.cpu()).numpy(), dims, None, 1, Ls)[0][0]
    everywhere = np.ones(odd.shape, dtype=bool)
    assert LY.rel_l2(got, O.mpc_in(Uc, fo, prm, everywhere)) <= 1e-13


@pytest.fixture(scope="module", params=["shamir", "mobius"])
def slab(request):
    prm = SHAMIR if request.param == "shamir" else MOBIUS
    rng = np.random.default_rng(35)
    U = inputs.gauge_field(SLAB, "haar", rng=rng)
    odd = O.parity_field(SLAB) == 1
    phis = [O.restrict(inputs.gaussian_source(SLAB, LS, rng=rng), odd) for _ in range(2)]
    box = O.band_box(SLAB, 2, dirs=(0,))
    h, hd = _pair(SLAB, LS, prm, [box], U, 2)
    return prm, U, phis, box, h, hd


def test_action_matches_oracle(slab):
    prm, U, phis, box, h, hd = slab
    S, st = h.one_flavour_action(hd, _odd_dev(phis, SLAB), R1, R2, nrhs=2, tol=1e-12)
    want = [one_flavour_action_dense(U, p, prm, box, R1, R2) for p in phis]
    assert np.allclose(S, want, rtol=1e-9, atol=0), (S, want)
    assert len(st) == (2 + 3) * 2 and all(s["true_resid"] <= 1e-11 for s in st)


@pytest.mark.parametrize("inner", [G.FP64, G.FP32], ids=["fp64", "fp32"])
def test_force_matches_oracle(slab, inner):
    prm, U, phis, box, h, hd = slab
    want = sum(one_flavour_force_dense(U, p, prm, box, R1, R2) for p in phis)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    tol = 1e-12 if inner == G.FP64 else 1e-11
    st = h.one_flavour_force(hd, out, _odd_dev(phis, SLAB), R1, R2, nrhs=2, tol=tol, inner=inner)
    assert len(st) == (2 * 2 + 3) * 2
    got = _force_host(out, U)
    assert LY.rel_l2(got, want) <= (1e-9 if inner == G.FP64 else 1e-8)
    assert np.abs(got + np.conj(np.swapaxes(got, -1, -2))).max() <= 1e-12 * np.abs(got).max()


def test_force_active_box_and_accumulate(slab):
    prm, U, phis, box, h, hd = slab
    act = box_links(SLAB, box)
    want = one_flavour_force_dense(U, phis[0], prm, box, R1, R2) * act[..., None, None]
    rng = np.random.default_rng(5)
    F0 = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    out = torch.view_as_real(torch.from_numpy(F0.reshape(-1, 3, 3).copy())).reshape(-1).cuda().contiguous()
    h.one_flavour_force(hd, out, _odd_dev(phis[:1], SLAB), R1, R2, nrhs=1, active=box, accumulate=True,
                        tol=1e-12)
    got = _force_host(out, U) - F0
    assert LY.rel_l2(got, want) <= 1e-9
    assert np.abs(got[~act]).max() <= 1e-12


def test_pair_checks():
    U = inputs.gauge_field(SLAB, "haar", rng=np.random.default_rng(1))
    box = O.band_box(SLAB, 2, dirs=(0,))
    h, hd = _pair(SLAB, LS, SHAMIR, [box], U, 1)
    phi = torch.zeros(h.cb_shape(1), dtype=torch.float64, device="cuda")
    with pytest.raises(G.DWFError):
        hd.one_flavour_action(h, phi, R1, R2)          # roles swapped
    with pytest.raises(G.DWFError):
        h.one_flavour_action(hd, phi, (0.1, [-1.0], [1.0]), R2)   # negative shift
    with pytest.raises(G.DWFError):
        G.Handle(SLAB, LS, _act(SHAMIR), cut=[((0, 0, 0, 0), (2, 2, 2, 2)), ((1, 0, 0, 0), (2, 2, 2, 2))])


# ------------------------------------------------------------- 8^4 x 8
DIMS8, LS8 = (8, 8, 8, 8), 8


def _lam_max(h, iters=60):
    g = torch.Generator(device="cuda").manual_seed(9)
    x = torch.randn(h.cb_shape(1), dtype=torch.float64, device="cuda", generator=g)
    t, y = torch.empty_like(x), torch.empty_like(x)
    lam = 0.0
    for _ in range(iters):
        x /= x.norm()
        h.mpc(t, x)
        h.mpc(y, t, dagger=True)
        lam = float((x * y).sum())
        x, y = y, x
    return lam


@pytest.fixture(scope="module")
def lattice8():
    rng = np.random.default_rng(77)
    U = inputs.gauge_field(DIMS8, "exp", eps=0.4, rng=rng)
    cut = [((0, 0, 0, 1), (8, 8, 8, 4))]           # two slabs in t: Omega and Omega-bar
    h, hd = _pair(DIMS8, LS8, MOBIUS, cut, U, 1)
    hi = 1.1 * max(_lam_max(h), _lam_max(hd))
    lo = 1e-6
    n = 24
    fit = {a: G.rational_power(a, n, lo, hi) for a in (0.25, -0.25, -0.5)}
    assert max(f[3] for f in fit.values()) < 1e-8
    rat = {a: (f[0], f[1], f[2]) for a, f in fit.items()}
    return U, cut, h, hd, rat, rng


def test_heatbath_gives_unit_action(lattice8):
    U, cut, h, hd, rat, rng = lattice8
    odd = O.parity_field(DIMS8) == 1
    eta_h = O.restrict(inputs.gaussian_source(DIMS8, LS8, rng=rng), odd)
    eta = _odd_dev([eta_h], DIMS8)
    phi = torch.empty_like(eta)
    h.one_flavour_heatbath(hd, phi, eta, rat[-0.25], rat[0.25], tol=1e-12)
    S, _ = h.one_flavour_action(hd, phi, rat[0.25], rat[-0.5], tol=1e-12)
    e2 = float((eta * eta).sum())
    assert abs(S[0] - e2) <= 1e-6 * e2, (S[0], e2)


def _expm_i_field(H, eps):
    """exp(i eps H) for a field of Hermitian 3 x 3 matrices (eigh)."""
    w, V = np.linalg.eigh(H)
    return np.einsum("...ij,...j,...kj->...ik", V, np.exp(1j * eps * w), V.conj())


def test_force_is_the_derivative_of_the_gpu_action(lattice8):
    U, cut, h, hd, rat, rng = lattice8
    odd = O.parity_field(DIMS8) == 1
    phi = _odd_dev([O.restrict(inputs.gaussian_source(DIMS8, LS8, rng=rng), odd)], DIMS8)
    r1, r2 = rat[0.25], rat[-0.5]
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    h.one_flavour_force(hd, out, phi, r1, r2, tol=1e-12)
    F = _force_host(out, U)
    A = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    H -= np.trace(H, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3
    want = float(np.sum(np.real(np.einsum("...ij,...ji->...", 1j * H, F))))
    eps = 1e-4
    vals = []
    for sg in (1, -1):
        Up = np.einsum("...ij,...jk->...ik", _expm_i_field(H, sg * eps), U)
        Ut = torch.from_numpy(np.ascontiguousarray(Up).reshape(-1)).cuda()
        h.set_gauge(Ut)
        hd.set_gauge(Ut)
        vals.append(h.one_flavour_action(hd, phi, r1, r2, tol=1e-12)[0][0])
    Ut = torch.from_numpy(U.reshape(-1)).cuda()
    h.set_gauge(Ut)
    hd.set_gauge(Ut)
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert abs(fd - want) <= 1e-5 * abs(want), (fd, want)
