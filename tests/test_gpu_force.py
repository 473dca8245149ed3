"""GPU parity of the link force (dwf_force) against the FP64 oracle.

Element by element against oracle.force.force_bilinear (FP64: relative L2
<= 1e-12; FP32 fields, links and arithmetic: <= 2e-5) on Shamir and Moebius
lattices with one and two right-hand sides, a ragged lattice, an active box
that wraps around the lattice, and accumulation.  At the bench size
(16^4 x 12 Moebius) the force is checked through the exact linearity of D in
the links: for U -> U + i H U on every link, Re <X, D Y> changes by
sum_links Re tr[i H F] (both sides on the GPU, D by dwf_apply_d in FP64)."""

import numpy as np
import pytest

from oracle import dwf as O
from oracle.force import box_links, force_bilinear
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

SHAMIR = O.DWFParams(M5=1.8, mf=0.01)
MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)

CASES = {
    "shamir_4444x8": ((4, 4, 4, 4), 8, SHAMIR, 1, "haar"),
    "mobius_6448x12_nrhs2": ((6, 4, 4, 8), 12, MOBIUS, 2, "exp"),
    "mobius_ragged_6622x6": ((6, 6, 2, 2), 6, MOBIUS, 1, "haar"),
}


def _setup(dims, Ls, prm, nrhs, kind, seed=21):
    rng = np.random.default_rng(seed)
    U = inputs.gauge_field(dims, kind, eps=0.3, rng=rng)
    Xs = [inputs.gaussian_source(dims, Ls, rng=rng) for _ in range(nrhs)]
    Ys = [inputs.gaussian_source(dims, Ls, rng=rng) for _ in range(nrhs)]
    h = G.Handle(dims, Ls, G.Action(prm.M5, prm.mf, prm.b5, prm.c5), nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    return rng, U, Xs, Ys, h


def _dev(fields, dims, prec=G.FP64):
    t = torch.view_as_real(torch.from_numpy(LY.to_full([fields], dims, None))).cuda().contiguous()
    return t if prec == G.FP64 else t.float()


def _force_host(out, U):
    return torch.view_as_complex(out.cpu()).numpy().reshape(U.shape)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [G.FP64, G.FP32], ids=["fp64", "fp32"])
def test_force_matches_oracle(name, prec):
    dims, Ls, prm, nrhs, kind = CASES[name]
    rng, U, Xs, Ys, h = _setup(dims, Ls, prm, nrhs, kind)
    want = force_bilinear(U, Xs, Ys, prm)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    h.force(out, _dev(Xs, dims, prec), _dev(Ys, dims, prec), prec=prec, nrhs=nrhs)
    got = _force_host(out.view(-1, 2), U)
    tol = 1e-12 if prec == G.FP64 else 2e-5
    assert LY.rel_l2(got, want) <= tol
    # traceless anti-Hermitian on every link
    assert np.abs(got + np.conj(np.swapaxes(got, -1, -2))).max() <= 1e-12 * np.abs(got).max() + 1e-14


def test_active_box_and_accumulate():
    dims, Ls, prm, nrhs, kind = CASES["mobius_6448x12_nrhs2"]
    rng, U, Xs, Ys, h = _setup(dims, Ls, prm, nrhs, kind, seed=22)
    box = ((4, 1, 0, 6), (4, 3, 4, 4))        # wraps in x and t
    act = box_links(dims, box)
    want = force_bilinear(U, Xs, Ys, prm, active=act)
    X, Y = _dev(Xs, dims), _dev(Ys, dims)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    h.force(out, X, Y, nrhs=nrhs, active=box)
    got = _force_host(out.view(-1, 2), U)
    assert LY.rel_l2(got, want) <= 1e-12
    assert np.abs(got[~act]).max() == 0.0 and act.sum() < act.size
    # accumulate: out += F(X, Y) + F(Y, X) (the force of Re <X, (D + D^+) Y>)
    h.force(out, Y, X, nrhs=nrhs, active=box, accumulate=True)
    got = _force_host(out.view(-1, 2), U)
    want2 = want + force_bilinear(U, Ys, Xs, prm, active=act)
    assert LY.rel_l2(got, want2) <= 1e-12


def test_bench_size_linearity():
    """16^4 x 12 Moebius, eps = 0.3 links: sum Re tr[i H F] = f(U + i H U) - f(U)."""
    dims, Ls = (16, 16, 16, 16), 12
    rng = np.random.default_rng(23)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    h = G.Handle(dims, Ls, G.Action(MOBIUS.M5, MOBIUS.mf, MOBIUS.b5, MOBIUS.c5))
    Ud = torch.from_numpy(U.reshape(-1)).cuda()
    h.set_gauge(Ud)
    n = 2 * 12 * Ls * int(np.prod(dims))
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    Y = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    h.force(out, X, Y)
    F = torch.view_as_complex(out.view(-1, 2)).view(-1, 3, 3)
    A = torch.randn(F.shape[0], 3, 3, dtype=torch.complex128, device="cuda", generator=g)
    H = 0.5 * (A + A.conj().transpose(-1, -2))
    H = H - torch.diagonal(H, dim1=-2, dim2=-1).sum(-1)[:, None, None] / 3 * torch.eye(3, device="cuda")
    lin = float((1j * H @ F).diagonal(dim1=-2, dim2=-1).sum().real)

    def f(Uflat):
        h.set_gauge(Uflat)
        DY = torch.zeros_like(Y)
        h.apply_d(DY, Y)
        return float(torch.dot(X, DY))

    Uc = Ud.view(-1, 3, 3)                      # complex128 [link][3][3]
    U2 = (Uc + 1j * H @ Uc).contiguous().view(-1)
    diff = f(U2) - f(Ud)
    assert abs(lin - diff) <= 1e-9 * abs(diff), (lin, diff)
    h.set_gauge(Ud)


def test_bad_arguments():
    dims, Ls, prm, nrhs, kind = CASES["shamir_4444x8"]
    rng, U, Xs, Ys, h = _setup(dims, Ls, prm, nrhs, kind)
    X = _dev(Xs, dims)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(G.DWFError):
        h.force(out, X, X, prec=G.BF16)
    with pytest.raises(G.DWFError):
        h.force(out, X, X, nrhs=2)
    hb = G.Handle(dims, Ls, G.Action(1.8, 0.1), boxes=[((0, 0, 0, 0), (2, 4, 4, 4))])
    hb.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    with pytest.raises(G.DWFError):
        hb.force(out, X, X)


def test_fp32_ls12_active_box_and_accumulate():
    """The FP32 path at N5 = 12 (one lane per thread, sixteen threads per
    site): against the oracle with an active box, then accumulating the
    adjoint bilinear's force."""
    dims, Ls = (4, 4, 4, 8), 12
    rng, U, Xs, Ys, h = _setup(dims, Ls, MOBIUS, 1, "exp", seed=24)
    box = ((3, 0, 1, 2), (3, 4, 2, 5))
    act = box_links(dims, box)
    want = force_bilinear(U, Xs, Ys, MOBIUS, active=act)
    X, Y = _dev(Xs, dims, G.FP32), _dev(Ys, dims, G.FP32)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    h.force(out, X, Y, prec=G.FP32, active=box)
    got = _force_host(out.view(-1, 2), U)
    assert LY.rel_l2(got, want) <= 2e-5
    assert np.abs(got[~act]).max() == 0.0
    h.force(out, Y, X, prec=G.FP32, active=box, accumulate=True)
    got = _force_host(out.view(-1, 2), U)
    assert LY.rel_l2(got, want + force_bilinear(U, Ys, Xs, MOBIUS, active=act)) <= 2e-5
