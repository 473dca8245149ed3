"""GPU parity of the two-level multigrid (dwf_mg_*) against oracle/multigrid.py:
the block-orthonormal basis, the transfer operators, the Galerkin coarse
operator, the V-cycle with and without a smoother, on the whole lattice and
on a Dirichlet box; and flexible GCR preconditioned by it reaching 1e-10 by
the oracle's residual in fewer iterations than GCR without preconditioner.
Tolerances: FP32 operator and fields (relative L2 1e-5 for single passes;
the V-cycle goes through A_c^-1, compared with the coarse matrix the device
built, 1e-4)."""

import zlib

import numpy as np
import pytest

from oracle import dwf as O
from oracle import multigrid as MGO
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)
SHAMIR = O.DWFParams(M5=1.8, mf=0.01)

CASES = {
    # name: dims, Ls, params, box (None: whole lattice), block, nvec
    "whole_mobius": ((4, 4, 4, 8), 8, MOBIUS, None, (2, 2, 2, 4), 4),
    "box_shamir": ((8, 4, 4, 8), 8, SHAMIR, ((1, 0, 1, 2), (6, 4, 2, 4)), (3, 2, 2, 2), 3),
}


def _host(t):
    return torch.view_as_complex(t.double().cpu().contiguous()).numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _lam_max(h, iters=40):
    """Top of the spectrum of A = M_pc^+ M_pc by power iteration (FP32, device)."""
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(h.cb_shape(1), device="cuda", generator=g)
    t, y = torch.empty_like(x), torch.empty_like(x)
    lam = 0.0
    for _ in range(iters):
        x /= x.norm()
        h.mpc(t, x, prec=G.FP32)
        h.mpc(y, t, dagger=True, prec=G.FP32)
        lam = float((x * y).sum())
        x, y = y, x
    return lam


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    dims, Ls, prm, box, block, nvec = CASES[request.param]
    rng = np.random.default_rng(zlib.crc32(request.param.encode()))
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    boxes = [box] if box else None
    h = G.Handle(dims, Ls, G.Action(prm.M5, prm.mf, prm.b5, prm.c5), boxes=boxes, nrhs_max=nvec)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    obox = box if box else ((0, 0, 0, 0), dims)
    mask = O.box_mask(dims, obox)
    bid, nb = MGO.block_index(dims, obox, block)
    A = lambda f: O.mpc_in(U, O.mpc_in(U, f, prm, mask), prm, mask, True)
    # near-null vectors: Gaussian vectors through a short Chebyshev filter on the device
    odd = (bid >= 0)[..., None, None, None]
    vs = [np.where(odd, inputs.gaussian_source(dims, Ls, rng=rng), 0) for _ in range(nvec)]
    V0 = torch.view_as_real(torch.from_numpy(LY.to_cb([vs], dims, boxes, 1))).cuda().float().contiguous()
    V = torch.empty_like(V0)
    lam = _lam_max(h)
    h.chebyshev_filter(V, V0, 8, lam / 30, 1.05 * lam, prec=G.FP32, nrhs=nvec)
    torch.cuda.synchronize()
    Vh = LY.from_cb(_host(V), dims, boxes, 1, Ls)[0]          # [k] oracle-layout fields
    mg = G.MG(h, block, nvec)
    mg.setup(V)
    return dims, Ls, prm, boxes, U, h, mg, A, bid, nb, Vh, rng, lam


def test_basis_and_transfers(case):
    dims, Ls, prm, boxes, U, h, mg, A, bid, nb, Vh, rng, lam = case
    B = MGO.block_orthonormalize(Vh, bid, nb)
    got = LY.from_cb(_host(mg.basis()), dims, boxes, 1, Ls)[0]
    assert _rel(np.stack(got), np.stack(B)) <= 1e-5
    assert mg.sizes() == (nb, nb * len(B))
    f = np.where((bid >= 0)[..., None, None, None], inputs.gaussian_source(dims, Ls, rng=rng), 0)
    fg = torch.view_as_real(torch.from_numpy(LY.to_cb([[f]], dims, boxes, 1))).cuda().float().contiguous()
    c = mg.restrict(fg)
    torch.cuda.synchronize()
    c_want = MGO.restrict(B, bid, nb, f)
    assert _rel(torch.view_as_complex(c.cpu()).numpy(), c_want) <= 1e-5
    pf = mg.prolong(c)
    torch.cuda.synchronize()
    p_want = MGO.prolong(B, bid, nb, c_want)
    got_p = LY.from_cb(_host(pf), dims, boxes, 1, Ls)[0][0]
    assert _rel(got_p, p_want) <= 1e-5


def test_galerkin_coarse_operator(case):
    dims, Ls, prm, boxes, U, h, mg, A, bid, nb, Vh, rng, lam = case
    B = MGO.block_orthonormalize(Vh, bid, nb)
    want = MGO.coarse_operator(A, B, bid, nb)
    got = mg.coarse_operator()
    assert _rel(got, want) <= 1e-5
    assert np.linalg.norm(got - got.conj().T) <= 1e-5 * np.linalg.norm(got)


@pytest.mark.parametrize("smoother", ["none", "chebyshev"])
def test_vcycle(case, smoother):
    dims, Ls, prm, boxes, U, h, mg, A, bid, nb, Vh, rng, lam = case
    B = LY.from_cb(_host(mg.basis()), dims, boxes, 1, Ls)[0]
    Ac_inv = np.linalg.inv(mg.coarse_operator())
    S = None
    if smoother == "chebyshev":
        lo, hi = lam / 10, 1.05 * lam
        mg.set_smoother("chebyshev", 3, lo, hi)
        S = lambda r: MGO.chebyshev_smoother(A, r, 3, lo, hi)
    else:
        mg.set_smoother("none")
    r = np.where((bid >= 0)[..., None, None, None], inputs.gaussian_source(dims, Ls, rng=rng), 0)
    rg = torch.view_as_real(torch.from_numpy(LY.to_cb([[r]], dims, boxes, 1))).cuda().float().contiguous()
    z = torch.empty_like(rg)
    for _ in range(2):                     # twice: the scratch of one call must not leak into the next
        mg.apply(z, rg)
        torch.cuda.synchronize()
        got = LY.from_cb(_host(z), dims, boxes, 1, Ls)[0][0]
        want = MGO.vcycle(A, B, bid, nb, Ac_inv, S, r)
        assert _rel(got, want) <= 1e-4, smoother
    mg.set_smoother("none")


def test_gcr_with_multigrid_converges_faster(case):
    dims, Ls, prm, boxes, U, h, mg, A, bid, nb, Vh, rng, lam = case
    mg.set_smoother("chebyshev", 3, lam / 10, 1.05 * lam)
    obox = boxes[0] if boxes else ((0, 0, 0, 0), dims)
    b = O.restrict(inputs.gaussian_source(dims, Ls, rng=rng), O.box_mask(dims, obox))
    bf = torch.view_as_real(torch.from_numpy(LY.to_full([[b]], dims, boxes))).cuda().contiguous()
    its = {}
    for name in ("mg", "plain"):
        x = torch.zeros_like(bf)
        if name == "mg":
            st, rc = h.gcr_solve_mg(x, bf, mg, tol=1e-10, max_seconds=300)
        else:
            st, rc = h.gcr_solve(x, bf, tol=1e-10, max_seconds=300)
        assert rc == 0 and st[0]["true_resid"] <= 1e-10, (name, st)
        assert st[0]["recorded"] != -1, (name, "fell back to CG")
        xf = LY.from_full(torch.view_as_complex(x.cpu()).numpy(), dims, boxes, Ls)[0][0]
        Dx = O.dirichlet_D(U, xf, prm, boxes) if boxes else O.apply_D(U, xf, prm)
        assert O.norm(b - Dx) / O.norm(b) <= 1e-10, name
        its[name] = st[0]["iters"]
    mg.set_smoother("none")
    assert its["mg"] < its["plain"], its
