"""GPU parity of the Chebyshev filter (dwf_chebyshev_filter) against the
FP64 oracle: T_n(z(A)) v with A = M_pc^+ M_pc of the whole lattice and of two
uneven Dirichlet boxes (each filtered with its own operator), FP64 (relative
L2 <= 1e-11) and FP32 (<= 1e-4), orders 0, 1 and 10; bad arguments rejected."""

import numpy as np
import pytest

from oracle import dwf as O
from oracle.chebyshev import chebyshev_filter
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)
SHAMIR = O.DWFParams(M5=1.8, mf=0.01)
LO, HI = 1.0, 120.0


def _problem(dims, Ls, prm, boxes, nrhs, seed):
    rng = np.random.default_rng(seed)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    masks = [O.box_mask(dims, b) for b in boxes] if boxes else [np.ones(dims[::-1], bool)]
    odd = O.parity_field(dims) == 1
    vs = [[O.restrict(inputs.gaussian_source(dims, Ls, rng=rng), masks[k] & odd) for _ in range(nrhs)]
          for k in range(len(masks))]
    h = G.Handle(dims, Ls, G.Action(prm.M5, prm.mf, prm.b5, prm.c5), boxes=boxes, nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    vcb = torch.view_as_real(torch.from_numpy(LY.to_cb(vs, dims, boxes, 1))).cuda().contiguous()
    return U, masks, vs, h, vcb


CASES = {
    "mobius_whole_4448x8": ((4, 4, 4, 8), 8, MOBIUS, None, 1),
    "shamir_boxes_nrhs2": ((4, 4, 6, 8), 8, SHAMIR, [((1, 1, 1, 1), (3, 2, 5, 6)), ((0, 0, 0, 0), (4, 4, 2, 8))], 2),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [G.FP64, G.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("order", [0, 1, 10])
def test_filter_matches_oracle(name, prec, order):
    dims, Ls, prm, boxes, nrhs = CASES[name]
    U, masks, vs, h, vcb = _problem(dims, Ls, prm, boxes, nrhs, 61)
    src = vcb if prec == G.FP64 else vcb.float()
    out = torch.zeros_like(src)
    h.chebyshev_filter(out, src, order, LO, HI, prec=prec, nrhs=nrhs)
    got = LY.from_cb(torch.view_as_complex(out.double().cpu()).numpy(), dims, boxes, 1, Ls)
    tol = 1e-11 if prec == G.FP64 else 1e-4
    for bi, mask in enumerate(masks):
        def A(f, mask=mask):
            return O.mpc_in(U, O.mpc_in(U, f, prm, mask), prm, mask, True)
        for r in range(nrhs):
            want = chebyshev_filter(A, vs[bi][r], order, LO, HI)
            assert LY.rel_l2(got[bi][r], want) <= tol, (bi, r)


def test_bad_arguments():
    dims, Ls, prm, boxes, nrhs = CASES["mobius_whole_4448x8"]
    U, masks, vs, h, vcb = _problem(dims, Ls, prm, boxes, nrhs, 62)
    out = torch.zeros_like(vcb)
    with pytest.raises(G.DWFError):
        h.chebyshev_filter(out, vcb, 4, 2.0, 1.0)
    with pytest.raises(G.DWFError):
        h.chebyshev_filter(out, vcb, -1, 1.0, 2.0)
    with pytest.raises(G.DWFError):
        h.chebyshev_filter(out, vcb, 4, 1.0, 2.0, prec=G.BF16)
    with pytest.raises(G.DWFError):
        h.chebyshev_filter(vcb, vcb, 4, 1.0, 2.0)
