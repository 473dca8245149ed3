"""GPU parity of the multi-shift CG (dwf_multishift_solve) against the FP64
oracle: every shifted solution x_s must satisfy |b - (A + sigma_s) x_s| /
|b| <= 2 tol with A = M_pc^+ M_pc evaluated by the oracle (boxes: the
Dirichlet block's Schur operator), and agree with the oracle's own
multi-shift solution; the FP32 operator reaches its own accuracy; bad
arguments are rejected."""

import numpy as np
import pytest

from oracle import dwf as O
from oracle.multishift import multishift_cg
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)
SHIFTS = [0.02, 0.0, 0.3, 2.5]


def _problem(dims, Ls, boxes, nrhs, seed):
    rng = np.random.default_rng(seed)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    masks = [O.box_mask(dims, b) for b in boxes] if boxes else [np.ones(dims[::-1], bool)]
    odd = O.parity_field(dims) == 1
    bs = [[O.restrict(inputs.gaussian_source(dims, Ls, rng=rng), masks[k] & odd) for _ in range(nrhs)]
          for k in range(len(masks))]
    h = G.Handle(dims, Ls, G.Action(MOBIUS.M5, MOBIUS.mf, MOBIUS.b5, MOBIUS.c5), boxes=boxes,
                 nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    bcb = torch.view_as_real(torch.from_numpy(LY.to_cb(bs, dims, boxes, 1))).cuda().contiguous()
    return U, masks, bs, h, bcb


def _A(U, mask):
    return lambda f: O.mpc_in(U, O.mpc_in(U, f, MOBIUS, mask), MOBIUS, mask, True)


@pytest.mark.parametrize("boxes,nrhs", [(None, 1),
                                        ([((1, 1, 1, 1), (3, 2, 3, 6)), ((0, 0, 0, 0), (4, 4, 2, 8))], 2)])
def test_fp64_shifts_match_oracle(boxes, nrhs):
    dims, Ls = (4, 4, 4, 8), 8
    U, masks, bs, h, bcb = _problem(dims, Ls, boxes, nrhs, 51)
    x = torch.zeros((len(SHIFTS),) + tuple(bcb.shape), dtype=torch.float64, device="cuda")
    stats, rc = h.multishift_solve(x, bcb, SHIFTS, nrhs=nrhs, tol=1e-10, inner=G.FP64)
    assert rc == 0
    for k, sig in enumerate(SHIFTS):
        got = LY.from_cb(torch.view_as_complex(x[k].cpu()).numpy(), dims, boxes, 1, Ls)
        for bi, mask in enumerate(masks):
            A = _A(U, mask)
            for r in range(nrhs):
                b = bs[bi][r]
                xs = got[bi][r]
                res = b - (A(xs) + sig * xs)
                assert O.norm(res) <= 2e-10 * O.norm(b), (k, bi, r)
                assert stats[k][bi * nrhs + r]["true_resid"] <= 2e-10
        # the oracle's multi-shift solution of the first system
        if k == 0:
            ref, _ = multishift_cg(_A(U, masks[0]), bs[0][0], SHIFTS, tol=1e-11)
            for kk in range(len(SHIFTS)):
                g = LY.from_cb(torch.view_as_complex(x[kk].cpu()).numpy(), dims, boxes, 1, Ls)[0][0]
                assert LY.rel_l2(g, ref[kk]) <= 1e-6
    # larger shifts converge no later than the smallest
    its = [stats[k][0]["iters"] for k in range(len(SHIFTS))]
    assert its[3] <= its[1]


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_fp32_operator_with_defect_correction(tol):
    """FP32 operator: to 1e-6 by the multi-shift iteration alone, to 1e-10
    with FP64 defect correction per shift."""
    dims, Ls = (4, 4, 4, 8), 8
    U, masks, bs, h, bcb = _problem(dims, Ls, None, 1, 52)
    x = torch.zeros((len(SHIFTS),) + tuple(bcb.shape), dtype=torch.float64, device="cuda")
    stats, rc = h.multishift_solve(x, bcb, SHIFTS, tol=tol, inner=G.FP32)
    assert rc == 0
    A = _A(U, masks[0])
    for k, sig in enumerate(SHIFTS):
        xs = LY.from_cb(torch.view_as_complex(x[k].cpu()).numpy(), dims, None, 1, Ls)[0][0]
        b = bs[0][0]
        assert O.norm(b - (A(xs) + sig * xs)) <= 2 * tol * O.norm(b)
        if tol < 1e-6:
            assert stats[k][0]["reliable_updates"] >= 1


def test_bad_arguments():
    dims, Ls = (4, 4, 4, 4), 4
    U, masks, bs, h, bcb = _problem(dims, Ls, None, 1, 53)
    x = torch.zeros((2,) + tuple(bcb.shape), dtype=torch.float64, device="cuda")
    with pytest.raises(G.DWFError):
        h.multishift_solve(x, bcb, [0.1, -1.0])
    with pytest.raises(G.DWFError):
        h.multishift_solve(x, bcb, [0.1, 0.2], inner=G.BF16)


@pytest.mark.parametrize("boxes,nrhs,inner", [(None, 1, "fp64"),
                                              ([((1, 1, 1, 1), (3, 2, 3, 6)), ((0, 0, 0, 0), (4, 4, 2, 8))], 2,
                                               "fp32")])
def test_rational_apply_matches_oracle(boxes, nrhs, inner):
    """a0 b + sum_i r_i (A + s_i)^-1 b on the GPU against the oracle's
    multi-shift partial fractions (each box with its own Dirichlet operator)."""
    from oracle.multishift import rational_apply
    dims, Ls = (4, 4, 4, 8), 8
    U, masks, bs, h, bcb = _problem(dims, Ls, boxes, nrhs, 55)
    a0, shifts, res = 0.3, [0.05, 0.4, 3.0], [0.7, -0.2, 1.5]
    out = torch.zeros_like(bcb)
    stats, rc = h.rational_apply(out, bcb, a0, shifts, res, nrhs=nrhs, tol=1e-11,
                                 inner=G.FP64 if inner == "fp64" else G.FP32)
    assert rc == 0
    got = LY.from_cb(torch.view_as_complex(out.cpu()).numpy(), dims, boxes, 1, Ls)
    for bi, mask in enumerate(masks):
        for r in range(nrhs):
            want = rational_apply(_A(U, mask), bs[bi][r], a0, shifts, res, tol=1e-12)
            assert LY.rel_l2(got[bi][r], want) <= 1e-9, (bi, r)


def test_zolotarev_inverse_square_root():
    """(M_pc^+ M_pc)^(-1/2) b by dwf_rational_apply with the library's
    Zolotarev coefficients, against the dense eigendecomposition, to within
    the approximation's delta."""
    from oracle import dense as Dn
    dims, Ls = (2, 2, 2, 4), 4
    rng = np.random.default_rng(57)
    U = inputs.gauge_field(dims, "haar", rng=rng)
    odd = O.parity_field(dims) == 1
    shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)

    def A(f):
        f = O.restrict(f, odd)
        return O.mpc(U, O.mpc(U, f, MOBIUS), MOBIUS, True)

    dofs = Dn.site_mask_to_dofs(odd, Ls * 12)
    Ad = Dn.dense_matrix(A, shape)[np.ix_(dofs, dofs)]
    w, V = np.linalg.eigh(Ad)
    shifts, res, delta = G.zolotarev_inv_sqrt(16, 0.9 * w[0], 1.1 * w[-1])
    assert delta < 1e-6
    b = O.restrict(inputs.gaussian_source(dims, Ls, rng=rng), odd)
    h = G.Handle(dims, Ls, G.Action(MOBIUS.M5, MOBIUS.mf, MOBIUS.b5, MOBIUS.c5))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    bcb = torch.view_as_real(torch.from_numpy(LY.to_cb([[b]], dims, None, 1))).cuda().contiguous()
    out = torch.zeros_like(bcb)
    stats, rc = h.rational_apply(out, bcb, 0.0, shifts, res, tol=1e-12)
    assert rc == 0
    got = LY.from_cb(torch.view_as_complex(out.cpu()).numpy(), dims, None, 1, Ls)[0][0]
    want = V @ ((w ** -0.5) * (V.conj().T @ b.reshape(-1)[dofs]))
    assert np.linalg.norm(got.reshape(-1)[dofs] - want) <= (2 * delta + 1e-9) * np.linalg.norm(want)
