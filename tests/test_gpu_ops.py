"""GPU parity of every operator entry point against the FP64 oracle.

Element-by-element relative-L2 comparisons at sizes the oracle finishes in
seconds, spanning several tiles with a ragged last tile, both parities,
adjoints, Shamir and Moebius, several right-hand sides and Dirichlet boxes
with odd extents and periodic wrap.  Tolerances (relative L2 per operator
application): FP64 1e-12, FP32 1e-6, BF16 1e-2.
"""

import zlib

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

SHAMIR = O.DWFParams(M5=1.8, mf=0.01)
MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)
TOL = {G.FP64: 1e-12, G.FP32: 1e-6, G.BF16: 1e-2}
# M_pc chains two hops and M_ee^-1: allow the FP32 rounding of three passes
TOL_MPC = {G.FP64: 1e-12, G.FP32: 2e-6, G.BF16: 1.5e-2}

CASES = {
    # name: dims, Ls, params, boxes, nrhs, gauge kind
    "shamir_haar_4444x8": ((4, 4, 4, 4), 8, SHAMIR, None, 1, "haar"),
    "mobius_ragged_6622x6": ((6, 6, 2, 2), 6, MOBIUS, None, 1, "haar"),
    "mobius_exp_4468x12_nrhs3": ((4, 4, 6, 8), 12, MOBIUS, None, 3, "exp"),
    "mobius_boxes_odd_wrap": ((6, 4, 6, 8), 8, MOBIUS,
                              [((1, 1, 1, 1), (3, 2, 5, 3)), ((5, 0, 3, 7), (4, 4, 4, 4)),
                               ((0, 0, 0, 0), (6, 4, 6, 1))], 2, "haar"),
}


def _setup(name):
    dims, Ls, prm, boxes, nrhs, kind = CASES[name]
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    U = inputs.gauge_field(dims, kind, eps=0.3, rng=rng)
    nb = len(boxes) if boxes else 1
    masks = [O.box_mask(dims, b) for b in boxes] if boxes else [np.ones(dims[::-1], bool)]
    psi = [[O.restrict(inputs.gaussian_source(dims, Ls, rng=rng), masks[b]) for _ in range(nrhs)]
           for b in range(nb)]
    h = G.Handle(dims, Ls, G.Action(prm.M5, prm.mf, prm.b5, prm.c5), boxes=boxes, nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    return dims, Ls, prm, boxes, nrhs, U, masks, psi, h


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    return _setup(request.param)


def _gpu(arr, prec):
    t = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(arr)))
    return t.to(device="cuda", dtype=G._DTYPE[prec]).contiguous()


def _host(t):
    return torch.view_as_complex(t.double().cpu().contiguous()).numpy()


PRECS = [G.FP64, G.FP32, G.BF16]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_dslash_eo(case, prec, dagger, out_parity):
    dims, Ls, prm, boxes, nrhs, U, masks, psi, h = case
    src = LY.to_cb(psi, dims, boxes, 1 - out_parity)
    want_f = [[O.eo_block_in(U, f, prm, masks[b], out_parity, dagger) for f in psi[b]]
              for b in range(len(psi))]
    want = LY.to_cb(want_f, dims, boxes, out_parity)
    out = h.empty_cb(out_parity, nrhs, prec)
    h.dslash_eo(out, _gpu(src, prec), out_parity, dagger, prec, nrhs)
    torch.cuda.synchronize()
    assert LY.rel_l2(_host(out), want) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("parity", [0, 1])
def test_mooee_and_inverse(case, prec, dagger, parity):
    dims, Ls, prm, boxes, nrhs, U, masks, psi, h = case
    src = LY.to_cb(psi, dims, boxes, parity)
    for fn, ofn in ((h.mooee, O.mooee), (h.mooee_inv, O.mooee_inv)):
        want = LY.to_cb([[ofn(f, prm, dagger) for f in psi[b]] for b in range(len(psi))],
                        dims, boxes, parity)
        out = h.empty_cb(parity, nrhs, prec)
        fn(out, _gpu(src, prec), parity, dagger, prec, nrhs)
        torch.cuda.synchronize()
        assert LY.rel_l2(_host(out), want) <= TOL[prec], fn.__name__


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [False, True])
def test_mpc(case, prec, dagger):
    dims, Ls, prm, boxes, nrhs, U, masks, psi, h = case
    po = [[O.parity_part(f, 1) for f in row] for row in psi]
    src = LY.to_cb(po, dims, boxes, 1)
    want = LY.to_cb([[O.mpc_in(U, f, prm, masks[b], dagger) for f in po[b]]
                     for b in range(len(po))], dims, boxes, 1)
    out = h.empty_cb(1, nrhs, prec)
    h.mpc(out, _gpu(src, prec), dagger, prec, nrhs)
    torch.cuda.synchronize()
    assert LY.rel_l2(_host(out), want) <= TOL_MPC[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [False, True])
def test_full_operator(case, prec, dagger):
    dims, Ls, prm, boxes, nrhs, U, masks, psi, h = case
    src = LY.to_full(psi, dims, boxes)
    if boxes:
        want_f = [[O.dirichlet_D(U, f, prm, [boxes[b]], dagger) for f in psi[b]]
                  for b in range(len(psi))]
    else:
        want_f = [[O.apply_D(U, f, prm, dagger) for f in psi[0]]]
    want = LY.to_full(want_f, dims, boxes)
    out = h.empty_full(nrhs, prec)
    if boxes:
        h.dirichlet_block(out, _gpu(src, prec), dagger, prec, nrhs)
    else:
        h.apply_d(out, _gpu(src, prec), dagger, prec, nrhs)
    torch.cuda.synchronize()
    assert LY.rel_l2(_host(out), want) <= TOL_MPC[prec]


def test_dirichlet_block_rejects_whole_lattice():
    h = G.Handle((4, 4, 4, 4), 4, G.Action(), nrhs_max=1)
    U = inputs.gauge_field((4, 4, 4, 4), "haar", seed=1)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    a, b = h.empty_full(), h.empty_full()
    with pytest.raises(G.DWFError):
        h.dirichlet_block(a, b)


@pytest.mark.parametrize("prec", PRECS)
def test_pack_unpack_layout(case, prec):
    """The library's layout kernels agree with the test-side layout rules."""
    dims, Ls, prm, boxes, nrhs, U, masks, psi, h = case
    canon = LY.canonical(psi, boxes, dims)
    full = h.pack(torch.from_numpy(canon).cuda(), nrhs, prec)
    torch.cuda.synchronize()
    assert LY.rel_l2(_host(full), LY.to_full(psi, dims, boxes)) <= TOL[prec]
    back = h.unpack(full, nrhs, prec)
    torch.cuda.synchronize()
    got = back.cpu().numpy().view(np.complex128).reshape(-1)
    assert LY.rel_l2(got, canon) <= TOL[prec]


@pytest.mark.parametrize("tile,vl,chunk,order", [(4, 1, 1, None), (8, 2, 1, (2, 2)), (48, 1, 1, None),
                                                  (64, 2, 1, (1, 3)), (4, 2, 8, (2, 2)), (8, 1, 3, None)])
def test_tile_and_lane_variants(tile, vl, chunk, order):
    """Every (tile size, lanes per thread, tile order, epilogue fusion) choice
    the autotuner can make gives the same operator: hop-based dslash_eo and
    M_pc (both adjoints) in FP32 and FP64, with the site-local factor of M_pc
    in the hop epilogue (8 lanes x 2 rhs: the site groups divide a warp) and
    without; tiles in lexicographic order or blocked in (z, t) inside each
    (odd-sized, wrapping) box."""
    dims, Ls, prm, boxes, nrhs, U, masks, psi, h = _setup("mobius_boxes_odd_wrap")
    h.set_tile(nrhs, tile, vl)
    h.set_hop_chunk(nrhs, chunk)
    if order:
        h.set_tile_order(1, *order)
    po = [[O.parity_part(f, 1) for f in row] for row in psi]
    src = LY.to_cb(po, dims, boxes, 1)
    for dagger in (False, True):
        want = LY.to_cb([[O.mpc_in(U, f, prm, masks[b], dagger) for f in po[b]] for b in range(len(po))],
                        dims, boxes, 1)
        for fuse in (False, True):
            h.set_fusion(nrhs, fuse)
            for prec in (G.FP64, G.FP32, G.BF16):
                out = h.empty_cb(1, nrhs, prec)
                h.mpc(out, _gpu(src, prec), dagger, prec, nrhs)
                torch.cuda.synchronize()
                assert LY.rel_l2(_host(out), want) <= TOL_MPC[prec], (prec, dagger, fuse)
    h.set_fusion(nrhs, False)
    want0 = LY.to_cb([[O.eo_block_in(U, f, prm, masks[b], 0) for f in psi[b]]
                      for b in range(len(psi))], dims, boxes, 0)
    out = h.empty_cb(0, nrhs, G.FP32)
    h.dslash_eo(out, _gpu(LY.to_cb(psi, dims, boxes, 1), G.FP32), 0, False, G.FP32, nrhs)
    torch.cuda.synchronize()
    assert LY.rel_l2(_host(out), want0) <= TOL[G.FP32]


def test_autotuned_solve_still_exact():
    """After dwf_autotune (which may pick the one-lane FP32 hop), a mixed
    solve still reaches 1e-10 by the oracle."""
    dims, Ls = (4, 4, 4, 8), 8
    rng = np.random.default_rng(31)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    b = inputs.gaussian_source(dims, Ls, rng=rng)
    h = G.Handle(dims, Ls, G.Action(MOBIUS.M5, MOBIUS.mf, MOBIUS.b5, MOBIUS.c5))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    h.autotune(1, G.FP32)
    bf = torch.view_as_real(torch.from_numpy(LY.to_full([[b]], dims, None))).cuda().contiguous()
    x = torch.zeros_like(bf)
    st, rc = h.cgne_solve(x, bf, tol=1e-10, inner=G.FP32)
    xf = LY.from_full(torch.view_as_complex(x.cpu()).numpy(), dims, None, Ls)[0][0]
    assert O.true_residual(U, xf, b, MOBIUS) <= 1e-10
    # tiles reordered in place under the solver's captured graphs: same solve
    h.set_tile_order(1, 2, 2)
    x.zero_()
    st2, rc = h.cgne_solve(x, bf, tol=1e-10, inner=G.FP32)
    xf = LY.from_full(torch.view_as_complex(x.cpu()).numpy(), dims, None, Ls)[0][0]
    assert O.true_residual(U, xf, b, MOBIUS) <= 1e-10
    assert abs(st2[0]["iters"] - st[0]["iters"]) <= 2


@pytest.mark.parametrize("dagger", [False, True])
def test_tensor_core_hop(case, dagger):
    """The BF16 operator on the tensor cores (dwf_set_hop_kernel = 1): every
    hop-based entry point against the FP64 oracle at the BF16 tolerances,
    and within the BF16 tolerance of the SIMT BF16 kernel."""
    dims, Ls, prm, boxes, nrhs, U, masks, psi, h = case
    po = [[O.parity_part(f, 1) for f in row] for row in psi]
    src1 = LY.to_cb(po, dims, boxes, 1)
    want_mpc = LY.to_cb([[O.mpc_in(U, f, prm, masks[b], dagger) for f in po[b]]
                         for b in range(len(po))], dims, boxes, 1)
    want_eo = LY.to_cb([[O.eo_block_in(U, f, prm, masks[b], 0, dagger) for f in psi[b]]
                        for b in range(len(psi))], dims, boxes, 0)
    src_eo = LY.to_cb(psi, dims, boxes, 1)
    got = {}
    try:
        for kern in (1, 0):
            h.set_hop_kernel(nrhs, kern)
            out = h.empty_cb(1, nrhs, G.BF16)
            h.mpc(out, _gpu(src1, G.BF16), dagger, G.BF16, nrhs)
            eo = h.empty_cb(0, nrhs, G.BF16)
            h.dslash_eo(eo, _gpu(src_eo, G.BF16), 0, dagger, G.BF16, nrhs)
            torch.cuda.synchronize()
            got[kern] = (_host(out), _host(eo))
    finally:
        h.set_hop_kernel(nrhs, 0)
    assert LY.rel_l2(got[1][0], want_mpc) <= TOL_MPC[G.BF16]
    assert LY.rel_l2(got[1][1], want_eo) <= TOL[G.BF16]
    assert LY.rel_l2(got[1][0], got[0][0]) <= TOL_MPC[G.BF16]


def test_autotune_cache_round_trip(tmp_path):
    """dwf_autotune_save writes the tuned choice; a fresh handle of the same
    domain picks it up with dwf_autotune_load (and gives the same operator);
    another nrhs or domain finds nothing."""
    dims, Ls = (4, 4, 4, 8), 8
    U = inputs.gauge_field(dims, "exp", eps=0.3, seed=73)
    act = G.Action(1.8, 0.01, 1.5, 0.5)
    h = G.Handle(dims, Ls, act, nrhs_max=2)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    h.autotune(1, G.FP32)
    h.set_tile_order(1, 2, 4)
    path = str(tmp_path / "tune.txt")
    h.autotune_save(path)
    h2 = G.Handle(dims, Ls, act, nrhs_max=2)
    h2.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    assert h2.autotune_load(path, 1, G.FP32)
    assert h2.tuning(1) == h.tuning(1)
    assert h2.tile_order() == (1, 2, 4)
    # a line without the tile-order fields loads as lexicographic
    old = str(tmp_path / "tune5.txt")
    with open(path) as f, open(old, "w") as g:
        for line in f:
            g.write(" ".join(line.split()[:6]) + "\n")
    h4 = G.Handle(dims, Ls, act, nrhs_max=2)
    h4.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    assert h4.autotune_load(old, 1, G.FP32)
    assert h4.tuning(1) == h.tuning(1) and h4.tile_order()[0] == 0
    assert not h2.autotune_load(path, 2, G.FP32)
    assert not h2.autotune_load(path, 1, G.BF16)
    h3 = G.Handle((4, 4, 4, 4), Ls, act)
    h3.set_gauge(torch.from_numpy(inputs.gauge_field((4, 4, 4, 4), "haar", seed=1).reshape(-1)).cuda())
    assert not h3.autotune_load(path, 1, G.FP32)
    x = torch.randn(h.cb_shape(1), device="cuda")
    y1, y2 = h.empty_cb(1, 1, G.FP32), h2.empty_cb(1, 1, G.FP32)
    h.mpc(y1, x, prec=G.FP32)
    h2.mpc(y2, x, prec=G.FP32)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
