"""GPU parity at the sizes and kernel configurations the benchmark times.

The small-lattice tests (test_gpu_ops.py) give each CTA of the persistent hop
at most one tile; here every CTA walks many tiles with the double buffer
cycling, in the compile-time lane counts the benchmark runs:

* Moebius 16^4 x Ls=12 (N5 = 12): dslash_eo and M_pc in FP64 / FP32 / BF16,
  both adjoints, tiles of 16 sites with one lane per thread (chunk 1) and two
  lanes per thread (chunk 8), compared element by element over the whole
  checkerboard with the oracle's lattice operators;
* Moebius 32^4 x Ls=16 (N5 = 16), FP32 and BF16: tiles of 64 sites, two lanes
  per thread, chunks of 8 tiles (the bare-hop configuration of the benchmark)
  and the autotuned one, at sampled sites against the oracle's per-site
  operators (eo_block_site, mpc_in_site);
* Moebius 24^4 x Ls=16, six uneven Dirichlet boxes 8^4 .. 16^4 with 16
  right-hand sides each (N5 = 256, the largest lane count), FP32 and BF16,
  sampled sites; and one mixed-precision solve of all 96 systems, two of
  which get their true residual |b - D_Omega x| / |b| recomputed by the
  oracle.

Sampled comparisons take the relative L2 error over all sampled outputs
(tolerances as in test_gpu_ops.py); samples include the first and last site
of every box and parity (the ragged tiles) and random sites in between.
"""

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

TOL = {G.FP64: 1e-12, G.FP32: 1e-6, G.BF16: 1e-2}
TOL_MPC = {G.FP64: 1e-12, G.FP32: 2e-6, G.BF16: 1.5e-2}
MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)
MOBIUS_LIGHT = O.DWFParams(M5=1.8, mf=0.005, b5=1.5, c5=0.5)
BOXES6 = [((0, 0, 0, 0), (8, 8, 8, 8)), ((0, 0, 0, 0), (8, 8, 12, 12)),
          ((0, 0, 0, 0), (12, 12, 12, 12)), ((0, 0, 0, 0), (12, 12, 16, 16)),
          ((0, 0, 0, 0), (16, 16, 16, 12)), ((0, 0, 0, 0), (16, 16, 16, 16))]


def _action(prm):
    return G.Action(prm.M5, prm.mf, prm.b5, prm.c5)


def _randn(shape, seed, dtype=torch.float64):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randn(shape, dtype=dtype, device="cuda", generator=g)


def _host(t):
    return torch.view_as_complex(t.double().cpu().contiguous()).numpy()


def _rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


# ------------------------------------------------ site bookkeeping (tests)
class Domain:
    """Sites of a handle's domain (the layout rules of include/dwf.h, restated
    by tests/layout.py): per parity the list of (box, global site) and the
    index of each."""

    def __init__(self, dims, boxes):
        self.dims = dims
        self.boxes = boxes or [LY.whole_lattice_box(dims)]
        self.sites = LY.domain_sites(dims, boxes)
        self.index = [{(b, x): i for i, (b, _, x) in enumerate(self.sites[p])} for p in range(2)]

    def inside(self, b):
        org, ext = self.boxes[b]
        L = self.dims
        return lambda s: all((s[m] - org[m]) % L[m] < ext[m] for m in range(4))

    def box_ranges(self, p):
        """[box] -> (first, last) index of its parity-p sites."""
        out = {}
        for i, (b, _, _) in enumerate(self.sites[p]):
            lo, hi = out.get(b, (i, i))
            out[b] = (min(lo, i), max(hi, i))
        return out


def _sample(dom, p, n, seed):
    """n sampled parity-p indices: first and last site of each box, the rest
    random."""
    rng = np.random.default_rng(seed)
    picks = set()
    for lo, hi in dom.box_ranges(p).values():
        picks.update((lo, hi))
    total = len(dom.sites[p])
    picks.update(rng.choice(total, size=max(n - len(picks), 0), replace=False).tolist())
    return sorted(picks)


def _neighbours(x, L, hops):
    """Global sites within `hops` hops of x (including x)."""
    seen = {tuple(x)}
    front = [tuple(x)]
    for _ in range(hops):
        nxt = []
        for s in front:
            for mu in range(4):
                for d in (1, -1):
                    y = list(s)
                    y[mu] = (y[mu] + d) % L[mu]
                    y = tuple(y)
                    if y not in seen:
                        seen.add(y)
                        nxt.append(y)
        front = nxt
    return seen


class Rows:
    """Oracle-side accessor of one right-hand side of a gathered cb field:
    psi[t, z, y, x] -> (Ls, 4, 3) for the gathered sites of one box, zero for
    every other site."""

    def __init__(self, dims, Ls, rows, rhs):
        self.shape = (dims[3], dims[2], dims[1], dims[0], Ls, 4, 3)
        self._rows = rows
        self._rhs = rhs
        self._zero = np.zeros((Ls, 4, 3), dtype=np.complex128)

    def __getitem__(self, key):
        t, z, y, x = key
        r = self._rows.get((x, y, z, t))
        return self._zero if r is None else r[self._rhs]


def _gather(field, dom, p, box, sites, nrhs, Ls):
    """Rows of the device cb field of parity p at the given global sites of
    one box (those that belong to it and to parity p), as a dict
    site -> (nrhs, Ls, 4, 3) complex128."""
    keys = [s for s in sites if (box, s) in dom.index[p]]
    if not keys:
        return {}
    idx = torch.tensor([dom.index[p][(box, s)] for s in keys], device=field.device)
    rows = _host(field.index_select(0, idx))          # (n, 12, nrhs, Ls)
    rows = rows.reshape(len(keys), 4, 3, nrhs, Ls).transpose(0, 3, 4, 1, 2)
    return dict(zip(keys, rows))


def _sampled_check(h, dom, U, prm, Ls, nrhs, fin, precs, cfgs, n_sample, seed, ops):
    """For each op ("eo": dslash_eo into even, "mpc": M_pc), dagger, kernel
    configuration and precision: run the device operator on the input `fin`
    (FP64 parity-1 cb field, cast to the precision), gather the sampled output
    rows and compare with the oracle's per-site evaluation (one right-hand
    side per sampled site, cycling over them)."""
    dims = dom.dims
    results = []
    for op in ops:
        p_out = 0 if op == "eo" else 1
        samples = _sample(dom, p_out, n_sample, seed + p_out)
        # what the oracle needs: per sampled site, its box, rhs and stencil
        hops = 1 if op == "eo" else 2
        need = {}
        plan = []
        for k, i in enumerate(samples):
            b, _, x = dom.sites[p_out][i]
            r = k % nrhs
            plan.append((i, b, x, r))
            need.setdefault(b, set()).update(_neighbours(x, dims, hops))
        rows = {b: _gather(fin, dom, 1, b, sorted(s), nrhs, Ls) for b, s in need.items()}
        for dagger in (False, True):
            want = []
            for i, b, x, r in plan:
                # the accessor is zero off the box's gathered sites, so the
                # hops that leave the box are cut
                acc = Rows(dims, Ls, rows[b], r)
                if op == "eo":
                    w = O.eo_block_site(U, acc, prm, x, dagger)
                else:
                    w = O.mpc_in_site(U, acc, prm, x, dom.inside(b), dagger)
                want.append(w)
            want = np.stack(want)
            idx = torch.tensor([i for i, _, _, _ in plan], device="cuda")
            for cfg in cfgs:
                if cfg is None:
                    h.autotune(nrhs, G.FP32)
                else:
                    T, vl, chunk, fuse = cfg
                    h.set_tile(nrhs, T, vl)
                    h.set_hop_chunk(nrhs, chunk)
                    h.set_fusion(nrhs, fuse)
                for prec in precs:
                    src = fin.to(G._DTYPE[prec])
                    out = h.empty_cb(p_out, nrhs, prec)
                    if op == "eo":
                        h.dslash_eo(out, src, 0, dagger, prec, nrhs)
                    else:
                        h.mpc(out, src, dagger, prec, nrhs)
                    torch.cuda.synchronize()
                    got = _host(out.index_select(0, idx))        # (n, 12, nrhs, Ls)
                    got = got.reshape(len(plan), 4, 3, nrhs, Ls).transpose(0, 3, 4, 1, 2)
                    got = np.stack([got[k, r] for k, (_, _, _, r) in enumerate(plan)])
                    tol = (TOL if op == "eo" else TOL_MPC)[prec]
                    err = _rel(got, want)
                    results.append((op, dagger, cfg, prec, err))
                    assert err <= tol, (op, dagger, cfg, prec, err)
                    del src, out
    return results


# ------------------------------------------------------- 16^4 x 12, whole
@pytest.fixture(scope="module")
def lat16():
    dims, Ls = (16, 16, 16, 16), 12
    U = inputs.gauge_field(dims, "exp", eps=0.3, seed=1001)
    h = G.Handle(dims, Ls, _action(MOBIUS))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    return dims, Ls, U, h


@pytest.mark.parametrize("cfg", [(16, 1, 1), (16, 2, 8)], ids=["t16_vl1", "t16_vl2_chunk8"])
def test_16x12_whole_field(lat16, cfg):
    """dslash_eo (both output parities) and M_pc, both adjoints, FP64 / FP32 /
    BF16 over the whole 16^4 x 12 checkerboard against the oracle's lattice
    operators (O.eo_block, O.mpc)."""
    dims, Ls, U, h = lat16
    h.set_tile(1, cfg[0], cfg[1])
    h.set_hop_chunk(1, cfg[2])
    h.set_fusion(1, False)
    for p_out in (0, 1):
        fin = _randn(h.cb_shape(1 - p_out), 17 + p_out)
        psi = LY.from_cb(_host(fin), dims, None, 1 - p_out, Ls)[0][0]
        for dagger in (False, True):
            want = LY.to_cb([[O.eo_block(U, psi, MOBIUS, p_out, dagger)]], dims, None, p_out)
            for prec in (G.FP64, G.FP32, G.BF16):
                out = h.empty_cb(p_out, 1, prec)
                h.dslash_eo(out, fin.to(G._DTYPE[prec]), p_out, dagger, prec, 1)
                torch.cuda.synchronize()
                assert LY.rel_l2(_host(out), want) <= TOL[prec], ("eo", p_out, dagger, prec)
    fin = _randn(h.cb_shape(1), 29)
    psi = LY.from_cb(_host(fin), dims, None, 1, Ls)[0][0]
    for dagger in (False, True):
        want = LY.to_cb([[O.mpc(U, psi, MOBIUS, dagger)]], dims, None, 1)
        for prec in (G.FP64, G.FP32, G.BF16):
            out = h.empty_cb(1, 1, prec)
            h.mpc(out, fin.to(G._DTYPE[prec]), dagger, prec, 1)
            torch.cuda.synchronize()
            assert LY.rel_l2(_host(out), want) <= TOL_MPC[prec], ("mpc", dagger, prec)


# ----------------------------------------------------- 32^4 x 16, sampled
def test_32x16_sampled():
    """The paper's per-GPU volume: 32^4 x Ls=16 FP32 and BF16 dslash_eo and
    M_pc at sampled sites, in the bench's bare-hop configuration (64-site
    tiles, two lanes per thread, chunks of 8), with the site-local factor of
    M_pc in the hop epilogue (32-site tiles), and the autotuned one."""
    dims, Ls = (32, 32, 32, 32), 16
    U = inputs.gauge_field(dims, "haar", seed=1003)
    h = G.Handle(dims, Ls, _action(MOBIUS_LIGHT))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    dom = Domain(dims, None)
    fin = _randn(h.cb_shape(1), 31)
    res = _sampled_check(h, dom, U, MOBIUS_LIGHT, Ls, 1, fin, (G.FP32, G.BF16),
                         [(64, 2, 8, False), (32, 2, 1, True), None], 256, 5, ("eo", "mpc"))
    assert len(res) == 2 * 2 * 3 * 2


# ------------------------------------------- 24^4 x 16, six boxes x 16 rhs
@pytest.fixture(scope="module")
def six_boxes():
    dims, Ls, nrhs = (24, 24, 24, 24), 16, 16
    U = inputs.gauge_field(dims, "haar", seed=1002)
    h = G.Handle(dims, Ls, _action(MOBIUS), boxes=BOXES6, nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    return dims, Ls, nrhs, U, h, Domain(dims, BOXES6)


def test_six_boxes_16rhs_sampled(six_boxes):
    """Six uneven Dirichlet boxes x 16 right-hand sides (N5 = 256 lanes):
    dslash_eo and M_pc of D_Omega in FP32 and BF16 at sampled sites, two
    kernel configurations (8-site tiles with two lanes per thread; 16-site
    tiles with one lane per thread and chunks of 8)."""
    dims, Ls, nrhs, U, h, dom = six_boxes
    fin = _randn(h.cb_shape(1, nrhs), 41)
    res = _sampled_check(h, dom, U, MOBIUS, Ls, nrhs, fin, (G.FP32, G.BF16),
                         [(8, 2, 1, False), (16, 1, 8, False)], 192, 9, ("eo", "mpc"))
    assert len(res) == 2 * 2 * 2 * 2


def _box_field(full, h, dom, box, rhs, Ls):
    """One box and right-hand side of a device full FP64 field as an oracle
    array on the box's own lattice padded by one site in every direction (so
    the hops that leave the box are cut, not wrapped)."""
    org, ext = dom.boxes[box]
    pad = tuple(e + 2 for e in ext)
    arr = np.zeros((pad[3], pad[2], pad[1], pad[0], Ls, 4, 3), dtype=np.complex128)
    n0 = h.nsite[0]
    for p in range(2):
        off, cnt = h.box_sites(box, p)
        rows = _host(full[(n0 if p else 0) + off:(n0 if p else 0) + off + cnt, :, rhs:rhs + 1])
        rows = rows.reshape(cnt, 4, 3, Ls).transpose(0, 3, 1, 2)
        for k, (b, l, x) in enumerate(s for s in dom.sites[p] if s[0] == box):
            loc = [(x[m] - org[m]) % dom.dims[m] for m in range(4)]
            arr[loc[3], loc[2], loc[1], loc[0]] = rows[k]
    return arr, pad


def test_six_boxes_16rhs_mixed_solve(six_boxes):
    """All 96 systems (six boxes x 16 right-hand sides) in one mixed-precision
    CGNE (FP32 operator, FP64 reliable updates) to 1e-10; for two systems the
    oracle recomputes |b - D_Omega x| / |b| on the box's own lattice with the
    crossing links cut."""
    dims, Ls, nrhs, U, h, dom = six_boxes
    h.autotune(nrhs, G.FP32)
    b = _randn(h.full_shape(nrhs), 53)
    x = torch.zeros_like(b)
    st, rc = h.cgne_solve(x, b, nrhs=nrhs, tol=1e-10, inner=G.FP32)
    assert rc == 0 and len(st) == 6 * nrhs
    assert max(s["true_resid"] for s in st) <= 1e-10
    for box, rhs in ((0, 3), (1, 11)):
        xb, pad = _box_field(x, h, dom, box, rhs, Ls)
        bb, _ = _box_field(b, h, dom, box, rhs, Ls)
        Ub = np.zeros((pad[3], pad[2], pad[1], pad[0], 4, 3, 3), dtype=np.complex128)
        org, ext = dom.boxes[box]
        t = (np.arange(pad[3]) + org[3]) % dims[3]
        z = (np.arange(pad[2]) + org[2]) % dims[2]
        y = (np.arange(pad[1]) + org[1]) % dims[1]
        xx = (np.arange(pad[0]) + org[0]) % dims[0]
        Ub[:] = U[t[:, None, None, None], z[None, :, None, None], y[None, None, :, None],
                  xx[None, None, None, :]]
        inner_box = ((0, 0, 0, 0), tuple(ext))
        r = bb - O.dirichlet_D(Ub, xb, MOBIUS, [inner_box])
        assert np.linalg.norm(r) / np.linalg.norm(bb) <= 1e-10, (box, rhs)
        assert st[box * nrhs + rhs]["true_resid"] <= 1e-10
