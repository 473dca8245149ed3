"""GPU parity of the learned preconditioner and of flexible GCR.

The network's forward pass and its analytic gradient are compared with the
FP64 oracle on the same weights (drawn BF16-representable, since the kernels
apply BF16 weights); GCR solves must reach a true residual <= 1e-10,
recomputed by the oracle; a short training run must lower the loss."""

import numpy as np
import pytest

from oracle import dwf as O
from oracle import nn as N
from paper_2203_17119_gb300 import inputs
from tests import layout as LY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

MOBIUS = O.DWFParams(M5=1.8, mf=0.01, b5=1.5, c5=0.5)


def bf16_exact(a):
    """Round float64 values to the nearest BF16 number (kept as float64)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def rand_weights(rng, C=16, scale=0.1):
    def c(shape):
        return bf16_exact(rng.standard_normal(shape) * scale) + 1j * bf16_exact(
            rng.standard_normal(shape) * scale)
    return c((11, C, 1, 4, 4)), c((11, 1, C, 4, 4))


def setup(dims, Ls, nrhs, seed, kind="haar"):
    rng = np.random.default_rng(seed)
    U = inputs.gauge_field(dims, kind, eps=0.3, rng=rng)
    h = G.Handle(dims, Ls, G.Action(MOBIUS.M5, MOBIUS.mf, MOBIUS.b5, MOBIUS.c5), nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    return rng, U, h


def odd_gpu(fields, dims):
    cb = LY.to_cb([fields], dims, None, 1)
    return torch.view_as_real(torch.from_numpy(cb)).to("cuda", torch.float32).contiguous()


def odd_host(t, dims, Ls):
    arr = torch.view_as_complex(t.double().cpu().contiguous()).numpy()
    return LY.from_cb(arr, dims, None, 1, Ls)[0]


@pytest.mark.parametrize("dims,Ls,nrhs", [((4, 4, 2, 4), 6, 2), ((4, 2, 2, 4), 16, 1)])
def test_forward_matches_oracle(dims, Ls, nrhs):
    rng, U, h = setup(dims, Ls, nrhs, 11)
    W1, W2 = rand_weights(rng)
    K = G.NN()
    K.set_weights(W1, W2)
    r = [O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1) for _ in range(nrhs)]
    out = torch.empty(h.cb_shape(1, nrhs), dtype=torch.float32, device="cuda")
    K.apply(h, out, odd_gpu(r, dims), nrhs)
    torch.cuda.synchronize()
    got = odd_host(out, dims, Ls)
    for k in range(nrhs):
        want = N.apply_K(U, r[k], W1, W2)
        assert LY.rel_l2(got[k], want) <= 2e-5, k


def test_identity_network_is_identity():
    dims, Ls = (4, 4, 4, 4), 8
    rng, U, h = setup(dims, Ls, 1, 12)
    K = G.NN()
    r = [O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1)]
    x = odd_gpu(r, dims)
    out = torch.empty_like(x)
    K.apply(h, out, x, 1)
    torch.cuda.synchronize()
    assert float((out - x).abs().max()) == 0.0


@pytest.mark.parametrize("energy", [False, True, "a2"])
def test_gradient_matches_oracle(energy):
    dims, Ls, nrhs = (4, 2, 2, 4), 4, 2
    rng, U, h = setup(dims, Ls, nrhs, 13)
    W1, W2 = rand_weights(rng, scale=0.2)
    K = G.NN()
    K.set_weights(W1, W2)
    A = (lambda f: O.mpc(U, O.mpc(U, f, MOBIUS), MOBIUS, True)) if energy else None
    es = [O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1) for _ in range(nrhs)]
    if energy:
        pairs = [(A(e), e) for e in es]
    else:
        pairs = [(O.parity_part(inputs.gaussian_source(dims, Ls, rng=rng), 1), e) for e in es]
    kind = "a2" if energy == "a2" else ("energy" if energy else "error")
    loss = K.train_step(h, odd_gpu([p[0] for p in pairs], dims), odd_gpu([p[1] for p in pairs], dims),
                        nrhs, lr=0.0, loss_kind=kind)
    g1, g2 = K.last_grad(h)
    L, w1, w2 = N.loss_and_grad(U, pairs, W1, W2, A, "a2" if energy == "a2" else None)
    assert abs(loss - L) <= 1e-5 * abs(L)
    assert np.linalg.norm(g1 - w1) <= 2e-4 * np.linalg.norm(w1)
    assert np.linalg.norm(g2 - w2) <= 2e-4 * np.linalg.norm(w2)


@pytest.mark.parametrize("use_k", [False, True])
def test_gcr_solve(use_k):
    dims, Ls = (4, 4, 4, 8), 8
    rng, U, h = setup(dims, Ls, 1, 14, kind="exp")
    b = inputs.gaussian_source(dims, Ls, rng=rng)
    bf = torch.view_as_real(torch.from_numpy(LY.to_full([[b]], dims, None))).cuda().contiguous()
    K = None
    if use_k:
        W1, W2 = N.identity_weights(16)
        W1[0, 0, 0] = np.eye(4) * bf16_exact(1 / 4.3)
        K = G.NN()
        K.set_weights(W1, W2)
    x = torch.zeros_like(bf)
    stats, rc = h.gcr_solve(x, bf, K=K, tol=1e-10, max_seconds=300)
    xf = LY.from_full(torch.view_as_complex(x.cpu()).numpy(), dims, None, Ls)[0][0]
    assert stats[0]["status"] == 0 and stats[0]["true_resid"] <= 1e-10
    assert O.true_residual(U, xf, b, MOBIUS) <= 1e-10


def test_training_generalises_and_gcr_converges():
    """Pairs (r, e) from the iterates of FP64 CGNE solves; Adam on the
    energy-norm loss must lower the held-out loss of the 1/d^2-initialised
    network by >= 30% (A^2-norm loss: the residual left by one GCR step);
    GCR with the trained K must reach 1e-10 by itself (no CG fallback) on a
    held-out source, in fewer iterations than GCR without the network (or
    where GCR without it needs the fallback)."""
    from paper_2203_17119_gb300 import train as TR
    dims, Ls, nrhs = (4, 4, 4, 8), 8, 4
    rng, U, h = setup(dims, Ls, nrhs, 15, kind="exp")
    h1 = G.Handle(dims, Ls, G.Action(MOBIUS.M5, MOBIUS.mf, MOBIUS.b5, MOBIUS.c5), nrhs_max=1)
    h1.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    pairs = [TR.make_pairs(h1, torch.from_numpy(inputs.gaussian_source(dims, Ls, rng=rng).reshape(-1)).cuda(),
                           n_iterates=24, record_every=4) for _ in range(3)]
    r_tr = torch.cat([pairs[0][0], pairs[1][0]])
    e_tr = torch.cat([pairs[0][1], pairs[1][1]])
    r_ho, e_ho = pairs[2]

    def held_out(K):
        n = (r_ho.shape[0] // nrhs) * nrhs
        return np.mean([K.train_step(h, TR._batch(r_ho, range(i, i + nrhs)),
                                     TR._batch(e_ho, range(i, i + nrhs)), nrhs, lr=0.0,
                                     loss_kind="a2")
                        for i in range(0, n, nrhs)])

    d = MOBIUS.d
    before = held_out(TR.initial_network(d))
    K = TR.initial_network(d)
    TR.train(K, h, r_tr, e_tr, steps=200, batch=nrhs, lr=1e-3, seed=0, loss_kind="a2")
    after = held_out(K)
    assert after < 0.7 * before, (before, after)
    b = inputs.gaussian_source(dims, Ls, rng=rng)
    bf = torch.view_as_real(torch.from_numpy(LY.to_full([[b]], dims, None))).cuda().contiguous()
    its, fell = {}, {}
    for name, KK in (("trained", K), ("none", None)):
        x = torch.zeros_like(bf)
        st, rc = h1.gcr_solve(x, bf, K=KK, tol=1e-10, max_seconds=300)
        assert st[0]["status"] == 0 and st[0]["true_resid"] <= 1e-10
        xf = LY.from_full(torch.view_as_complex(x.cpu()).numpy(), dims, None, Ls)[0][0]
        assert O.true_residual(U, xf, b, MOBIUS) <= 1e-10
        its[name] = st[0]["iters"]
        fell[name] = st[0]["recorded"] == -1
    print("held-out A^2 loss", before, "->", after, "GCR iterations", its, "CG fallback", fell)
    assert not fell["trained"]
    assert fell["none"] or its["trained"] < its["none"], its


def test_weights_file_round_trip(tmp_path):
    """dwf_nn_save / dwf_nn_load: the weights come back exactly (in the FP32
    copy the network holds), and a file of another kind is refused."""
    rng = np.random.default_rng(71)
    W1, W2 = rand_weights(rng)
    K = G.NN()
    K.set_weights(W1, W2)
    path = str(tmp_path / "k.dwfnn")
    K.save(path)
    K2 = G.NN()
    K2.load(path)
    a1, a2 = K.get_weights()
    b1, b2 = K2.get_weights()
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    bad = tmp_path / "bad.dwfnn"
    bad.write_bytes(b"not a weight file")
    with pytest.raises(G.DWFError):
        K2.load(str(bad))
