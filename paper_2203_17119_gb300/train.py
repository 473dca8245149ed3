"""Training and evaluation of the learned preconditioner K.

Training pairs come from the solver itself: an FP64 CGNE solve records its
odd iterates x_k; with the converged x* the pair is (r_k, e_k) with
e_k = x* - x_k and r_k = M_pc^+ M_pc e_k (the residual of the normal
equations that CGNE iterates on and that flexible GCR is preconditioned
for), both divided by |e_k|.  The network is
then fitted with Adam on the energy-norm error mean <d, A d> / <e, r>,
d = K r - e, A = M_pc^+ M_pc (or on |K r - e|^2 / |e|^2), batches of pairs laid out
as right-hand-side lanes of one field.  All arithmetic runs in the library
(``dwf_cgne_solve``, ``dwf_mpc``, ``dwf_nn_train_step``); this module only
moves tensors and loops.

    python -m paper_2203_17119_gb300.train --train-dims 16 16 16 16 --train-Ls 12 \\
        --sources 64 --iterates 64 --out K.dwfnn --eval-dims 24 24 24 24 --eval-Ls 16
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from paper_2203_17119_gb300 import dwf as G
from paper_2203_17119_gb300 import inputs


def make_pairs(h, b_canon, n_iterates=64, record_every=4, tol=1e-10):
    """Pairs from one FP64 solve of D x = b on a whole-lattice handle with
    nrhs = 1.  Returns (r, e): FP32 odd cb fields, shape (n, *cb_shape(1))."""
    b = h.pack(b_canon)
    x = torch.zeros_like(b)
    rec = torch.empty((n_iterates,) + h.cb_shape(1), dtype=torch.float64, device=b.device)
    st, _ = h.cgne_solve(x, b, tol=tol, inner=G.FP64, record=rec, record_every=record_every,
                         check_every=min(record_every, 8))
    n = st[0]["recorded"]
    xs = x[h.nsite[0]:].contiguous()
    r_out, e_out = [], []
    for k in range(n):
        r = torch.empty(h.cb_shape(1), dtype=torch.float32, device=b.device)
        e = torch.empty_like(r)
        if h.make_pair(r, e, xs, rec[k]) == 0.0:
            continue
        r_out.append(r)
        e_out.append(e)
    return torch.stack(r_out), torch.stack(e_out)


def _batch(fields, idx):
    """Stack single-rhs cb fields (n, site, 12, 1, Ls, 2) into lanes."""
    return torch.cat([fields[i] for i in idx], dim=2).contiguous()


def train(K, h, r, e, steps=100, batch=4, lr=1e-3, seed=0, energy=True, loss_kind=None):
    """Adam steps on random minibatches of the pairs (r, e) (energy-norm loss
    by default, see NN.train_step); returns the losses."""
    g = np.random.default_rng(seed)
    n = r.shape[0]
    losses = []
    for _ in range(steps):
        idx = g.choice(n, size=batch, replace=n < batch)
        losses.append(K.train_step(h, _batch(r, idx), _batch(e, idx), batch, lr=lr, energy=energy,
                                   loss_kind=loss_kind))
    return losses


def initial_network(d):
    """K = 1/d^2 on the identity transport: the scale of the inverse of the
    diagonal of M_pc^+ M_pc (M_oo = d + e S5, |e| << d), plus a small
    symmetry-breaking start for the other channels."""
    K = G.NN()
    W1 = np.zeros((11, 16, 1, 4, 4), dtype=np.complex128)
    W2 = np.zeros((11, 1, 16, 4, 4), dtype=np.complex128)
    W1[0, 0, 0] = np.eye(4) / d ** 2
    W2[0, 0, 0] = np.eye(4)
    rng = np.random.default_rng(7)
    W1[:, 1:] += 1e-3 * (rng.standard_normal(W1[:, 1:].shape) + 1j * rng.standard_normal(W1[:, 1:].shape))
    W2[:, :, 1:] += 1e-3 * (rng.standard_normal(W2[:, :, 1:].shape)
                            + 1j * rng.standard_normal(W2[:, :, 1:].shape))
    K.set_weights(W1, W2)
    return K


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-dims", type=int, nargs=4, default=[16, 16, 16, 16])
    ap.add_argument("--train-Ls", type=int, default=12)
    ap.add_argument("--sources", type=int, default=64)
    ap.add_argument("--iterates", type=int, default=64)
    ap.add_argument("--steps-per-source", type=int, default=16)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--mf", type=float, default=0.005)
    ap.add_argument("--out", default="K.dwfnn")
    ap.add_argument("--eval-dims", type=int, nargs=4, default=None)
    ap.add_argument("--eval-Ls", type=int, default=16)
    ap.add_argument("--loss", default="a2", choices=["error", "energy", "a2"])
    a = ap.parse_args()
    act = G.Action(1.8, a.mf, 1.5, 0.5)
    d = 1.5 * (4 - 1.8) + 1
    dims = tuple(a.train_dims)
    rng = np.random.default_rng(1004)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    Ut = torch.from_numpy(U.reshape(-1)).cuda()
    h1 = G.Handle(dims, a.train_Ls, act, nrhs_max=1)
    h1.set_gauge(Ut)
    hb = G.Handle(dims, a.train_Ls, act, nrhs_max=a.batch)
    hb.set_gauge(Ut)
    K = initial_network(d)
    t0 = time.time()
    log = []
    npairs = 0
    for s in range(a.sources):
        b = inputs.gaussian_source(dims, a.train_Ls, rng=rng)
        r, e = make_pairs(h1, torch.from_numpy(b.reshape(-1)).cuda(), a.iterates,
                          record_every=4)
        npairs += r.shape[0]
        losses = train(K, hb, r, e, steps=a.steps_per_source, batch=a.batch, lr=a.lr, seed=s,
                       loss_kind=a.loss)
        log.append({"source": s, "pairs": int(r.shape[0]), "loss_first": losses[0],
                    "loss_last": losses[-1], "t": time.time() - t0})
        print(json.dumps(log[-1]), flush=True)
        del r, e
    K.save(a.out)
    res = {"train_pairs": npairs, "train_seconds": time.time() - t0, "weights": a.out}
    if a.eval_dims:
        res["eval"] = evaluate(K, tuple(a.eval_dims), a.eval_Ls, act)
    print(json.dumps(res), flush=True)


def lam_max(h, iters=30, seed=3):
    """Top of the spectrum of A = M_pc^+ M_pc by power iteration (FP32 operator
    calls of the library; the vector scaling is plumbing)."""
    g = torch.Generator(device="cuda").manual_seed(seed)
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


def multigrid(h, nvec, block, order, seed=5):
    """Two-level multigrid of Sec. 4 on handle h: nvec Gaussian vectors through
    the Chebyshev filter of order `order` on [hi/50, hi], block aggregation,
    Galerkin coarse operator.  Returns (MG, hi)."""
    hi = 1.05 * lam_max(h)
    g = torch.Generator(device="cuda").manual_seed(seed)
    V0 = torch.randn(h.cb_shape(1, nvec), device="cuda", generator=g)
    V = torch.empty_like(V0)
    h.chebyshev_filter(V, V0, order, hi / 50, hi, prec=G.FP32, nrhs=nvec)
    mg = G.MG(h, block, nvec)
    mg.setup(V)
    return mg, hi


def evaluate(K, dims, Ls, act, seed=1004, nvec=12, block=(8, 8, 8, 8), order=30, restart=64):
    """Time to 1e-10 on one Gaussian source: GCR with K, GCR without K, GCR
    with the two-level multigrid (Chebyshev smoother, and K as smoother; the
    multigrid set-up timed separately), mixed CG and FP64 CG.  `restart`: the
    GCR restart length (short restarts stall on these normal equations: at
    24^4 x 16, GCR(16) + K needs over 2900 iterations where GCR(64) + K needs
    320).  `fallback` marks a GCR that handed over to CG."""
    rng = np.random.default_rng(seed + 10)
    U = inputs.gauge_field(dims, "exp", eps=0.3, rng=rng)
    h = G.Handle(dims, Ls, act, nrhs_max=nvec)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    h.autotune(1, G.FP32)
    b = h.pack(torch.from_numpy(inputs.gaussian_source(dims, Ls, rng=rng).reshape(-1)).cuda())
    out = {}
    torch.cuda.synchronize()
    t = time.time()
    mg, hi = multigrid(h, nvec, block, order)
    torch.cuda.synchronize()
    out["mg_setup_seconds"] = time.time() - t
    out["mg"] = {"nvec": nvec, "block": list(block), "filter_order": order, "coarse": mg.sizes()[1]}

    def with_smoother(kind):
        if kind == "nn":
            mg.set_smoother("nn", K=K)
        else:
            mg.set_smoother("chebyshev", 3, hi / 10, hi)
        return mg

    out["restart"] = restart
    for name, fn in (("gcr_K", lambda x: h.gcr_solve(x, b, K=K, tol=1e-10, restart=restart)),
                     ("gcr", lambda x: h.gcr_solve(x, b, K=None, tol=1e-10, restart=restart)),
                     ("gcr_mg_chebyshev", lambda x: h.gcr_solve_mg(x, b, with_smoother("chebyshev"), tol=1e-10,
                                                                  restart=restart)),
                     ("gcr_mg_K", lambda x: h.gcr_solve_mg(x, b, with_smoother("nn"), tol=1e-10, restart=restart)),
                     ("cg_mixed_fp32", lambda x: h.cgne_solve(x, b, tol=1e-10, inner=G.FP32)),
                     ("cg_fp64", lambda x: h.cgne_solve(x, b, tol=1e-10, inner=G.FP64))):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t = time.time()
        st, rc = fn(x)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.time() - t, "iters": st[0]["iters"],
                     "true_resid": st[0]["true_resid"], "status": st[0]["status"],
                     "fallback": st[0]["recorded"] == -1}
    return out


if __name__ == "__main__":
    main()
