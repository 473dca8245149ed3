"""Oracle: the gauge-covariant parallel-transport convolutional preconditioner
K and its training step, in plain FP64 numpy (test infrastructure only).

Reading (the paper does not describe a learned preconditioner; the network
is the learned form added to the paper's local solves):

* Fields phi^a(x, s), a = channel, each a 4-spin x 3-colour complex field on
  the whole lattice (arrays (t, z, y, x, Ls, 4, 3)).
* Eleven transports T_d, d = 0..10:  T_0 = 1;
  T_{1+mu} phi(x) = U_mu(x) phi(x + mu)          (mu = 0..3);
  T_{5+mu} phi(x) = U_mu(x - mu)^+ phi(x - mu);
  T_9 phi(x, s) = phi(x, s + 1),  T_10 phi(x, s) = phi(x, s - 1), zero
  outside [0, Ls) (open ends, so the weights do not depend on Ls).
  Adjoints: T_{1+mu}^+ = T_{5+mu}, T_9^+ = T_10.
* Layer: phi_out^a = sum_b sum_d W_d^{ab} T_d phi_in^b, W_d^{ab} a complex
  4 x 4 matrix acting on spin (it commutes with colour and with T_d, so the
  layer is gauge covariant).
* Network: 1 -> C -> 1 channels, two linear layers.  K acts on the odd
  checkerboard: the input is embedded with zeros on even sites and the
  output is restricted to odd sites.
* Loss for a batch of pairs (r_k, e_k):  mean_k |K r_k - e_k|^2 / |e_k|^2,
  or, given the operator A with A e_k = r_k, the error in the energy norm
  mean_k <d_k, A d_k> / <e_k, r_k>, d_k = K r_k - e_k, whose gradient in
  z = K r is 2 (A z - r) / <e, r>: it weighs each mode of the error by its
  eigenvalue, the part a short-range K can represent; or in the A^2 norm,
  |A (K r - e)|^2 / |A e|^2 = |A K r - r|^2 / |r|^2, the residual left by one
  GCR step with z = K r.
  Gradients treat Re and Im of every weight as real parameters; with
  g = dL/dz (dL = Re<g, dz>) a layer z = W x back-propagates g_x = W^+ g and
  g_W = g x^+.
* Adam with bias correction on the real and imaginary parts.

Weight arrays: W1 (11, C, 1, 4, 4), W2 (11, 1, C, 4, 4), complex.
"""

from __future__ import annotations

import numpy as np

from oracle.dwf import AXIS, parity_part

NDIR = 11


def transport(U, phi, d):
    """T_d phi for one field phi (t, z, y, x, Ls, 4, 3)."""
    if d == 0:
        return phi.copy()
    if 1 <= d <= 4:
        mu = d - 1
        fwd = np.roll(phi, -1, axis=AXIS[mu])
        return np.einsum("tzyxab,tzyxsib->tzyxsia", U[..., mu, :, :], fwd)
    if 5 <= d <= 8:
        mu = d - 5
        Ub = np.roll(U[..., mu, :, :], 1, axis=AXIS[mu])
        bwd = np.roll(phi, 1, axis=AXIS[mu])
        return np.einsum("tzyxba,tzyxsib->tzyxsia", np.conj(Ub), bwd)
    out = np.zeros_like(phi)
    if d == 9:
        out[..., :-1, :, :] = phi[..., 1:, :, :]
    elif d == 10:
        out[..., 1:, :, :] = phi[..., :-1, :, :]
    else:
        raise ValueError(d)
    return out


ADJ = [0, 5, 6, 7, 8, 1, 2, 3, 4, 10, 9]   # T_d^+ = T_{ADJ[d]}


def layer(U, phis, W):
    """phi_out^a = sum_b sum_d W[d, a, b] (spin matrix) T_d phi_in^b."""
    nd, cout, cin = W.shape[:3]
    out = [np.zeros_like(phis[0]) for _ in range(cout)]
    for d in range(nd):
        T = [transport(U, p, d) for p in phis]
        for a in range(cout):
            for b in range(cin):
                out[a] += np.einsum("ij,tzyxsja->tzyxsia", W[d, a, b], T[b])
    return out


def apply_K(U, r, W1, W2):
    """K r on the odd checkerboard (input restricted to odd sites first)."""
    phi1 = layer(U, [parity_part(r, 1)], W1)
    z = layer(U, phi1, W2)[0]
    return parity_part(z, 1)


def loss_and_grad(U, pairs, W1, W2, apply_A=None, kind=None):
    """Mean relative squared error over (r, e) pairs (or, with ``apply_A``,
    the relative energy-norm error) and its gradients (dL/dW1, dL/dW2) as
    complex arrays (real part / imaginary part of each entry = derivative
    w.r.t. the real / imaginary part of the weight).  ``kind`` "a2" (with
    ``apply_A``) measures the error in the A^2 norm instead:
    |A (K r - e)|^2 / |A e|^2 = |A z - r|^2 / |r|^2, gradient 2 A (A z - r) / |r|^2."""
    nd, C = W1.shape[0], W1.shape[1]
    gW1 = np.zeros_like(W1)
    gW2 = np.zeros_like(W2)
    L = 0.0
    n = len(pairs)
    for r, e in pairs:
        x0 = parity_part(r, 1)
        T0 = [transport(U, x0, d) for d in range(nd)]
        phi1 = [sum(np.einsum("ij,tzyxsja->tzyxsia", W1[d, a, 0], T0[d]) for d in range(nd))
                for a in range(C)]
        T1 = [[transport(U, phi1[b], d) for b in range(C)] for d in range(nd)]
        z = sum(np.einsum("ij,tzyxsja->tzyxsia", W2[d, 0, b], T1[d][b])
                for d in range(nd) for b in range(C))
        z = parity_part(z, 1)
        if apply_A is None:
            en = np.vdot(e, e).real
            diff = z - e
            L += np.vdot(diff, diff).real / en / n
            gz = parity_part(2.0 * diff / en / n, 1)
        elif kind == "a2":
            res = apply_A(z) - r
            rr = np.vdot(r, r).real
            L += np.vdot(res, res).real / rr / n
            gz = parity_part(2.0 * apply_A(res) / rr / n, 1)
        else:
            Az = apply_A(z)
            er = np.vdot(e, r).real
            L += (np.vdot(z, Az).real - 2 * np.vdot(z, r).real + er) / er / n
            gz = parity_part(2.0 * (Az - r) / er / n, 1)
        # layer 2: z = sum_{d,b} W2[d,0,b] T_d phi1^b
        gphi1 = [np.zeros_like(x0) for _ in range(C)]
        for d in range(nd):
            for b in range(C):
                gW2[d, 0, b] += np.einsum("tzyxsia,tzyxsja->ij", gz, np.conj(T1[d][b]))
                gphi1[b] += transport(U, np.einsum("ji,tzyxsja->tzyxsia",
                                                   np.conj(W2[d, 0, b]), gz), ADJ[d])
        # layer 1: phi1^a = sum_d W1[d,a,0] T_d x0
        for d in range(nd):
            for a in range(C):
                gW1[d, a, 0] += np.einsum("tzyxsia,tzyxsja->ij", gphi1[a], np.conj(T0[d]))
    return L, gW1, gW2


class Adam:
    """Adam on the real and imaginary parts of complex parameters."""

    def __init__(self, shapes, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros(s, dtype=np.complex128) for s in shapes]
        self.v = [np.zeros(s, dtype=np.complex128) for s in shapes]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for k, (p, g) in enumerate(zip(params, grads)):
            gr = np.stack([g.real, g.imag])
            m = np.stack([self.m[k].real, self.m[k].imag])
            v = np.stack([self.v[k].real, self.v[k].imag])
            m = self.b1 * m + (1 - self.b1) * gr
            v = self.b2 * v + (1 - self.b2) * gr * gr
            self.m[k] = m[0] + 1j * m[1]
            self.v[k] = v[0] + 1j * v[1]
            mh = m / (1 - self.b1 ** self.t)
            vh = v / (1 - self.b2 ** self.t)
            upd = self.lr * mh / (np.sqrt(vh) + self.eps)
            out.append(p - (upd[0] + 1j * upd[1]))
        return out


def identity_weights(C):
    """W1[0, a] = 1 for a = 0, W2[0, 0, 0] = 1, everything else 0: K = 1."""
    W1 = np.zeros((NDIR, C, 1, 4, 4), dtype=np.complex128)
    W2 = np.zeros((NDIR, 1, C, 4, 4), dtype=np.complex128)
    W1[0, 0, 0] = np.eye(4)
    W2[0, 0, 0] = np.eye(4)
    return W1, W2


def gcr(U, b_odd, p, apply_mpc, K=None, tol=1e-10, restart=16, maxiter=2000, bnorm=None):
    """Right-preconditioned flexible GCR(restart) on A x = b (odd sites),
    A = ``apply_mpc`` (M_pc, or M_pc^+ M_pc for the normal equations):
    z = K r, q = A z, modified Gram-Schmidt of q against the previous q's
    (the same combination applied to z), x += a z, r -= a q with
    a = <q, r> / <q, q>.  Returns (x, iterations)."""
    x = np.zeros_like(b_odd)
    bn = bnorm if bnorm is not None else np.linalg.norm(b_odd)
    r = b_odd.copy()
    it = 0
    while it < maxiter:
        Q, Z = [], []
        for _ in range(restart):
            z = K(r) if K is not None else r.copy()
            q = apply_mpc(z)
            for qi, zi in zip(Q, Z):
                beta = np.vdot(qi, q)
                q = q - beta * qi
                z = z - beta * zi
            nq = np.sqrt(np.vdot(q, q).real)
            q, z = q / nq, z / nq
            a = np.vdot(q, r)
            x = x + a * z
            r = r - a * q
            Q.append(q)
            Z.append(z)
            it += 1
            if np.linalg.norm(r) <= tol * bn:
                break
        r = b_odd - apply_mpc(x)
        if np.linalg.norm(r) <= tol * bn:
            break
    return x, it
