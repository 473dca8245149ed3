"""Test-side restatement of the field layouts documented in include/dwf.h.

Independent of the library's own tables: sites of box b are visited in
box-local lexicographic order, global coordinate (origin + l) mod L, and the
parity-p site list is the concatenation over boxes of the sites with global
parity p.  A cb field is [site][c = spin*3 + colour][rhs][s][re, im]; a full
field is the parity-0 cb field followed by the parity-1 cb field.
"""

from __future__ import annotations

import numpy as np


def whole_lattice_box(dims):
    return ((0, 0, 0, 0), tuple(dims))


def domain_sites(dims, boxes):
    """[parity] -> list of (box, local lex, (x, y, z, t))."""
    boxes = boxes or [whole_lattice_box(dims)]
    out = ([], [])
    for b, (org, ext) in enumerate(boxes):
        e0, e1, e2, e3 = ext
        for l3 in range(e3):
            for l2 in range(e2):
                for l1 in range(e1):
                    for l0 in range(e0):
                        lc = (l0, l1, l2, l3)
                        x = tuple((org[m] + lc[m]) % dims[m] for m in range(4))
                        l = l0 + e0 * (l1 + e1 * (l2 + e2 * l3))
                        out[sum(x) % 2].append((b, l, x))
    return out


def _site_arrays(dims, boxes):
    sites = domain_sites(dims, boxes)
    res = []
    for p in range(2):
        if sites[p]:
            b = np.array([s[0] for s in sites[p]])
            x = np.array([s[2] for s in sites[p]])
        else:
            b = np.zeros(0, dtype=int)
            x = np.zeros((0, 4), dtype=int)
        res.append((b, x))
    return res


def to_cb(fields, dims, boxes, parity):
    """fields[box][rhs] = full-lattice oracle array (t,z,y,x,Ls,4,3) ->
    cb field of the given parity (complex128, [site][12][nrhs][Ls])."""
    b, x = _site_arrays(dims, boxes)[parity]
    nrhs = len(fields[0])
    Ls = fields[0][0].shape[4]
    out = np.zeros((len(b), 12, nrhs, Ls), dtype=np.complex128)
    for r in range(nrhs):
        for bi in range(len(fields)):
            sel = np.flatnonzero(b == bi)
            if sel.size == 0:
                continue
            xs = x[sel]
            vals = fields[bi][r][xs[:, 3], xs[:, 2], xs[:, 1], xs[:, 0]]   # (n, Ls, 4, 3)
            out[sel, :, r, :] = vals.reshape(len(sel), Ls, 12).transpose(0, 2, 1)
    return out


def to_full(fields, dims, boxes):
    return np.concatenate([to_cb(fields, dims, boxes, 0), to_cb(fields, dims, boxes, 1)])


def from_cb(cb, dims, boxes, parity, Ls, nbox_fields=None):
    """cb field -> fields[box][rhs] full-lattice arrays (zero elsewhere)."""
    b, x = _site_arrays(dims, boxes)[parity]
    nrhs = cb.shape[2]
    nb = len(boxes) if boxes else 1
    Lx, Ly, Lz, Lt = dims
    fields = [[np.zeros((Lt, Lz, Ly, Lx, Ls, 4, 3), dtype=np.complex128) for _ in range(nrhs)]
              for _ in range(nb)]
    for r in range(nrhs):
        for bi in range(nb):
            sel = np.flatnonzero(b == bi)
            if sel.size == 0:
                continue
            xs = x[sel]
            vals = cb[sel, :, r, :].transpose(0, 2, 1).reshape(len(sel), Ls, 4, 3)
            fields[bi][r][xs[:, 3], xs[:, 2], xs[:, 1], xs[:, 0]] = vals
    return fields


def from_full(full, dims, boxes, Ls):
    n0 = len(domain_sites(dims, boxes)[0])
    f0 = from_cb(full[:n0], dims, boxes, 0, Ls)
    f1 = from_cb(full[n0:], dims, boxes, 1, Ls)
    return [[f0[b][r] + f1[b][r] for r in range(len(f0[b]))] for b in range(len(f0))]


def canonical(fields, boxes, dims):
    """fields[box][rhs] -> canonical complex128 [box][r][l][s][spin][colour]."""
    boxes = boxes or [whole_lattice_box(dims)]
    parts = []
    for bi, (org, ext) in enumerate(boxes):
        e0, e1, e2, e3 = ext
        t = (np.arange(e3)[:, None, None, None] + org[3]) % dims[3]
        z = (np.arange(e2)[None, :, None, None] + org[2]) % dims[2]
        y = (np.arange(e1)[None, None, :, None] + org[1]) % dims[1]
        xx = (np.arange(e0)[None, None, None, :] + org[0]) % dims[0]
        for f in fields[bi]:
            parts.append(f[t, z, y, xx].reshape(-1))
    return np.concatenate(parts)


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
