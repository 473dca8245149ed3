"""Thin ctypes binding of ``include/dwf.h`` (argument marshalling only).

Every operator and solver step runs inside ``libdwf.so``; this module only
passes device pointers, sizes and the current CUDA stream.  It raises
``DWFError`` when the library has not been built or a call fails -- there
is no CPU fallback.  Fields are ``torch`` CUDA tensors in the layouts that
``include/dwf.h`` documents; torch is used for device memory and streams.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# DWF_DEBUG=1 in the environment loads the debug build (host-side bounds checks
# of every caller buffer, python -m paper_2203_17119_gb300.build --debug)
LIB_PATH = (os.path.join(_PKG, "_build_debug", "libdwf_debug.so") if os.environ.get("DWF_DEBUG") == "1"
            else os.path.join(_PKG, "_build", "libdwf.so"))

FP64, FP32, BF16 = 0, 1, 2
_DTYPE = {FP64: torch.float64, FP32: torch.float32, BF16: torch.bfloat16}
PREC = {"f64": FP64, "fp64": FP64, "f32": FP32, "fp32": FP32, "bf16": BF16}

STATUS = {0: "DWF_OK", 1: "DWF_ERR_ARG", 2: "DWF_ERR_CUDA", 3: "DWF_ERR_NOT_CONVERGED",
          4: "DWF_ERR_TIMEOUT", 5: "DWF_ERR_NAN", 6: "DWF_ERR_UNSUPPORTED", 7: "DWF_ERR_DEVICE"}


class DWFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("Ls", C.c_int), ("M5", C.c_double),
                ("mf", C.c_double), ("b5", C.c_double), ("c5", C.c_double)]


class Box(C.Structure):
    _fields_ = [("origin", C.c_int * 4), ("extent", C.c_int * 4)]


class Rational(C.Structure):
    _fields_ = [("a0", C.c_double), ("shifts", C.POINTER(C.c_double)), ("residues", C.POINTER(C.c_double)),
                ("n", C.c_int)]


class SolverParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("delta", C.c_double),
                ("restart", C.c_int), ("use_x0", C.c_int), ("inner_prec", C.c_int),
                ("max_seconds", C.c_double), ("check_every", C.c_int),
                ("record_x", C.c_void_p), ("record_every", C.c_int), ("record_max", C.c_int)]


class SolverStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("reliable_updates", C.c_int), ("op_applies", C.c_int),
                ("status", C.c_int), ("true_resid", C.c_double), ("seconds", C.c_double),
                ("recorded", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def signatures():
    """argtypes of every entry point of include/dwf.h (restype: dwf_status)."""
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    return {
        "dwf_create": [C.POINTER(vp), C.POINTER(Params), C.POINTER(Box), i, i],
        "dwf_create_cut": [C.POINTER(vp), C.POINTER(Params), C.POINTER(Box), i, i],
        "dwf_debug_build": [C.POINTER(C.c_int)],
        "dwf_copy": [vp, vp, C.c_size_t, vp],
        "dwf_set_tile_order": [vp, i, i, i],
        "dwf_get_tile_order": [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "dwf_check_range": [vp, C.c_size_t],
        "dwf_one_flavour_action": [vp, vp, vp, i, C.POINTER(Rational), C.POINTER(Rational), C.POINTER(SolverParams),
                                   C.POINTER(C.c_double), C.POINTER(SolverStats), vp],
        "dwf_one_flavour_force": [vp, vp, vp, vp, i, C.POINTER(Rational), C.POINTER(Rational), C.POINTER(Box), i,
                                  C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
        "dwf_one_flavour_heatbath": [vp, vp, vp, vp, i, C.POINTER(Rational), C.POINTER(Rational),
                                     C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
        "dwf_destroy": [vp],
        "dwf_domain_sites": [vp, i, C.POINTER(C.c_int64)],
        "dwf_box_sites": [vp, i, i, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
        "dwf_set_gauge": [vp, vp, vp],
        "dwf_pack": [vp, vp, vp, i, i, vp],
        "dwf_unpack": [vp, vp, vp, i, i, vp],
        "dwf_dslash_eo": [vp, vp, vp, i, i, i, i, vp],
        "dwf_mooee": [vp, vp, vp, i, i, i, i, vp],
        "dwf_mooee_inv": [vp, vp, vp, i, i, i, i, vp],
        "dwf_mpc": [vp, vp, vp, i, i, i, vp],
        "dwf_apply_d": [vp, vp, vp, i, i, i, vp],
        "dwf_dirichlet_block": [vp, vp, vp, i, i, i, vp],
        "dwf_cgne_solve": [vp, vp, vp, i, C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
        "dwf_check_device": [vp],
        "dwf_hop": [vp, vp, vp, i, i, i, i, vp],
        "dwf_launch_count": [C.POINTER(C.c_uint64)],
        "dwf_alloc_count": [C.POINTER(C.c_uint64)],
        "dwf_autotune": [vp, i, i, C.POINTER(C.c_int)],
        "dwf_set_tile": [vp, i, i, i],
        "dwf_set_hop_kernel": [vp, i, i],
        "dwf_set_hop_chunk": [vp, i, i],
        "dwf_get_tuning": [vp, i, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                           C.POINTER(C.c_int)],
        "dwf_mpc_noalloc": [vp, vp, vp, i, i, i, vp],
        "dwf_gcr_solve": [vp, vp, vp, i, vp, C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
        "dwf_multishift_solve": [vp, vp, vp, C.POINTER(C.c_double), i, i, C.POINTER(SolverParams),
                                 C.POINTER(SolverStats), vp],
        "dwf_boundary_project": [vp, C.POINTER(Box), vp, vp, i, vp],
        "dwf_force": [vp, vp, vp, vp, i, i, C.POINTER(Box), i, vp],
        "dwf_zolotarev_inv_sqrt": [i, C.c_double, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)],
        "dwf_rational_power": [C.c_double, i, C.c_double, C.c_double, C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "dwf_rational_apply": [vp, vp, vp, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double), i, i,
                               C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
        "dwf_chebyshev_filter": [vp, vp, vp, i, C.c_double, C.c_double, i, i, vp],
        "dwf_boundary_r": [vp, C.POINTER(Box), vp, vp, i, C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
        "dwf_boundary_ratio_force": [vp, vp, C.POINTER(Box), vp, vp, i, C.POINTER(Box), i,
                                     C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
        "dwf_boundary_force": [vp, C.POINTER(Box), vp, vp, i, C.POINTER(Box), i, C.POINTER(SolverParams),
                               C.POINTER(SolverStats), vp],
        "dwf_boundary_rinv": [vp, C.POINTER(Box), vp, vp, i, C.POINTER(SolverParams),
                              C.POINTER(SolverStats), vp],
        "dwf_nn_create": [C.POINTER(vp), i],
        "dwf_nn_destroy": [vp],
        "dwf_nn_set_weights": [vp, vp, C.c_size_t],
        "dwf_nn_get_weights": [vp, vp, C.c_size_t],
        "dwf_nn_apply": [vp, vp, vp, vp, i, vp],
        "dwf_nn_train_step": [vp, vp, vp, vp, i, i, d, C.POINTER(C.c_double), vp],
        "dwf_nn_last_grad": [vp, vp, C.c_size_t],
        "dwf_nn_make_pair": [vp, vp, vp, vp, vp, C.POINTER(C.c_double), vp],
        "dwf_nn_save": [vp, C.c_char_p],
        "dwf_autotune_save": [vp, C.c_char_p],
        "dwf_set_fusion": [vp, i, i],
        "dwf_get_fusion": [vp, i, C.POINTER(C.c_int)],
        "dwf_autotune_load": [vp, C.c_char_p, i, i, C.POINTER(C.c_int)],
        "dwf_nn_load": [vp, C.c_char_p],
        "dwf_mg_create": [C.POINTER(vp), vp, C.POINTER(C.c_int), i],
        "dwf_mg_destroy": [vp],
        "dwf_mg_setup": [vp, vp, vp],
        "dwf_mg_set_smoother": [vp, i, i, d, d, vp],
        "dwf_mg_apply": [vp, vp, vp, vp],
        "dwf_mg_restrict": [vp, vp, vp, vp],
        "dwf_mg_prolong": [vp, vp, vp, vp],
        "dwf_mg_info": [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "dwf_mg_copy": [vp, i, vp, vp],
        "dwf_mg_handle": [vp, C.POINTER(vp)],
        "dwf_gcr_solve_mg": [vp, vp, vp, vp, C.POINTER(SolverParams), C.POINTER(SolverStats), vp],
    }


def lib():
    """The loaded ``libdwf.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise DWFError(2, f"{LIB_PATH} is missing: run __graft_entry__.build() or "
                              "python -m paper_2203_17119_gb300.build")
        L = C.CDLL(LIB_PATH)
        sig = signatures()
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.dwf_last_error.restype = C.c_char_p
        L.dwf_last_error.argtypes = []
        _lib = L
    return _lib


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    n = C.c_uint64()
    _check(lib().dwf_launch_count(C.byref(n)))
    return n.value


def alloc_count() -> int:
    """Device allocations (cudaMalloc) made by the library so far in this process."""
    n = C.c_uint64()
    _check(lib().dwf_alloc_count(C.byref(n)))
    return n.value


def _check(st: int, allow=()):
    if st != 0 and st not in allow:
        raise DWFError(st, lib().dwf_last_error().decode())
    return st


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    if not t.is_cuda:
        raise DWFError(1, "field tensors must live on the GPU")
    if not t.is_contiguous():
        raise DWFError(1, "field tensors must be contiguous")
    return C.c_void_p(t.data_ptr())


@dataclass
class Action:
    """Operator parameters; Shamir is b5 = 1, c5 = 0."""
    M5: float = 1.8
    mf: float = 0.01
    b5: float = 1.0
    c5: float = 0.0


def zolotarev_inv_sqrt(n, lo, hi):
    """Zolotarev's 1/sqrt(x) on [lo, hi] in partial fractions: (shifts, residues, delta)."""
    sh = (C.c_double * n)()
    rs = (C.c_double * n)()
    dl = C.c_double()
    _check(lib().dwf_zolotarev_inv_sqrt(int(n), float(lo), float(hi), sh, rs, C.byref(dl)))
    return list(sh), list(rs), dl.value


def copy(dst: torch.Tensor, src: torch.Tensor, stream=None):
    """dst <- src (same byte size; device or pinned host tensors) with the GPU's
    own loads and stores (dwf_copy)."""
    nb = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nb or not dst.is_contiguous() or not src.is_contiguous():
        raise DWFError(1, "copy: contiguous tensors of the same byte size")
    _check(lib().dwf_copy(C.c_void_p(dst.data_ptr()), C.c_void_p(src.data_ptr()), nb, _stream(stream)))
    return dst


def rational_power(alpha, n, lo, hi):
    """Best relative type (n, n) approximation of x**alpha on [lo, hi] in
    partial fractions: (a0, shifts, residues, delta)."""
    a0 = C.c_double()
    sh = (C.c_double * n)()
    rs = (C.c_double * n)()
    dl = C.c_double()
    _check(lib().dwf_rational_power(float(alpha), int(n), float(lo), float(hi), C.byref(a0), sh, rs,
                                    C.byref(dl)))
    return a0.value, list(sh), list(rs), dl.value


class Handle:
    """A ``dwf_handle``: the whole lattice (``boxes=None``) or the Dirichlet
    blocks of a list of boxes ((origin[4], extent[4]) in x, y, z, t order)."""

    def __init__(self, dims, Ls, action: Action, boxes=None, nrhs_max=1, cut=None):
        """``cut``: a list of boxes making this the whole-lattice handle of
        D_dirichlet (the links between those domains and the rest left out,
        ``dwf_create_cut``); not together with ``boxes``."""
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.action = action
        self.nrhs_max = int(nrhs_max)
        self.boxes = [tuple(map(tuple, b)) for b in boxes] if boxes else []
        self.cut = [tuple(map(tuple, b)) for b in cut] if cut else []
        if self.boxes and self.cut:
            raise ValueError("a handle has either Dirichlet boxes or cut domains")
        p = Params((C.c_int * 4)(*self.dims), self.Ls, action.M5, action.mf, action.b5, action.c5)
        lst = self.boxes or self.cut
        nb = len(lst)
        arr = (Box * max(nb, 1))()
        for k, (o, e) in enumerate(lst):
            arr[k] = Box((C.c_int * 4)(*o), (C.c_int * 4)(*e))
        h = C.c_void_p()
        if self.cut:
            _check(lib().dwf_create_cut(C.byref(h), C.byref(p), arr, nb, self.nrhs_max))
        else:
            _check(lib().dwf_create(C.byref(h), C.byref(p), arr if nb else None, nb, self.nrhs_max))
        self._h = h
        n0, n1 = C.c_int64(), C.c_int64()
        _check(lib().dwf_domain_sites(h, 0, C.byref(n0)))
        _check(lib().dwf_domain_sites(h, 1, C.byref(n1)))
        self.nsite = (n0.value, n1.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().dwf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ fields
    def cb_shape(self, parity, nrhs=1):
        return (self.nsite[parity], 12, nrhs, self.Ls, 2)

    def full_shape(self, nrhs=1):
        return (self.nsite[0] + self.nsite[1], 12, nrhs, self.Ls, 2)

    def empty_cb(self, parity, nrhs=1, prec=FP64):
        return torch.empty(self.cb_shape(parity, nrhs), dtype=_DTYPE[prec], device="cuda")

    def empty_full(self, nrhs=1, prec=FP64):
        return torch.empty(self.full_shape(nrhs), dtype=_DTYPE[prec], device="cuda")

    def box_sites(self, box, parity):
        o, c = C.c_int64(), C.c_int64()
        _check(lib().dwf_box_sites(self._h, box, parity, C.byref(o), C.byref(c)))
        return o.value, c.value

    # -------------------------------------------------------------- calls
    def set_gauge(self, U: torch.Tensor, stream=None):
        """U: complex128 or float64 CUDA tensor, canonical [site][mu][3][3]."""
        if U.dtype == torch.complex128:
            U = torch.view_as_real(U)
        if U.dtype != torch.float64:
            raise DWFError(1, "gauge field must be complex128 / float64")
        _check(lib().dwf_set_gauge(self._h, _ptr(U), _stream(stream)))

    def pack(self, canon: torch.Tensor, nrhs=1, prec=FP64, out=None, stream=None):
        """canonical complex128 [box][r][l][s][spin][colour] -> full field."""
        if canon.dtype == torch.complex128:
            canon = torch.view_as_real(canon)
        out = self.empty_full(nrhs, prec) if out is None else out
        _check(lib().dwf_pack(self._h, _ptr(out), _ptr(canon), nrhs, prec, _stream(stream)))
        return out

    def unpack(self, field: torch.Tensor, nrhs=1, prec=FP64, out=None, stream=None):
        n = (self.nsite[0] + self.nsite[1]) * 12 * nrhs * self.Ls
        out = torch.empty((n, 2), dtype=torch.float64, device="cuda") if out is None else out
        _check(lib().dwf_unpack(self._h, _ptr(out), _ptr(field), nrhs, prec, _stream(stream)))
        return out

    def dslash_eo(self, out, inp, out_parity, dagger=False, prec=FP64, nrhs=1, stream=None):
        _check(lib().dwf_dslash_eo(self._h, _ptr(out), _ptr(inp), out_parity, int(dagger), prec,
                                   nrhs, _stream(stream)))
        return out

    def hop(self, out, inp, out_parity, dagger=False, prec=FP64, nrhs=1, stream=None):
        """Bare Wilson hop Dh (the dominant kernel)."""
        _check(lib().dwf_hop(self._h, _ptr(out), _ptr(inp), out_parity, int(dagger), prec, nrhs,
                             _stream(stream)))
        return out

    def mooee(self, out, inp, parity, dagger=False, prec=FP64, nrhs=1, stream=None):
        _check(lib().dwf_mooee(self._h, _ptr(out), _ptr(inp), parity, int(dagger), prec, nrhs,
                               _stream(stream)))
        return out

    def mooee_inv(self, out, inp, parity, dagger=False, prec=FP64, nrhs=1, stream=None):
        _check(lib().dwf_mooee_inv(self._h, _ptr(out), _ptr(inp), parity, int(dagger), prec, nrhs,
                                   _stream(stream)))
        return out

    def mpc(self, out, inp, dagger=False, prec=FP64, nrhs=1, stream=None):
        _check(lib().dwf_mpc(self._h, _ptr(out), _ptr(inp), int(dagger), prec, nrhs,
                             _stream(stream)))
        return out

    def mpc_noalloc(self, out, inp, dagger=False, prec=FP64, nrhs=1, stream=None):
        """M_pc with its temporaries in the library's static scratch array."""
        _check(lib().dwf_mpc_noalloc(self._h, _ptr(out), _ptr(inp), int(dagger), prec, nrhs,
                                     _stream(stream)))
        return out

    def apply_d(self, out, inp, dagger=False, prec=FP64, nrhs=1, stream=None):
        _check(lib().dwf_apply_d(self._h, _ptr(out), _ptr(inp), int(dagger), prec, nrhs,
                                 _stream(stream)))
        return out

    def dirichlet_block(self, out, inp, dagger=False, prec=FP64, nrhs=1, stream=None):
        _check(lib().dwf_dirichlet_block(self._h, _ptr(out), _ptr(inp), int(dagger), prec, nrhs,
                                         _stream(stream)))
        return out

    def cgne_solve(self, x, b, nrhs=1, tol=1e-10, maxiter=100000, inner=FP64, delta=0.0,
                   use_x0=False, max_seconds=0.0, check_every=8, stream=None, allow_fail=False,
                   record=None, record_every=8):
        """Solve D x = b (D_Omega x = b on a box handle); x, b full FP64
        fields.  ``record``: optional FP64 device tensor of shape
        (n, *cb_shape(1, nrhs)) receiving the odd iterates every
        ``record_every`` iterations (FP64 inner solves).  Returns the list of
        per-system stats dicts (box-major) and the status code."""
        rp = C.c_void_p(record.data_ptr()) if record is not None else None
        rmax = record.shape[0] if record is not None else 0
        sp = SolverParams(tol, maxiter, delta, 16, int(use_x0), inner, max_seconds, check_every,
                          rp, record_every, rmax)
        nsys = max(len(self.boxes), 1) * nrhs
        st = (SolverStats * nsys)()
        rc = lib().dwf_cgne_solve(self._h, _ptr(x), _ptr(b), nrhs, C.byref(sp), st,
                                  _stream(stream))
        if not allow_fail:
            _check(rc)
        return [s.as_dict() for s in st], rc

    def autotune(self, nrhs=1, prec=FP32):
        """Pick the tile size (sites per CTA) for this nrhs by timing the hop."""
        t = C.c_int()
        _check(lib().dwf_autotune(self._h, nrhs, prec, C.byref(t)))
        return t.value


    def autotune_save(self, path):
        """Append / update this handle's tunings in the autotune file ``path``."""
        _check(lib().dwf_autotune_save(self._h, os.fsencode(path)))

    def autotune_load(self, path, nrhs=1, prec=FP32):
        """Apply the cached tuning for (nrhs, prec) if ``path`` has one; True if found."""
        f = C.c_int()
        _check(lib().dwf_autotune_load(self._h, os.fsencode(path), nrhs, prec, C.byref(f)))
        return bool(f.value)
    def gcr_solve(self, x, b, K=None, nrhs=1, tol=1e-10, maxiter=100000, restart=16,
                  max_seconds=0.0, stream=None, allow_fail=False):
        """Flexible GCR with the learned preconditioner ``K`` (an ``NN``) or none."""
        sp = SolverParams(tol, maxiter, 0.1, restart, 0, FP32, max_seconds, 8, None, 0, 0)
        nsys = max(len(self.boxes), 1) * nrhs
        st = (SolverStats * nsys)()
        rc = lib().dwf_gcr_solve(self._h, _ptr(x), _ptr(b), nrhs, K._k if K is not None else None,
                                 C.byref(sp), st, _stream(stream))
        if not allow_fail:
            _check(rc)
        return [s.as_dict() for s in st], rc

    def gcr_solve_mg(self, x, b, mg, tol=1e-10, maxiter=100000, restart=16, max_seconds=0.0,
                     stream=None, allow_fail=False):
        """Flexible GCR with the multigrid preconditioner ``mg`` (an ``MG``)."""
        sp = SolverParams(tol, maxiter, 0.1, restart, 0, FP32, max_seconds, 8, None, 0, 0)
        st = (SolverStats * max(len(self.boxes), 1))()
        rc = lib().dwf_gcr_solve_mg(self._h, _ptr(x), _ptr(b), mg._m, C.byref(sp), st, _stream(stream))
        if not allow_fail:
            _check(rc)
        return [v.as_dict() for v in st], rc

    def multishift_solve(self, x, b, shifts, nrhs=1, tol=1e-10, maxiter=100000, inner=FP64,
                         max_seconds=0.0, stream=None, allow_fail=False):
        """(M_pc^+ M_pc + sigma_s) x_s = b for every shift: ``b`` an odd cb FP64
        field, ``x`` a FP64 tensor of shape (len(shifts), *cb_shape(1, nrhs)).
        Returns ([per shift: [per system: stats dict]], status)."""
        sh = (C.c_double * len(shifts))(*[float(v) for v in shifts])
        sp = SolverParams(tol, maxiter, 0.0, 0, 0, inner, max_seconds, 0, None, 0, 0)
        nsys = max(len(self.boxes), 1) * nrhs
        st = (SolverStats * (nsys * len(shifts)))()
        rc = lib().dwf_multishift_solve(self._h, _ptr(x), _ptr(b), sh, len(shifts), nrhs,
                                        C.byref(sp), st, _stream(stream))
        if not allow_fail:
            _check(rc)
        d = [s.as_dict() for s in st]
        return [d[k * nsys:(k + 1) * nsys] for k in range(len(shifts))], rc

    @staticmethod
    def _box(omega):
        o, e = omega
        return Box((C.c_int * 4)(*o), (C.c_int * 4)(*e))

    def boundary_project(self, out, inp, omega, nrhs=1, stream=None):
        """out = P in: Luescher's projector for the box ``omega`` = (origin, extent)."""
        _check(lib().dwf_boundary_project(self._h, C.byref(self._box(omega)), _ptr(out), _ptr(inp),
                                          nrhs, _stream(stream)))
        return out

    def boundary_rinv(self, out, inp, omega, nrhs=1, tol=1e-10, inner=FP32, stream=None):
        """out = R^-1 in = P in - P D^-1 D_partialbar P in; returns the D solve's stats."""
        sp = SolverParams(tol, 100000, 0.0, 16, 0, inner, 0.0, 8, None, 0, 0)
        st = (SolverStats * nrhs)()
        _check(lib().dwf_boundary_rinv(self._h, C.byref(self._box(omega)), _ptr(out), _ptr(inp), nrhs,
                                       C.byref(sp), st, _stream(stream)))
        return [s.as_dict() for s in st]

    def boundary_r(self, out, inp, omega, nrhs=1, tol=1e-10, maxiter=20000, inner=FP32, stream=None):
        """out = R in (Dirichlet solves on Omega-bar and Omega: FP64 CGNR, or
        FP32 CGNR with FP64 defect correction); returns the stats of the two
        solves (2 * nrhs dicts)."""
        sp = SolverParams(tol, maxiter, 0.0, 16, 0, inner, 0.0, 8, None, 0, 0)
        st = (SolverStats * (2 * nrhs))()
        _check(lib().dwf_boundary_r(self._h, C.byref(self._box(omega)), _ptr(out), _ptr(inp), nrhs,
                                    C.byref(sp), st, _stream(stream)))
        return [s.as_dict() for s in st]

    def boundary_ratio_force(self, pv, out, phi, omega, nrhs=1, active=None, accumulate=False, tol=1e-10,
                             inner=FP32, stream=None):
        """out[lex, mu] = link force of |R^-1 R_pv phi|^2, R on this handle,
        R_pv on the Pauli-Villars handle ``pv``; returns the stats of the six
        solves (6 * nrhs dicts: b, d, y, adjoint light, eta, kappa)."""
        sp = SolverParams(tol, 100000, 0.0, 16, 0, inner, 0.0, 8, None, 0, 0)
        st = (SolverStats * (6 * nrhs))()
        box = C.byref(self._box(active)) if active is not None else None
        _check(lib().dwf_boundary_ratio_force(self._h, pv._h, C.byref(self._box(omega)), _ptr(out), _ptr(phi),
                                              nrhs, box, int(accumulate), C.byref(sp), st, _stream(stream)))
        return [s.as_dict() for s in st]

    def boundary_force(self, out, phi, omega, nrhs=1, active=None, accumulate=False, tol=1e-10,
                       inner=FP32, stream=None):
        """out[lex, mu] = link force of |R^-1 phi|^2 for the box ``omega``;
        returns the stats of the two solves (2 * nrhs dicts)."""
        sp = SolverParams(tol, 100000, 0.0, 16, 0, inner, 0.0, 8, None, 0, 0)
        st = (SolverStats * (2 * nrhs))()
        box = C.byref(self._box(active)) if active is not None else None
        _check(lib().dwf_boundary_force(self._h, C.byref(self._box(omega)), _ptr(out), _ptr(phi), nrhs, box,
                                        int(accumulate), C.byref(sp), st, _stream(stream)))
        return [s.as_dict() for s in st]

    def rational_apply(self, out, inp, a0, shifts, residues, nrhs=1, tol=1e-10, maxiter=100000, inner=FP64,
                       stream=None):
        """out = a0 in + sum_i residues[i] (M_pc^+ M_pc + shifts[i])^-1 in (odd
        cb FP64 fields); returns ([per shift: [per system: stats dict]], status)."""
        n = len(shifts)
        sh = (C.c_double * n)(*[float(v) for v in shifts])
        rs = (C.c_double * n)(*[float(v) for v in residues])
        sp = SolverParams(tol, maxiter, 0.0, 0, 0, inner, 0.0, 0, None, 0, 0)
        nsys = max(len(self.boxes), 1) * nrhs
        st = (SolverStats * (nsys * n))()
        rc = lib().dwf_rational_apply(self._h, _ptr(out), _ptr(inp), float(a0), sh, rs, n, nrhs, C.byref(sp), st,
                                      _stream(stream))
        _check(rc)
        return [[st[k * nsys + i].as_dict() for i in range(nsys)] for k in range(n)], rc

    # ------------------------------------------- one-flavour DD-RHMC term
    @staticmethod
    def _rational(r):
        a0, shifts, residues = r
        n = len(shifts)
        sh = (C.c_double * n)(*[float(v) for v in shifts])
        rs = (C.c_double * n)(*[float(v) for v in residues])
        return Rational(float(a0), sh, rs, n), (sh, rs)

    def one_flavour_action(self, hd, phi, r1, r2, nrhs=1, tol=1e-10, maxiter=100000, inner=FP64,
                           stream=None):
        """S[r] = phi_r^+ r1(A_d) r2(A) r1(A_d) phi_r with A of this handle (D)
        and A_d of ``hd`` (the cut handle of D_dirichlet); r1, r2 = (a0,
        shifts, residues).  Returns (list of S, stats dicts)."""
        R1, keep1 = self._rational(r1)
        R2, keep2 = self._rational(r2)
        sp = SolverParams(tol, maxiter, 0.0, 0, 0, inner, 0.0, 0, None, 0, 0)
        st = (SolverStats * ((R1.n + R2.n) * nrhs))()
        S = (C.c_double * nrhs)()
        _check(lib().dwf_one_flavour_action(self._h, hd._h, _ptr(phi), nrhs, C.byref(R1), C.byref(R2), C.byref(sp),
                                            S, st, _stream(stream)))
        return list(S), [s.as_dict() for s in st]

    def one_flavour_force(self, hd, out, phi, r1, r2, nrhs=1, active=None, accumulate=False, tol=1e-10,
                          maxiter=100000, inner=FP64, stream=None):
        """out[lex, mu] = link force of the one-flavour term (summed over
        right-hand sides); returns the stats dicts of the three multi-shift solves."""
        R1, keep1 = self._rational(r1)
        R2, keep2 = self._rational(r2)
        sp = SolverParams(tol, maxiter, 0.0, 0, 0, inner, 0.0, 0, None, 0, 0)
        st = (SolverStats * ((2 * R1.n + R2.n) * nrhs))()
        box = C.byref(self._box(active)) if active is not None else None
        _check(lib().dwf_one_flavour_force(self._h, hd._h, _ptr(out), _ptr(phi), nrhs, C.byref(R1), C.byref(R2),
                                           box, int(accumulate), C.byref(sp), st, _stream(stream)))
        return [s.as_dict() for s in st]

    def one_flavour_heatbath(self, hd, phi, eta, q1, q2, nrhs=1, tol=1e-10, maxiter=100000, inner=FP64,
                             stream=None):
        """phi = q1(A_d) q2(A) eta (q1 ~ x^-1/4, q2 ~ x^1/4); returns stats dicts."""
        Q1, keep1 = self._rational(q1)
        Q2, keep2 = self._rational(q2)
        sp = SolverParams(tol, maxiter, 0.0, 0, 0, inner, 0.0, 0, None, 0, 0)
        st = (SolverStats * ((Q1.n + Q2.n) * nrhs))()
        _check(lib().dwf_one_flavour_heatbath(self._h, hd._h, _ptr(phi), _ptr(eta), nrhs, C.byref(Q1), C.byref(Q2),
                                              C.byref(sp), st, _stream(stream)))
        return [s.as_dict() for s in st]

    def chebyshev_filter(self, out, inp, order, lo, hi, prec=FP64, nrhs=1, stream=None):
        """out = T_order(z(A)) in, A = M_pc^+ M_pc, z(lam) = (hi + lo - 2 lam)/(hi - lo)."""
        _check(lib().dwf_chebyshev_filter(self._h, _ptr(out), _ptr(inp), int(order), float(lo), float(hi),
                                          prec, nrhs, _stream(stream)))
        return out

    def force(self, out, X, Y, prec=FP64, nrhs=1, active=None, accumulate=False, stream=None):
        """out[lex, mu] = link force of sum_r Re <X_r, D Y_r> (traceless
        anti-Hermitian 3 x 3, FP64 canonical gauge layout); ``active`` an
        optional box (origin, extent) outside which links get 0."""
        box = C.byref(self._box(active)) if active is not None else None
        _check(lib().dwf_force(self._h, _ptr(out), _ptr(X), _ptr(Y), prec, nrhs, box, int(accumulate),
                               _stream(stream)))
        return out

    def set_tile(self, nrhs=1, tile_sites=32, lanes_per_thread=2):
        """Fix the tile size and FP32 hop lanes per thread for this nrhs."""
        _check(lib().dwf_set_tile(self._h, nrhs, tile_sites, lanes_per_thread))

    def set_hop_kernel(self, nrhs=1, kernel=1):
        """BF16-operator hop for this nrhs: 0 = FP32 SIMT, 1 = tensor cores."""
        _check(lib().dwf_set_hop_kernel(self._h, nrhs, kernel))

    def set_fusion(self, nrhs=1, fuse=True):
        """dwf_set_fusion: site-local factors of M_pc in the hop epilogues (where possible)."""
        _check(lib().dwf_set_fusion(self._h, nrhs, 1 if fuse else 0))

    def fusion(self, nrhs=1):
        f = C.c_int()
        _check(lib().dwf_get_fusion(self._h, nrhs, C.byref(f)))
        return bool(f.value)

    def set_tile_order(self, order=1, bz=8, bt=8):
        """Tile order of every kernel on this handle: 0 lexicographic, 1
        blocked in (z, t) by bz x bt planes."""
        _check(lib().dwf_set_tile_order(self._h, int(order), int(bz), int(bt)))

    def tile_order(self):
        """(order, bz, bt) of this handle's tiles."""
        o, z, t = C.c_int(), C.c_int(), C.c_int()
        _check(lib().dwf_get_tile_order(self._h, C.byref(o), C.byref(z), C.byref(t)))
        return o.value, z.value, t.value

    def set_hop_chunk(self, nrhs=1, chunk=1):
        """Consecutive tiles per CTA of the hop before striding by the grid."""
        _check(lib().dwf_set_hop_chunk(self._h, nrhs, chunk))

    def tuning(self, nrhs=1):
        """(tile sites, lanes per thread, chunk, tensor cores) used for this nrhs."""
        v = [C.c_int() for _ in range(4)]
        _check(lib().dwf_get_tuning(self._h, nrhs, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def make_pair(self, r, e, x_star, x_k, stream=None):
        """One training pair of the learned preconditioner (dwf_nn_make_pair):
        e = (x* - x_k)/|x* - x_k|, r = M_pc^+ M_pc e into the FP32 odd cb
        tensors r, e; returns |x* - x_k| (0: nothing written)."""
        n = C.c_double()
        _check(lib().dwf_nn_make_pair(self._h, _ptr(x_star), _ptr(x_k), _ptr(r), _ptr(e), C.byref(n),
                                      _stream(stream)))
        return n.value

    def check_device(self):
        return _check(lib().dwf_check_device(self._h))


class MG:
    """Two-level multigrid preconditioner of A = M_pc^+ M_pc (``dwf_mg``) on a
    handle: blocks (x, y, z, t) extents, nvec near-null vectors."""

    SMOOTHER = {"none": 0, "chebyshev": 1, "nn": 2}

    def __init__(self, h: "Handle", block, nvec):
        m = C.c_void_p()
        _check(lib().dwf_mg_create(C.byref(m), h._h, (C.c_int * 4)(*block), int(nvec)))
        self._m = m
        self.h = h
        self.nvec = int(nvec)
        self.block = tuple(block)
        self._K = None

    def close(self):
        if getattr(self, "_m", None):
            lib().dwf_mg_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, V, stream=None):
        """V: odd cb FP32 field with nvec lanes, shape cb_shape(1, nvec)."""
        _check(lib().dwf_mg_setup(self._m, _ptr(V), _stream(stream)))

    def set_smoother(self, kind="none", steps=0, lo=0.0, hi=0.0, K=None):
        self._K = K
        _check(lib().dwf_mg_set_smoother(self._m, self.SMOOTHER[kind], int(steps), float(lo), float(hi),
                                         K._k if K is not None else None))

    def apply(self, z, r, stream=None):
        _check(lib().dwf_mg_apply(self._m, _ptr(z), _ptr(r), _stream(stream)))
        return z

    def sizes(self):
        nb, nc = C.c_int(), C.c_int()
        _check(lib().dwf_mg_info(self._m, C.byref(nb), C.byref(nc)))
        return nb.value, nc.value

    def restrict(self, f, stream=None):
        nb, nc = self.sizes()
        c = torch.empty((nb, self.nvec, 2), dtype=torch.float64, device="cuda")
        _check(lib().dwf_mg_restrict(self._m, _ptr(c), _ptr(f), _stream(stream)))
        return c

    def prolong(self, c, stream=None):
        f = self.h.empty_cb(1, 1, FP32)
        _check(lib().dwf_mg_prolong(self._m, _ptr(f), _ptr(c), _stream(stream)))
        return f

    def basis(self):
        """Copy of the orthonormal basis: odd cb FP32 field with nvec lanes."""
        out = torch.empty(self.h.cb_shape(1, self.nvec), dtype=torch.float32, device="cuda")
        _check(lib().dwf_mg_copy(self._m, 0, _ptr(out), _stream(None)))
        torch.cuda.synchronize()
        return out

    def coarse_operator(self):
        """A_c = P^+ A P as a complex128 numpy array (nc x nc, (block, k) order)."""
        nb, nc = self.sizes()
        out = torch.empty((nc, nc, 2), dtype=torch.float64, device="cuda")
        _check(lib().dwf_mg_copy(self._m, 1, _ptr(out), _stream(None)))
        torch.cuda.synchronize()
        return torch.view_as_complex(out.cpu()).numpy()


class NN:
    """The learned preconditioner K (``dwf_nn``): 1 -> 16 -> 1 channels."""

    CHANNELS = 16

    def __init__(self, channels=16):
        k = C.c_void_p()
        _check(lib().dwf_nn_create(C.byref(k), channels))
        self._k = k
        self.C = channels
        self.nweights = 2 * 11 * channels * 16

    def close(self):
        if getattr(self, "_k", None):
            lib().dwf_nn_destroy(self._k)
            self._k = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, W1, W2):
        """W1 (11, C, 1, 4, 4) and W2 (11, 1, C, 4, 4) complex numpy arrays."""
        import numpy as np
        w = np.concatenate([np.ascontiguousarray(W1, dtype=np.complex128).reshape(-1),
                            np.ascontiguousarray(W2, dtype=np.complex128).reshape(-1)])
        _check(lib().dwf_nn_set_weights(self._k, w.ctypes.data_as(C.c_void_p), w.size))

    def get_weights(self):
        import numpy as np
        w = np.zeros(self.nweights, dtype=np.complex128)
        _check(lib().dwf_nn_get_weights(self._k, w.ctypes.data_as(C.c_void_p), w.size))
        n1 = 11 * self.C * 16
        return w[:n1].reshape(11, self.C, 1, 4, 4), w[n1:].reshape(11, 1, self.C, 4, 4)

    def apply(self, h, out, inp, nrhs=1, stream=None):
        _check(lib().dwf_nn_apply(self._k, h._h, _ptr(out), _ptr(inp), nrhs, _stream(stream)))
        return out

    LOSS = {"error": 0, "energy": 1, "a2": 2}

    def train_step(self, h, r, e, nrhs=1, lr=1e-3, energy=True, loss_kind=None, stream=None):
        """One Adam step.  loss_kind: "error" |K r - e|^2/|e|^2, "energy"
        (default; energy=False selects "error"), or "a2" |A K r - r|^2/|r|^2."""
        kind = self.LOSS[loss_kind] if loss_kind else (1 if energy else 0)
        loss = C.c_double()
        _check(lib().dwf_nn_train_step(self._k, h._h, _ptr(r), _ptr(e), nrhs, kind, lr,
                                       C.byref(loss), _stream(stream)))
        return loss.value

    def last_grad(self, h):
        import numpy as np
        g = np.zeros(self.nweights, dtype=np.complex128)
        _check(lib().dwf_nn_last_grad(h._h, g.ctypes.data_as(C.c_void_p), g.size))
        n1 = 11 * self.C * 16
        return g[:n1].reshape(11, self.C, 1, 4, 4), g[n1:].reshape(11, 1, self.C, 4, 4)

    def save(self, path):
        """dwf_nn_save: the weights to a file."""
        _check(lib().dwf_nn_save(self._k, os.fsencode(path)))

    def load(self, path):
        """dwf_nn_load: the weights from a file written by save."""
        _check(lib().dwf_nn_load(self._k, os.fsencode(path)))
