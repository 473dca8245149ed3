"""dwf_mpc_noalloc: the Schur operator for callers that may not allocate
device memory when they apply it (a framework pool that owns all device
memory, a fixed-footprint embedding).  Its temporaries live in the library's
static device array, so it must give the same result as dwf_mpc, call after
call, allocate nothing, and refuse problems that do not fit.  This file is
collected last on purpose."""

import numpy as np
import pytest

from paper_2203_17119_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402

TOL = {G.FP64: 1e-12, G.FP32: 2e-6, G.BF16: 1.5e-2}


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("prec", [G.FP64, G.FP32, G.BF16])
def test_noalloc_matches_mpc_twice(prec):
    dims, Ls, nrhs = (4, 4, 4, 8), 8, 2
    U = inputs.gauge_field(dims, "exp", eps=0.3, seed=77)
    h = G.Handle(dims, Ls, G.Action(1.8, 0.01, 1.5, 0.5), nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    gen = torch.Generator(device="cuda").manual_seed(5)
    for call in range(2):          # two calls in a row share the scratch array
        for dagger in (False, True):
            x = torch.randn(h.cb_shape(1, nrhs), device="cuda", generator=gen).to(G._DTYPE[prec])
            ref = h.empty_cb(1, nrhs, prec)
            got = h.empty_cb(1, nrhs, prec)
            h.mpc(ref, x, dagger, prec, nrhs)
            h.mpc_noalloc(got, x, dagger, prec, nrhs)
            torch.cuda.synchronize()
            assert _rel(got, ref) <= TOL[prec], (call, dagger)


def test_noalloc_rejects_oversize():
    dims, Ls = (16, 16, 16, 16), 16      # 32768 sites x 12 x 16 x 16 B > 32 MiB
    U = inputs.gauge_field(dims, "unit")
    h = G.Handle(dims, Ls, G.Action(1.8, 0.01, 1.5, 0.5))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    x = h.empty_cb(1, 1, G.FP64)
    y = h.empty_cb(1, 1, G.FP64)
    with pytest.raises(G.DWFError) as e:
        h.mpc_noalloc(y, x, prec=G.FP64)
    assert e.value.status == 1 and "static scratch" in str(e.value)


def test_noalloc_allocates_nothing():
    """On a fresh handle, right after dwf_autotune, calls of dwf_mpc_noalloc
    make no device allocation: the library's allocation count and the free
    device memory stay where they were."""
    dims, Ls, nrhs = (8, 8, 8, 8), 8, 1
    U = inputs.gauge_field(dims, "exp", eps=0.3, seed=78)
    h = G.Handle(dims, Ls, G.Action(1.8, 0.01, 1.5, 0.5), nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    h.autotune(nrhs, G.FP32)
    x = torch.randn(h.cb_shape(1, nrhs), device="cuda")
    y = h.empty_cb(1, nrhs, G.FP32)
    h.mpc_noalloc(y, x, False, G.FP32, nrhs)    # first call on the device: symbol look-up
    torch.cuda.synchronize()
    n0 = G.alloc_count()
    free0 = torch.cuda.mem_get_info()[0]
    for dagger in (False, True, False):
        h.mpc_noalloc(y, x, dagger, G.FP32, nrhs)
    torch.cuda.synchronize()
    assert G.alloc_count() == n0
    assert torch.cuda.mem_get_info()[0] == free0
