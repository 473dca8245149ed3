"""The DWF_DEBUG build (libdwf_debug.so): its range check against the
driver's allocation ranges, and that a sequence of entry points through the
checks gives bit-identical results to the release library (no false
refusals, no change to the arithmetic).  Run in child processes: DWF_DEBUG=1
selects the debug library at import, PYTORCH_NO_CUDA_MEMORY_CACHING=1 makes
every tensor its own allocation.  An entry point handed an undersized buffer
is not exercised here: were the check broken, its kernel would overrun the
buffer on the GPU; the check itself is what is tested."""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes as C, json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2203_17119_gb300 import dwf as G, inputs
out = {}
L = G.lib()
on = C.c_int(-1)
assert L.dwf_debug_build(C.byref(on)) == 0
out["debug"] = on.value
if on.value:
    t = torch.zeros(4096, dtype=torch.float64, device="cuda")
    nb = t.numel() * 8
    out["range_ok"] = L.dwf_check_range(C.c_void_p(t.data_ptr()), nb)
    out["range_over"] = L.dwf_check_range(C.c_void_p(t.data_ptr()), nb + 8)
    out["range_offset"] = L.dwf_check_range(C.c_void_p(t.data_ptr() + 64), nb)
    host = np.zeros(16)
    out["range_host"] = L.dwf_check_range(C.c_void_p(host.ctypes.data), 128)
    out["range_null"] = L.dwf_check_range(None, 8)
dims, Ls = (4, 4, 4, 4), 4
rng = np.random.default_rng(3)
U = inputs.gauge_field(dims, "haar", rng=rng)
h = G.Handle(dims, Ls, G.Action(1.8, 0.05, 1.5, 0.5))
h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
full = h.pack(torch.from_numpy(inputs.gaussian_source(dims, Ls, rng=rng).reshape(-1)).cuda())
b = full[h.nsite[0]:].contiguous()
y = torch.empty_like(b)
h.mpc(y, b)
z = torch.empty_like(full)
h.apply_d(z, full)
x = torch.zeros_like(full)
st = h.cgne_solve(x, full, tol=1e-10)
F = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
h.force(F, full, z)
out["mpc"] = y.cpu().numpy().tobytes().hex()
out["apply_d"] = z.cpu().numpy().tobytes().hex()
out["solve"] = x.cpu().numpy().tobytes().hex()
out["force"] = F.cpu().numpy().tobytes().hex()
print("RESULT " + json.dumps(out))
'''


def _child(debug):
    env = dict(os.environ, PYTORCH_NO_CUDA_MEMORY_CACHING="1", DWF_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    import json
    return json.loads(line[len("RESULT "):])


@pytest.fixture(scope="module")
def runs():
    from paper_2203_17119_gb300 import build
    build.build(debug=True)
    return _child(True), _child(False)


def test_range_check(runs):
    dbg, rel = runs
    assert dbg["debug"] == 1 and rel["debug"] == 0
    assert dbg["range_ok"] == 0
    for k in ("range_over", "range_offset", "range_host", "range_null"):
        assert dbg[k] == 1, k          # DWF_ERR_ARG


def test_debug_build_results_are_identical(runs):
    dbg, rel = runs
    for k in ("mpc", "apply_d", "solve", "force"):
        assert dbg[k] == rel[k], k
