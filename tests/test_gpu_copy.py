"""dwf_copy: host <-> device copies with the GPU's own loads and stores.
Bit-exact against the source in all three directions (pinned host to device,
device to pinned host, device to device), at sizes that are not a multiple of
the grid; refused, before any launch, for pageable host memory, misaligned
pointers and sizes that are not a multiple of 16 bytes."""

import ctypes as C

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2203_17119_gb300 import dwf as G  # noqa: E402


@pytest.mark.parametrize("n", [2, 1000, 3 * 1024 * 1024 + 6])
def test_copies_are_exact(n):
    g = torch.Generator().manual_seed(n)
    host = torch.randn(n, dtype=torch.float64, generator=g).pin_memory()
    dev = torch.empty(n, dtype=torch.float64, device="cuda")
    G.copy(dev, host)
    back = torch.empty(n, dtype=torch.float64).pin_memory()
    G.copy(back, dev)
    dev2 = torch.empty_like(dev)
    G.copy(dev2, dev)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)
    assert torch.equal(back, host)
    assert torch.equal(dev2, dev)


def test_refusals():
    n0 = G.launch_count()
    dev = torch.zeros(64, dtype=torch.float64, device="cuda")
    pageable = torch.zeros(64, dtype=torch.float64)
    with pytest.raises(G.DWFError, match="page-locked"):
        G.copy(dev, pageable)
    with pytest.raises(G.DWFError, match="page-locked"):
        G.copy(pageable, dev)
    L = G.lib()
    assert L.dwf_copy(C.c_void_p(dev.data_ptr() + 8), C.c_void_p(dev.data_ptr() + 256), 64, None) == 1
    assert L.dwf_copy(C.c_void_p(dev.data_ptr()), C.c_void_p(dev.data_ptr() + 256), 24, None) == 1
    assert L.dwf_copy(None, C.c_void_p(dev.data_ptr()), 16, None) == 1
    torch.cuda.synchronize()
    assert G.launch_count() == n0
