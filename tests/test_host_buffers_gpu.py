"""Page-locked host buffers of isis_host_alloc: pinned, zero-filled, huge-page aligned when large enough, and
a round trip through the device by asynchronous copies returns what was written."""
import ctypes
import gc

import pytest
import torch

from paper_1307_6748_gb300 import isis

pytestmark = pytest.mark.gpu


def _page_locked(ptr: int) -> bool:
    """The runtime's view: cudaPointerGetAttributes gives cudaMemoryTypeHost (1) for page-locked (allocated or
    registered) host memory, cudaMemoryTypeUnregistered (0) for pageable memory.  (torch's is_pinned() knows
    only its own allocator's blocks.)"""
    isis.load()  # maps the CUDA runtime the library links
    rt = None
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    assert rt is not None
    attr = (ctypes.c_int * 64)()  # the attribute struct begins with its memory type (an enum), room to spare
    assert rt.cudaPointerGetAttributes(ctypes.byref(attr), ctypes.c_void_p(ptr)) == 0
    return attr[0] == 1


def _thp_size():
    try:
        with open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size") as f:
            return int(f.read().strip())
    except (OSError, ValueError):
        return 0


@pytest.mark.parametrize("n", [1000, 1 << 27])
def test_host_empty_round_trip(n):
    t = isis.host_empty(n)
    assert t.numel() == n and t.dtype == torch.float32
    assert _page_locked(t.data_ptr())
    assert not _page_locked(torch.empty(n, dtype=torch.float32).data_ptr())
    assert int(t.abs().max()) == 0
    hp = _thp_size()
    if hp and n * 4 >= hp:
        assert t.data_ptr() % hp == 0
    src = torch.arange(n, dtype=torch.float32) * 0.5
    t.copy_(src)
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    back = isis.host_empty(n)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d.copy_(t, non_blocking=True)
        d.mul_(2.0)
        back.copy_(d, non_blocking=True)
    s.synchronize()
    assert torch.equal(back, src * 2.0)
    del t, back
    gc.collect()


def test_host_free_twice_is_rejected():
    L = isis.load()
    p = ctypes.c_void_p()
    assert L.isis_host_alloc(4096, ctypes.byref(p)) == isis.ISIS_OK
    assert p.value
    assert L.isis_host_free(p) == isis.ISIS_OK
    assert L.isis_host_free(p) == isis.ISIS_EINVAL
