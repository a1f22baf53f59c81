"""Host-side logic of the serving engine (no GPU): the device-memory arena allocator."""
import pytest

from paper_2307_03017_gb300.serve import DeviceArena, _align


def test_arena_first_fit_release_and_merge():
    a = DeviceArena(10_000, "cpu")
    o1 = a.alloc(1000)
    o2 = a.alloc(3000)
    o3 = a.alloc(500)
    assert (o1, o2, o3) == (0, _align(1000), _align(1000) + _align(3000))
    assert all(o % 256 == 0 for o in (o1, o2, o3))
    a.release(o2, 3000)
    assert a.alloc(2000) == o2  # first fit reuses the hole
    a.release(o2, 2000)
    a.release(o1, 1000)
    a.release(o3, 500)
    assert a.free == [(0, a.size)]  # fully merged back
    assert a.alloc(a.size + 1) is None
    assert a.can_alloc(a.size) and not a.can_alloc(a.size + 256)


def test_arena_views_are_aligned_typed_windows():
    import torch
    a = DeviceArena(1 << 16, "cpu")
    off = a.alloc(4096)
    v = a.view(off, (8, 16), torch.float32)
    v.fill_(2.0)
    assert v.shape == (8, 16) and float(a.buf[off:off + 4].view(torch.float32)[0]) == 2.0
