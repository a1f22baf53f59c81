"""Host-side logic of the serving engine (no GPU): the device-memory arena allocator."""
import pytest

from paper_2307_03017_gb300.serve import DeviceArena, Request, _align, reject_oversized, request_bytes


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


def test_oversized_requests_are_rejected_and_the_rest_kept():
    import numpy as np
    import torch
    import scenegen as sg
    cam = sg.Camera(sg.intrinsics(64, 48), np.eye(3), np.zeros(3))

    def req(i, H, W, D):
        return Request(id=i, arrival=0.01 * i, coarse=torch.zeros((D, H, W, 4)), images=torch.zeros((2, H, W, 3)),
                       ref=cam, src=[cam, cam], near=1.0, far=10.0, schedule=(2, 1, 0))

    small = request_bytes(8, 48, 64, 2, 5, torch.float32)
    big = request_bytes(32, 384, 512, 2, 5, torch.float32)
    arena = small * 4
    assert big > arena
    reqs = [req(0, 48, 64, 8), req(1, 384, 512, 32), req(2, 48, 64, 8)]
    rejected, fits = reject_oversized(reqs, arena)
    assert [r.id for r in rejected] == [1] and [r.id for r in fits] == [0, 2]
    assert rejected[0].error and rejected[0].t_done == rejected[0].arrival
    assert all(r.error is None for r in fits)
