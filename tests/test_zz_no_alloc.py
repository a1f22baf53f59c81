"""The fixed-scratch HSGD step, for callers that cannot allocate device memory (a plugin
whose host application owns the GPU heap, a frame loop that must not call cudaMalloc).

It is checked through the C ABI against the workspace entry point on the same inputs,
for two calls in a row, and for its size limit.  The file sorts last so that a run that
stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def test_noalloc_step_matches_workspace_step_on_two_calls():
    import paper_2307_03017_gb300 as rl
    sc = sg.workload("small", 3)[0]
    k = 5
    images = torch.from_numpy(sc.images).cuda()
    A = torch.from_numpy(sc.coarse_mpi).cuda().contiguous()
    B = A.clone()
    ma = rl.make_mpi(A, sc.near, sc.far, sc.ref)
    mb = rl.make_mpi(B, sc.near, sc.far, sc.ref)
    ws = rl.workspace(len(sc.src), sc.D, sc.H, sc.W, k)
    for call, level in enumerate((1, 0)):
        if call:
            B.copy_(A)  # both calls of the pair start from the same MPI
        h, w = sc.H >> level, sc.W >> level
        la, lb = torch.empty(1, device="cuda"), torch.empty(1, device="cuda")
        Sa = torch.empty((k, h, w), dtype=torch.uint8, device="cuda")
        Sb = torch.empty_like(Sa)
        rl.reallife_hsgd_step(ma, images, sc.src, k, level=level, loss_out=la, S_out=Sa, ws=ws)
        rl.reallife_hsgd_step_noalloc(mb, images, sc.src, k, level=level, loss_out=lb, S_out=Sb)
        torch.cuda.synchronize()
        assert torch.equal(Sa, Sb), f"call {call}: selections differ"
        err = (A - B).abs().max().item()
        assert err <= TOL32, f"call {call}: MPIs differ by {err}"
        assert abs(la.item() - lb.item()) <= 1e-5 * abs(la.item()), f"call {call}: losses differ"
        assert err < 1.0 and (A != torch.from_numpy(sc.coarse_mpi).cuda()).any()  # the step did change M


def test_noalloc_step_rejects_problems_beyond_its_scratch():
    import paper_2307_03017_gb300 as rl
    from paper_2307_03017_gb300 import _lib
    lib = _lib.lib()
    small = torch.zeros((1, 16, 16, 4), dtype=torch.float32, device="cuda")
    m = _lib.RlMpi()
    m.D, m.H, m.W, m.near_, m.far_, m.dtype = 64, 1024, 2048, 1.0, 100.0, 0
    m.data = ctypes.c_void_p(small.data_ptr())
    m.ref = _lib.camera(sg.Camera(sg.intrinsics(2048, 1024), np.eye(3), np.zeros(3)))
    cams = _lib.cameras([sg.Camera(sg.intrinsics(2048, 1024), np.eye(3), np.zeros(3))])
    P = _lib.RlHsgdParams()
    P.k, P.lambda_, P.clamp01, P.level = 5, 1.0, 1, 0
    st = lib.reallife_hsgd_step_noalloc(ctypes.byref(m), ctypes.c_void_p(small.data_ptr()), cams, 1,
                                        ctypes.byref(P), None, None, None)
    assert st == 2  # RL_ENOMEM, nothing launched
    assert b"fixed scratch" in lib.reallife_last_error()
    need = rl.reallife_workspace_bytes(1, 64, 1024, 2048, 5)
    assert need > (64 << 20)
