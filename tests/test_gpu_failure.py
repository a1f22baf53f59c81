"""Failure detection on the GPU without a fault: a bounded device wait that nothing completes
gives up after its limit, the host reads the timeout through the device status word, and the
context stays usable (a render launched afterwards still matches the FP64 oracle)."""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import paper_2307_03017_gb300 as rl
    rl._lib.lib()
    assert rl.reallife_device_status(clear=True) == 0  # starts clean
    rl.reallife_selftest_wait_timeout(2000)  # 2 ms on a barrier nothing completes
    with pytest.raises(rl.RealLifeError, match="timed out"):
        rl.reallife_device_status(clear=True)
    assert rl.reallife_device_status(clear=True) == 0  # the word was cleared
    sc = sg.make_scene(3, 16, 24, 4, 2, n_layers=(1, 2))
    m = rl.make_mpi(torch.from_numpy(sc.coarse_mpi).cuda(), sc.near, sc.far, sc.ref)
    out = rl.reallife_render(m, sc.src).cpu().numpy()
    for j, cam in enumerate(sc.src):
        ref = oracle.render(sc.coarse_mpi, sc.near, sc.far, sc.ref, cam)
        assert np.abs(out[j] - ref).max() <= 1e-5
    assert rl.reallife_device_status(clear=True) == 0


def test_selftest_rejects_bad_limits():
    import paper_2307_03017_gb300 as rl
    for us in (0, 2_000_000):
        with pytest.raises(rl.RealLifeError):
            rl.reallife_selftest_wait_timeout(us)
