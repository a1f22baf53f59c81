"""The bounds-checked debug build (-DRL_DEBUG) and the slot cap of caller-supplied masks.

* The release library compiles the checks out: its bounds self-test reports RL_ENOTIMPL.
* The debug library's self-test sets the bounds bit (4) of the device status word without a
  fault; reallife_device_status then reports RL_EBOUNDS, and the context stays usable.
* The small-shape GPU parity, batch and volume suites run under the debug library with no
  check tripped (a child pytest with REALLIFE_DEBUG=1; conftest.py checks the bounds bit
  after every GPU test there).
* A mask with more than k bits in a pixel keeps its k lowest planes (the compact gradient of
  Sec. 3.3 holds k slots): the gradient equals the oracle's dense gradient at those planes.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEBUG = os.environ.get("REALLIFE_DEBUG", "0") not in ("", "0")


@pytest.fixture(scope="module")
def rl():
    import paper_2307_03017_gb300 as rl
    rl._lib.lib()
    rl.reallife_set_kernel_path(0)
    yield rl


def test_loss_grad_mask_with_more_than_k_bits_keeps_the_k_lowest(rl):
    sc = sg.workload("small", 0)[0]
    D, H, W, k = sc.D, sc.H, sc.W, 3
    rng = np.random.default_rng(11)
    # k + 2 distinct planes per pixel
    bits = np.argsort(rng.random((H, W, D)), axis=-1)[..., :k + 2]
    mask = np.zeros((H, W), dtype=np.int64)
    for j in range(k + 2):
        mask |= np.left_shift(np.int64(1), bits[..., j].astype(np.int64))
    low = np.sort(bits, axis=-1)[..., :k]  # [H][W][k]
    M = torch.from_numpy(sc.coarse_mpi).cuda().contiguous()
    m = rl.make_mpi(M, sc.near, sc.far, sc.ref)
    _, G = rl.reallife_loss_grad(m, torch.from_numpy(sc.images).cuda(), sc.src,
                                 mask=torch.from_numpy(mask).cuda(), k=k)
    _, g_o, _ = oracle.loss_grad(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images)
    want = np.take_along_axis(g_o, np.transpose(low, (2, 0, 1))[..., None], axis=0)  # [k][H][W][4]
    assert np.abs(G.cpu().numpy() - want).max() <= 1e-5


@pytest.mark.skipif(DEBUG, reason="release-build behaviour")
def test_release_build_has_no_bounds_checks(rl):
    assert not rl.reallife_debug_build()
    with pytest.raises(rl.RealLifeError, match="debug build"):
        rl.reallife_selftest_bounds()


@pytest.mark.skipif(not DEBUG, reason="runs in the child pytest under REALLIFE_DEBUG=1")
@pytest.mark.trips_bounds
def test_debug_selftest_sets_the_bounds_bit(rl):
    assert rl.reallife_debug_build()
    assert rl.reallife_device_status(clear=True) == 0
    rl.reallife_selftest_bounds()
    with pytest.raises(rl.RealLifeError, match="bounds check"):
        rl.reallife_device_status(clear=False)
    with pytest.raises(rl.RealLifeError, match="bounds check"):
        rl.reallife_device_status(clear=True)  # reports once more, and clears
    assert rl.reallife_device_status(clear=True) == 0
    x = torch.arange(8, device="cuda", dtype=torch.float32)
    assert float((x * 2).sum()) == 56.0  # the context is usable


@pytest.mark.skipif(DEBUG, reason="this is the parent of the debug run")
def test_small_gpu_suites_under_the_debug_build():
    from paper_2307_03017_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, REALLIFE_DEBUG="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py", "tests/test_gpu_batch.py", "tests/test_gpu_volume.py",
           "tests/test_gpu_debug.py", "-k", "not paper and not display"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = r.stdout[-3000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout.splitlines()[-1], tail
