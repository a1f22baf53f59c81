"""GPU parity of the metric kernels (metrics.cu) against the FP64 metric oracle.

* MSE and mean SSIM of image pairs: random and rendered images, a ragged size that spans
  several 16 x 16 window tiles, the smallest valid size (11 x 11), identical images;
  MSE within 1e-6 relative, mean SSIM within 1e-5 absolute (FP32 windows, FP64 sums).
* Kept mass of the GPU's own selection on FP32 and BF16 MPIs, and of a keep-all mask:
  both sums within 1e-6 relative of the oracle (the oracle is given the BF16-rounded MPI).
* Both calls are deterministic (fixed reduction order): repeated calls agree bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from oracle import metrics as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    import paper_2307_03017_gb300 as rl
    rl._lib.lib()
    yield rl


def _pair(rng, N, H, W):
    x = rng.random((N, H, W, 3)).astype(np.float32)
    # smooth structure plus noise so that windows have both flat and textured parts
    yy, xx = np.mgrid[0:H, 0:W]
    base = 0.5 + 0.4 * np.sin(xx / 5.0)[..., None] * np.cos(yy / 7.0)[..., None]
    x = (0.5 * x + 0.5 * base[None]).astype(np.float32)
    y = np.clip(x + 0.05 * rng.standard_normal(x.shape), 0, 1).astype(np.float32)
    return x, y


@pytest.mark.parametrize("shape", [(2, 37, 53), (1, 11, 11), (3, 64, 48)])
def test_image_metrics_match_oracle(rl, shape):
    rng = np.random.default_rng(sum(shape))
    x, y = _pair(rng, *shape)
    out = rl.reallife_image_metrics(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
    mse, ssim = om.image_metrics(x, y)
    assert abs(out[0] - mse) <= 1e-6 * mse
    assert abs(out[1] - ssim) <= 1e-5


def test_image_metrics_of_rendered_views(rl):
    sc = sg.workload("small", 0)[0]
    M = torch.from_numpy(sc.coarse_mpi).cuda().contiguous()
    m = rl.make_mpi(M, sc.near, sc.far, sc.ref)
    r = rl.reallife_render(m, sc.novel)
    truth = np.stack([sg.raycast(sc.layers, sc.ref.K, c, sc.H, sc.W)[0] for c in sc.novel]).astype(np.float32)
    gt = torch.from_numpy(truth).cuda()
    out = rl.reallife_image_metrics(r, gt).cpu().numpy()
    mse, ssim = om.image_metrics(r.cpu().numpy(), truth)
    assert abs(out[0] - mse) <= 1e-6 * mse
    assert abs(out[1] - ssim) <= 1e-5
    again = rl.reallife_image_metrics(r, gt).cpu().numpy()
    assert np.array_equal(out, again)


def test_identical_images(rl):
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.random((1, 20, 30, 3)).astype(np.float32)).cuda()
    out = rl.reallife_image_metrics(x, x.clone()).cpu().numpy()
    assert out[0] == 0.0
    assert abs(out[1] - 1.0) <= 1e-6


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_kept_mass_matches_oracle(rl, dtype):
    sc = sg.workload("small", 0)[0]
    M = torch.from_numpy(sc.coarse_mpi).cuda().to(dtype).contiguous()
    m = rl.make_mpi(M, sc.near, sc.far, sc.ref)
    k = 3
    _, mask = rl.reallife_select(m, k)
    out = rl.reallife_kept_mass(m, mask).cpu().numpy()
    Mo = M.float().cpu().numpy()
    kept, total = om.kept_mass(Mo, mask.cpu().numpy())
    assert abs(out[0] - kept) <= 1e-6 * kept
    assert abs(out[1] - total) <= 1e-6 * total
    assert 0.0 < out[0] <= out[1]
    full = torch.full_like(mask, (1 << sc.D) - 1)
    both = rl.reallife_kept_mass(m, full).cpu().numpy()
    assert both[0] == both[1] and abs(both[1] - total) <= 1e-6 * total
    assert np.array_equal(rl.reallife_kept_mass(m, mask).cpu().numpy(), out)


def test_kept_mass_on_the_paper_scene(rl):
    sc = sg.workload("paper", 0)[0]
    M = torch.from_numpy(sc.coarse_mpi).cuda().contiguous()
    m = rl.make_mpi(M, sc.near, sc.far, sc.ref)
    _, mask = rl.reallife_select(m, 5)
    out = rl.reallife_kept_mass(m, mask).cpu().numpy()
    kept, total = om.kept_mass(sc.coarse_mpi, mask.cpu().numpy())
    assert abs(out[0] - kept) <= 1e-6 * kept
    assert abs(out[1] - total) <= 1e-6 * total
