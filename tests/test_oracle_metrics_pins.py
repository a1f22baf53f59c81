"""Pins of the metric oracle (oracle/metrics.py) against closed forms, a library filter and
invariants, so that a dropped term, a wrong sign or a misplaced index in it fails a test.

SSIM (Wang et al. 2004 form, Sec. 5.1's quality metric):
* the window equals scipy's separable Gaussian filter (sigma 1.5, radius 5), and the whole
  SSIM map equals one built from scipy.ndimage.gaussian_filter moments;
* constant images a, b give (2ab + C1) / (a^2 + b^2 + C1) in every window;
* ssim(x, x) = 1, symmetry, a brightness shift keeps only the luminance term, and an inverted
  image gives the closed-form contrast-structure term (C2 - 2 s^2) / (2 s^2 + C2);
* MSE / PSNR of a constant offset.
Kept mass (Eq. eq_gradient's alpha weights):
* keep-all equals the telescoping sum 1 - prod(1 - alpha) per pixel, an empty mask gives 0,
  an opaque plane carries all the weight, and the top-k selection keeps at least as much mass
  as any other k planes.
"""
import numpy as np
import pytest

import oracle
from oracle import metrics as om

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def _gauss_moments(x, y):
    f = lambda a: scipy_ndimage.gaussian_filter(a, sigma=om.SSIM_SIGMA, radius=om.SSIM_RADIUS, mode="constant")
    r = om.SSIM_RADIUS
    crop = lambda a: a[r:a.shape[0] - r, r:a.shape[1] - r]
    mx, my = crop(f(x)), crop(f(y))
    return mx, my, crop(f(x * x)) - mx * mx, crop(f(y * y)) - my * my, crop(f(x * y)) - mx * my


def test_window_is_the_separable_gaussian():
    w = om.ssim_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    delta = np.zeros((11, 11))
    delta[5, 5] = 1.0
    ref = scipy_ndimage.gaussian_filter(delta, sigma=1.5, radius=5, mode="constant")
    assert np.abs(w - ref).max() < 1e-16


def test_ssim_map_equals_one_from_a_library_filter():
    rng = np.random.default_rng(3)
    x = rng.random((29, 37))
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1)
    mx, my, sxx, syy, sxy = _gauss_moments(x, y)
    want = ((2 * mx * my + om.SSIM_C1) * (2 * sxy + om.SSIM_C2)) / (
        (mx ** 2 + my ** 2 + om.SSIM_C1) * (sxx + syy + om.SSIM_C2))
    got = om.ssim_map(x, y)
    assert got.shape == (19, 27)
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("a,b", [(0.2, 0.7), (0.0, 1.0), (0.5, 0.5), (0.9, 0.1)])
def test_constant_images_closed_form(a, b):
    x = np.full((13, 16), a)
    y = np.full((13, 16), b)
    want = (2 * a * b + om.SSIM_C1) / (a * a + b * b + om.SSIM_C1)
    assert np.abs(om.ssim_map(x, y) - want).max() < 1e-12


def test_identity_symmetry_shift_and_inversion():
    rng = np.random.default_rng(5)
    x = rng.random((24, 31)) * 0.6 + 0.2
    y = rng.random((24, 31))
    assert np.abs(om.ssim_map(x, x) - 1.0).max() < 1e-12
    assert np.abs(om.ssim_map(x, y) - om.ssim_map(y, x)).max() < 1e-13
    # brightness shift: contrast-structure term is 1, the luminance term remains
    c = 0.15
    mx = _gauss_moments(x, x)[0]
    want = (2 * mx * (mx + c) + om.SSIM_C1) / (mx ** 2 + (mx + c) ** 2 + om.SSIM_C1)
    assert np.abs(om.ssim_map(x, x + c) - want).max() < 1e-12
    # inversion y = 1 - x: s_xy = -s_x^2, s_y^2 = s_x^2
    mx, _, sxx, _, _ = _gauss_moments(x, 1 - x)
    lum = (2 * mx * (1 - mx) + om.SSIM_C1) / (mx ** 2 + (1 - mx) ** 2 + om.SSIM_C1)
    cs = (om.SSIM_C2 - 2 * sxx) / (2 * sxx + om.SSIM_C2)
    assert np.abs(om.ssim_map(x, 1 - x) - lum * cs).max() < 1e-12


def test_mse_and_psnr_of_an_offset():
    rng = np.random.default_rng(7)
    x = rng.random((2, 16, 20, 3)) * 0.5
    mse, s = om.image_metrics(x, x + 0.01)
    assert abs(mse - 1e-4) < 1e-15
    assert abs(om.psnr(mse) - 40.0) < 1e-9
    mse0, s0 = om.image_metrics(x, x)
    assert mse0 == 0.0 and abs(s0 - 1.0) < 1e-12
    # image_metrics averages the per-channel maps
    y = np.clip(x + 0.05 * rng.standard_normal(x.shape), 0, 1)
    per = [om.ssim_map(x[n, :, :, c], y[n, :, :, c]).mean() for n in range(2) for c in range(3)]
    assert abs(om.image_metrics(x, y)[1] - np.mean(per)) < 1e-15


def _mpi(rng, D, H, W):
    M = rng.random((D, H, W, 4))
    M[..., 3] = np.where(rng.random((D, H, W)) < 0.3, 0.0, M[..., 3])
    return M


def test_kept_mass_keep_all_is_the_telescoping_sum():
    rng = np.random.default_rng(9)
    M = _mpi(rng, 7, 5, 6)
    full = np.full((5, 6), (1 << 7) - 1, dtype=np.int64)
    kept, total = om.kept_mass(M, full)
    want = np.sum(1.0 - np.prod(1.0 - M[..., 3], axis=0))
    assert abs(kept - want) < 1e-12 and abs(total - want) < 1e-12
    assert om.kept_mass(M, np.zeros((5, 6), dtype=np.int64))[0] == 0.0


def test_kept_mass_of_an_opaque_plane():
    D, H, W, d0 = 6, 4, 5, 2
    M = np.zeros((D, H, W, 4))
    M[d0, ..., 3] = 1.0
    M[:d0, ..., 3] = 0.8  # behind the opaque plane: no weight
    kept, total = om.kept_mass(M, np.full((H, W), 1 << d0, dtype=np.int64))
    assert kept == H * W and total == H * W
    kept, _ = om.kept_mass(M, np.full((H, W), 1 << (d0 - 1), dtype=np.int64))
    assert kept == 0.0


def test_top_k_keeps_the_most_mass():
    rng = np.random.default_rng(11)
    D, H, W, k = 9, 6, 7, 3
    M = _mpi(rng, D, H, W)
    A = oracle.alpha_weights(M)
    _, mask = oracle.select_topk(A, k)
    best, total = om.kept_mass(M, mask)
    for _ in range(20):
        other = np.zeros((H, W), dtype=np.int64)
        for y in range(H):
            for x in range(W):
                for d in rng.choice(D, k, replace=False):
                    other[y, x] |= 1 << int(d)
        assert om.kept_mass(M, other)[0] <= best + 1e-12
    assert 0.0 < best <= total
