"""FP64 oracle of the quality and selection metrics (test infrastructure only: the test-suite,
the package smoke check and the CPU-baseline leg of the benchmark may use it; the product path
never does).

* ``image_metrics``: mean squared error and mean SSIM of image pairs.  Sec. 5.1 names PSNR
  and SSIM as the quality metrics without fixing SSIM's form; the reading here is the
  original one of Wang et al. (2004): an 11 x 11 Gaussian window of standard deviation 1.5
  (weights normalised to sum 1), the weighted (biased) moments, C1 = (0.01 L)^2 and
  C2 = (0.03 L)^2 with dynamic range L = 1, per colour channel over the windows that lie
  inside the image ("valid"), averaged over windows, channels and images.
  PSNR = 10 log10(L^2 / MSE).
* ``kept_mass``: the share of the reference view's alpha weights (Eq. eq_gradient,
  A_d = alpha_d prod_{j>d} (1 - alpha_j), plane D-1 nearest) that a selection keeps,
  summed over all pixels: (sum of A over the kept voxels, sum of A over all voxels).

Parity status: pinned by ``tests/test_oracle_metrics_pins.py`` (closed forms for constant
images, identity and symmetry, a separable Gaussian filter from scipy, the telescoping sum of
the alpha weights, keep-all, and the maximality of the top-k selection).
"""
from __future__ import annotations

import numpy as np

SSIM_RADIUS = 5
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def ssim_window() -> np.ndarray:
    """The 11 x 11 Gaussian window (sigma 1.5), normalised to sum 1, FP64."""
    r = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    g = np.exp(-(r * r) / (2.0 * SSIM_SIGMA * SSIM_SIGMA))
    w = np.outer(g, g)
    return w / w.sum()


def _window_sums(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_{i,j} w[i][j] img[y + i][x + j] for every window inside img [H][W] (valid)."""
    n = w.shape[0]
    H, W = img.shape
    out = np.zeros((H - n + 1, W - n + 1), dtype=np.float64)
    for i in range(n):
        for j in range(n):
            out += w[i, j] * img[i:i + H - n + 1, j:j + W - n + 1]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM of every valid window of two single-channel images [H][W] (FP64)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = ssim_window()
    mx, my = _window_sums(x, w), _window_sums(y, w)
    sxx = _window_sums(x * x, w) - mx * mx
    syy = _window_sums(y * y, w) - my * my
    sxy = _window_sums(x * y, w) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def image_metrics(x, y) -> tuple[float, float]:
    """(MSE, mean SSIM) of image stacks x, y [N][H][W][3] with values in [0, 1]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.shape != y.shape or x.ndim != 4 or x.shape[3] != 3:
        raise ValueError("x and y must both be [N][H][W][3]")
    mse = float(np.mean((x - y) ** 2))
    vals = [ssim_map(x[n, :, :, c], y[n, :, :, c]).mean() for n in range(x.shape[0]) for c in range(3)]
    return mse, float(np.mean(vals))


def psnr(mse: float) -> float:
    """PSNR in dB for dynamic range 1."""
    return float(10.0 * np.log10(1.0 / mse))


def kept_mass(M, mask) -> tuple[float, float]:
    """(sum of A over the voxels whose plane bit is set in mask [H][W], sum of A over all voxels),
    A from the oracle's alpha weights (Eq. eq_gradient)."""
    from . import alpha_weights
    A = np.asarray(alpha_weights(M), np.float64)
    D = A.shape[0]
    m = np.ascontiguousarray(mask)
    m = m.view(np.uint64) if m.dtype == np.int64 else m.astype(np.uint64)
    bits = np.stack([((m >> np.uint64(d)) & np.uint64(1)).astype(bool) for d in range(D)])
    return float(A[bits].sum()), float(A.sum())
