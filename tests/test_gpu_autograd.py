"""Differentiation workload: 512x384, D=32, 4 views, BF16 MPI storage, FP32 accumulation.

The hand-written forward/backward of warp + composite, exposed as a torch.autograd.Function,
is checked against central finite differences (step 1e-3, FP64 oracle evaluations at the
BF16-rounded values) on 64 seeded MPI entries and against the FP64 oracle gradient; dense
and sparse-mask HSGD are compared at 2 and 3 iterations.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    return sg.make_scene(0, 384, 512, 32, 4, n_layers=(3, 8), render_novel_gt=True)


@pytest.fixture(scope="module")
def rl():
    import paper_2307_03017_gb300 as rl
    rl._lib.lib()
    return rl


def _project(cam, X):
    x = cam.R @ X + cam.t
    u = cam.K @ x
    return u[:2] / u[2]


def _windowed_loss(M64, sc, views, d, y, x, rho, rad=3):
    """1/(2N) sum |render - I|^2 over the view pixels whose samples can touch voxel (d, y, x)."""
    Kinv = np.linalg.inv(sc.ref.K)
    X = (1.0 / rho[d]) * (Kinv @ np.array([x, y, 1.0]))
    L = 0.0
    for i, cam in enumerate(views):
        q = _project(cam, X)
        xs = np.arange(int(np.floor(q[0])) - rad, int(np.floor(q[0])) + rad + 2)
        ys = np.arange(int(np.floor(q[1])) - rad, int(np.floor(q[1])) + rad + 2)
        xs, ys = xs[(xs >= 0) & (xs < sc.W)], ys[(ys >= 0) & (ys < sc.H)]
        if len(xs) == 0 or len(ys) == 0:
            continue
        gx, gy = np.meshgrid(xs, ys)
        gx, gy = gx.ravel(), gy.ravel()
        out = oracle.render_pixels(M64, sc.near, sc.far, sc.ref, cam, gx, gy)
        L += np.sum((out - sc.images[i][gy, gx].astype(np.float64)) ** 2)
    return L / (2 * len(views))


def test_autograd_bf16_matches_finite_differences_and_oracle(rl, scene):
    from paper_2307_03017_gb300.autograd import warp_composite
    sc = scene
    N = len(sc.src)
    M = torch.from_numpy(sc.coarse_mpi).cuda().to(torch.bfloat16).requires_grad_(True)
    I = torch.from_numpy(sc.images).cuda()
    out = warp_composite(M, sc.near, sc.far, sc.ref, sc.src)
    loss = 0.5 / N * ((out - I) ** 2).sum()
    loss.backward()
    assert M.grad is not None and M.grad.dtype == torch.bfloat16

    # FP32 gradient of the same backward kernel (BF16 storage, FP32 accumulation)
    m = rl.make_mpi(M.detach().contiguous(), sc.near, sc.far, sc.ref)
    g32 = rl.reallife_render_backward(m, sc.src, ((out.detach() - I) / N).contiguous()).cpu().numpy()
    M64 = M.detach().float().cpu().numpy().astype(np.float64)  # the BF16-rounded values

    # against the FP64 oracle gradient at the BF16-rounded values
    L_o, g_o, _ = oracle.loss_grad(M64, sc.near, sc.far, sc.ref, sc.src, sc.images)
    gmax = np.abs(g_o).max()
    err_o = np.abs(g32 - g_o).max()
    assert err_o <= 1e-4 * gmax, (err_o, gmax)
    assert abs(loss.item() - L_o) <= 1e-4 * L_o
    # the autograd gradient is the FP32 one rounded to BF16
    gb = M.grad.float().cpu().numpy()
    assert np.abs(gb - g32).max() <= 2 ** -8 * gmax

    # central finite differences on 64 seeded entries (FP64 at the BF16-rounded values)
    rng = np.random.default_rng(2024)
    rho = oracle.plane_inverse_depths(sc.D, sc.near, sc.far)
    h = 1e-3
    worst = 0.0
    # 32 uniformly drawn entries and 32 drawn among the 2000 largest |gradient| entries
    flat_top = np.argsort(np.abs(g_o).ravel())[-2000:]
    picks = [tuple(int(v) for v in (rng.integers(0, sc.D), rng.integers(0, sc.H), rng.integers(0, sc.W),
                                    rng.integers(0, 4))) for _ in range(32)]
    picks += [tuple(int(v) for v in np.unravel_index(i, g_o.shape)) for i in rng.choice(flat_top, 32, replace=False)]
    for d, y, x, c in picks:
        old = M64[d, y, x, c]
        M64[d, y, x, c] = old + h
        lp = _windowed_loss(M64, sc, sc.src, d, y, x, rho)
        M64[d, y, x, c] = old - h
        lm = _windowed_loss(M64, sc, sc.src, d, y, x, rho)
        M64[d, y, x, c] = old
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - g32[d, y, x, c]))
    assert worst <= 2e-5 + 1e-4 * gmax, (worst, gmax)
    print(f"\nautograd BF16: max|g_gpu - g_oracle| = {err_o:.2e} (max|g| = {gmax:.3e}); "
          f"max|g_gpu - FD| over 64 entries = {worst:.2e}")


def test_autograd_fp32_gradient_flows_through_torch(rl, scene):
    from paper_2307_03017_gb300.autograd import warp_composite
    sc = scene
    M = torch.from_numpy(sc.coarse_mpi[:, :96, :128].copy()).cuda().requires_grad_(True)
    K = sc.ref.K.copy()
    cams = [sg.Camera(K, c.R, c.t) for c in sc.src[:2]]
    out = warp_composite(M, sc.near, sc.far, sc.ref, cams)
    w = torch.linspace(0, 1, out.numel(), device="cuda").reshape(out.shape)
    (out * w).sum().backward()
    want = oracle.vjp(M.detach().cpu().numpy(), sc.near, sc.far, sc.ref, cams, w.cpu().numpy())
    assert np.abs(M.grad.cpu().numpy() - want).max() <= 1e-4 * max(1.0, np.abs(want).max())


def _psnr(a, b):
    return -10.0 * np.log10(np.mean((a - b) ** 2))


@pytest.mark.parametrize("schedule", [(2, 0), (2, 1, 0)])
def test_dense_vs_sparse_hsgd_bf16(rl, scene, schedule):
    """Dense (k = D) and sparse (k = 5) HSGD with BF16 storage: both lower the loss and the
    novel-view error against the ray-cast ground truth; numbers are printed for the record."""
    sc = scene
    images = torch.from_numpy(sc.images).cuda()
    coarse = torch.from_numpy(sc.coarse_mpi).cuda().to(torch.bfloat16)
    m0 = rl.make_mpi(coarse.clone(), sc.near, sc.far, sc.ref)
    psnr0 = np.mean([_psnr(v, t) for v, t in zip(rl.reallife_render(m0, sc.novel).cpu().numpy(), sc.novel_images)])
    res = {}
    for k in (5, sc.D):
        m = rl.make_mpi(coarse.clone(), sc.near, sc.far, sc.ref)
        losses = torch.empty(len(schedule), device="cuda")
        rl.reallife_refine(m, images, sc.src, k, schedule, loss_per_iter=losses)
        final = torch.empty(1, device="cuda")
        probe = rl.make_mpi(m.data.clone(), sc.near, sc.far, sc.ref)
        rl.reallife_hsgd_step(probe, images, sc.src, 1, lam=0.0, loss_out=final)  # loss of the result, no update
        views = rl.reallife_render(m, sc.novel).cpu().numpy()
        res[k] = (losses.cpu().numpy(), final.item(), np.mean([_psnr(v, t) for v, t in zip(views, sc.novel_images)]))
    loss0 = torch.empty(1, device="cuda")
    rl.reallife_hsgd_step(rl.make_mpi(coarse.clone(), sc.near, sc.far, sc.ref), images, sc.src, 1, lam=0.0,
                          loss_out=loss0)
    for k, (li, lf, ps) in res.items():
        assert lf < loss0.item()
        assert ps > psnr0
    print(f"\nschedule {schedule}: coarse loss {loss0.item():.1f} PSNR {psnr0:.2f} dB; "
          + "; ".join(f"k={k}: loss {lf:.1f} PSNR {ps:.2f} dB" for k, (li, lf, ps) in res.items()))
