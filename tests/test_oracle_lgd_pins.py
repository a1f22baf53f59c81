"""Pins of the learned-update oracle (oracle/lgd.py): BF16 rounding against torch's conversion,
the convolution against scipy's correlate and torch's conv3d, batch-norm folding against the
unfolded form, the whole network against a torch composition, and the restore operator against
the separately pinned analytic HSGD step.  CPU only."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from oracle import lgd
import scenegen as sg


def test_round_bf16_matches_torch_including_ties():
    rng = np.random.default_rng(50)
    x = rng.standard_normal(20000).astype(np.float32) * np.float32(3.0)
    # exact ties: low 16 bits 0x8000, with even and odd kept parts
    ties = (rng.integers(0, 1 << 15, 2000, dtype=np.uint32) << 17 | np.uint32(0x8000)
            | (rng.integers(0, 2, 2000, dtype=np.uint32) << 16)).view(np.float32)
    x = np.concatenate([x, ties[np.isfinite(ties)], np.array([0.0, -0.0, 1e-40, 3.4e38], np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(lgd.round_bf16(x), want)


def test_conv_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(51)
    x = rng.standard_normal((1, 5, 7, 9))
    w = rng.standard_normal((1, 1, 3, 3, 3))
    got = lgd.conv3d_same(x, w, np.zeros(1))[0]
    want = ndimage.correlate(x[0], w[0, 0], mode="constant", cval=0.0)
    assert np.max(np.abs(got - want)) < 1e-12


def test_conv_matches_torch_conv3d_multichannel():
    rng = np.random.default_rng(52)
    x = rng.standard_normal((6, 4, 5, 8))
    w = rng.standard_normal((3, 6, 3, 3, 3))
    b = rng.standard_normal(3)
    got = lgd.conv3d_same(x, w, b)
    want = F.conv3d(torch.from_numpy(x)[None], torch.from_numpy(w), torch.from_numpy(b), padding=1)[0].numpy()
    assert np.max(np.abs(got - want)) < 1e-12


def test_delta_kernel_shifts_with_zero_padding():
    rng = np.random.default_rng(53)
    x = rng.standard_normal((2, 4, 5, 6))
    w = np.zeros((2, 2, 3, 3, 3))
    w[1, 0, 2, 0, 1] = 1.0  # out channel 1 reads in channel 0 at (z+1, y-1, x)
    got = lgd.conv3d_same(x, w, np.zeros(2))
    want = np.zeros((4, 5, 6))
    want[:3, 1:, :] = x[0, 1:, :4, :]
    assert np.array_equal(got[1], want) and np.all(got[0] == 0.0)


def test_batch_norm_folding():
    rng = np.random.default_rng(54)
    x = rng.standard_normal((3, 3, 4, 5))
    w, b = rng.standard_normal((4, 3, 3, 3, 3)), rng.standard_normal(4)
    g, be = rng.uniform(0.5, 1.5, 4), rng.standard_normal(4)
    mu, var, eps = rng.standard_normal(4), rng.uniform(0.5, 2.0, 4), 1e-5
    y = lgd.conv3d_same(x, w, b)
    bn = g[:, None, None, None] * (y - mu[:, None, None, None]) / np.sqrt(var[:, None, None, None] + eps) \
        + be[:, None, None, None]
    wf, bf = lgd.bn_fold(w, b, g, be, mu, var, eps)
    assert np.max(np.abs(lgd.conv3d_same(x, wf, bf) - bn)) < 1e-12


def test_network_matches_torch_composition():
    """fp64 forward = torch conv3d + batch_norm (inference) + relu blocks, then the 1x1x1 layer."""
    rng = np.random.default_rng(55)
    net = sg.lgd_weights(3, 12, width=8)
    V = rng.uniform(0, 1, (12, 3, 6, 7))
    got = lgd.lgd_forward(V, net, storage="fp64")
    x = torch.from_numpy(V)[None]
    for l in range(5):
        x = F.conv3d(x, torch.from_numpy(net.conv_w[l]).double(), torch.from_numpy(net.conv_b[l]).double(), padding=1)
        x = F.batch_norm(x, torch.from_numpy(net.bn_mean[l]).double(), torch.from_numpy(net.bn_var[l]).double(),
                         torch.from_numpy(net.bn_gamma[l]).double(), torch.from_numpy(net.bn_beta[l]).double(),
                         training=False, eps=net.eps)
        x = torch.relu(x)
    x = F.conv3d(x, torch.from_numpy(net.out_w).double()[:, :, None, None, None], torch.from_numpy(net.out_b).double())
    want = x[0].permute(1, 2, 3, 0).numpy()
    assert got.shape == (3, 6, 7, 4)
    assert np.max(np.abs(got - want)) < 1e-10


def test_bf16_storage_rounds_only_where_stated():
    """One block on a BF16-valued input: its output feeds the 1x1x1 layer unrounded, so the bf16
    forward differs from the fp64 forward by the folded weights' rounding alone (bounded by half
    a BF16 ulp of the largest weight over the 27 x C taps), and does differ."""
    rng = np.random.default_rng(56)
    net = sg.lgd_weights(4, 6, width=8, blocks=1)
    V = lgd.round_bf16(rng.uniform(0, 1, (6, 2, 4, 5)))
    wf, _ = lgd.bn_fold(net.conv_w[0], net.conv_b[0], net.bn_gamma[0], net.bn_beta[0], net.bn_mean[0],
                        net.bn_var[0], net.eps)
    r64 = lgd.lgd_forward(V, net, "fp64")
    r16 = lgd.lgd_forward(V, net, "bf16")
    scale = np.abs(wf).max() * 2.0 ** -8 * 27 * 6 * np.abs(net.out_w).sum(1).max()
    assert 0 < np.max(np.abs(r16 - r64)) <= scale


@pytest.mark.parametrize("level", [0, 1])
def test_restore_update_with_the_gradient_step_is_the_hsgd_step(level):
    """R(-lambda g_S, S) added and clamped is exactly the analytic HSGD update of the pinned oracle."""
    sc = sg.make_scene(2, 16, 24, 4, 2, n_layers=(1, 2))
    k, lam = 2, 0.7
    M1, _, S = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k, lam, True, level)
    Ml = oracle.down(sc.coarse_mpi, level)
    Il = oracle.down(sc.images, level)
    refl = sg.Camera(*oracle.camera_at_level(sc.ref, level))
    views = [sg.Camera(*oracle.camera_at_level(c, level)) for c in sc.src]
    _, g, _ = oracle.loss_grad(Ml, sc.near, sc.far, refl, views, Il)
    h, w = S.shape[1:]
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    res = np.stack([-lam * g[S[j], yy, xx] for j in range(k)])
    M2 = lgd.restore_update(sc.coarse_mpi, res, S, level)
    assert np.max(np.abs(M2 - M1)) < 1e-13
