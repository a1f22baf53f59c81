"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs.

Tolerances: FP32 renders, gradients and refined MPIs within 1e-5 max-abs; BF16-stored
MPIs within 2e-2; selections bit-exact when the GPU selects from the oracle's keys
rounded to FP32 (both sides then decide in FP32).  Where the GPU selects from its own
FP32 keys, near-ties may flip against FP64, so the refinement is compared with the
oracle fed the GPU's selection, and the GPU selection is checked to be a valid top-k
under the oracle's keys.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 2e-2


@pytest.fixture(scope="module")
def rl():
    import paper_2307_03017_gb300 as rl
    rl._lib.lib()  # loud failure if the library is missing
    rl.reallife_set_kernel_path(0)
    yield rl
    assert rl.reallife_device_status(clear=True) == 0  # no bounded wait gave up


@pytest.fixture(params=[3, 4, 5, 2], ids=["planepar", "planepar4", "planepar8", "gather"])
def kernel_path(request, rl):
    """Run a test with each warp-kernel family: plane-parallel (8 or 4 warps a block), per-pixel gather."""
    rl.reallife_set_kernel_path(request.param)
    yield request.param
    rl.reallife_set_kernel_path(0)


@pytest.fixture(scope="module")
def small():
    return sg.workload("small", 0)[0]


@pytest.fixture(scope="module")
def paper():
    return sg.workload("paper", 0)[0]


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def _mpi(rl, sc, dtype=torch.float32, M=None):
    data = _dev(sc.coarse_mpi if M is None else M, dtype).contiguous()
    return rl.make_mpi(data, sc.near, sc.far, sc.ref)


def _valid_topk(keys, S):
    """Every GPU-selected plane's oracle key is >= every unselected key, up to FP32 rounding."""
    D = keys.shape[0]
    sel = np.zeros(keys.shape, dtype=bool)
    for j in range(S.shape[0]):
        np.put_along_axis(sel, S[j][None].astype(np.int64), True, axis=0)
    kmin = np.where(sel, keys, np.inf).min(0)
    kmax_out = np.where(sel, -np.inf, keys).max(0)
    slack = 4e-6 * np.maximum(np.abs(keys).max(0), 1e-30)
    return np.all(kmin >= kmax_out - slack) and np.all(sel.sum(0) == S.shape[0]) and D >= S.shape[0]


# ---------------------------------------------------------------- warp geometry

def test_warp_offsets_match_ray_plane_intersection(rl, paper):
    sc = paper
    m = _mpi(rl, sc)
    rng = np.random.default_rng(0)
    rho = oracle.plane_inverse_depths(sc.D, sc.near, sc.far)
    worst = 0.0
    for cam in sc.src + sc.novel[:2]:
        off = rl.reallife_warp_offsets(m, cam).cpu().numpy()
        for _ in range(400):
            d, y, x = rng.integers(0, sc.D), rng.integers(0, sc.H), rng.integers(0, sc.W)
            px, py = oracle.view_to_ref(sc.ref, cam, 1.0 / rho[d], x, y)
            worst = max(worst, abs(off[d, y, x, 0] - (px - x)), abs(off[d, y, x, 1] - (py - y)))
    assert worst < 2e-5, worst


# ---------------------------------------------------------------------- render

@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_render_matches_oracle_small(rl, kernel_path, small, dtype):
    sc = small
    m = _mpi(rl, sc, dtype)
    Mq = m.data.float().cpu().numpy()  # the values the GPU stores (BF16-rounded when BF16)
    cams = sc.novel + sc.src
    out = rl.reallife_render(m, cams).cpu().numpy()
    for j, cam in enumerate(cams):
        ref = oracle.render(Mq, sc.near, sc.far, sc.ref, cam)
        assert np.abs(out[j] - ref).max() <= TOL32


def test_render_matches_oracle_paper_sampled(rl, kernel_path, paper):
    """Full-size render (the benchmark's 9 views), checked on 3000 sampled pixels per view."""
    sc = paper
    m = _mpi(rl, sc)
    out = rl.reallife_render(m, sc.novel).cpu().numpy()
    rng = np.random.default_rng(1)
    for j, cam in enumerate(sc.novel):
        xs, ys = rng.integers(0, sc.W, 3000), rng.integers(0, sc.H, 3000)
        xs[:4], ys[:4] = [0, sc.W - 1, 0, sc.W - 1], [0, 0, sc.H - 1, sc.H - 1]
        ref = oracle.render_pixels(sc.coarse_mpi, sc.near, sc.far, sc.ref, cam, xs, ys)
        assert np.abs(out[j][ys, xs] - ref).max() <= TOL32


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_shift_render_equals_general_render(rl, small, dtype):
    """Views that are pure shifts of the reference take a kernel with per-plane shifts and
    weights (formed in FP64 once per plane); rendered in one launch with a rotated view they take
    the general kernel (per-pixel FP32 coordinates at these offsets, up to ~115 px).  The same
    samples up to the coordinates' rounding: within 1e-5 of each other and of the oracle."""
    rl.reallife_set_kernel_path(2)
    try:
        sc = small
        m = _mpi(rl, sc, dtype)
        far = sg.Camera(sc.ref.K, np.eye(3), np.array([0.9, -0.4, 0.0]))  # mostly outside the MPI
        shifts = sc.novel + [far]
        a = rl.reallife_render(m, shifts).cpu().numpy()
        b = rl.reallife_render(m, shifts + [sc.src[0]]).cpu().numpy()
        assert np.abs(a - b[:len(shifts)]).max() <= TOL32
        M64 = m.data.float().cpu().numpy().astype(np.float64)
        for j, cam in enumerate(shifts):
            assert np.abs(a[j] - oracle.render(M64, sc.near, sc.far, sc.ref, cam)).max() <= TOL32
    finally:
        rl.reallife_set_kernel_path(0)


def test_render_edge_cases(rl, kernel_path):
    # ragged tile tails (W % 32, H % 4 != 0), one plane, a view that sees mostly outside the MPI
    sc = sg.make_scene(5, 23, 37, 1, 2, n_layers=(1, 2), f=30.0, n_novel=3)
    m = _mpi(rl, sc)
    far = sg.Camera(sc.ref.K, np.eye(3), np.array([3.0, 0.0, 0.0]))
    cams = sc.novel + [far]
    out = rl.reallife_render(m, cams).cpu().numpy()
    for j, cam in enumerate(cams):
        assert np.abs(out[j] - oracle.render(sc.coarse_mpi, sc.near, sc.far, sc.ref, cam)).max() <= TOL32
    # more than one launch chunk of target views
    many = [sc.novel[j % 3] for j in range(20)]
    out2 = rl.reallife_render(m, many).cpu().numpy()
    assert np.array_equal(out2[19], out[19 % 3])


# -------------------------------------------------------------------- selection

def test_select_keys_bit_exact_against_oracle(rl, small, paper):
    rng = np.random.default_rng(2)
    for sc in (small, paper):
        M = sc.coarse_mpi.astype(np.float64).copy()
        # exact ties: quantised alphas and fully transparent / fully occluded planes
        M[..., 3] = np.round(M[..., 3] * 8) / 8
        M[:, : sc.H // 4, : sc.W // 4, 3] = 0.0
        keys32 = oracle.alpha_weights(M).astype(np.float32)
        for k in sorted(k for k in {1, 3, 5, 8, 9, sc.D // 2, sc.D} if k <= sc.D):
            S_g, mask_g = rl.reallife_select_keys(_dev(keys32), k)
            S_o, mask_o = oracle.select_topk(keys32.astype(np.float64), k)
            assert np.array_equal(S_g.cpu().numpy(), S_o), k
            assert np.array_equal(mask_g.cpu().numpy().view(np.uint64), mask_o), k
    # random keys with many duplicates
    keys = rng.choice(np.float32([0, 0, 0.25, 0.5, 1e-30, 3.0]), size=(17, 9, 13)).astype(np.float32)
    for k in (1, 4, 8, 9, 17):
        S_g, _ = rl.reallife_select_keys(_dev(keys), k)
        assert np.array_equal(S_g.cpu().numpy(), oracle.select_topk(keys.astype(np.float64), k)[0])


def test_select_from_mpi_is_valid_topk(rl, paper):
    sc = paper
    for dtype in (torch.float32, torch.bfloat16):
        m = _mpi(rl, sc, dtype)
        Mq = m.data.float().cpu().numpy()
        keys = oracle.alpha_weights(Mq)
        S_g, mask_g = rl.reallife_select(m, 5)
        S_g = S_g.cpu().numpy()
        assert np.all(np.diff(S_g.astype(int), axis=0) > 0)
        assert _valid_topk(keys, S_g)
        S_o, _ = oracle.select_topk(keys, 5)
        flips = np.mean(np.any(S_g != S_o, axis=0))
        assert flips < 1e-3, flips


# -------------------------------------------------------------------- gradient

def test_dense_gradient_and_loss_match_oracle(rl, kernel_path, small):
    sc = small
    m = _mpi(rl, sc)
    loss, G = rl.reallife_loss_grad(m, _dev(sc.images), sc.src)
    L_o, g_o, _ = oracle.loss_grad(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images)
    assert abs(loss.item() - L_o) <= 1e-5 * L_o
    assert np.abs(G.cpu().numpy() - g_o).max() <= TOL32


def test_sparse_gradient_is_masked_dense_gradient(rl, kernel_path, small):
    sc = small
    m = _mpi(rl, sc)
    k = 3
    S, mask = rl.reallife_select(m, k)
    _, Gs = rl.reallife_loss_grad(m, _dev(sc.images), sc.src, mask=mask, k=k)
    _, g_o, _ = oracle.loss_grad(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images)
    S = S.cpu().numpy().astype(np.int64)
    want = np.take_along_axis(g_o, S[..., None], axis=0)  # [k][H][W][4]
    assert np.abs(Gs.cpu().numpy() - want).max() <= TOL32


def test_render_backward_matches_oracle_vjp(rl, kernel_path, small):
    sc = small
    m = _mpi(rl, sc)
    rng = np.random.default_rng(3)
    g_out = rng.normal(size=(len(sc.src), sc.H, sc.W, 3)).astype(np.float32)
    G = rl.reallife_render_backward(m, sc.src, _dev(g_out)).cpu().numpy()
    want = oracle.vjp(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, g_out)
    assert np.abs(G - want).max() <= 1e-4 * max(1.0, np.abs(want).max())


# ------------------------------------------------------------------ HSGD steps

@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 5, 8])
def test_hsgd_step_matches_oracle_with_selection_pinned(rl, kernel_path, small, level, k):
    sc = small
    m = _mpi(rl, sc)
    h, w = sc.H >> level, sc.W >> level
    S = torch.empty((k, h, w), dtype=torch.uint8, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rl.reallife_hsgd_step(m, _dev(sc.images), sc.src, k, level=level, loss_out=loss, S_out=S)
    S = S.cpu().numpy()
    M_o, L_o, S_free = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k, level=level,
                                        S_pin=S)
    assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32
    assert abs(loss.item() - L_o) <= 1e-5 * L_o
    Ml = oracle.down(sc.coarse_mpi, level)
    assert _valid_topk(oracle.alpha_weights(Ml), S)


def test_keep_everything_equals_dense_gd(rl, small):
    sc = small
    m = _mpi(rl, sc)
    rl.reallife_hsgd_step(m, _dev(sc.images), sc.src, sc.D, level=1)
    M_o, _ = oracle.gd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, level=1)
    assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32


def test_unclamped_step_and_lambda(rl, small):
    sc = small
    m = _mpi(rl, sc)
    S = torch.empty((4, sc.H, sc.W), dtype=torch.uint8, device="cuda")
    rl.reallife_hsgd_step(m, _dev(sc.images), sc.src, 4, lam=0.37, clamp=False, S_out=S)
    M_o, _, _ = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, 4, lam=0.37,
                                 clamp=False, S_pin=S.cpu().numpy())
    assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32


def _gpu_refine_steps(rl, sc, k, schedule, dtype=torch.float32):
    m = _mpi(rl, sc, dtype)
    M0 = m.data.float().cpu().numpy()
    ws = rl.workspace(len(sc.src), sc.D, sc.H, sc.W, k, dtype)
    images = _dev(sc.images)
    sels, losses = [], []
    for level in schedule:
        S = torch.empty((k, sc.H >> level, sc.W >> level), dtype=torch.uint8, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        rl.reallife_hsgd_step(m, images, sc.src, k, level=level, loss_out=loss, S_out=S, ws=ws)
        sels.append(S.cpu().numpy())
        losses.append(loss.item())
    return m, M0, sels, losses


def test_refine_small_matches_oracle(rl, kernel_path, small):
    sc = small
    m, M0, sels, losses = _gpu_refine_steps(rl, sc, 5, (2, 1, 0))
    M_o, L_o, _ = oracle.refine(M0, sc.near, sc.far, sc.ref, sc.src, sc.images, 5, (2, 1, 0), S_pins=sels)
    assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32
    np.testing.assert_allclose(losses, L_o, rtol=1e-5)


def test_refine_call_equals_step_sequence(rl, small):
    sc = small
    m1, _, _, losses = _gpu_refine_steps(rl, sc, 5, (2, 1, 0))
    m2 = _mpi(rl, sc)
    lpi = torch.empty(3, dtype=torch.float32, device="cuda")
    rl.reallife_refine(m2, _dev(sc.images), sc.src, 5, (2, 1, 0), loss_per_iter=lpi)
    assert torch.allclose(m1.data, m2.data, rtol=0, atol=1e-6)
    np.testing.assert_allclose(lpi.cpu().numpy(), losses, rtol=1e-6)


def test_refine_paper_size_matches_oracle(rl, kernel_path, paper):
    """The benchmark's workload (512x384, D=32, N=4, k=5, levels 2,1,0) at full size."""
    sc = paper
    m, M0, sels, losses = _gpu_refine_steps(rl, sc, 5, (2, 1, 0))
    M_o, L_o, free = oracle.refine(M0, sc.near, sc.far, sc.ref, sc.src, sc.images, 5, (2, 1, 0), S_pins=sels)
    assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32
    np.testing.assert_allclose(losses, L_o, rtol=1e-5)


def test_refine_bf16_storage_within_tolerance(rl, kernel_path, small):
    sc = small
    m, M0, sels, losses = _gpu_refine_steps(rl, sc, 5, (2, 1, 0), torch.bfloat16)
    M_o, L_o, _ = oracle.refine(M0, sc.near, sc.far, sc.ref, sc.src, sc.images, 5, (2, 1, 0), S_pins=sels)
    err = np.abs(m.data.float().cpu().numpy() - M_o)
    assert err.max() <= TOL16, err.max()
    np.testing.assert_allclose(losses, L_o, rtol=2e-2)


def test_refine_bf16_paper_size_within_tolerance(rl, paper):
    """BF16 storage at the benchmark's size: 3-level refine (512x384, D=32, N=4, k=5) against the
    FP64 oracle fed the GPU's selections (the oracle on all host cores, bit-identical)."""
    sc = paper
    m, M0, sels, losses = _gpu_refine_steps(rl, sc, 5, (2, 1, 0), torch.bfloat16)
    oracle.set_threads(True)
    try:
        M_o, L_o, _ = oracle.refine(M0, sc.near, sc.far, sc.ref, sc.src, sc.images, 5, (2, 1, 0), S_pins=sels)
    finally:
        oracle.set_threads(False)
    err = np.abs(m.data.float().cpu().numpy() - M_o)
    assert err.max() <= TOL16, err.max()
    np.testing.assert_allclose(losses, L_o, rtol=2e-2)


def test_degenerate_one_plane_and_one_view(rl):
    sc = sg.make_scene(9, 12, 20, 1, 1, n_layers=(1, 1), f=20.0)
    m = _mpi(rl, sc)
    S = torch.empty((1, 12, 20), dtype=torch.uint8, device="cuda")
    rl.reallife_hsgd_step(m, _dev(sc.images), sc.src, 1, S_out=S)
    assert np.all(S.cpu().numpy() == 0)
    M_o, _ = oracle.gd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images)
    assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32


def test_ragged_sizes_and_level_tails(rl, kernel_path):
    sc = sg.make_scene(4, 20, 44, 5, 2, n_layers=(2, 3), f=40.0)  # W/4 = 11: ragged tiles at every level
    m, M0, sels, _ = _gpu_refine_steps(rl, sc, 2, (2, 1, 0))
    M_o, _, _ = oracle.refine(M0, sc.near, sc.far, sc.ref, sc.src, sc.images, 2, (2, 1, 0), S_pins=sels)
    assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32


def test_large_offsets_take_anchored_coordinates(rl):
    """Views whose warp offsets exceed 128 px (here up to ~190 px: a wide baseline and a rotated
    view) take the per-block FP64 anchored coordinates; renders, the dense and sparse adjoints and
    an HSGD step match the oracle at 1e-5 in every kernel family."""
    rng = np.random.default_rng(17)
    sc = sg.make_scene(16, 48, 384, 8, 2, n_layers=(2, 3), novel="none")
    cams = [sg.Camera(sc.ref.K, sg.random_rotation(rng, 6.0), np.array([0.45, -0.04, 0.02])),
            sg.Camera(sc.ref.K, np.eye(3), np.array([-0.5, 0.0, 0.0]))]
    images = oracle.render(sc.coarse_mpi, sc.near, sc.far, sc.ref, cams[0])[None].repeat(2, 0).astype(np.float32)
    g_out = _dev(rng.normal(size=(2, sc.H, sc.W, 3)).astype(np.float32))
    want_r = [oracle.render(sc.coarse_mpi, sc.near, sc.far, sc.ref, c) for c in cams]
    want_g = oracle.vjp(sc.coarse_mpi, sc.near, sc.far, sc.ref, cams, g_out.cpu().numpy())
    for path in (2, 3, 5):
        rl.reallife_set_kernel_path(path)
        m = _mpi(rl, sc)
        out = rl.reallife_render(m, cams).cpu().numpy()
        for j in range(2):
            assert np.abs(out[j] - want_r[j]).max() <= TOL32
        g = rl.reallife_render_backward(m, cams, g_out).cpu().numpy()
        assert np.abs(g - want_g).max() <= 1e-5 * max(1.0, np.abs(want_g).max())
        S = torch.empty((3, sc.H, sc.W), dtype=torch.uint8, device="cuda")
        rl.reallife_hsgd_step(m, _dev(images), cams, 3, S_out=S)
        M_o, _, _ = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, cams, images, 3, S_pin=S.cpu().numpy())
        assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32
    rl.reallife_set_kernel_path(0)


def test_kernel_families_agree_on_extreme_warps(rl):
    """Large rotations and translations: far-off taps, planes met behind the views."""
    rng = np.random.default_rng(7)
    sc = sg.make_scene(6, 64, 96, 6, 3, n_layers=(2, 3), f=96.0)
    cams = [sg.Camera(sc.ref.K, sg.random_rotation(rng, 25.0), rng.uniform(-0.6, 0.6, 3)) for _ in range(3)]
    g_out = _dev(rng.normal(size=(3, sc.H, sc.W, 3)).astype(np.float32))
    outs, grads = [], []
    for path in (3, 4, 5, 2):
        rl.reallife_set_kernel_path(path)
        m = _mpi(rl, sc)
        outs.append(rl.reallife_render(m, cams).cpu().numpy())
        grads.append(rl.reallife_render_backward(m, cams, g_out).cpu().numpy())
    rl.reallife_set_kernel_path(0)
    for j, cam in enumerate(cams):
        assert np.abs(outs[0][j] - oracle.render(sc.coarse_mpi, sc.near, sc.far, sc.ref, cam)).max() <= TOL32
    want = oracle.vjp(sc.coarse_mpi, sc.near, sc.far, sc.ref, cams, g_out.cpu().numpy())
    for p in range(1, len(outs)):
        assert np.abs(outs[0] - outs[p]).max() <= TOL32
    for p in range(len(grads)):
        assert np.abs(grads[p] - want).max() <= 1e-4 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("D", [16, 64])
def test_bf16_odd_width_and_large_plane_counts(rl, D):
    """BF16 MPIs with odd W cannot be described for TMA (gather kernels); D=64 fills the mask word."""
    sc = sg.make_scene(8, 24, 45 if D == 16 else 48, D, 2, n_layers=(2, 3), f=45.0)
    m = _mpi(rl, sc, torch.bfloat16)
    Mq = m.data.float().cpu().numpy()
    out = rl.reallife_render(m, sc.src).cpu().numpy()
    for j, cam in enumerate(sc.src):
        assert np.abs(out[j] - oracle.render(Mq, sc.near, sc.far, sc.ref, cam)).max() <= TOL32
    S = torch.empty((9, sc.H, sc.W), dtype=torch.uint8, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rl.reallife_hsgd_step(m, _dev(sc.images), sc.src, 9, loss_out=loss, S_out=S)
    M_o, L_o, _ = oracle.hsgd_step(Mq, sc.near, sc.far, sc.ref, sc.src, sc.images, 9, S_pin=S.cpu().numpy())
    assert np.abs(m.data.float().cpu().numpy() - M_o).max() <= TOL16
    assert abs(loss.item() - L_o) <= 1e-5 * L_o


# ------------------------------------------- MVS-sampling selection and sparsity prior

def test_mvs_selection_bit_exact_against_oracle(rl, small):
    sc = small
    M = sc.coarse_mpi.astype(np.float64).copy()
    M[..., 3] = np.round(M[..., 3] * 8) / 8  # ties
    keys32 = oracle.alpha_weights(M).astype(np.float32)
    for k in (1, 3, 5, sc.D):
        S_g, mask_g = rl.reallife_select_keys(_dev(keys32), k, selection=rl.SELECT_MVS)
        S_o, mask_o = oracle.select_mvs(keys32.astype(np.float64), k)
        assert np.array_equal(S_g.cpu().numpy(), S_o), k
        assert np.array_equal(mask_g.cpu().numpy().view(np.uint64), mask_o), k


@pytest.mark.parametrize("level", [0, 1])
def test_hsgd_mvs_and_sparsity_prior_match_oracle(rl, small, level):
    sc = small
    k, lam_s = 3, 4000.0
    for selection in (rl.SELECT_TOPK, rl.SELECT_MVS):
        m = _mpi(rl, sc)
        S = torch.empty((k, sc.H >> level, sc.W >> level), dtype=torch.uint8, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        rl.reallife_hsgd_step(m, _dev(sc.images), sc.src, k, level=level, loss_out=loss, S_out=S, selection=selection,
                              lambda_s=lam_s)
        S = S.cpu().numpy()
        M_o, L_o, _ = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k, level=level,
                                       S_pin=S, lambda_s=lam_s)
        assert np.abs(m.data.cpu().numpy() - M_o).max() <= TOL32
        if selection == rl.SELECT_MVS:
            Ml = oracle.down(sc.coarse_mpi, level)
            best = np.argmax(oracle.alpha_weights(Ml), axis=0)  # first maximum
            assert np.all(np.diff(S.astype(int), axis=0) == 1)
            assert np.mean(np.any(S == best[None], axis=0)) > 0.999  # FP32 vs FP64 near-ties aside
