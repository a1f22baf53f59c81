"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formula: each checks a closed form, an
invariant, a special case, brute force, finite differences or a hand-derived
fixture (``tests/golden/``).  A plausible slip in the oracle (a dropped term, a
flipped sign, a transposed index, a wrong tie rule, a wrong pixel-centre
convention) fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cam(K, R=None, t=None):
    return sg.Camera(K, np.eye(3) if R is None else R, np.zeros(3) if t is None else t)


def _rand_mpi(rng, D, H, W, lo=0.0, hi=1.0):
    return rng.uniform(lo, hi, size=(D, H, W, 4))


def _small_views(rng, K, N, t_scale=0.1, rot_deg=2.0):
    return [sg.Camera(K, sg.random_rotation(rng, rot_deg), rng.uniform(-t_scale, t_scale, 3)) for _ in range(N)]


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=")
            vals[k.strip()] = np.array([float(x) for x in v.split()])
    return vals


# --------------------------------------------------------------- golden fixture

def test_golden_one_pixel_three_planes():
    """Hand-derived values of Eq. (eq_over), (eq_gradient) and top-k on one pixel."""
    g = _read_golden("over_operator_1px_3planes.txt")
    M = np.zeros((3, 1, 1, 4))
    for d in range(3):
        M[d, 0, 0, :3] = g[f"colour_{d}"]
        M[d, 0, 0, 3] = g["alpha"][d]
    K = np.eye(3)
    ref = _cam(K)
    out = oracle.render(M, 1.0, 100.0, ref, ref)
    np.testing.assert_allclose(out[0, 0], g["render"], rtol=0, atol=1e-15)
    A = oracle.alpha_weights(M)
    np.testing.assert_allclose(A[:, 0, 0], g["A"], rtol=0, atol=1e-15)
    assert abs(A.sum() - g["sum_A"][0]) < 1e-15
    grad = oracle.vjp(M, 1.0, 100.0, ref, [ref], np.ones((1, 1, 1, 3)))
    np.testing.assert_allclose(grad[:, 0, 0, 3], g["dL_dalpha_for_unit_residual"], rtol=0, atol=1e-15)
    for d in range(3):  # dL/dc_d = A_d * residual
        np.testing.assert_allclose(grad[d, 0, 0, :3], g["A"][d], rtol=0, atol=1e-15)
    S, mask = oracle.select_topk(A, 2)
    assert list(S[:, 0, 0]) == list(g["top2"].astype(int))
    assert int(mask[0, 0]) == (1 << 0) | (1 << 2)


# ------------------------------------------------------------------ composite

def test_single_opaque_plane_identity_pose_reproduces_plane():
    rng = np.random.default_rng(1)
    D, H, W = 5, 7, 9
    K = sg.intrinsics(W, H)
    ref = _cam(K)
    for d in range(D):
        M = _rand_mpi(rng, D, H, W)
        M[..., 3] = 0.0
        M[d, ..., 3] = 1.0
        out = oracle.render(M, 1.0, 50.0, ref, ref)
        np.testing.assert_allclose(out, M[d, ..., :3], rtol=0, atol=1e-12)


def test_transparent_planes_are_invisible():
    rng = np.random.default_rng(2)
    D, H, W = 6, 10, 12
    K = sg.intrinsics(W, H)
    ref = _cam(K)
    view = _small_views(rng, K, 1, 0.2)[0]
    M = _rand_mpi(rng, D, H, W)
    M[[1, 4], ..., 3] = 0.0
    a = oracle.render(M, 1.0, 20.0, ref, view)
    M2 = M.copy()
    M2[[1, 4], ..., :3] = rng.uniform(size=(2, H, W, 3))
    b = oracle.render(M2, 1.0, 20.0, ref, view)
    assert np.array_equal(a, b)


def test_compositing_weights_sum_to_one_minus_transmittance():
    rng = np.random.default_rng(3)
    M = _rand_mpi(rng, 9, 5, 6)
    A = oracle.alpha_weights(M)
    telescoped = 1.0 - np.prod(1.0 - M[..., 3], axis=0)
    np.testing.assert_allclose(A.sum(0), telescoped, rtol=0, atol=1e-15)


def test_alpha_weight_is_colour_derivative_at_reference_view():
    """A_d = dO/dc_d (Eq. eq_gradient): render is linear in colour, so a finite difference is exact."""
    rng = np.random.default_rng(4)
    D, H, W = 4, 5, 6
    K = sg.intrinsics(W, H)
    ref = _cam(K)
    M = _rand_mpi(rng, D, H, W)
    A = oracle.alpha_weights(M)
    base = oracle.render(M, 1.0, 10.0, ref, ref)
    for d in range(D):
        Mp = M.copy()
        Mp[d, ..., 1] += 0.5
        diff = (oracle.render(Mp, 1.0, 10.0, ref, ref) - base)[..., 1] / 0.5
        np.testing.assert_allclose(diff, A[d], rtol=0, atol=1e-12)


# ----------------------------------------------------------------- homography

def _eq_homo(Ki, Ri, ti, Kr, Rr, tr, z):
    """Eq. (eq_homo) as printed: maps a reference pixel at depth z to source view i (n = (0,0,1))."""
    n = np.array([0.0, 0.0, 1.0])
    inner = np.eye(3) + np.outer(np.linalg.inv(Ri) @ ti - np.linalg.inv(Rr) @ tr, n) @ Rr / z
    return Ki @ Ri @ inner @ np.linalg.inv(Rr) @ np.linalg.inv(Kr)


def test_reference_view_warp_is_identity():
    rng = np.random.default_rng(5)
    K = sg.intrinsics(64, 48)
    ref = sg.Camera(K, sg.random_rotation(rng, 10.0), rng.uniform(-1, 1, 3))
    for z in (1.0, 3.7, 100.0):
        for (u, v) in ((0, 0), (63, 47), (17.25, 30.5)):
            px, py = oracle.view_to_ref(ref, ref, z, u, v)
            assert abs(px - u) < 1e-11 and abs(py - v) < 1e-11


def test_paper_homography_matrix_agrees_with_ray_plane_intersection():
    rng = np.random.default_rng(6)
    Kr = sg.intrinsics(512, 384)
    Ki = sg.intrinsics(512, 384, 480.0)
    Ki[0, 2] += 3.0
    for trial in range(5):
        Rr, tr = sg.random_rotation(rng, 5.0), rng.uniform(-0.3, 0.3, 3)
        Ri, ti = sg.random_rotation(rng, 5.0), rng.uniform(-0.3, 0.3, 3)
        ref, src = sg.Camera(Kr, Rr, tr), sg.Camera(Ki, Ri, ti)
        for z in (1.0, 2.5, 40.0):
            Hm = _eq_homo(Ki, Ri, ti, Kr, Rr, tr, z)
            for _ in range(10):
                u, v = rng.uniform(0, 511), rng.uniform(0, 383)
                q = Hm @ np.array([u, v, 1.0])
                q = q[:2] / q[2]
                px, py = oracle.view_to_ref(ref, src, z, q[0], q[1])
                assert abs(px - u) < 1e-9 and abs(py - v) < 1e-9


def test_pure_translation_shifts_by_disparity():
    K = sg.intrinsics(40, 30, 32.0)
    ref = _cam(K)
    tx = 0.15
    view = _cam(K, t=np.array([tx, 0.0, 0.0]))  # camera centre at (-tx, 0, 0)
    rho = oracle.plane_inverse_depths(6, 1.0, 30.0)
    for r in rho:
        px, py = oracle.view_to_ref(ref, view, 1.0 / r, 10.0, 7.0)
        assert abs(px - (10.0 - 32.0 * tx * r)) < 1e-12 and abs(py - 7.0) < 1e-12


def test_integer_shift_reproduces_plane():
    """An opaque plane seen from a camera translated by an integer disparity is the shifted plane."""
    rng = np.random.default_rng(7)
    D, H, W = 2, 6, 10
    K = sg.intrinsics(W, H, 8.0)
    ref = _cam(K)
    # far = 2 -> plane 0 at z = 2; t_x = 0.5 -> disparity f t / z = 2 px
    view = _cam(K, t=np.array([0.5, 0.0, 0.0]))
    M = _rand_mpi(rng, D, H, W)
    M[..., 3] = 0.0
    M[0, ..., 3] = 1.0
    out = oracle.render(M, 1.0, 2.0, ref, view)
    np.testing.assert_allclose(out[:, 2:], M[0, :, :-2, :3], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, :2], 0.0, rtol=0, atol=1e-12)


def test_plane_spacing_is_uniform_in_inverse_depth():
    rho = oracle.plane_inverse_depths(8, 1.0, 100.0)
    assert rho[0] == pytest.approx(1 / 100.0, abs=1e-16) and rho[-1] == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(np.diff(rho), (1.0 - 0.01) / 7, rtol=1e-13)
    assert oracle.plane_inverse_depths(1, 1.0, 100.0)[0] == pytest.approx(0.01)


def test_camera_at_level_matches_box_average_pixel_centres():
    """A point seen at pixel u at level 0 lands at (u + 0.5)/2^l - 0.5 at level l."""
    K = sg.intrinsics(512, 384)
    cam = _cam(K)
    X = np.array([0.3, -0.2, 2.0])
    u0 = K @ X
    u0 = u0[:2] / u0[2]
    for l in (1, 2, 3):
        Kl, _, _ = oracle.camera_at_level(cam, l)
        ul = Kl @ X
        ul = ul[:2] / ul[2]
        np.testing.assert_allclose(ul, (u0 + 0.5) / 2**l - 0.5, rtol=0, atol=1e-12)


# ------------------------------------------------------------------- adjoint

def test_warp_composite_adjoint_dot_product():
    """For fixed alpha the render is linear in colour: <J x, y> = <x, J^T y> (colour part of the VJP)."""
    rng = np.random.default_rng(8)
    D, H, W, N = 4, 9, 11, 2
    K = sg.intrinsics(W, H, 10.0)
    ref = _cam(K)
    views = _small_views(rng, K, N, 0.3, 5.0)
    M = _rand_mpi(rng, D, H, W)
    y = rng.normal(size=(N, H, W, 3))
    lhs = sum(np.sum(oracle.render(M, 1.0, 10.0, ref, v) * y[i]) for i, v in enumerate(views))
    rhs = np.sum(oracle.vjp(M, 1.0, 10.0, ref, views, y)[..., :3] * M[..., :3])
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_full_adjoint_matches_central_differences():
    """dL/dM (colour and alpha) against central differences, step 1e-3, on a tiny problem."""
    rng = np.random.default_rng(9)
    D, H, W, N = 3, 6, 8, 2
    K = sg.intrinsics(W, H, 8.0)
    ref = _cam(K)
    views = _small_views(rng, K, N, 0.2, 4.0)
    M = _rand_mpi(rng, D, H, W, 0.1, 0.9)
    I = rng.uniform(size=(N, H, W, 3))
    _, g, _ = oracle.loss_grad(M, 1.0, 8.0, ref, views, I)
    h = 1e-3
    fd = np.empty_like(M)
    for idx in np.ndindex(M.shape):
        Mp, Mm = M.copy(), M.copy()
        Mp[idx] += h
        Mm[idx] -= h
        fd[idx] = (oracle.loss_grad(Mp, 1.0, 8.0, ref, views, I, want_grad=False)[0]
                   - oracle.loss_grad(Mm, 1.0, 8.0, ref, views, I, want_grad=False)[0]) / (2 * h)
    assert np.abs(g).max() > 1e-2  # non-trivial
    np.testing.assert_allclose(g, fd, rtol=0, atol=2e-6)


def test_loss_definition_on_identity_views():
    """With all views at the reference pose, L = 1/(2N) sum (O(M) - I)^2 of the unwarped composite."""
    rng = np.random.default_rng(10)
    D, H, W = 3, 4, 5
    K = sg.intrinsics(W, H)
    ref = _cam(K)
    M = _rand_mpi(rng, D, H, W)
    I = rng.uniform(size=(2, H, W, 3))
    A = oracle.alpha_weights(M)
    C = np.einsum("dhw,dhwc->hwc", A, M[..., :3])  # Eq. (eq_overA): O = sum_d c_d A_d
    expect = (np.sum((C - I[0]) ** 2) + np.sum((C - I[1]) ** 2)) / 4.0
    L, _, _ = oracle.loss_grad(M, 1.0, 5.0, ref, [ref, ref], I, want_grad=False)
    assert abs(L - expect) < 1e-12


# ---------------------------------------------------------------- selection

def _brute_force_topk(keys, k):
    """The unique k-subset whose every member beats every non-member under (key desc, index asc)."""
    D = len(keys)
    found = []
    for sub in itertools.combinations(range(D), k):
        rest = [e for e in range(D) if e not in sub]
        if all(keys[s] > keys[e] or (keys[s] == keys[e] and s < e) for s in sub for e in rest):
            found.append(sub)
    assert len(found) == 1
    return found[0]


def test_selection_matches_brute_force_with_ties():
    rng = np.random.default_rng(11)
    D, H, W = 6, 3, 4
    keys = rng.choice([0.0, 0.0, 0.0, 0.125, 0.25, 0.5, 0.75], size=(D, H, W))
    keys[:, 0, 0] = 0.0  # all tied
    keys[:, 0, 1] = -0.0
    keys[2, 0, 1] = 0.0  # -0 == +0
    for k in range(1, D + 1):
        S, mask = oracle.select_topk(keys, k)
        for y in range(H):
            for x in range(W):
                want = _brute_force_topk(list(keys[:, y, x]), k)
                assert tuple(S[:, y, x]) == want
                assert int(mask[y, x]) == sum(1 << d for d in want)


def test_selection_sorted_unique_and_keep_all():
    rng = np.random.default_rng(12)
    D, H, W = 8, 5, 5
    keys = rng.uniform(size=(D, H, W))
    for k in (1, 3, 8):
        S, mask = oracle.select_topk(keys, k)
        assert np.all(np.diff(S.astype(int), axis=0) > 0)
        assert np.all(np.vectorize(lambda m: bin(int(m)).count("1"))(mask) == k)
    S, mask = oracle.select_topk(keys, D)
    assert np.all(S == np.arange(D)[:, None, None]) and np.all(mask == (1 << D) - 1)


# ---------------------------------------------------------- update and levels

@pytest.fixture(scope="module")
def tiny_scene():
    sc = sg.make_scene(3, 16, 24, 6, 2, n_layers=(2, 3), f=24.0)
    return sc


def test_keep_everything_hsgd_equals_dense_gd_bitwise(tiny_scene):
    sc = tiny_scene
    for level in (0, 1):
        a, La, _ = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k=sc.D, level=level)
        b, Lb = oracle.gd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, level=level)
        assert np.array_equal(a, b) and La == Lb


def test_small_step_descends(tiny_scene):
    sc = tiny_scene
    L0, _, _ = oracle.loss_grad(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, want_grad=False)
    for k in (1, 3, sc.D):
        M1, Lstep, _ = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k=k,
                                        lam=1e-3, clamp=False)
        assert Lstep == pytest.approx(L0, rel=1e-14)
        L1, _, _ = oracle.loss_grad(M1, sc.near, sc.far, sc.ref, sc.src, sc.images, want_grad=False)
        assert L1 < L0


def test_masked_update_touches_only_selected_planes(tiny_scene):
    sc = tiny_scene
    k = 2
    M1, _, S = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k=k, clamp=False)
    changed = np.any(M1 != sc.coarse_mpi.astype(np.float64), axis=-1)  # [D][H][W]
    sel = np.zeros_like(changed)
    for j in range(k):
        for y in range(sc.H):
            for x in range(sc.W):
                sel[S[j, y, x], y, x] = True
    assert not np.any(changed & ~sel)


def test_level_step_is_upsampled_coarse_step(tiny_scene):
    """Down^l of the level-l update equals the masked coarse gradient step (Down o U_l = id)."""
    sc = tiny_scene
    level, k, lam = 1, 3, 0.7
    M0 = sc.coarse_mpi.astype(np.float64)
    M1, _, S = oracle.hsgd_step(M0, sc.near, sc.far, sc.ref, sc.src, sc.images, k=k, lam=lam, clamp=False,
                                level=level)
    delta = M1 - M0
    # block-constant: every 2x2 block changed by one value (up to the rounding of M - lam g)
    blocks = delta.reshape(sc.D, sc.H // 2, 2, sc.W // 2, 2, 4)
    np.testing.assert_allclose(blocks, np.broadcast_to(blocks[:, :, :1, :, :1, :], blocks.shape), rtol=0, atol=1e-15)
    Ml = oracle.down(M0, level)
    Il = oracle.down(sc.images, level)
    refl = sg.Camera(*oracle.camera_at_level(sc.ref, level))
    vl = [sg.Camera(*oracle.camera_at_level(v, level)) for v in sc.src]
    _, g, _ = oracle.loss_grad(Ml, sc.near, sc.far, refl, vl, Il)
    mask = np.zeros(g.shape[:3], dtype=bool)
    for j in range(k):
        for y in range(g.shape[1]):
            for x in range(g.shape[2]):
                mask[S[j, y, x], y, x] = True
    np.testing.assert_allclose(oracle.down(delta, level), -lam * g * mask[..., None], rtol=0, atol=1e-14)


def test_downsample_box_average():
    rng = np.random.default_rng(13)
    x = rng.uniform(size=(2, 8, 12, 3))
    y = oracle.down(x, 1)
    np.testing.assert_allclose(y, x.reshape(2, 4, 2, 6, 2, 3).mean(axis=(2, 4)), rtol=0, atol=1e-15)
    # a ramp in x sampled at pixel centres stays a ramp at the coarse centres (2u + 0.5)
    ramp = np.broadcast_to(np.arange(16.0)[None, None, :, None], (1, 4, 16, 1)).copy()
    np.testing.assert_allclose(oracle.down(ramp, 2)[0, 0, :, 0], 4 * np.arange(4) + 1.5, rtol=0, atol=1e-14)
    np.testing.assert_allclose(oracle.down(x, 2), oracle.down(oracle.down(x, 1), 1), rtol=0, atol=0)


def test_flat_schedule_equals_repeated_level0_steps(tiny_scene):
    sc = tiny_scene
    Ma, La, _ = oracle.refine(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k=2, schedule=(0, 0))
    M = sc.coarse_mpi
    Lb = []
    for _ in range(2):
        M, L, _ = oracle.hsgd_step(M, sc.near, sc.far, sc.ref, sc.src, sc.images, k=2)
        Lb.append(L)
    assert np.array_equal(Ma, M) and La == Lb


def test_refinement_improves_novel_views():
    """End-to-end sanity (not a parity pin): refinement lowers the novel-view error vs ray-cast views."""
    sc = sg.make_scene(0, 48, 64, 8, 3, n_layers=(3, 5), render_novel_gt=True, n_novel=3)
    def err(M):
        return np.mean([np.mean((oracle.render(M, sc.near, sc.far, sc.ref, c) - sc.novel_images[j]) ** 2)
                        for j, c in enumerate(sc.novel)])
    e0 = err(sc.coarse_mpi)
    M, losses, _ = oracle.refine(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k=5,
                                 schedule=(2, 1, 0, 0, 0))
    assert err(M) < e0


# ------------------------------------------------- MVS-sampling and sparsity prior

def test_mvs_sampling_window_definition():
    """Argmax plane (ties to the lower index) plus (k-1)/2 neighbours each side, shifted into [0, D)."""
    rng = np.random.default_rng(14)
    D, H, W = 9, 4, 5
    keys = rng.choice([0.0, 0.1, 0.2, 0.5], size=(D, H, W))
    keys[:, 0, 0] = 0.0                      # all tied: argmax = 0, window at the back
    keys[:, 0, 1] = np.arange(D)             # argmax = D-1: window at the front
    keys[4, 0, 2], keys[6, 0, 2] = 1.0, 1.0  # tie between 4 and 6: argmax 4
    for k in (1, 3, 5, D):
        S, mask = oracle.select_mvs(keys, k)
        for y in range(H):
            for x in range(W):
                col = list(keys[:, y, x])
                best = col.index(max(col))  # first maximum = lowest index
                start = min(max(best - (k - 1) // 2, 0), D - k)
                assert list(S[:, y, x]) == list(range(start, start + k))
                assert best in S[:, y, x]
                assert int(mask[y, x]) == sum(1 << d for d in range(start, start + k))
    assert list(oracle.select_mvs(keys, 3)[0][:, 0, 0]) == [0, 1, 2]
    assert list(oracle.select_mvs(keys, 3)[0][:, 0, 1]) == [D - 3, D - 2, D - 1]
    assert list(oracle.select_mvs(keys, 3)[0][:, 0, 2]) == [3, 4, 5]


def test_sparsity_prior_gradient_matches_finite_differences():
    """dL_s/dalpha of Sec. 3.4's L_s = mean log(1.5 - |0.5 - alpha|), by central differences."""
    rng = np.random.default_rng(15)
    D, H, W = 3, 4, 5
    M = rng.uniform(0.02, 0.98, size=(D, H, W, 4))
    M[..., 3][np.abs(M[..., 3] - 0.5) < 0.02] = 0.3  # keep away from the kink
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (2, 3, 4), (0, 1, 2)]:
        Mp, Mm = M.copy(), M.copy()
        Mp[idx + (3,)] += h
        Mm[idx + (3,)] -= h
        fd = (oracle.sparsity_loss(Mp) - oracle.sparsity_loss(Mm)) / (2 * h)
        assert abs(fd - oracle.sparsity_grad(M[idx + (3,)], D, H, W)) < 1e-8
    # closed form at the ends: log(1) = 0 at alpha in {0, 1}, log(1.5) at 0.5
    Z = np.zeros((1, 1, 1, 4))
    assert oracle.sparsity_loss(Z) == 0.0
    Z[..., 3] = 0.5
    assert abs(oracle.sparsity_loss(Z) - np.log(1.5)) < 1e-15
    assert oracle.sparsity_grad(0.5, 1, 1, 1) == 0.0


def test_sparsity_prior_pushes_alpha_to_the_ends(tiny_scene):
    """With only the prior (photometric step lambda = 0 would also freeze it, so use a huge
    lambda_s and a tiny lambda), selected alphas below 0.5 fall and above 0.5 rise."""
    sc = tiny_scene
    M0 = sc.coarse_mpi.astype(np.float64)
    M1, _, S = oracle.hsgd_step(M0, sc.near, sc.far, sc.ref, sc.src, sc.images, k=sc.D, lam=1e-12, clamp=False,
                                lambda_s=1e12 * sc.D * sc.H * sc.W)
    a0, a1 = M0[..., 3], M1[..., 3]
    assert np.all(a1[a0 < 0.49] < a0[a0 < 0.49]) and np.all(a1[a0 > 0.51] > a0[a0 > 0.51])


def test_hsgd_with_mvs_selection_updates_only_the_window(tiny_scene):
    sc = tiny_scene
    k = 3
    M1, _, S = oracle.hsgd_step(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k=k, clamp=False,
                                selection=1)
    A = oracle.alpha_weights(sc.coarse_mpi)
    S_want, _ = oracle.select_mvs(A, k)
    assert np.array_equal(S, S_want)
    assert np.all(np.diff(S.astype(int), axis=0) == 1)  # consecutive planes


@pytest.mark.parametrize("poses", ["random", "grid4x2"])
def test_voxel_gradient_equals_dense_gradient(poses):
    """The brute-force gradient at chosen voxels (over the view pixels near each voxel's
    projection) equals the dense adjoint of loss_grad bit for bit, at every voxel: borders,
    planes behind nothing, rotated and translated views."""
    if poses == "random":
        sc = sg.make_scene(21, 18, 26, 5, 3, n_layers=(2, 3), novel="none")
    else:
        sc = sg.make_scene(22, 16, 24, 4, 8, n_layers=(2, 3), src_poses="grid4x2", novel="none", f=24.0)
    _, G, _ = oracle.loss_grad(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images)
    D, H, W = sc.D, sc.H, sc.W
    dd, yy, xx = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    g = oracle.grad_voxels(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, dd.ravel(), yy.ravel(),
                           xx.ravel())
    assert np.array_equal(g.reshape(D, H, W, 4), G)
    assert np.abs(G).max() > 0
