"""Pins of the oracle's gradient-volume functions (Sec. 3.2 PSV, Sec. 3.3 gradient formulation
and sparsification) against closed forms, the paper's homography matrix, the separately pinned
render and brute-force shifted indexing.  CPU only."""
import numpy as np
import pytest

import oracle
import scenegen as sg


def _cam(K, R=None, t=None):
    return sg.Camera(K, np.eye(3) if R is None else R, np.zeros(3) if t is None else t)


def _eq_homo(Ki, Ri, ti, Kr, Rr, tr, z):
    """Eq. (eq_homo) as printed: the reference pixel at depth z -> source view i (n = (0,0,1))."""
    n = np.array([0.0, 0.0, 1.0])
    inner = np.eye(3) + np.outer(np.linalg.inv(Ri) @ ti - np.linalg.inv(Rr) @ tr, n) @ Rr / z
    return Ki @ Ri @ inner @ np.linalg.inv(Rr) @ np.linalg.inv(Kr)


def _rand_mpi(rng, D, H, W):
    M = rng.uniform(0.0, 1.0, (D, H, W, 4))
    M[..., 3] = rng.uniform(0.0, 1.0, (D, H, W)) ** 2
    return M


def test_inverse_warp_is_the_paper_homography():
    rng = np.random.default_rng(31)
    Kr = sg.intrinsics(512, 384)
    Ki = sg.intrinsics(512, 384, 470.0)
    Ki[1, 2] -= 2.0
    for _ in range(5):
        Rr, tr = sg.random_rotation(rng, 5.0), rng.uniform(-0.3, 0.3, 3)
        Ri, ti = sg.random_rotation(rng, 5.0), rng.uniform(-0.3, 0.3, 3)
        ref, src = sg.Camera(Kr, Rr, tr), sg.Camera(Ki, Ri, ti)
        for z in (1.0, 3.0, 50.0):
            Hm = _eq_homo(Ki, Ri, ti, Kr, Rr, tr, z)
            for _ in range(10):
                u, v = rng.uniform(0, 511), rng.uniform(0, 383)
                q = Hm @ np.array([u, v, 1.0])
                x, y = oracle.ref_to_view(ref, src, z, u, v)
                assert abs(x - q[0] / q[2]) < 1e-9 and abs(y - q[1] / q[2]) < 1e-9


def test_inverse_warp_round_trip_and_behind_view():
    rng = np.random.default_rng(32)
    K = sg.intrinsics(64, 48)
    ref = _cam(K)
    view = sg.Camera(K, sg.random_rotation(rng, 3.0), rng.uniform(-0.2, 0.2, 3))
    for z in (1.5, 4.0, 20.0):
        for _ in range(20):
            u, v = rng.uniform(0, 63), rng.uniform(0, 47)
            x, y = oracle.ref_to_view(ref, view, z, u, v)
            pu, pv = oracle.view_to_ref(ref, view, z, x, y)
            assert abs(pu - u) < 1e-10 and abs(pv - v) < 1e-10
    # a camera 5 units in front of the reference sees the plane z = 1 behind it
    ahead = _cam(K, t=np.array([0.0, 0.0, -5.0]))
    assert oracle.ref_to_view(ref, ahead, 1.0, 10.0, 10.0) is None
    P = oracle.psv_view(np.ones((48, 64, 3)), 2, 1.0, 10.0, ref, ahead)
    assert np.all(P[1] == 0.0)  # plane d = 1 is the near plane z = 1


def test_psv_of_the_reference_view_is_the_image():
    rng = np.random.default_rng(33)
    K = sg.intrinsics(12, 9)
    ref = sg.Camera(K, sg.random_rotation(rng, 10.0), rng.uniform(-1, 1, 3))
    img = rng.uniform(0, 1, (9, 12, 3))
    P = oracle.psv_view(img, 4, 1.0, 20.0, ref, ref)
    assert np.max(np.abs(P - img[None])) < 1e-12


def test_psv_integer_disparity_is_the_shifted_image():
    """Camera translated by t_x: reference pixel u of plane d lands on u + f t_x rho_d."""
    rng = np.random.default_rng(34)
    H, W = 5, 12
    K = sg.intrinsics(W, H, 8.0)
    ref = _cam(K)
    view = _cam(K, t=np.array([0.5, 0.0, 0.0]))  # f t_x = 4; rho = 0.5, 0.75, 1 -> shifts 2, 3, 4 px
    img = rng.uniform(0, 1, (H, W, 3))
    P = oracle.psv_view(img, 3, 1.0, 2.0, ref, view)
    for d, s in enumerate((2, 3, 4)):
        want = np.zeros_like(img)
        want[:, :W - s] = img[:, s:]
        assert np.max(np.abs(P[d] - want)) < 1e-12


def test_psv_of_a_constant_image_is_constant_where_the_footprint_is_inside():
    rng = np.random.default_rng(35)
    H, W, D = 10, 14, 3
    K = sg.intrinsics(W, H, 12.0)
    ref = _cam(K)
    view = sg.Camera(K, sg.random_rotation(rng, 2.0), rng.uniform(-0.1, 0.1, 3))
    rho = oracle.plane_inverse_depths(D, 1.0, 10.0)
    P = oracle.psv_view(np.full((H, W, 3), 0.37), D, 1.0, 10.0, ref, view)
    inside = 0
    for d in range(D):
        for y in range(H):
            for x in range(W):
                vx, vy = oracle.ref_to_view(ref, view, 1.0 / rho[d], x, y)
                if 0 <= np.floor(vx) and np.floor(vx) + 1 <= W - 1 and 0 <= np.floor(vy) and np.floor(vy) + 1 <= H - 1:
                    inside += 1
                    assert np.max(np.abs(P[d, y, x] - 0.37)) < 1e-14
    assert inside > D * H * W // 2


def test_view_alpha_weights_sum_to_the_white_render():
    """sum_d A_{i,d}(q) is the render of the MPI with every colour set to 1 (Eq. eq_overA)."""
    rng = np.random.default_rng(36)
    D, H, W = 4, 8, 11
    K = sg.intrinsics(W, H, 10.0)
    ref = _cam(K)
    view = sg.Camera(K, sg.random_rotation(rng, 2.0), rng.uniform(-0.1, 0.1, 3))
    M = _rand_mpi(rng, D, H, W)
    M[..., :3] = 1.0
    A = oracle.view_alpha_weights(M, 1.0, 8.0, ref, view)
    C = oracle.render(M, 1.0, 8.0, ref, view)
    # zero padding scales a sampled colour by the weight inside the frame: compare the pixels
    # whose samples are inside on every plane
    rho = oracle.plane_inverse_depths(D, 1.0, 8.0)
    inside = np.ones((H, W), dtype=bool)
    for d in range(D):
        for y in range(H):
            for x in range(W):
                px, py = oracle.view_to_ref(ref, view, 1.0 / rho[d], x, y)
                inside[y, x] &= bool(0 <= np.floor(px) and np.floor(px) + 1 <= W - 1 and 0 <= np.floor(py)
                                     and np.floor(py) + 1 <= H - 1)
    assert inside.sum() > H * W // 3
    assert np.max(np.abs(A.sum(0) - C[..., 0])[inside]) < 1e-12


def test_view_alpha_weight_is_the_colour_derivative_of_the_view_render():
    """Eq. (eq_gradient): A_{i,d} = dO(M_i)/dc_d, by central differences of the pinned render
    (exact: the render is linear in the colours), where the sample's four taps are inside."""
    rng = np.random.default_rng(37)
    D, H, W = 3, 7, 9
    K = sg.intrinsics(W, H, 9.0)
    ref = _cam(K)
    view = sg.Camera(K, sg.random_rotation(rng, 2.0), rng.uniform(-0.08, 0.08, 3))
    near, far = 1.0, 6.0
    M = _rand_mpi(rng, D, H, W)
    A = oracle.view_alpha_weights(M, near, far, ref, view)
    rho = oracle.plane_inverse_depths(D, near, far)
    h = 1e-3
    checked = 0
    for d in range(D):
        Mp, Mm = M.copy(), M.copy()
        Mp[d, ..., :3] += h
        Mm[d, ..., :3] -= h
        fd = (oracle.render(Mp, near, far, ref, view) - oracle.render(Mm, near, far, ref, view)) / (2 * h)
        for y in range(H):
            for x in range(W):
                px, py = oracle.view_to_ref(ref, view, 1.0 / rho[d], x, y)
                if 0 <= np.floor(px) and np.floor(px) + 1 <= W - 1 and 0 <= np.floor(py) and np.floor(py) + 1 <= H - 1:
                    checked += 1
                    assert np.max(np.abs(fd[y, x] - A[d, y, x])) < 1e-10
    assert checked > D * H * W // 3


def test_inverse_warped_alpha_weights_integer_disparity_closed_form():
    """Pure x-translation, integer disparities s_d: the view sees plane j of reference column
    q - s_j, so A^{w^-1}[d](p) = alpha_d(p) prod_{j>d} (1 - alpha_j(p + s_d - s_j)), zero where the
    shifted columns leave the image."""
    rng = np.random.default_rng(38)
    D, H, W = 3, 4, 13
    K = sg.intrinsics(W, H, 8.0)
    ref = _cam(K)
    view = _cam(K, t=np.array([0.5, 0.0, 0.0]))
    near, far = 1.0, 2.0
    s = (2, 3, 4)
    M = _rand_mpi(rng, D, H, W)
    Av = oracle.view_alpha_weights(M, near, far, ref, view)
    Ainv = oracle.inverse_warp_stack(Av, near, far, ref, view)
    alpha = M[..., 3]

    def a(j, y, x):
        return alpha[j, y, x] if 0 <= x < W else 0.0

    for d in range(D):
        for y in range(H):
            for x in range(W):
                q = x + s[d]  # view column of reference pixel x on plane d
                if q > W - 1:
                    want = 0.0
                else:
                    want = a(d, y, q - s[d])
                    for j in range(d + 1, D):
                        want *= 1.0 - a(j, y, q - s[j])
                assert abs(Ainv[d, y, x] - want) < 1e-12


def _scene(rng, D=4, H=8, W=12, N=2, identity=False):
    K = sg.intrinsics(W, H, 10.0)
    ref = _cam(K)
    views = [ref if identity else sg.Camera(K, sg.random_rotation(rng, 2.0), rng.uniform(-0.1, 0.1, 3))
             for _ in range(N)]
    M = _rand_mpi(rng, D, H, W)
    images = rng.uniform(0, 1, (N, H, W, 3))
    return M, ref, views, images


@pytest.mark.parametrize("level", [0, 1])
def test_gradient_volume_of_identity_views(level):
    """Source views at the reference camera: P_l = Down^l(I), A^{w^-1}_i = the reference alpha
    weights of M_l, and the last four channels are M_l, all at the planes of S."""
    rng = np.random.default_rng(39)
    M, ref, views, images = _scene(rng, identity=True)
    N, k = len(views), 3
    Vs, S = oracle.gradient_volume(M, 1.0, 9.0, ref, views, images, k, level)
    Ml = oracle.down(M, level)
    Il = oracle.down(images, level)
    A = oracle.alpha_weights(Ml)
    S_want, _ = oracle.select_topk(A, k)
    assert np.array_equal(S, S_want)
    _, h, w, _ = Ml.shape
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    for j in range(k):
        d = S[j]
        for i in range(N):
            for c in range(3):
                assert np.max(np.abs(Vs[3 * i + c, j] - Il[i, ..., c])) < 1e-12
            assert np.max(np.abs(Vs[3 * N + i, j] - A[d, yy, xx])) < 1e-12
        for c in range(4):
            assert np.array_equal(Vs[4 * N + c, j], Ml[d, yy, xx, c])


def test_gradient_volume_keep_all_is_the_dense_volume_in_plane_order():
    """k = D keeps every plane in ascending order; the compacted volume is then the stack of
    the separately pinned parts: the PSV, the inverse-warped view alpha weights and M."""
    rng = np.random.default_rng(40)
    M, ref, views, images = _scene(rng)
    D, N = M.shape[0], len(views)
    near, far = 1.0, 9.0
    Vs, S = oracle.gradient_volume(M, near, far, ref, views, images, D, 0)
    assert np.array_equal(S, np.broadcast_to(np.arange(D, dtype=np.uint8)[:, None, None], S.shape))
    for i, v in enumerate(views):
        P = oracle.psv_view(images[i], D, near, far, ref, v)
        Ainv = oracle.inverse_warp_stack(oracle.view_alpha_weights(M, near, far, ref, v), near, far, ref, v)
        for c in range(3):
            assert np.array_equal(Vs[3 * i + c], P[..., c])
        assert np.array_equal(Vs[3 * N + i], Ainv)
    for c in range(4):
        assert np.array_equal(Vs[4 * N + c], M[..., c])


def test_gradient_volume_level_psv_is_the_downsampled_full_resolution_psv():
    """Sec. 3.2: the level-l PSV is Down^l of the full-resolution PSV (not a PSV of Down^l(I))."""
    rng = np.random.default_rng(41)
    M, ref, views, images = _scene(rng, D=3, H=8, W=8, N=1)
    near, far = 1.0, 9.0
    Vs, S = oracle.gradient_volume(M, near, far, ref, views, images, 3, 1)
    P = oracle.down(oracle.psv_view(images[0], 3, near, far, ref, views[0]), 1)
    for c in range(3):
        assert np.array_equal(Vs[c], P[..., c])
