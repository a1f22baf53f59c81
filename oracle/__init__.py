"""FP64 CPU oracle of the RealLiFe HSGD hot path (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never loads it and shares no code with it; the two meet only
through the seeded inputs of ``scenegen``.

The arithmetic lives in ``reallife_oracle.c`` (plain loops, ``double``), built
here with gcc and loaded through ctypes.  Each wrapper below states the equation
of the paper it follows; see the C file's header for the readings of the paper
it fixes (plane spacing, camera convention, loss, tie rule, level schedule).

Parity status: every function is pinned by the tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, brute force, finite
differences, hand-derived fixtures under ``tests/golden/``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "reallife_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libreallife_oracle.so")
_lock = threading.Lock()
_lib = None


class _Cam(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


_LIB_OMP_PATH = os.path.join(_HERE, "libreallife_oracle_omp.so")
_lib_omp = None
_use_threads = False


def _compile(path: str, extra: list[str]):
    tmp = path + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", *extra,
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, path)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction) if needed: the serial
    library and the OpenMP one (bit-identical results, all host cores)."""
    for path, extra in ((_LIB_PATH, []), (_LIB_OMP_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            _compile(path, extra)
    return _LIB_PATH


def set_threads(on: bool) -> None:
    """Run the oracle's parallel loops on all host cores (the OpenMP build) or on one."""
    global _use_threads
    _use_threads = bool(on)


def num_threads() -> int:
    """Threads of the build in use (OpenMP: OMP_NUM_THREADS or the cores this process may use)."""
    return int(_load().orc_num_threads())


def _load():
    with _lock:
        return _load_locked()


def _load_locked():
    global _lib, _lib_omp
    if _use_threads:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(ctypes.CDLL(_LIB_OMP_PATH))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(lib):
    P = ctypes.POINTER
    d, i, dp = ctypes.c_double, ctypes.c_int, P(ctypes.c_double)
    cam = P(_Cam)
    u8p, u64p = P(ctypes.c_uint8), P(ctypes.c_uint64)
    lib.orc_plane_inverse_depths.argtypes = [i, d, d, dp]
    lib.orc_camera_at_level.argtypes = [cam, i, cam]
    lib.orc_view_to_ref.argtypes = [cam, cam, d, d, d, dp, dp]
    lib.orc_view_to_ref.restype = i
    lib.orc_render.argtypes = [dp, i, i, i, d, d, cam, cam, dp]
    ip = P(ctypes.c_int)
    lib.orc_render_pixels.argtypes = [dp, i, i, i, d, d, cam, cam, i, ip, ip, dp]
    lib.orc_vjp.argtypes = [dp, i, i, i, d, d, cam, cam, i, dp, dp]
    lib.orc_loss_grad.argtypes = [dp, i, i, i, d, d, cam, dp, cam, i, dp, dp]
    lib.orc_loss_grad.restype = d
    lib.orc_alpha_weights.argtypes = [dp, i, i, i, dp]
    lib.orc_select_topk.argtypes = [dp, i, i, i, i, u8p, u64p]
    lib.orc_downsample2.argtypes = [dp, i, i, i, i, dp]
    lib.orc_down_levels.argtypes = [dp, i, i, i, i, i, dp]
    lib.orc_hsgd_step.argtypes = [dp, i, i, i, d, d, cam, dp, cam, i, i, d, i, i, u8p, u8p, dp]
    lib.orc_hsgd_step.restype = i
    lib.orc_hsgd_step2.argtypes = [dp, i, i, i, d, d, cam, dp, cam, i, i, d, i, i, i, d, u8p, u8p, dp]
    lib.orc_hsgd_step2.restype = i
    lib.orc_select_mvs.argtypes = [dp, i, i, i, i, u8p, u64p]
    lib.orc_sparsity_grad.argtypes = [d, i, i, i]
    lib.orc_sparsity_grad.restype = d
    lib.orc_sparsity_loss.argtypes = [dp, i, i, i]
    lib.orc_sparsity_loss.restype = d
    lib.orc_gd_step.argtypes = [dp, i, i, i, d, d, cam, dp, cam, i, d, i, i, dp]
    lib.orc_gd_step.restype = i
    lib.orc_ref_to_view.argtypes = [cam, cam, d, d, d, dp, dp]
    lib.orc_ref_to_view.restype = i
    lib.orc_view_alpha_weights.argtypes = [dp, i, i, i, d, d, cam, cam, dp]
    lib.orc_psv_view.argtypes = [dp, i, i, i, d, d, cam, cam, dp]
    lib.orc_inverse_warp_stack.argtypes = [dp, i, i, i, d, d, cam, cam, dp]
    lib.orc_gradient_volume.argtypes = [dp, i, i, i, d, d, cam, dp, cam, i, i, i, i, u8p, u8p, dp]
    lib.orc_gradient_volume.restype = i
    lib.orc_num_threads.restype = i
    lib.orc_grad_voxels.argtypes = [dp, i, i, i, d, d, cam, dp, cam, i, i, ip, ip, ip, i, dp]
    return lib


def _cam(c) -> _Cam:
    s = _Cam()
    s.K[:] = np.asarray(c.K, dtype=np.float64).reshape(9).tolist()
    s.R[:] = np.asarray(c.R, dtype=np.float64).reshape(9).tolist()
    s.t[:] = np.asarray(c.t, dtype=np.float64).reshape(3).tolist()
    return s


def _cams(cs):
    arr = (_Cam * len(cs))()
    for j, c in enumerate(cs):
        arr[j] = _cam(c)
    return arr


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def plane_inverse_depths(D: int, near: float, far: float) -> np.ndarray:
    """rho_d, uniform in inverse depth from 1/far (d=0) to 1/near (d=D-1)."""
    out = np.empty(D)
    _load().orc_plane_inverse_depths(D, near, far, _ptr(out))
    return out


def camera_at_level(cam, level: int):
    """(K, R, t) of ``cam`` at pyramid level ``level`` (f / 2^l, c' = (c+0.5)/2^l - 0.5)."""
    out = _Cam()
    _load().orc_camera_at_level(ctypes.byref(_cam(cam)), level, ctypes.byref(out))
    return (np.array(out.K[:]).reshape(3, 3), np.array(out.R[:]).reshape(3, 3), np.array(out.t[:]))


def view_to_ref(ref, view, z: float, u: float, v: float):
    """Reference pixel hit by the view's ray through (u, v) on the plane at depth z; None if not met."""
    px, py = ctypes.c_double(), ctypes.c_double()
    ok = _load().orc_view_to_ref(ctypes.byref(_cam(ref)), ctypes.byref(_cam(view)), z, u, v,
                                 ctypes.byref(px), ctypes.byref(py))
    return (px.value, py.value) if ok else None


def render(M, near: float, far: float, ref, view) -> np.ndarray:
    """Eq. (eq_render) / (eq_over): view of the MPI ``M[D][H][W][4]`` -> ``[H][W][3]``."""
    M = _f64(M)
    D, H, W, _ = M.shape
    out = np.empty((H, W, 3))
    _load().orc_render(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), ctypes.byref(_cam(view)), _ptr(out))
    return out


def render_pixels(M, near: float, far: float, ref, view, xs, ys) -> np.ndarray:
    """Eq. (eq_render) at the listed view pixels only -> ``[n][3]``."""
    M = _f64(M)
    D, H, W, _ = M.shape
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    out = np.empty((len(xs), 3))
    _load().orc_render_pixels(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), ctypes.byref(_cam(view)),
                              len(xs), _ptr(xs, ctypes.c_int), _ptr(ys, ctypes.c_int), _ptr(out))
    return out


def vjp(M, near: float, far: float, ref, views, g_out) -> np.ndarray:
    """dL/dM given dL/dC for each view (``g_out[N][H][W][3]``): the exact adjoint of warp + composite."""
    M = _f64(M)
    D, H, W, _ = M.shape
    g_out = _f64(g_out)
    grad = np.zeros_like(M)
    _load().orc_vjp(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), _cams(views), len(views),
                    _ptr(g_out), _ptr(grad))
    return grad


def loss_grad(M, near: float, far: float, ref, views, images, want_grad: bool = True, want_renders: bool = False):
    """Photometric loss 1/(2N) sum (C - I)^2 and its gradient dL/dM (dense)."""
    M = _f64(M)
    D, H, W, _ = M.shape
    images = _f64(images)
    N = len(views)
    grad = np.empty_like(M) if want_grad else None
    rend = np.empty((N, H, W, 3)) if want_renders else None
    L = _load().orc_loss_grad(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), _ptr(images), _cams(views), N,
                              _ptr(grad) if want_grad else None, _ptr(rend) if want_renders else None)
    return L, grad, rend


def alpha_weights(M) -> np.ndarray:
    """Reference-view A_d = alpha_d prod_{j>d} (1 - alpha_j) -> ``[D][H][W]`` (Eq. eq_gradient)."""
    M = _f64(M)
    D, H, W, _ = M.shape
    A = np.empty((D, H, W))
    _load().orc_alpha_weights(_ptr(M), D, H, W, _ptr(A))
    return A


def select_topk(A, k: int):
    """Top-k planes per pixel by key (ties to lower d), ascending: (S[k][H][W] uint8, mask[H][W] uint64)."""
    A = _f64(A)
    D, H, W = A.shape
    S = np.empty((k, H, W), dtype=np.uint8)
    mask = np.empty((H, W), dtype=np.uint64)
    _load().orc_select_topk(_ptr(A), D, H, W, k, _ptr(S, ctypes.c_uint8), _ptr(mask, ctypes.c_uint64))
    return S, mask


def select_mvs(A, k: int):
    """MVS-sampling window: argmax plane (ties to lower d) and (k-1)/2 neighbours each side."""
    A = _f64(A)
    D, H, W = A.shape
    S = np.empty((k, H, W), dtype=np.uint8)
    mask = np.empty((H, W), dtype=np.uint64)
    _load().orc_select_mvs(_ptr(A), D, H, W, k, _ptr(S, ctypes.c_uint8), _ptr(mask, ctypes.c_uint64))
    return S, mask


def sparsity_loss(M) -> float:
    """L_s = mean log(1.5 - |0.5 - alpha|) over all voxels (Sec. 3.4)."""
    M = _f64(M)
    D, H, W, _ = M.shape
    return _load().orc_sparsity_loss(_ptr(M), D, H, W)


def sparsity_grad(alpha: float, D: int, H: int, W: int) -> float:
    """dL_s/dalpha of one voxel."""
    return _load().orc_sparsity_grad(float(alpha), D, H, W)


def down(x, level: int) -> np.ndarray:
    """Down^l over the two spatial axes of ``x[P][H][W][C]`` (l successive 2x2 box averages)."""
    x = _f64(x)
    P, H, W, C = x.shape
    out = np.empty((P, H >> level, W >> level, C))
    _load().orc_down_levels(_ptr(x), P, H, W, C, level, _ptr(out))
    return out


def grad_voxels(M, near: float, far: float, ref, views, images, ds, ys, xs, radius: int = 3) -> np.ndarray:
    """dL/dM of the photometric loss at the voxels (ds[j], ys[j], xs[j]): ``[n][4]``, equal to the
    dense gradient of ``loss_grad`` there, by brute force over the view pixels near the voxel's
    projection (for problems whose dense gradient is too large to form)."""
    M = _f64(M)
    D, H, W, _ = M.shape
    images = _f64(images)
    ds, ys, xs = (np.ascontiguousarray(a, dtype=np.int32) for a in (ds, ys, xs))
    n = len(ds)
    assert len(ys) == n and len(xs) == n
    assert np.all((ds >= 0) & (ds < D) & (ys >= 0) & (ys < H) & (xs >= 0) & (xs < W))
    out = np.empty((n, 4))
    ip = ctypes.POINTER(ctypes.c_int)
    _load().orc_grad_voxels(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), _ptr(images), _cams(views),
                            len(views), n, ds.ctypes.data_as(ip), ys.ctypes.data_as(ip), xs.ctypes.data_as(ip),
                            int(radius), _ptr(out))
    return out


def hsgd_step(M, near, far, ref, views, images, k: int, lam: float = 1.0, clamp: bool = True, level: int = 0,
              S_pin=None, selection: int = 0, lambda_s: float = 0.0):
    """One HSGD iteration (Sec. 3.3) at ``level`` on a copy of ``M``: returns (M_new, loss, S).

    selection 0: top-k by the reference alpha weight; 1: MVS-sampling window.
    lambda_s: weight of the sparsity prior L_s (Sec. 3.4) added to the descent direction."""
    M = _f64(M).copy()
    D, H, W, _ = M.shape
    images = _f64(images)
    h, w = H >> level, W >> level
    S = np.empty((k, h, w), dtype=np.uint8)
    pin = None
    if S_pin is not None:
        pin = np.ascontiguousarray(S_pin, dtype=np.uint8)
        assert pin.shape == (k, h, w)
    L = ctypes.c_double()
    rc = _load().orc_hsgd_step2(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), _ptr(images), _cams(views),
                                len(views), k, lam, int(clamp), level, int(selection), float(lambda_s),
                                _ptr(pin, ctypes.c_uint8) if pin is not None else None, _ptr(S, ctypes.c_uint8),
                                ctypes.byref(L))
    if rc:
        raise ValueError("oracle hsgd_step: invalid arguments")
    return M, L.value, S


def gd_step(M, near, far, ref, views, images, lam: float = 1.0, clamp: bool = True, level: int = 0):
    """Dense analytic gradient-descent step (Sec. 3.1) at ``level``: returns (M_new, loss)."""
    M = _f64(M).copy()
    D, H, W, _ = M.shape
    images = _f64(images)
    L = ctypes.c_double()
    rc = _load().orc_gd_step(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), _ptr(images), _cams(views),
                             len(views), lam, int(clamp), level, ctypes.byref(L))
    if rc:
        raise ValueError("oracle gd_step: invalid arguments")
    return M, L.value


def refine(M, near, far, ref, views, images, k: int, schedule=(2, 1, 0), lam: float = 1.0, clamp: bool = True,
           S_pins=None, selection: int = 0, lambda_s: float = 0.0):
    """HSGD refinement: one ``hsgd_step`` per entry of ``schedule``; returns (M, losses, selections)."""
    losses, sels = [], []
    for it, level in enumerate(schedule):
        M, L, S = hsgd_step(M, near, far, ref, views, images, k, lam, clamp, level,
                            None if S_pins is None else S_pins[it], selection, lambda_s)
        losses.append(L)
        sels.append(S)
    return M, losses, sels


def ref_to_view(ref, view, z: float, u: float, v: float):
    """Inverse warp of Eq. (eq_homo): view pixel of reference pixel (u, v) on the plane at depth z; None if
    the point is behind the view."""
    x, y = ctypes.c_double(), ctypes.c_double()
    ok = _load().orc_ref_to_view(ctypes.byref(_cam(ref)), ctypes.byref(_cam(view)), z, u, v,
                                 ctypes.byref(x), ctypes.byref(y))
    return (x.value, y.value) if ok else None


def view_alpha_weights(M, near: float, far: float, ref, view) -> np.ndarray:
    """Alpha weights of the MPI warped into ``view`` (Eq. eq_gradient on M_i) -> ``[D][H][W]``."""
    M = _f64(M)
    D, H, W, _ = M.shape
    A = np.empty((D, H, W))
    _load().orc_view_alpha_weights(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), ctypes.byref(_cam(view)),
                                   _ptr(A))
    return A


def psv_view(image, D: int, near: float, far: float, ref, view) -> np.ndarray:
    """Plane sweep volume of one source view (Sec. 3.2): ``image[H][W][3]`` -> ``[D][H][W][3]``."""
    image = _f64(image)
    H, W, _ = image.shape
    P = np.empty((D, H, W, 3))
    _load().orc_psv_view(_ptr(image), D, H, W, near, far, ctypes.byref(_cam(ref)), ctypes.byref(_cam(view)), _ptr(P))
    return P


def inverse_warp_stack(X, near: float, far: float, ref, view) -> np.ndarray:
    """Inverse warp of view-frame maps ``X[D][H][W]`` into the reference frame (Sec. 3.3)."""
    X = _f64(X)
    D, H, W = X.shape
    out = np.empty((D, H, W))
    _load().orc_inverse_warp_stack(_ptr(X), D, H, W, near, far, ctypes.byref(_cam(ref)), ctypes.byref(_cam(view)),
                                   _ptr(out))
    return out


def gradient_volume(M, near, far, ref, views, images, k: int, level: int = 0, selection: int = 0, S_pin=None):
    """Sparsified gradient volume V_s (Sec. 3.3, Eq. eq_simplifiedGradients / eq_V) at ``level``:
    returns (Vs[4N+4][k][h][w], S[k][h][w]).  Channels: P_l (3N, view-major), A^{w^-1} (N), M_l (4)."""
    M = _f64(M)
    D, H, W, _ = M.shape
    images = _f64(images)
    N = len(views)
    h, w = H >> level, W >> level
    S = np.empty((k, h, w), dtype=np.uint8)
    Vs = np.empty((4 * N + 4, k, h, w))
    pin = None
    if S_pin is not None:
        pin = np.ascontiguousarray(S_pin, dtype=np.uint8)
        assert pin.shape == (k, h, w)
    rc = _load().orc_gradient_volume(_ptr(M), D, H, W, near, far, ctypes.byref(_cam(ref)), _ptr(images),
                                     _cams(views), N, k, level, int(selection),
                                     _ptr(pin, ctypes.c_uint8) if pin is not None else None,
                                     _ptr(S, ctypes.c_uint8), _ptr(Vs))
    if rc:
        raise ValueError("oracle gradient_volume: invalid arguments")
    return Vs, S
