"""Seeded synthetic scenes: the only input source shared by the CUDA path and the oracle.

This module draws cameras, source images, a ground-truth multi-plane image (MPI)
and a perturbed coarse MPI for the workloads the method is evaluated on.  It
holds none of the method's arithmetic: source and novel-view images come from
ray casting an analytic layered scene (each layer a 3D plane restricted to an
elliptical region of the reference image, with a smooth analytic colour field),
not from warping or compositing an MPI.  The ground-truth MPI is a
discretisation of the same scene onto D fronto-parallel planes in the reference
frustum (Sec. 3.1).

Camera convention (shared with the library and the oracle): world -> camera,
``x_cam = R @ X + t``; pixel = ``K @ x_cam / z`` with pixel centres on integer
coordinates.  The reference camera is ``K, R=I, t=0``, so the world frame is the
reference camera frame.

Shapes: images ``[N][H][W][3]`` float32 in [0,1]; MPIs ``[D][H][W][4]`` float32
(RGB, alpha), plane ``d=0`` farthest, ``d=D-1`` nearest.  Plane depths are
uniform in inverse depth between ``near`` and ``far``.

Workloads (stand-ins for the paper's forward-facing datasets, Sec. 5.2):
``small`` 128x96 D=8 N=3; ``paper`` 512x384 D=32 N=4 with 9 novel views;
``display`` 1920x1080 D=64 N=8 on a 4x2 grid with 45 views on an arc;
``serve_requests`` draws the Poisson request stream of the batched-serving
workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Camera", "Layer", "Scene", "intrinsics", "random_rotation", "look_at",
    "plane_inverse_depths", "make_scene", "raycast", "workload", "serve_requests",
    "WORKLOADS", "LgdWeights", "lgd_weights",
]


@dataclass
class Camera:
    """Pinhole camera, world->camera (``x_cam = R X + t``)."""

    K: np.ndarray
    R: np.ndarray
    t: np.ndarray

    def __post_init__(self):
        self.K = np.asarray(self.K, dtype=np.float64).reshape(3, 3)
        self.R = np.asarray(self.R, dtype=np.float64).reshape(3, 3)
        self.t = np.asarray(self.t, dtype=np.float64).reshape(3)

    @property
    def centre(self) -> np.ndarray:
        return -self.R.T @ self.t


def intrinsics(W: int, H: int, f: float | None = None) -> np.ndarray:
    """fx = fy = f (default W), principal point at the image centre."""
    f = float(W) if f is None else float(f)
    return np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])


def random_rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    """Rotation about an axis uniform on the sphere by an angle uniform in [0, max_deg]."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = math.radians(rng.uniform(0.0, max_deg))
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * Kx + (1 - math.cos(ang)) * (Kx @ Kx)


def look_at(centre: np.ndarray, target: np.ndarray, up=(0.0, -1.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """World->camera (R, t) for a camera at ``centre`` looking at ``target`` (+z forward, +y down)."""
    centre = np.asarray(centre, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - centre
    z /= np.linalg.norm(z)
    upv = np.asarray(up, dtype=np.float64)
    x = np.cross(-upv, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])  # rows: camera axes in world coordinates
    return R, -R @ centre


def plane_inverse_depths(D: int, near: float, far: float) -> np.ndarray:
    """Inverse depths of the D planes, uniform between 1/far (d=0) and 1/near (d=D-1)."""
    if D == 1:
        return np.array([1.0 / far])
    d = np.arange(D, dtype=np.float64)
    return 1.0 / far + d / (D - 1) * (1.0 / near - 1.0 / far)


@dataclass
class Layer:
    """A scene surface: plane ``n . X = 1`` (reference frame) inside an ellipse of the reference image."""

    n: np.ndarray
    ellipse: tuple | None  # (uc, vc, ru, rv, theta) in reference pixels; None = unbounded background
    colour: np.ndarray  # [3][T][4] cosine terms: amplitude, ku, kv, phase (plus base in colour_base)
    colour_base: np.ndarray  # [3]


@dataclass
class Scene:
    H: int
    W: int
    D: int
    near: float
    far: float
    ref: Camera
    src: list
    novel: list
    layers: list
    images: np.ndarray          # [N][H][W][3] float32, ray-cast + noise, clamped
    gt_mpi: np.ndarray          # [D][H][W][4] float32
    coarse_mpi: np.ndarray      # [D][H][W][4] float32 = clamp(gt + noise)
    novel_images: np.ndarray | None = None  # [T][H][W][3] float32 ray-cast, noise-free
    meta: dict = field(default_factory=dict)


def _colour_terms(rng, W, n_terms=4):
    """Smooth colour field parameters: per channel a base plus cosines of period >= W/4 px."""
    base = rng.uniform(0.2, 0.8, size=3)
    terms = np.empty((3, n_terms, 4))
    for c in range(3):
        for j in range(n_terms):
            period = rng.uniform(W / 4.0, W * 1.5)
            ang = rng.uniform(0, 2 * math.pi)
            k = 2 * math.pi / period
            terms[c, j] = (rng.uniform(0.03, 0.12), k * math.cos(ang), k * math.sin(ang), rng.uniform(0, 2 * math.pi))
    return base, terms


def _eval_colour(base, terms, u, v):
    out = np.empty(u.shape + (3,), dtype=np.float64)
    for c in range(3):
        acc = np.full(u.shape, base[c])
        for a, ku, kv, ph in terms[c]:
            acc += a * np.cos(ku * u + kv * v + ph)
        out[..., c] = acc
    return np.clip(out, 0.0, 1.0)


def _make_layers(rng, H, W, K, near, far, n_layers):
    fx, fy, cx, cy = K[0, 0], K[1, 1], K[0, 2], K[1, 2]
    layers = []
    # background: a gently slanted plane far away, covering everything
    rho_bg = rng.uniform(1.0 / far, min(0.1, 0.5 / near))
    gx, gy = rng.uniform(-0.2, 0.2, size=2) * rho_bg / W
    a = rho_bg
    base, terms = _colour_terms(rng, W)
    layers.append(Layer(n=np.array([gx * fx, gy * fy, a]), ellipse=None, colour=terms, colour_base=base))
    rho_lo, rho_hi = 1.0 / far, 1.0 / near
    for _ in range(n_layers):
        uc, vc = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        ru, rv = rng.uniform(0.08, 0.35) * W, rng.uniform(0.08, 0.35) * H
        theta = rng.uniform(0, math.pi)
        rho_c = rng.uniform(rho_lo + 0.1 * (rho_hi - rho_lo), rho_hi * 0.95)
        # slope keeps inverse depth inside [rho_lo, rho_hi] over the ellipse
        smax = 0.15 * min(rho_c - rho_lo, rho_hi - rho_c) / max(ru, rv)
        gx, gy = rng.uniform(-smax, smax, size=2)
        a = rho_c - gx * (uc - cx) - gy * (vc - cy)
        base, terms = _colour_terms(rng, W)
        layers.append(Layer(n=np.array([gx * fx, gy * fy, a]), ellipse=(uc, vc, ru, rv, theta),
                            colour=terms, colour_base=base))
    return layers


def raycast(layers, ref_K: np.ndarray, cam: Camera, H: int, W: int):
    """First-hit ray cast of the layered scene from ``cam``.

    Returns (colour [H][W][3] float64, depth_in_reference_frame [H][W], hit_u, hit_v) where
    hit_u/hit_v are the reference-image coordinates of each hit point.
    """
    fx, fy, cx, cy = ref_K[0, 0], ref_K[1, 1], ref_K[0, 2], ref_K[1, 2]
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    Kinv = np.linalg.inv(cam.K)
    m = np.stack([u, v, np.ones_like(u)], axis=-1) @ Kinv.T  # camera-frame directions
    dirs = m @ cam.R  # R^T applied to each row: world (= reference) frame
    C = cam.centre
    best_s = np.full((H, W), np.inf)
    best_l = np.full((H, W), -1, dtype=np.int64)
    for li, L in enumerate(layers):
        den = dirs @ L.n
        num = 1.0 - L.n @ C
        with np.errstate(divide="ignore", invalid="ignore"):
            s = num / den
        ok = np.isfinite(s) & (s > 0)
        X = C[None, None, :] + s[..., None] * dirs
        Z = X[..., 2]
        ok &= Z > 1e-9
        if L.ellipse is not None:
            uc, vc, ru, rv, th = L.ellipse
            with np.errstate(divide="ignore", invalid="ignore"):
                ur = fx * X[..., 0] / Z + cx - uc
                vr = fy * X[..., 1] / Z + cy - vc
            a = (ur * math.cos(th) + vr * math.sin(th)) / ru
            b = (-ur * math.sin(th) + vr * math.cos(th)) / rv
            ok &= (a * a + b * b) <= 1.0
        better = ok & (s < best_s)
        best_s = np.where(better, s, best_s)
        best_l = np.where(better, li, best_l)
    X = C[None, None, :] + best_s[..., None] * dirs
    Z = X[..., 2]
    hu = fx * X[..., 0] / Z + cx
    hv = fy * X[..., 1] / Z + cy
    col = np.zeros((H, W, 3))
    for li, L in enumerate(layers):
        sel = best_l == li
        if np.any(sel):
            col[sel] = _eval_colour(L.colour_base, L.colour, hu[sel], hv[sel])
    return col, Z, hu, hv


def _plane_colour_fields(rng, D, H, W):
    """Smooth random colours for every plane: [D][H][W][3] float32 (separable cosine sums)."""
    out = np.empty((D, H, W, 3), dtype=np.float32)
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[:, None]
    for d in range(D):
        acc = np.broadcast_to(rng.uniform(0.2, 0.8, size=3).astype(np.float32), (H, W, 3)).copy()
        for _ in range(2):
            kx = 2 * math.pi / rng.uniform(W / 4.0, 2.0 * W, size=3) * rng.choice([-1, 1], size=3)
            ky = 2 * math.pi / rng.uniform(H / 4.0, 2.0 * H, size=3) * rng.choice([-1, 1], size=3)
            ph = rng.uniform(0, 2 * math.pi, size=3)
            a = rng.uniform(0.05, 0.2, size=3)
            # cos(kx x + ky y + ph) = cos(kx x + ph) cos(ky y) - sin(kx x + ph) sin(ky y), per channel
            cxp, sxp = (a * np.cos(kx * x + ph)).astype(np.float32), (a * np.sin(kx * x + ph)).astype(np.float32)
            cy_, sy_ = np.cos(ky * y).astype(np.float32), np.sin(ky * y).astype(np.float32)
            acc += cy_[:, None, :] * cxp[None, :, :]
            acc -= sy_[:, None, :] * sxp[None, :, :]
        np.clip(acc, 0.0, 1.0, out=out[d])
    return out


def make_scene(seed: int, H: int, W: int, D: int, N: int, *, near: float = 1.0, far: float = 100.0,
               n_layers: tuple = (3, 8), src_poses: str = "random", novel: str = "grid3x3",
               n_novel: int = 9, image_noise: float = 0.01, mpi_noise: float = 0.05,
               render_novel_gt: bool = False, f: float | None = None) -> Scene:
    """Draw one synthetic scene (all arrays host numpy, fixed by ``seed``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = intrinsics(W, H, f)
    ref = Camera(K, np.eye(3), np.zeros(3))
    layers = _make_layers(rng, H, W, K, near, far, int(rng.integers(n_layers[0], n_layers[1] + 1)))

    src = []
    if src_poses == "random":
        for _ in range(N):
            R = random_rotation(rng, 2.0)
            t = rng.uniform(-0.1, 0.1, size=3)
            src.append(Camera(K, R, t))
    elif src_poses == "grid4x2":
        xs, ys = (-0.3, -0.1, 0.1, 0.3), (-0.1, 0.1)
        for yy in ys:
            for xx in xs:
                C = np.array([xx, yy, 0.0])
                src.append(Camera(K, np.eye(3), -C))
        src = src[:N]
    else:
        raise ValueError(src_poses)

    images = np.empty((N, H, W, 3), dtype=np.float32)
    for i, cam in enumerate(src):
        col, _, _, _ = raycast(layers, K, cam, H, W)
        col += image_noise * rng.standard_normal(size=col.shape)
        images[i] = np.clip(col, 0.0, 1.0)

    # ground-truth MPI: reference depth map discretised onto the planes
    col_r, Z, _, _ = raycast(layers, K, ref, H, W)
    rho = plane_inverse_depths(D, near, far)
    inv = np.clip(1.0 / Z, rho[0], rho[-1])
    gt = np.zeros((D, H, W, 4), dtype=np.float32)
    gt[..., :3] = _plane_colour_fields(rng, D, H, W)
    if D == 1:
        gt[0, ..., 3] = 1.0
        gt[0, ..., :3] = col_r
    else:
        dlo = np.clip(np.searchsorted(rho, inv, side="right") - 1, 0, D - 2)
        w = (inv - rho[dlo]) / (rho[dlo + 1] - rho[dlo])
        yy, xx = np.mgrid[0:H, 0:W]
        gt[dlo, yy, xx, 3] = 1.0
        gt[dlo + 1, yy, xx, 3] = w.astype(np.float32)
        gt[dlo, yy, xx, :3] = col_r
        gt[dlo + 1, yy, xx, :3] = col_r
    coarse = np.empty_like(gt)
    rng.standard_normal(dtype=np.float32, out=coarse)
    coarse *= np.float32(mpi_noise)
    coarse += gt
    np.clip(coarse, 0.0, 1.0, out=coarse)

    novel_cams = []
    if novel == "grid3x3":
        cs = np.array([c.centre for c in src])
        gx = np.linspace(cs[:, 0].min(), cs[:, 0].max(), 3)
        gy = np.linspace(cs[:, 1].min(), cs[:, 1].max(), 3)
        for yy_ in gy:
            for xx_ in gx:
                C = np.array([xx_, yy_, 0.0])
                novel_cams.append(Camera(K, np.eye(3), -C))
        novel_cams = novel_cams[:n_novel]
    elif novel == "arc":
        zf = 2.0 / (1.0 / near + 1.0 / far)  # harmonic mean of near and far
        target = np.array([0.0, 0.0, zf])
        for x in np.linspace(-0.2, 0.2, n_novel):
            # on a circle of radius zf about the target, through the reference centre
            phi = math.asin(x / zf)
            C = np.array([zf * math.sin(phi), 0.0, zf - zf * math.cos(phi)])
            R, t = look_at(C, target)
            novel_cams.append(Camera(K, R, t))
    elif novel == "none":
        pass
    else:
        raise ValueError(novel)

    novel_images = None
    if render_novel_gt and novel_cams:
        novel_images = np.stack([raycast(layers, K, c, H, W)[0] for c in novel_cams]).astype(np.float32)

    return Scene(H=H, W=W, D=D, near=near, far=far, ref=ref, src=src, novel=novel_cams, layers=layers,
                 images=images, gt_mpi=gt, coarse_mpi=coarse, novel_images=novel_images,
                 meta={"seed": seed, "n_layers": len(layers) - 1})


# The evaluated workloads: (H, W, D, N, k, schedule, novel views, dtype)
WORKLOADS = {
    "small": dict(H=96, W=128, D=8, N=3, k=5, schedule=(2, 1, 0), n_layers=(3, 6), src_poses="random",
                  novel="grid3x3", n_novel=9, dtype="f32"),
    "paper": dict(H=384, W=512, D=32, N=4, k=5, schedule=(2, 1, 0), n_layers=(3, 8), src_poses="random",
                  novel="grid3x3", n_novel=9, dtype="f32"),
    "paper_bf16": dict(H=384, W=512, D=32, N=4, k=5, schedule=(2, 1, 0), n_layers=(3, 8), src_poses="random",
                       novel="grid3x3", n_novel=9, dtype="bf16"),
    "display": dict(H=1080, W=1920, D=64, N=8, k=5, schedule=(2, 1, 0), n_layers=(5, 12), src_poses="grid4x2",
                    novel="arc", n_novel=45, dtype="bf16"),
}


def workload(name: str, seed: int = 0, **overrides) -> tuple[Scene, dict]:
    """Scene and settings of a named workload."""
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    sc = make_scene(seed, cfg["H"], cfg["W"], cfg["D"], cfg["N"], n_layers=cfg["n_layers"],
                    src_poses=cfg["src_poses"], novel=cfg["novel"], n_novel=cfg["n_novel"])
    return sc, cfg


def serve_requests(n: int = 2000, rate: float = 200.0, seed: int = 12345) -> list[dict]:
    """Poisson request stream of the batched-serving workload (arrival times in seconds)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    res = [(192, 256), (384, 512), (576, 768), (768, 1024)]
    t = 0.0
    out = []
    for r in range(n):
        t += rng.exponential(1.0 / rate)
        H, W = res[int(rng.integers(0, 4))]
        out.append(dict(id=r, arrival=t, H=H, W=W, D=int(rng.choice([16, 32, 48, 64])),
                        N=int(rng.integers(2, 7)), iters=int(rng.integers(2, 4)), seed=int(rng.integers(0, 2**31))))
    return out


@dataclass
class LgdWeights:
    """Random parameters of the learned-update network (no trained weights exist here):
    ``conv_w[l]`` [F][C_l][3][3][3] and ``conv_b[l]`` [F] for the five 3x3x3 blocks, their
    batch-norm statistics and affine terms ``bn_gamma/bn_beta/bn_mean/bn_var[l]`` [F], and the
    final 1x1x1 layer ``out_w`` [4][F], ``out_b`` [4].  All float32."""
    conv_w: list
    conv_b: list
    bn_gamma: list
    bn_beta: list
    bn_mean: list
    bn_var: list
    out_w: np.ndarray
    out_b: np.ndarray
    eps: float = 1e-5


def lgd_weights(seed: int, c_in: int, width: int = 32, blocks: int = 5) -> LgdWeights:
    """He-normal convolution weights and plausible batch-norm statistics, fixed by ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cw, cb, g, b, m, v = [], [], [], [], [], []
    c = c_in
    for _ in range(blocks):
        fan_in = c * 27
        cw.append((rng.standard_normal((width, c, 3, 3, 3)) * math.sqrt(2.0 / fan_in)).astype(np.float32))
        cb.append((rng.standard_normal(width) * 0.05).astype(np.float32))
        g.append(rng.uniform(0.5, 1.5, width).astype(np.float32))
        b.append((rng.standard_normal(width) * 0.1).astype(np.float32))
        m.append((rng.standard_normal(width) * 0.1).astype(np.float32))
        v.append(rng.uniform(0.5, 2.0, width).astype(np.float32))
        c = width
    out_w = (rng.standard_normal((4, width)) * math.sqrt(1.0 / width) * 0.1).astype(np.float32)
    out_b = np.zeros(4, dtype=np.float32)
    return LgdWeights(cw, cb, g, b, m, v, out_w, out_b)
