"""Python binding of libreallife: the GB300 (sm_103a) RealLiFe hot path.

Argument marshalling only.  Every step (warp, composite, loss, adjoint, selection,
update, rendering) runs in the CUDA kernels behind the C ABI of ``include/reallife.h``;
the functions here carry the same names as the C entry points, take CUDA tensors
(PyTorch supplies device memory and streams) and host cameras, and raise
``RealLifeError`` when the library reports a failure.  There is no CPU fallback:
importing works without a GPU, but every call needs the built library and a CUDA
device.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

__all__ = [
    "RealLifeError", "Mpi", "make_mpi",
    "reallife_workspace_bytes", "reallife_render", "reallife_hsgd_step", "reallife_refine",
    "reallife_downsample_f32", "reallife_select", "reallife_select_keys", "reallife_loss_grad",
    "reallife_sparse_update", "reallife_render_backward", "reallife_warp_offsets",
    "reallife_trace_enable", "reallife_trace_read", "reallife_strerror", "workspace", "library_path",
    "reallife_set_kernel_path", "reallife_device_status", "reallife_hsgd_step_noalloc",
    "reallife_trace_release_captured", "reallife_selftest_wait_timeout", "reallife_selftest_bounds",
    "reallife_debug_build", "reallife_metrics_workspace_bytes", "reallife_image_metrics", "reallife_kept_mass",
    "BatchItem", "BatchTable", "batch_c_item", "reallife_batch_table_bytes", "reallife_batch_prepare", "reallife_hsgd_step_batch",
]

RealLifeError = _lib.RealLifeError
F32, BF16 = 0, 1
SELECT_TOPK, SELECT_MVS = 0, 1
_DT = {torch.float32: F32, torch.bfloat16: BF16}


def library_path() -> str:
    return _lib.path()


class Mpi:
    """A device MPI ``[D][H][W][4]`` (float32 or bfloat16) in the frustum of ``ref``."""

    def __init__(self, data: torch.Tensor, near: float, far: float, ref):
        if data.dim() != 4 or data.shape[-1] != 4:
            raise ValueError("MPI tensor must be [D][H][W][4]")
        if data.dtype not in _DT:
            raise ValueError("MPI dtype must be float32 or bfloat16")
        if not data.is_cuda or not data.is_contiguous():
            raise ValueError("MPI tensor must be a contiguous CUDA tensor")
        self.data = data
        self.near = float(near)
        self.far = float(far)
        self.ref = ref

    @property
    def D(self):
        return self.data.shape[0]

    @property
    def H(self):
        return self.data.shape[1]

    @property
    def W(self):
        return self.data.shape[2]

    def c_struct(self) -> _lib.RlMpi:
        s = _lib.RlMpi()
        s.D, s.H, s.W = self.D, self.H, self.W
        s.near_, s.far_ = self.near, self.far
        s.dtype = _DT[self.data.dtype]
        s.data = ctypes.c_void_p(self.data.data_ptr())
        s.ref = _lib.camera(self.ref)
        return s


def make_mpi(data: torch.Tensor, near: float, far: float, ref) -> Mpi:
    return Mpi(data, near, far, ref)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check_f32(t: torch.Tensor, shape, name):
    if t.dtype != torch.float32 or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be float32 {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")


def _params(k, lam, clamp, level, selection=SELECT_TOPK, lambda_s=0.0) -> _lib.RlHsgdParams:
    p = _lib.RlHsgdParams()
    p.k, p.lambda_, p.clamp01, p.level = int(k), float(lam), int(bool(clamp)), int(level)
    p.selection, p.lambda_s = int(selection), float(lambda_s)
    return p


# ------------------------------------------------------------------ entry points

def reallife_workspace_bytes(N: int, D: int, H: int, W: int, k: int, dtype=torch.float32) -> int:
    return int(_lib.lib().reallife_workspace_bytes(N, D, H, W, k, _DT[dtype]))


def workspace(N: int, D: int, H: int, W: int, k: int, dtype=torch.float32, device="cuda") -> torch.Tensor:
    """A caller-owned workspace tensor (uint8, 256-byte aligned) for hsgd_step / refine."""
    n = reallife_workspace_bytes(N, D, H, W, k, dtype)
    return torch.empty(n, dtype=torch.uint8, device=device)


def reallife_render(m: Mpi, cams, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Novel views of the MPI for every camera in ``cams``: ``[T][H][W][3]`` float32."""
    T = len(cams)
    if out is None:
        out = torch.empty((T, m.H, m.W, 3), dtype=torch.float32, device=m.data.device)
    _check_f32(out, (T, m.H, m.W, 3), "out")
    ms = m.c_struct()
    _lib.check("reallife_render", _lib.lib().reallife_render(ctypes.byref(ms), _lib.cameras(cams), T,
                                                            _ptr(out), _stream(stream)))
    return out


def reallife_hsgd_step(m: Mpi, images: torch.Tensor, src, k: int, lam: float = 1.0, clamp: bool = True,
                       level: int = 0, loss_out: torch.Tensor | None = None, S_out: torch.Tensor | None = None,
                       ws: torch.Tensor | None = None, stream=None, selection: int = SELECT_TOPK,
                       lambda_s: float = 0.0):
    """One HSGD iteration on ``m`` in place; returns (loss_out, S_out)."""
    N = len(src)
    _check_f32(images, (N, m.H, m.W, 3), "images")
    if ws is None:
        ws = workspace(N, m.D, m.H, m.W, k, m.data.dtype, m.data.device)
    ms = m.c_struct()
    p = _params(k, lam, clamp, level, selection, lambda_s)
    _lib.check("reallife_hsgd_step", _lib.lib().reallife_hsgd_step(
        ctypes.byref(ms), _ptr(images), _lib.cameras(src), N, ctypes.byref(p), _ptr(loss_out), _ptr(S_out),
        _ptr(ws), ws.numel(), _stream(stream)))
    return loss_out, S_out


def reallife_hsgd_step_noalloc(m: Mpi, images: torch.Tensor, src, k: int, lam: float = 1.0, clamp: bool = True,
                               level: int = 0, loss_out: torch.Tensor | None = None,
                               S_out: torch.Tensor | None = None, stream=None, selection: int = SELECT_TOPK,
                               lambda_s: float = 0.0):
    """One HSGD iteration without a caller workspace (for callers that cannot allocate):
    the library's fixed per-device scratch array is used instead.  Same results as
    ``reallife_hsgd_step``; calls that overlap on the GPU race on the shared array."""
    N = len(src)
    _check_f32(images, (N, m.H, m.W, 3), "images")
    ms = m.c_struct()
    p = _params(k, lam, clamp, level, selection, lambda_s)
    _lib.check("reallife_hsgd_step_noalloc", _lib.lib().reallife_hsgd_step_noalloc(
        ctypes.byref(ms), _ptr(images), _lib.cameras(src), N, ctypes.byref(p), _ptr(loss_out), _ptr(S_out),
        _stream(stream)))
    return loss_out, S_out


def reallife_refine(m: Mpi, images: torch.Tensor, src, k: int, schedule=(2, 1, 0), lam: float = 1.0,
                    clamp: bool = True, loss_per_iter: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                    stream=None, selection: int = SELECT_TOPK, lambda_s: float = 0.0):
    """HSGD refinement of ``m`` in place over the level schedule; returns ``loss_per_iter``."""
    N = len(src)
    _check_f32(images, (N, m.H, m.W, 3), "images")
    if ws is None:
        ws = workspace(N, m.D, m.H, m.W, k, m.data.dtype, m.data.device)
    sched = (ctypes.c_int * len(schedule))(*[int(s) for s in schedule])
    ms = m.c_struct()
    p = _params(k, lam, clamp, 0, selection, lambda_s)
    _lib.check("reallife_refine", _lib.lib().reallife_refine(
        ctypes.byref(ms), _ptr(images), _lib.cameras(src), N, ctypes.byref(p), sched, len(schedule),
        _ptr(loss_per_iter), _ptr(ws), ws.numel(), _stream(stream)))
    return loss_per_iter


class BatchItem:
    """One request's HSGD iteration in a batched step: the arguments of ``reallife_hsgd_step``."""

    def __init__(self, m: Mpi, images: torch.Tensor, src, k: int, ws: torch.Tensor, level: int = 0,
                 loss_out: torch.Tensor | None = None, lam: float = 1.0, clamp: bool = True,
                 selection: int = SELECT_TOPK, lambda_s: float = 0.0):
        _check_f32(images, (len(src), m.H, m.W, 3), "images")
        self.m, self.images, self.src, self.k, self.ws, self.level = m, images, src, int(k), ws, int(level)
        self.loss_out, self.lam, self.clamp, self.selection, self.lambda_s = loss_out, lam, clamp, selection, lambda_s


class BatchTable:
    """Work table of a batched step for up to ``max_items`` requests: page-locked host memory
    (written by ``reallife_batch_prepare``) and its device copy."""

    def __init__(self, max_items: int, device="cuda"):
        self.max_items = int(max_items)
        self.nbytes = reallife_batch_table_bytes(self.max_items)
        if self.nbytes == 0:
            raise ValueError(f"max_items={max_items} outside the library's range")
        self.host = torch.empty(self.nbytes, dtype=torch.uint8).pin_memory()
        self.dev = torch.empty(self.nbytes, dtype=torch.uint8, device=device)


def reallife_batch_table_bytes(max_items: int) -> int:
    return int(_lib.lib().reallife_batch_table_bytes(int(max_items)))


def batch_c_item(it: BatchItem):
    """The C struct of one batch item and the host objects it points to (keep them alive while
    the struct is in use); its ``params.level`` and ``loss_out`` may be changed in place."""
    ms = it.m.c_struct()
    cams = _lib.cameras(it.src)
    b = _lib.RlBatchItem()
    b.mpi = ctypes.pointer(ms)
    b.images = _ptr(it.images)
    b.src = ctypes.cast(cams, ctypes.POINTER(_lib.RlCamera))
    b.N = len(it.src)
    b.params = _params(it.k, it.lam, it.clamp, it.level, it.selection, it.lambda_s)
    b.loss_out = _ptr(it.loss_out)
    b.ws = _ptr(it.ws)
    b.ws_bytes = it.ws.numel()
    return b, (ms, cams)


def reallife_batch_prepare(items, table: BatchTable):
    """Write the work table of one HSGD iteration of every item (host only).  ``items``:
    ``BatchItem`` objects, or C structs from ``batch_c_item``."""
    n = len(items)
    keep = []
    cs = []
    for it in items:
        if isinstance(it, _lib.RlBatchItem):
            cs.append(it)
        else:
            b, k = batch_c_item(it)
            cs.append(b)
            keep.append(k)
    arr = (_lib.RlBatchItem * max(n, 1))(*cs)
    _lib.check("reallife_batch_prepare", _lib.lib().reallife_batch_prepare(
        arr, n, ctypes.c_void_p(table.host.data_ptr()), table.nbytes))


def reallife_hsgd_step_batch(table: BatchTable, items=None, stream=None):
    """One HSGD iteration of every request of the table in one launch per stage (selection,
    gradient, update); with ``items`` the table is first written from them."""
    if items is not None:
        reallife_batch_prepare(items, table)
    _lib.check("reallife_hsgd_step_batch", _lib.lib().reallife_hsgd_step_batch(
        ctypes.c_void_p(table.host.data_ptr()), _ptr(table.dev), table.nbytes, _stream(stream)))


def reallife_gradient_volume_workspace_bytes(N: int, D: int, H: int, W: int, k: int, dtype=torch.float32) -> int:
    return int(_lib.lib().reallife_gradient_volume_workspace_bytes(N, D, H, W, k, _DT[dtype]))


def reallife_gradient_volume(m: Mpi, images: torch.Tensor, src, k: int, level: int = 0,
                             selection: int = SELECT_TOPK, V: torch.Tensor | None = None,
                             S_out: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """Sparsified gradient volume of Sec. 3.3 at ``level``: returns (V [4N+4][k][h][w] float32,
    S [k][h][w] uint8).  Channels: PSV (3N, view-major), inverse-warped alpha weights (N),
    the level MPI (4).  ``m`` is not modified."""
    N = len(src)
    _check_f32(images, (N, m.H, m.W, 3), "images")
    h, w = m.H >> level, m.W >> level
    dev = m.data.device
    if V is None:
        V = torch.empty((4 * N + 4, k, h, w), dtype=torch.float32, device=dev)
    _check_f32(V, (4 * N + 4, k, h, w), "V")
    if S_out is None:
        S_out = torch.empty((k, h, w), dtype=torch.uint8, device=dev)
    if S_out.dtype != torch.uint8 or tuple(S_out.shape) != (k, h, w):
        raise ValueError(f"S_out must be uint8 {(k, h, w)}")
    if ws is None:
        ws = torch.empty(reallife_gradient_volume_workspace_bytes(N, m.D, m.H, m.W, k, m.data.dtype),
                         dtype=torch.uint8, device=dev)
    ms = m.c_struct()
    _lib.check("reallife_gradient_volume", _lib.lib().reallife_gradient_volume(
        ctypes.byref(ms), _ptr(images), _lib.cameras(src), N, int(k), int(level), int(selection), _ptr(S_out),
        _ptr(V), _ptr(ws), ws.numel(), _stream(stream)))
    return V, S_out


class LgdNet:
    """The learned-update network on the device: the trained parameters (FP32 tensors, kept
    alive here) packed by ``reallife_lgd_prepare`` into ``packed`` (BF16 weights with batch norm
    folded).  ``params`` is any object with the fields of ``scenegen.LgdWeights``."""

    def __init__(self, params, device="cuda", stream=None):
        def t(a):
            return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(device)
        self.c_in = int(params.conv_w[0].shape[1])
        self._keep = []
        p = _lib.RlLgdParams()
        p.c_in, p.eps = self.c_in, float(params.eps)
        for name in ("conv_w", "conv_b", "bn_gamma", "bn_beta", "bn_mean", "bn_var"):
            arr = getattr(p, name)
            for l, a in enumerate(getattr(params, name)):
                ta = t(a)
                self._keep.append(ta)
                arr[l] = ta.data_ptr()
        ow, ob = t(params.out_w), t(params.out_b)
        self._keep += [ow, ob]
        p.out_w, p.out_b = ow.data_ptr(), ob.data_ptr()
        self.packed = torch.empty(int(_lib.lib().reallife_lgd_net_bytes()), dtype=torch.uint8, device=device)
        _lib.check("reallife_lgd_prepare", _lib.lib().reallife_lgd_prepare(ctypes.byref(p), _ptr(self.packed),
                                                                          _stream(stream)))


def reallife_lgd_forward(net: LgdNet, V: torch.Tensor, residual: torch.Tensor | None = None,
                         ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """N_w(V): V [C][k][h][w] float32 (C <= 32) -> residual [k][h][w][4] float32."""
    C, k, h, w = V.shape
    if V.dtype != torch.float32:
        raise ValueError("V must be float32")
    if residual is None:
        residual = torch.empty((k, h, w, 4), dtype=torch.float32, device=V.device)
    _check_f32(residual, (k, h, w, 4), "residual")
    if ws is None:
        ws = torch.empty(int(_lib.lib().reallife_lgd_workspace_bytes(k, h, w)), dtype=torch.uint8, device=V.device)
    _lib.check("reallife_lgd_forward", _lib.lib().reallife_lgd_forward(
        _ptr(net.packed), _ptr(V), C, k, h, w, _ptr(residual), _ptr(ws), ws.numel(), _stream(stream)))
    return residual


def reallife_lgd_step_workspace_bytes(N: int, D: int, H: int, W: int, k: int, dtype=torch.float32) -> int:
    return int(_lib.lib().reallife_lgd_step_workspace_bytes(N, D, H, W, k, _DT[dtype]))


def reallife_lgd_step(m: Mpi, images: torch.Tensor, src, k: int, net: LgdNet, level: int = 0,
                      selection: int = SELECT_TOPK, clamp: bool = True, S_out: torch.Tensor | None = None,
                      ws: torch.Tensor | None = None, stream=None):
    """One learned HSGD iteration on ``m`` in place: M <- M + R(N_w(V_s), S); returns S_out."""
    N = len(src)
    _check_f32(images, (N, m.H, m.W, 3), "images")
    if ws is None:
        ws = torch.empty(reallife_lgd_step_workspace_bytes(N, m.D, m.H, m.W, k, m.data.dtype), dtype=torch.uint8,
                         device=m.data.device)
    ms = m.c_struct()
    _lib.check("reallife_lgd_step", _lib.lib().reallife_lgd_step(
        ctypes.byref(ms), _ptr(images), _lib.cameras(src), N, int(k), int(level), int(selection), int(bool(clamp)),
        _ptr(net.packed), _ptr(S_out), _ptr(ws), ws.numel(), _stream(stream)))
    return S_out


def reallife_downsample_f32(x: torch.Tensor, level: int, out: torch.Tensor | None = None, stream=None):
    """Down^l of ``x[P][H][W][C]`` float32 (2^l x 2^l box average)."""
    P, H, W, C = x.shape
    if out is None:
        out = torch.empty((P, H >> level, W >> level, C), dtype=torch.float32, device=x.device)
    _lib.check("reallife_downsample_f32", _lib.lib().reallife_downsample_f32(
        _ptr(x), P, H, W, C, level, _ptr(out), _stream(stream)))
    return out


def reallife_select(m: Mpi, k: int, S: torch.Tensor | None = None, mask: torch.Tensor | None = None, stream=None,
                    selection: int = SELECT_TOPK):
    """k planes per pixel by the reference-view alpha weight (top-k or MVS-sampling window):
    (S uint8 [k][H][W], mask int64 [H][W])."""
    dev = m.data.device
    if S is None:
        S = torch.empty((k, m.H, m.W), dtype=torch.uint8, device=dev)
    if mask is None:
        mask = torch.empty((m.H, m.W), dtype=torch.int64, device=dev)
    ms = m.c_struct()
    _lib.check("reallife_select", _lib.lib().reallife_select(ctypes.byref(ms), k, int(selection), _ptr(S), _ptr(mask),
                                                            _stream(stream)))
    return S, mask


def reallife_select_keys(keys: torch.Tensor, k: int, stream=None, selection: int = SELECT_TOPK):
    """Selection from caller-supplied float32 keys ``[D][H][W]``: (S, mask)."""
    D, H, W = keys.shape
    if keys.dtype != torch.float32:
        raise ValueError("keys must be float32")
    S = torch.empty((k, H, W), dtype=torch.uint8, device=keys.device)
    mask = torch.empty((H, W), dtype=torch.int64, device=keys.device)
    _lib.check("reallife_select_keys", _lib.lib().reallife_select_keys(_ptr(keys), D, H, W, k, int(selection), _ptr(S),
                                                                      _ptr(mask), _stream(stream)))
    return S, mask


def reallife_loss_grad(m: Mpi, images: torch.Tensor, src, mask: torch.Tensor | None = None, k: int | None = None,
                       stream=None):
    """Photometric loss and its gradient at the MPI's resolution: (loss [1], G).

    Dense ``G [D][H][W][4]`` when ``mask`` is None, else compact ``G [k][H][W][4]``."""
    N = len(src)
    _check_f32(images, (N, m.H, m.W, 3), "images")
    slots = m.D if mask is None else int(k)
    G = torch.empty((slots, m.H, m.W, 4), dtype=torch.float32, device=m.data.device)
    loss = torch.empty(1, dtype=torch.float32, device=m.data.device)
    ws = workspace(N, m.D, m.H, m.W, 1, m.data.dtype, m.data.device)
    ms = m.c_struct()
    _lib.check("reallife_loss_grad", _lib.lib().reallife_loss_grad(
        ctypes.byref(ms), _ptr(images), _lib.cameras(src), N, _ptr(mask), slots, _ptr(G), _ptr(loss), _ptr(ws),
        ws.numel(), _stream(stream)))
    return loss, G


def reallife_sparse_update(m: Mpi, S: torch.Tensor, G: torch.Tensor, k: int, level: int, lam: float,
                           clamp: bool = True, stream=None):
    ms = m.c_struct()
    _lib.check("reallife_sparse_update", _lib.lib().reallife_sparse_update(
        ctypes.byref(ms), _ptr(S), _ptr(G), k, level, float(lam), int(bool(clamp)), _stream(stream)))


def reallife_render_backward(m: Mpi, cams, grad_out: torch.Tensor, grad_mpi: torch.Tensor | None = None,
                             stream=None) -> torch.Tensor:
    """dL/dM (float32 ``[D][H][W][4]``) given dL/dC of the views ``grad_out [N][H][W][3]``."""
    N = len(cams)
    _check_f32(grad_out, (N, m.H, m.W, 3), "grad_out")
    if grad_mpi is None:
        grad_mpi = torch.empty((m.D, m.H, m.W, 4), dtype=torch.float32, device=m.data.device)
    ms = m.c_struct()
    _lib.check("reallife_render_backward", _lib.lib().reallife_render_backward(
        ctypes.byref(ms), _lib.cameras(cams), N, _ptr(grad_out), _ptr(grad_mpi), _stream(stream)))
    return grad_mpi


def reallife_warp_offsets(m: Mpi, cam, stream=None) -> torch.Tensor:
    out = torch.empty((m.D, m.H, m.W, 2), dtype=torch.float32, device=m.data.device)
    ms = m.c_struct()
    _lib.check("reallife_warp_offsets", _lib.lib().reallife_warp_offsets(
        ctypes.byref(ms), _lib.cameras([cam]), _ptr(out), _stream(stream)))
    return out


def reallife_metrics_workspace_bytes(N: int, H: int, W: int) -> int:
    return int(_lib.lib().reallife_metrics_workspace_bytes(int(N), int(H), int(W)))


def reallife_image_metrics(x: torch.Tensor, y: torch.Tensor, ws: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
    """Device ``double[2]``: (mean squared difference, mean SSIM) of ``x, y [N][H][W][3]`` float32."""
    if x.dim() != 4 or x.shape[3] != 3:
        raise ValueError("x must be [N][H][W][3]")
    N, H, W = (int(v) for v in x.shape[:3])
    _check_f32(x, (N, H, W, 3), "x")
    _check_f32(y, (N, H, W, 3), "y")
    out = torch.empty(2, dtype=torch.float64, device=x.device)
    if ws is None:
        ws = torch.empty(max(reallife_metrics_workspace_bytes(N, H, W), 8), dtype=torch.uint8, device=x.device)
    _lib.check("reallife_image_metrics", _lib.lib().reallife_image_metrics(
        _ptr(x), _ptr(y), N, H, W, _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def reallife_kept_mass(m: Mpi, mask: torch.Tensor, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Device ``double[2]``: (alpha weight of the planes kept by ``mask [H][W]`` int64, all alpha weight)."""
    if mask.dtype != torch.int64 or tuple(mask.shape) != (m.H, m.W):
        raise ValueError(f"mask must be int64 {(m.H, m.W)}")
    out = torch.empty(2, dtype=torch.float64, device=m.data.device)
    if ws is None:
        ws = torch.empty(max(reallife_metrics_workspace_bytes(1, m.H, m.W), 8), dtype=torch.uint8,
                         device=m.data.device)
    ms = m.c_struct()
    _lib.check("reallife_kept_mass", _lib.lib().reallife_kept_mass(
        ctypes.byref(ms), _ptr(mask), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def reallife_trace_enable(on: bool = True):
    _lib.check("reallife_trace_enable", _lib.lib().reallife_trace_enable(int(bool(on))))


def reallife_trace_read() -> dict:
    """{kernel name: (launches, total device ms)} since the last read (synchronises)."""
    arr = (_lib.RlTraceEntry * 64)()
    n = ctypes.c_int()
    _lib.check("reallife_trace_read", _lib.lib().reallife_trace_read(arr, 64, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, 64))}


def reallife_trace_release_captured():
    """Return the events of captured launches to the tracer (after their graphs are gone)."""
    _lib.check("reallife_trace_release_captured", _lib.lib().reallife_trace_release_captured())


def reallife_strerror(status: int) -> str:
    return _lib.lib().reallife_strerror(status).decode()


def reallife_set_kernel_path(path: int):
    """0: automatic (default); 2: per-pixel gather; 3-5: plane-parallel (1 is not used)."""
    _lib.check("reallife_set_kernel_path", _lib.lib().reallife_set_kernel_path(int(path)))


def reallife_selftest_wait_timeout(wait_us: int = 2000, stream=None) -> None:
    """Enqueue the bounded-wait self-test: a wait that nothing completes gives up after
    wait_us microseconds and sets the timeout bit that reallife_device_status reports."""
    _lib.check("reallife_selftest_wait_timeout", _lib.lib().reallife_selftest_wait_timeout(int(wait_us),
                                                                                             _stream(stream)))


def reallife_selftest_bounds(stream=None) -> None:
    """Enqueue the bounds-check self-test of the debug build: a store one past the end of a
    device buffer is stopped by its check, which sets the bounds bit (4) of the status word.
    Raises RL_ENOTIMPL on the release build."""
    _lib.check("reallife_selftest_bounds", _lib.lib().reallife_selftest_bounds(_stream(stream)))


def reallife_debug_build() -> bool:
    """True when the loaded library is the bounds-checked debug build (REALLIFE_DEBUG=1)."""
    return bool(_lib.lib().reallife_debug_build())


def reallife_device_status(clear: bool = True) -> int:
    """Synchronise the device and return the device status bits (raises on a timeout, and on
    a failed bounds check of the debug build)."""
    flags = ctypes.c_uint()
    _lib.check("reallife_device_status", _lib.lib().reallife_device_status(int(bool(clear)), ctypes.byref(flags)))
    return int(flags.value)
