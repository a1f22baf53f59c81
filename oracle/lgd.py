"""FP64 oracle of the learned-update network of Sec. 3.3 ("Sparse Gradient Update") and of one
learned HSGD iteration (test infrastructure only: the test-suite, the package smoke check and
the CPU-baseline leg of the benchmark may use it; the product path never does).

The paper fixes the network only as five basic blocks (3D convolution, batch norm, ReLU)
followed by a 1x1x1 3D convolution (Sec. 4, implementation details), fed the sparsified volume
V_s [C][k][h][w] and producing the sparse MPI residual, which the restore operator R(., S) puts
back at the kept planes: M_{n+1} = M_n + R(N_w(V_s), S).  Readings fixed here (the figure with
the layer sizes is not available): 3x3x3 kernels with zero padding 1 ("same"), 32 channels in
every block, batch norm in inference form with running statistics, a 4-channel (R, G, B, alpha)
residual, and the coarse-to-fine nearest-neighbour upsampling plus [0, 1] clamp of the HSGD
update for levels >= 1.

``storage="bf16"`` rounds, to nearest even, exactly where a BF16-storing implementation holds
values: the network input, every block's folded weights and every block's output except the
last block's (which feeds the 1x1x1 layer directly); everything else is FP64.
``storage="fp64"`` is the plain definition.
"""
from __future__ import annotations

import numpy as np


def round_bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def bn_fold(w, b, gamma, beta, mean, var, eps):
    """Convolution followed by inference batch norm as one convolution:
    BN(y) = gamma (y - mean) / sqrt(var + eps) + beta with y = w * x + b."""
    w = np.asarray(w, np.float64)
    s = np.asarray(gamma, np.float64) / np.sqrt(np.asarray(var, np.float64) + eps)
    wf = w * s.reshape((-1,) + (1,) * (w.ndim - 1))
    bf = (np.asarray(b, np.float64) - np.asarray(mean, np.float64)) * s + np.asarray(beta, np.float64)
    return wf, bf


def conv3d_same(x, w, b) -> np.ndarray:
    """out[o][z][y][x] = b[o] + sum_{c,dz,dy,dx} w[o][c][dz][dy][dx] x[c][z+dz-r][y+dy-r][x+dx-r], with
    zero outside the volume (r = kernel radius).  x [C][K][H][W], w [O][C][s][s][s] (s odd)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    C, K, H, W = x.shape
    s = w.shape[2]
    r = s // 2
    xp = np.zeros((C, K + 2 * r, H + 2 * r, W + 2 * r))
    xp[:, r:r + K, r:r + H, r:r + W] = x
    out = np.zeros((w.shape[0], K, H, W))
    for dz in range(s):
        for dy in range(s):
            for dx in range(s):
                tap = xp[:, dz:dz + K, dy:dy + H, dx:dx + W].reshape(C, -1)
                out += (w[:, :, dz, dy, dx] @ tap).reshape(-1, K, H, W)
    return out + np.asarray(b, np.float64).reshape(-1, 1, 1, 1)


def lgd_forward(V, net, storage: str = "bf16") -> np.ndarray:
    """N_w(V_s): five (3x3x3 conv, BN, ReLU) blocks then the 1x1x1 layer.  V [C][k][h][w]
    (C <= 32); returns the residual [k][h][w][4]."""
    rnd = round_bf16 if storage == "bf16" else (lambda a: np.asarray(a, np.float64))
    x = rnd(V)
    nb = len(net.conv_w)
    for l in range(nb):
        wf, bf = bn_fold(net.conv_w[l], net.conv_b[l], net.bn_gamma[l], net.bn_beta[l], net.bn_mean[l],
                         net.bn_var[l], net.eps)
        x = np.maximum(conv3d_same(x, rnd(wf), bf), 0.0)
        if l < nb - 1:
            x = rnd(x)
    out = conv3d_same(x, np.asarray(net.out_w, np.float64)[:, :, None, None, None], net.out_b)
    return np.moveaxis(out, 0, -1)


def restore_update(M, residual, S, level: int, clamp: bool = True) -> np.ndarray:
    """M + R(residual, S) at full resolution (Sec. 3.3 "Sparse Gradient Update"): the residual of
    slot j of level pixel p goes to plane S[j][p] of every full-resolution pixel of p's 2^l x 2^l
    block (nearest-neighbour upsampling), clamped to [0, 1].  residual [k][h][w][4]."""
    M = np.array(M, np.float64, copy=True)
    k, h, w = S.shape
    s = 1 << level
    for j in range(k):
        for yy in range(h):
            for xx in range(w):
                d = int(S[j, yy, xx])
                blk = M[d, yy * s:(yy + 1) * s, xx * s:(xx + 1) * s]
                v = blk + residual[j, yy, xx]
                M[d, yy * s:(yy + 1) * s, xx * s:(xx + 1) * s] = np.clip(v, 0.0, 1.0) if clamp else v
    return M


def lgd_step(M, near, far, ref, views, images, net, k: int, level: int = 0, selection: int = 0, S_pin=None,
             storage: str = "bf16", clamp: bool = True):
    """One learned HSGD iteration: V_s and S (Sec. 3.3), the residual N_w(V_s), and the restore
    update.  Returns (M_new, residual, S)."""
    import oracle
    Vs, S = oracle.gradient_volume(M, near, far, ref, views, images, k, level, selection, S_pin)
    res = lgd_forward(Vs, net, storage)
    return restore_update(M, res, S, level, clamp), res, S
