"""Batched HSGD step: one launch per stage (selection, gradient, update; the gradient one per
kernel family) serves one iteration of several independent requests of different sizes, plane
and view counts and levels.

Every item's refined MPI, selection and loss equal those of reallife_hsgd_step on that item
alone (FP32: 1e-5; BF16 storage: 2e-2; selection bit-exact), one item is checked against the
FP64 oracle with its selection pinned, and a graph captured from one batched call serves a
rewritten table.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu
TOL32, TOL16 = 1e-5, 2e-2

SHAPES = [(96, 128, 8, 3, 5, 0), (48, 64, 16, 2, 3, 1), (64, 96, 12, 4, 5, 2), (32, 32, 5, 1, 5, 0)]


def _scenes():
    return [sg.make_scene(70 + i, H, W, D, N, n_layers=(2, 4), novel="none")
            for i, (H, W, D, N, _, _) in enumerate(SHAPES)]


@pytest.fixture(scope="module")
def scenes():
    return _scenes()


def _request(rl, sc, k, level, dtype, dev):
    M = torch.from_numpy(sc.coarse_mpi).to(dev).to(dtype).contiguous()
    images = torch.from_numpy(sc.images).to(dev)
    ws = rl.workspace(len(sc.src), sc.D, sc.H, sc.W, k, dtype, dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    return M, images, ws, loss


def _alone(rl, scenes, dtype, dev):
    out = []
    for sc, (_, _, _, _, k, level) in zip(scenes, SHAPES):
        M, images, ws, loss = _request(rl, sc, k, level, dtype, dev)
        S = torch.empty((k, sc.H >> level, sc.W >> level), dtype=torch.uint8, device=dev)
        rl.reallife_hsgd_step(rl.make_mpi(M, sc.near, sc.far, sc.ref), images, sc.src, k, level=level, loss_out=loss,
                              S_out=S, ws=ws)
        out.append((M, S, loss))
    torch.cuda.synchronize()
    return out


def _batch_items(rl, scenes, dtype, dev):
    reqs, items = [], []
    for sc, (_, _, _, _, k, level) in zip(scenes, SHAPES):
        M, images, ws, loss = _request(rl, sc, k, level, dtype, dev)
        reqs.append((M, ws, loss, k, level, sc))
        items.append(rl.BatchItem(rl.make_mpi(M, sc.near, sc.far, sc.ref), images, sc.src, k, ws, level=level,
                                  loss_out=loss))
    return reqs, items


def _kept_planes(ws, rl, sc, k, level, dtype):
    """The selection S [k][h][w] the batched step left in the request's workspace."""
    h, w = sc.H >> level, sc.W >> level
    off = 0
    if sc.H % 2 == 0 and sc.W % 2 == 0:
        elt = 4 if dtype == torch.float32 else 2
        off = (sc.D * (sc.H // 2) * (sc.W // 2) * 4 * elt + 255) // 256 * 256
    return ws[off:off + k * h * w].view(k, h, w)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_batched_step_equals_each_request_alone(scenes, dtype):
    import paper_2307_03017_gb300 as rl
    dev = torch.device("cuda")
    alone = _alone(rl, scenes, dtype, dev)
    reqs, items = _batch_items(rl, scenes, dtype, dev)
    table = rl.BatchTable(8, dev)
    rl.reallife_trace_enable(True)
    rl.reallife_trace_read()
    rl.reallife_hsgd_step_batch(table, items)
    torch.cuda.synchronize()
    tr = rl.reallife_trace_read()
    rl.reallife_trace_enable(False)
    # one launch per stage served all four requests (the gradient: one per kernel family used)
    sfx = "f32" if dtype == torch.float32 else "bf16"
    counts = {n: c for n, (c, _) in tr.items()}
    assert counts.pop(f"select_batch_{sfx}") == 1 and counts.pop(f"update_batch_{sfx}") == 1
    assert counts and set(counts) <= {f"grad_batch_{sfx}", f"grad_pp_batch_{sfx}"}
    assert all(c == 1 for c in counts.values())
    tol = TOL32 if dtype == torch.float32 else TOL16
    for (M, ws, loss, k, level, sc), (Ma, Sa, la) in zip(reqs, alone):
        assert torch.equal(_kept_planes(ws, rl, sc, k, level, dtype), Sa)
        assert (M.float() - Ma.float()).abs().max().item() <= tol
        assert abs(loss.item() - la.item()) <= 1e-5 * max(1.0, abs(la.item()))
    assert rl.reallife_device_status(clear=True) == 0


def test_batched_step_matches_oracle(scenes):
    import paper_2307_03017_gb300 as rl
    dev = torch.device("cuda")
    reqs, items = _batch_items(rl, scenes, torch.float32, dev)
    table = rl.BatchTable(4, dev)
    rl.reallife_hsgd_step_batch(table, items)
    torch.cuda.synchronize()
    for (M, ws, loss, k, level, sc) in reqs:
        S = _kept_planes(ws, rl, sc, k, level, torch.float32).cpu().numpy()
        Mo, Lo, _ = oracle.hsgd_step(sc.coarse_mpi.astype(np.float64), sc.near, sc.far, sc.ref, sc.src, sc.images, k,
                                     level=level, S_pin=S)
        assert np.abs(M.cpu().numpy() - Mo).max() <= TOL32
        assert abs(loss.item() - Lo) <= 1e-5 * max(1.0, abs(Lo))


def test_captured_batch_serves_a_rewritten_table(scenes):
    """A graph captured from one batched call (items 0 and 1) replays another table (items
    2 and 3, then 1, 2 and 3) with the results of the direct calls."""
    import paper_2307_03017_gb300 as rl
    dev = torch.device("cuda")
    dtype = torch.float32
    alone = _alone(rl, scenes, dtype, dev)
    reqs, items = _batch_items(rl, scenes, dtype, dev)
    table = rl.BatchTable(4, dev)
    s = torch.cuda.Stream()
    rl.reallife_batch_prepare(items[:2], table)
    rl.reallife_hsgd_step_batch(table, stream=s)  # kernels load before the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rl.reallife_hsgd_step_batch(table, stream=s)
    # fresh inputs for items 2 and 3, then replay with the table rewritten
    reqs, items = _batch_items(rl, scenes, dtype, dev)
    rl.reallife_batch_prepare(items[2:], table)
    g.replay()
    torch.cuda.synchronize()
    for i in (2, 3):
        M, ws, loss, k, level, sc = reqs[i]
        assert (M - alone[i][0]).abs().max().item() <= TOL32
        assert abs(loss.item() - alone[i][2].item()) <= 1e-5 * max(1.0, abs(alone[i][2].item()))
    # untouched by the replay: items 0 and 1 still hold their coarse MPIs
    for i in (0, 1):
        M = reqs[i][0]
        assert torch.equal(M.cpu(), torch.from_numpy(scenes[i].coarse_mpi))
    reqs, items = _batch_items(rl, scenes, dtype, dev)
    rl.reallife_batch_prepare(items[1:], table)
    g.replay()
    torch.cuda.synchronize()
    for i in (1, 2, 3):
        assert (reqs[i][0] - alone[i][0]).abs().max().item() <= TOL32
    assert rl.reallife_device_status(clear=True) == 0


def test_batch_rejects_shared_buffers_and_mixed_storage(scenes):
    import paper_2307_03017_gb300 as rl
    dev = torch.device("cuda")
    reqs, items = _batch_items(rl, scenes[:2], torch.float32, dev)
    table = rl.BatchTable(4, dev)
    with pytest.raises(rl.RealLifeError, match="share"):
        rl.reallife_batch_prepare([items[0], items[0]], table)
    _, items16 = _batch_items(rl, scenes[:2], torch.bfloat16, dev)
    with pytest.raises(rl.RealLifeError, match="storage"):
        rl.reallife_batch_prepare([items[0], items16[1]], table)
    # a table of BF16 items given to kernels captured for FP32 sets the batch bit and changes nothing
    s = torch.cuda.Stream()
    rl.reallife_batch_prepare(items, table)
    rl.reallife_hsgd_step_batch(table, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rl.reallife_hsgd_step_batch(table, stream=s)
    reqs16, items16 = _batch_items(rl, scenes[:2], torch.bfloat16, dev)
    rl.reallife_batch_prepare(items16, table)
    g.replay()
    torch.cuda.synchronize()
    flags = rl.reallife_device_status(clear=True)
    assert flags & 2
    for i in range(2):
        assert torch.equal(reqs16[i][0].cpu(), torch.from_numpy(scenes[i].coarse_mpi).to(torch.bfloat16))
