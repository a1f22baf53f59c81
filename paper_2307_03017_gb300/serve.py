"""Continuous-batching reconstruction server for the HSGD hot path.

A persistent host loop serves reconstruction requests of different resolutions, plane
counts and view counts.  A request is admitted as soon as a slot and enough device memory
are free; requests that arrive while others are on the GPU join them, so the work of
concurrent requests overlaps on the device.

- **Memory.** Admission is by device memory: every request takes its MPI, source images,
  loss buffer and HSGD workspace from one preallocated device arena (first fit, 256-byte
  granularity), and gives them back when its result has reached the host.
- **Work.** Each slot owns a CUDA stream.  An admitted request's work is enqueued on its
  slot's stream in one go: the host-to-device copy of its coarse MPI and images, its HSGD
  iterations (``reallife_refine``; the MPI stays resident across them) and the
  device-to-host copy of the refined MPI and the losses.
- **Graphs.** With ``graphs=True`` the compute part is a CUDA graph captured once per
  (slot, request shape, geometry) on buffers pinned to that slot, and replayed as a single
  launch for every later request with the same key in that slot.  The camera constants
  travel in the kernels' parameters, so a graph is only reused for identical geometry.
- **Batched steps.** With ``batched=True`` the engine schedules by iteration instead: every
  engine step runs the next HSGD iteration of every active request (each at its own level)
  in one launch per stage through ``reallife_hsgd_step_batch``, whose work table lists the
  requests.  Requests join at the next step after their inputs are copied in and leave after
  their last iteration.  Requests go to ``lanes`` size classes (by pixels x planes x views),
  each with its own stream and tables, so that small requests are not held behind the steps
  of large ones.  A lane's table is double-buffered (page-locked host and device copies), at
  most two of its steps are in flight, and with ``graphs=True`` each buffer's step is one
  captured graph replayed with the table rewritten, whatever the requests' shapes and cameras.
- **Latency.** A request's latency is the time from its arrival to the moment the host sees
  its result, including queueing and both copies.
- **Oversized requests.** A request that needs more memory than the whole arena is never
  admitted: it is marked failed (``req.error``) and returned with the others.
"""
from __future__ import annotations

import collections
import gc
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (BatchItem, BatchTable, batch_c_item, make_mpi, reallife_batch_prepare, reallife_hsgd_step_batch,
               reallife_refine, reallife_workspace_bytes)

ALIGN = 256


def _align(n: int) -> int:
    return (n + ALIGN - 1) // ALIGN * ALIGN


class DeviceArena:
    """First-fit allocator over one device buffer; offsets are 256-byte aligned."""

    def __init__(self, nbytes: int, device):
        self.size = _align(nbytes)
        self.buf = torch.empty(self.size, dtype=torch.uint8, device=device)
        self.free = [(0, self.size)]  # sorted, non-adjacent (offset, length)

    def alloc(self, n: int):
        n = _align(n)
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                return off
        return None

    def release(self, off: int, n: int):
        n = _align(n)
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    def bytes_free(self) -> int:
        return sum(ln for _, ln in self.free)

    def can_alloc(self, n: int) -> bool:
        n = _align(n)
        return any(ln >= n for _, ln in self.free)

    def view(self, off: int, shape, dtype):
        n = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        return self.buf[off:off + n].view(dtype).view(*shape)


@dataclass
class Request:
    """One reconstruction: refine ``coarse`` (pinned host, [D][H][W][4]) against ``images``
    (pinned host, [N][H][W][3] float32) from cameras ``src`` over ``schedule``."""
    id: int
    arrival: float
    coarse: torch.Tensor
    images: torch.Tensor
    ref: object
    src: list
    near: float
    far: float
    schedule: tuple
    k: int = 5
    t_admit: float = -1.0
    t_done: float = -1.0
    slot: int = -1
    error: str | None = None
    losses: np.ndarray | None = None
    result: torch.Tensor | None = None
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        D, H, W, _ = self.coarse.shape
        return (D, H, W, len(self.src), tuple(self.schedule), self.k, self.coarse.dtype)

    @property
    def geometry(self):
        """Everything the captured kernels take by value besides the buffers."""
        cams = [self.ref] + list(self.src)
        return (self.near, self.far) + tuple(np.concatenate(
            [np.concatenate([np.ravel(c.K), np.ravel(c.R), np.ravel(c.t)]) for c in cams]).tolist())

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def request_bytes(D, H, W, N, k, dtype) -> int:
    elt = torch.tensor([], dtype=dtype).element_size()
    return (_align(D * H * W * 4 * elt) + _align(N * H * W * 3 * 4) + _align(64)
            + _align(reallife_workspace_bytes(N, D, H, W, k, dtype)))


def reject_oversized(requests, arena_bytes: int):
    """Split ``requests`` into (rejected, admissible): a request whose buffers alone exceed the
    whole arena could never be admitted and would hold up every request behind it, so it is
    marked failed (``error`` set, done at its arrival) instead of queued."""
    rejected, fits = [], []
    for r in requests:
        if request_bytes(*r.shape[:4], r.k, r.coarse.dtype) > arena_bytes:
            r.error = "needs more device memory than the whole arena"
            r.t_done = r.arrival
            rejected.append(r)
        else:
            fits.append(r)
    return rejected, fits


class ServeEngine:
    """Admits requests by device memory into up to ``max_slots`` concurrent slots."""

    def __init__(self, arena_bytes: int, max_slots: int = 8, device="cuda", graphs: bool = False,
                 keep_results: bool = False, max_result_elems: int = 0, result_dtype=torch.bfloat16,
                 batched: bool = False, lanes: int = 2, lane_split: int = 512 * 384 * 32 * 4):
        """``max_result_elems``: preallocate every slot's pinned result buffer for MPIs of up to
        this many elements, so that no pinned allocation happens while serving.  ``batched``:
        iteration-level scheduling with one batched launch per stage for all active requests."""
        self.device = torch.device(device)
        self.batched = batched
        self.lanes = max(1, int(lanes)) if batched else 1
        self.lane_split = lane_split  # pixels x planes x views at which a request takes the next lane
        self.steps = 0  # batched engine steps run
        self.max_items_per_step = 0
        self.arena = DeviceArena(arena_bytes, self.device)
        self.max_slots = max_slots
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(max_slots)]
        self.graphs = graphs
        self.keep_results = keep_results
        self.graph_cache = {}  # (slot, shape, geometry) -> (graph, buffers, offset, nbytes)
        self.slot_result = [torch.empty(max_result_elems, dtype=result_dtype).pin_memory() if max_result_elems
                            else None for _ in range(max_slots)]  # pinned host result buffer per slot
        self.slot_loss = [torch.empty(8, dtype=torch.float32).pin_memory() for _ in range(max_slots)]
        self.captures = 0
        self.replays = 0

    # ------------------------------------------------------------ buffers
    def _carve(self, req, off):
        D, H, W, _ = req.coarse.shape
        N = len(req.src)
        elt_dtype = req.coarse.dtype
        M = self.arena.view(off, (D, H, W, 4), elt_dtype)
        o = off + _align(M.numel() * M.element_size())
        images = self.arena.view(o, (N, H, W, 3), torch.float32)
        o += _align(images.numel() * 4)
        loss = self.arena.view(o, (len(req.schedule),), torch.float32)
        o += _align(64)
        nws = reallife_workspace_bytes(N, D, H, W, req.k, elt_dtype)
        ws = self.arena.buf[o:o + nws]
        return M, images, loss, ws

    def _host_result(self, slot, req):
        need = req.coarse.numel()
        buf = self.slot_result[slot]
        if buf is None or buf.numel() < need or buf.dtype != req.coarse.dtype:
            buf = torch.empty(need, dtype=req.coarse.dtype).pin_memory()
            self.slot_result[slot] = buf
        return buf[:need].view(req.coarse.shape)

    # ------------------------------------------------------------ launch
    def _compute(self, req, M, images, loss, ws, stream):
        mpi = make_mpi(M, req.near, req.far, req.ref)
        reallife_refine(mpi, images, req.src, req.k, req.schedule, loss_per_iter=loss, ws=ws, stream=stream)

    def _launch(self, req, slot):
        """Enqueue a request on its slot's stream; None when its memory is not available."""
        s = self.streams[slot]
        n = request_bytes(*req.shape[:4], req.k, req.coarse.dtype)
        key = (slot, req.shape, req.geometry)
        g = None
        owned = False
        if self.graphs and key in self.graph_cache:
            g, bufs, off, n = self.graph_cache[key]
            M, images, loss, ws = bufs
        else:
            if not self.arena.can_alloc(n) and self.graphs:
                self._evict_idle_graphs(n)
            off = self.arena.alloc(n)
            if off is None:
                return None
            M, images, loss, ws = self._carve(req, off)
            owned = True
        host_out = self._host_result(slot, req)
        host_loss = self.slot_loss[slot][:len(req.schedule)]
        with torch.cuda.stream(s):
            M.copy_(req.coarse, non_blocking=True)
            images.copy_(req.images, non_blocking=True)
            if self.graphs:
                if g is None:
                    # capture this slot's compute for this shape; its buffers stay with the slot
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=s):
                        self._compute(req, M, images, loss, ws, s)
                    self.graph_cache[key] = (g, (M, images, loss, ws), off, n)
                    owned = False
                    self.captures += 1
                g.replay()
                self.replays += 1
            else:
                self._compute(req, M, images, loss, ws, s)
            host_out.copy_(M, non_blocking=True)
            host_loss.copy_(loss, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return ev, (off if owned else None), n, host_out, host_loss

    def _evict_idle_graphs(self, need: int):
        """Give back the buffers of cached graphs of idle slots until ``need`` bytes fit."""
        for key in list(self.graph_cache):
            if self.arena.can_alloc(need):
                return
            if key[0] in self._busy:
                continue
            _, _, off, n = self.graph_cache.pop(key)
            self.arena.release(off, n)

    # ------------------------------------------------------------ loop
    def run(self, requests, realtime: bool = True, poll_s: float = 20e-6):
        """Serve ``requests`` (sorted by arrival, seconds).  ``realtime``: admit a request no
        earlier than its arrival time; otherwise all are available at once (closed loop)."""
        requests = sorted(requests, key=lambda r: r.arrival)
        done, fits = reject_oversized(requests, self.arena.size)
        if self.batched:
            return done + self._run_batched(fits, realtime, poll_s)
        pending = collections.deque(fits)
        active = {}
        free_slots = list(range(self.max_slots - 1, -1, -1))
        self._busy = set()
        t0 = time.perf_counter()
        if not realtime:
            for r in pending:
                r.arrival = 0.0
        gc_was_enabled = gc.isenabled()
        gc.disable()  # no collector pauses inside the serving loop
        try:
            self._loop(pending, active, free_slots, t0, done, poll_s)
        finally:
            if gc_was_enabled:
                gc.enable()
        return done

    def _loop(self, pending, active, free_slots, t0, done, poll_s):
        while pending or active:
            now = time.perf_counter() - t0
            progressed = False
            for slot in list(active):
                req, ev, off, n, host_out, host_loss = active[slot]
                if ev.query():
                    req.t_done = time.perf_counter() - t0
                    req.losses = host_loss.numpy().copy()
                    if self.keep_results:
                        req.result = host_out.clone()
                    if off is not None:
                        self.arena.release(off, n)
                    del active[slot]
                    self._busy.discard(slot)
                    free_slots.append(slot)
                    done.append(req)
                    progressed = True
            while pending and free_slots and pending[0].arrival <= now:
                req = pending[0]
                # prefer a free slot that already holds a graph for this shape
                slot = free_slots[-1]
                if self.graphs:
                    for cand in free_slots:
                        if (cand, req.shape, req.geometry) in self.graph_cache:
                            slot = cand
                            break
                launched = self._launch(req, slot)
                if launched is None:
                    break  # first come, first served: wait for memory
                pending.popleft()
                free_slots.remove(slot)
                self._busy.add(slot)
                req.slot = slot
                req.t_admit = time.perf_counter() - t0
                active[slot] = (req,) + launched
                progressed = True
            if not progressed:
                if pending and not active and pending[0].arrival > now:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 1e-3)))
                else:
                    time.sleep(poll_s)


    # ------------------------------------------------------------ batched steps
    def _run_batched(self, requests, realtime, poll_s):
        if not requests:
            return []
        dtypes = {r.coarse.dtype for r in requests}
        if len(dtypes) != 1:
            raise ValueError("batched serving takes requests of one storage type")
        if not hasattr(self, "_lane_state"):
            self._s_in = torch.cuda.Stream(device=self.device)
            self._s_out = torch.cuda.Stream(device=self.device)
            self._lane_state = [{"tables": [BatchTable(self.max_slots, self.device) for _ in range(2)],
                                 "graphs": [None, None], "ev": [None, None], "steps": 0,
                                 "stream": torch.cuda.Stream(device=self.device)} for _ in range(self.lanes)]
            self._table_dtype = None
        if self._table_dtype not in (None, next(iter(dtypes))):
            for ln in self._lane_state:
                ln["graphs"] = [None, None]  # captured for the other storage type
        self._table_dtype = next(iter(dtypes))
        pending = collections.deque(requests)
        t0 = time.perf_counter()
        if not realtime:
            for r in pending:
                r.arrival = 0.0
        done = []
        gc_was_enabled = gc.isenabled()
        gc.disable()
        try:
            self._loop_batched(pending, t0, done, poll_s)
        finally:
            if gc_was_enabled:
                gc.enable()
        return done

    def _lane_of(self, req) -> int:
        D, H, W, N = req.shape[:4]
        work = H * W * D * N
        return min(self.lanes - 1, int(work >= self.lane_split))

    def _admit_batched(self, req, t0):
        n = request_bytes(*req.shape[:4], req.k, req.coarse.dtype)
        off = self.arena.alloc(n)
        if off is None:
            return None
        M, images, loss, ws = self._carve(req, off)
        ev = torch.cuda.Event()
        with torch.cuda.stream(self._s_in):
            M.copy_(req.coarse, non_blocking=True)
            images.copy_(req.images, non_blocking=True)
            ev.record(self._s_in)
        req.t_admit = time.perf_counter() - t0
        mpi = make_mpi(M, req.near, req.far, req.ref)
        citem, keep = batch_c_item(BatchItem(mpi, images, req.src, req.k, ws, level=req.schedule[0],
                                             loss_out=loss[0:1]))
        return {"req": req, "off": off, "n": n, "M": M, "loss": loss, "citem": citem, "keep": keep,
                "loss_ptr": loss.data_ptr(), "it": 0, "ev_in": ev, "waited": False, "ready": False,
                "lane": self._lane_of(req)}

    def _step_batched(self, lane, group):
        ln = self._lane_state[lane]
        b = ln["steps"] & 1
        if ln["ev"][b] is not None:
            ln["ev"][b].synchronize()  # the step that used this table buffer is done
        comp = ln["stream"]
        for a in group:
            if not a["waited"]:
                comp.wait_event(a["ev_in"])
                a["waited"] = True
            c = a["citem"]
            c.params.level = a["req"].schedule[a["it"]]
            c.loss_out = a["loss_ptr"] + 4 * a["it"]
        table = ln["tables"][b]
        reallife_batch_prepare([a["citem"] for a in group], table)
        if self.graphs:
            g = ln["graphs"][b]
            if g is None:
                comp.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=comp):
                    reallife_hsgd_step_batch(table, stream=comp)
                ln["graphs"][b] = g
                self.captures += 1
            with torch.cuda.stream(comp):
                g.replay()
            self.replays += 1
        else:
            reallife_hsgd_step_batch(table, stream=comp)
        ev = torch.cuda.Event()
        ev.record(comp)
        ln["ev"][b] = ev
        ln["steps"] += 1
        self.steps += 1
        self.max_items_per_step = max(self.max_items_per_step, len(group))
        return ev

    def _loop_batched(self, pending, t0, done, poll_s):
        active = []     # requests with iterations left
        leaving = []    # requests whose result is on its way to the host
        while pending or active or leaving:
            now = time.perf_counter() - t0
            progressed = False
            for a in list(leaving):
                if a["ev_out"].query():
                    req = a["req"]
                    req.t_done = time.perf_counter() - t0
                    req.losses = a["host_loss"].numpy().copy()
                    if self.keep_results:
                        req.result = a["host_out"].clone()
                    self.arena.release(a["off"], a["n"])
                    self.slot_result[a["slot"]] = a["host_buf"]
                    leaving.remove(a)
                    done.append(req)
                    progressed = True
            used = {x["slot"] for x in active + leaving}
            free = [i for i in range(self.max_slots) if i not in used]
            while pending and pending[0].arrival <= now and free:
                a = self._admit_batched(pending[0], t0)
                if a is None:
                    break  # first come, first served: wait for memory
                pending.popleft()
                a["slot"] = free.pop()
                a["req"].slot = a["slot"]
                active.append(a)
                progressed = True
            for a in active:
                # a request joins the steps once its upload has landed, so that one large upload
                # never holds up the other requests of its lane
                if not a["ready"] and a["ev_in"].query():
                    a["ready"] = True
            for lane in range(self.lanes):
                group = [a for a in active if a["lane"] == lane and a["ready"]]
                ln = self._lane_state[lane]
                if not group or sum(1 for e in ln["ev"] if e is not None and not e.query()) >= 2:
                    continue
                ev = self._step_batched(lane, group)
                for a in group:
                    a["it"] += 1
                    if a["it"] == len(a["req"].schedule):
                        self._send_result(a, ev)
                        active.remove(a)
                        leaving.append(a)
                progressed = True
            if not progressed:
                if pending and not active and not leaving and pending[0].arrival > now:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 1e-3)))
                else:
                    time.sleep(poll_s)

    def _send_result(self, a, ev):
        req = a["req"]
        host_buf = self.slot_result[a["slot"]]
        need = req.coarse.numel()
        if host_buf is None or host_buf.numel() < need or host_buf.dtype != req.coarse.dtype:
            host_buf = torch.empty(need, dtype=req.coarse.dtype).pin_memory()
        a["host_buf"] = host_buf
        a["host_out"] = host_buf[:need].view(req.coarse.shape)
        a["host_loss"] = self.slot_loss[a["slot"]][:len(req.schedule)]
        with torch.cuda.stream(self._s_out):
            self._s_out.wait_event(ev)
            a["host_out"].copy_(a["M"], non_blocking=True)
            a["host_loss"].copy_(a["loss"], non_blocking=True)
            a["ev_out"] = torch.cuda.Event()
            a["ev_out"].record(self._s_out)


def latency_stats(done) -> dict:
    done = [r for r in done if r.error is None]
    lat = np.array([r.latency for r in done]) * 1e3
    queue = np.array([r.t_admit - r.arrival for r in done]) * 1e3
    t_first = min(r.arrival for r in done)
    t_last = max(r.t_done for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "queue_p50_ms": float(np.percentile(queue, 50)), "queue_p99_ms": float(np.percentile(queue, 99)),
            "reconstructions_per_s": len(done) / (t_last - t_first)}
