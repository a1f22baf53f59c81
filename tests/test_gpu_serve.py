"""Serving: continuous batching of heterogeneous reconstruction requests on one GPU.

Each request's result is the same alone and in the mix (BF16 tolerance 2e-2); admission
by device memory bounds the concurrent requests; graph replay gives the direct results.
"""
import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu
TOL16 = 2e-2


@pytest.fixture(scope="module")
def pool():
    out = {}
    for i, (H, W, D, N) in enumerate([(96, 128, 8, 3), (192, 256, 16, 2), (96, 128, 16, 4), (192, 256, 8, 3)]):
        sc = sg.make_scene(40 + i, H, W, D, N, n_layers=(2, 4), novel="none")
        out[i] = (sc, torch.from_numpy(sc.coarse_mpi).to(torch.bfloat16).pin_memory(),
                  torch.from_numpy(sc.images).pin_memory())
    return out


def _requests(pool, n, seed=0, only=None):
    from paper_2307_03017_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n):
        sc, M, I = pool[int(rng.integers(0, len(pool))) if only is None else only]
        sched = (2, 1, 0) if rng.integers(0, 2) else (2, 0)
        reqs.append(Request(id=r, arrival=0.0, coarse=M, images=I, ref=sc.ref, src=sc.src, near=sc.near, far=sc.far,
                            schedule=sched, k=5))
    return reqs


def test_result_alone_equals_result_in_the_mix(pool):
    from paper_2307_03017_gb300.serve import ServeEngine
    reqs = _requests(pool, 12)
    alone = {}
    eng1 = ServeEngine(1 << 30, max_slots=1, keep_results=True)
    for r in _requests(pool, 12):
        (d,) = eng1.run([r], realtime=False)
        alone[d.id] = (d.result.float().numpy(), d.losses)
    eng = ServeEngine(1 << 30, max_slots=8, keep_results=True)
    mix = eng.run(reqs, realtime=False)
    assert len(mix) == 12
    # the mix really overlapped: some request was admitted before another one finished
    spans = sorted((r.t_admit, r.t_done) for r in mix)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    for r in mix:
        ref, ref_losses = alone[r.id]
        assert np.abs(r.result.float().numpy() - ref).max() <= TOL16
        np.testing.assert_allclose(r.losses, ref_losses, rtol=1e-3)


def test_admission_is_bounded_by_device_memory(pool):
    from paper_2307_03017_gb300.serve import ServeEngine, request_bytes
    reqs = _requests(pool, 10, seed=1, only=1)  # one shape: the arena holds exactly two
    need = request_bytes(*reqs[0].shape[:4], reqs[0].k, reqs[0].coarse.dtype)
    eng = ServeEngine(2 * need + 4096, max_slots=8)
    done = eng.run(reqs, realtime=False)
    assert len(done) == 10
    events = sorted([(r.t_admit, 1) for r in done] + [(r.t_done, -1) for r in done])
    live = peak = 0
    for _, e in events:
        live += e
        peak = max(peak, live)
    assert peak <= 2  # never more than the two that fit
    assert max(r.t_admit for r in done) > min(r.t_done for r in done)  # later ones waited for memory
    assert eng.arena.bytes_free() == eng.arena.size


def test_graph_replay_matches_direct_launches(pool):
    from paper_2307_03017_gb300.serve import ServeEngine
    reqs_a = _requests(pool, 10, seed=2)
    reqs_b = _requests(pool, 10, seed=2)
    direct = {r.id: r for r in ServeEngine(1 << 30, max_slots=4, keep_results=True).run(reqs_a, realtime=False)}
    eng = ServeEngine(1 << 30, max_slots=4, graphs=True, keep_results=True)
    graphed = eng.run(reqs_b, realtime=False)
    assert eng.captures >= 1 and eng.replays == 10
    for r in graphed:
        assert np.abs(r.result.float().numpy() - direct[r.id].result.float().numpy()).max() <= TOL16


def test_realtime_poisson_stream_reports_latency(pool):
    from paper_2307_03017_gb300.serve import ServeEngine, latency_stats
    reqs = _requests(pool, 40, seed=3)
    rng = np.random.default_rng(4)
    t = 0.0
    for r in reqs:
        t += rng.exponential(1 / 400.0)
        r.arrival = t
    done = ServeEngine(1 << 30, max_slots=8).run(reqs, realtime=True)
    st = latency_stats(done)
    assert st["requests"] == 40 and 0 < st["p50_ms"] <= st["p99_ms"]
    assert all(r.t_done >= r.arrival for r in done)


@pytest.mark.parametrize("graphs", [False, True])
def test_batched_steps_result_alone_equals_result_in_the_mix(pool, graphs):
    """Iteration-level batching: one batched launch per stage serves the next iteration of every
    active request; each result equals the request served alone."""
    from paper_2307_03017_gb300.serve import ServeEngine
    alone = {}
    eng1 = ServeEngine(1 << 30, max_slots=1, keep_results=True)
    for r in _requests(pool, 12, seed=5):
        (d,) = eng1.run([r], realtime=False)
        alone[d.id] = (d.result.float().numpy(), d.losses)
    eng = ServeEngine(1 << 30, max_slots=8, keep_results=True, batched=True, graphs=graphs)
    mix = eng.run(_requests(pool, 12, seed=5), realtime=False)
    assert len(mix) == 12 and all(r.error is None for r in mix)
    iters = sum(len(r.schedule) for r in mix)
    assert eng.max_items_per_step >= 2 and eng.steps < iters  # launches served several requests
    if graphs:
        assert eng.captures <= 2 * eng.lanes and eng.replays == eng.steps
    for r in mix:
        ref, ref_losses = alone[r.id]
        assert np.abs(r.result.float().numpy() - ref).max() <= TOL16
        np.testing.assert_allclose(r.losses, ref_losses, rtol=1e-3)
    assert eng.arena.bytes_free() == eng.arena.size


def test_batched_realtime_stream_and_oversized_request(pool):
    """A Poisson stream through the batched engine; a request larger than the whole arena is
    returned failed while the others are served."""
    from paper_2307_03017_gb300.serve import ServeEngine, latency_stats, request_bytes
    reqs = _requests(pool, 30, seed=6)
    rng = np.random.default_rng(7)
    t = 0.0
    for r in reqs:
        t += rng.exponential(1 / 400.0)
        r.arrival = t
    big = max(request_bytes(*r.shape[:4], r.k, r.coarse.dtype) for r in reqs)
    small = [r for r in reqs if request_bytes(*r.shape[:4], r.k, r.coarse.dtype) < big]
    eng = ServeEngine(big - 256, max_slots=8, batched=True)
    done = eng.run(reqs, realtime=True)
    assert len(done) == 30
    failed = [r for r in done if r.error is not None]
    assert failed and all(request_bytes(*r.shape[:4], r.k, r.coarse.dtype) == big for r in failed)
    assert len(failed) + len(small) == 30
    st = latency_stats(done)
    assert st["requests"] == len(small) and 0 < st["p50_ms"] <= st["p99_ms"]
    assert all(r.t_done >= r.arrival for r in done)
    # the same for the per-stream engine
    done2 = ServeEngine(big - 256, max_slots=8).run(_requests(pool, 30, seed=6), realtime=False)
    assert sum(r.error is not None for r in done2) == len(failed)
