"""The OpenMP build of the oracle (used to time it on all host cores) gives bit-identical
results to the serial build: renders, the loss and its dense gradient, HSGD steps at every
level and a full refinement, on a scene with ragged sizes and planes behind a view."""
import numpy as np
import pytest

import oracle
import scenegen as sg


@pytest.fixture
def both():
    oracle.build()
    yield
    oracle.set_threads(False)


def _run(threads: bool, sc, k):
    oracle.set_threads(threads)
    out = {"threads": oracle.num_threads()}
    out["render"] = oracle.render(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src[0])
    out["loss_grad"] = oracle.loss_grad(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images)
    M = sc.coarse_mpi.astype(np.float64)
    for level in (1, 0):
        M, L, S = oracle.hsgd_step(M, sc.near, sc.far, sc.ref, sc.src, sc.images, k, level=level)
        out[f"step{level}"] = (M.copy(), L, S)
    out["refine"] = oracle.refine(sc.coarse_mpi, sc.near, sc.far, sc.ref, sc.src, sc.images, k, (2, 1, 0))
    return out


def _same(a, b):
    if isinstance(a, (tuple, list)):
        assert len(a) == len(b)
        for x, y in zip(a, b):
            _same(x, y)
    elif isinstance(a, np.ndarray):
        assert a.dtype == b.dtype and a.shape == b.shape
        assert np.array_equal(a, b)  # bit for bit (no NaN in these outputs)
    else:
        assert a == b


def test_openmp_build_is_bit_identical_to_serial(both, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    sc = sg.make_scene(5, 36, 44, 6, 3, n_layers=(2, 3), novel="none")
    serial = _run(False, sc, 3)
    par = _run(True, sc, 3)
    assert serial.pop("threads") == 1
    assert par.pop("threads") >= 1
    for key in serial:
        _same(serial[key], par[key])
