import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "trips_bounds: sets the bounds bit on purpose (debug-build self-test)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _debug_bounds_word(request):
    """Under the bounds-checked debug build (REALLIFE_DEBUG=1) no GPU test may trip a check:
    after each one the bounds bit (4) of the device status word must be clear."""
    yield
    if os.environ.get("REALLIFE_DEBUG", "0") in ("", "0") or "gpu" not in request.keywords:
        return
    if request.node.get_closest_marker("trips_bounds"):
        return
    import ctypes

    from paper_2307_03017_gb300 import _lib
    flags = ctypes.c_uint()
    _lib.lib().reallife_device_status(0, ctypes.byref(flags))
    if flags.value & 4:
        _lib.lib().reallife_device_status(1, ctypes.byref(flags))
        pytest.fail("a bounds check of the debug build failed during this test")
