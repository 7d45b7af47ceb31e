import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O


@pytest.fixture(autouse=True)
def _collect_after_gpu_test(request):
    """Finalise the solver handles a GPU test leaves behind on the main thread,
    between tests, rather than inside a later test's worker threads."""
    yield
    if request.node.get_closest_marker("gpu") is not None:
        import gc
        gc.collect()
