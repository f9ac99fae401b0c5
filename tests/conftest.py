import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _bounds_checked(request):
    """Under PFREG_DEBUG=1 (the bounds-checked library) every GPU test must
    end with no out-of-bounds gather index recorded by the kernels."""
    yield
    if os.environ.get("PFREG_DEBUG") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import paper_2504_19930_gb300 as pk
    on, hits, first = pk.pf_debug_bounds(clear=True)
    assert on, "PFREG_DEBUG=1 but the loaded library has no bounds checks"
    assert hits == 0, f"{hits} out-of-bounds gather indices (first: {first})"
