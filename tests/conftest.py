import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def repo_root():
    return ROOT


@pytest.fixture(autouse=True)
def _device_checks(request):
    """Under the checked build (DETLSH_CHECKED=1) a GPU test fails if any device
    index check failed while it ran."""
    yield
    if os.environ.get("DETLSH_CHECKED") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import paper_2406_10938_gb300 as pkg
    st = pkg.detlsh_check_status()
    assert st is not None, "DETLSH_CHECKED=1 but the loaded library is not the checked build"
    assert st[0] == 0, f"{st[0]} device index checks failed (first: site {st[1]}, index {st[2]})"
