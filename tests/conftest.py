import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built engine")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session", autouse=True)
def _private_autotune_cache(tmp_path_factory):
    """Tunings made by tests (on small probes) go to a file of the session's own,
    never to the cache that real runs read."""
    old = os.environ.get("SDE_AUTOTUNE_CACHE")
    os.environ["SDE_AUTOTUNE_CACHE"] = str(tmp_path_factory.mktemp("autotune") / "autotune.json")
    yield
    if old is None:
        os.environ.pop("SDE_AUTOTUNE_CACHE", None)
    else:
        os.environ["SDE_AUTOTUNE_CACHE"] = old
