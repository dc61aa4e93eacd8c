import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# The property tests of the configuration rules need hypothesis, which not
# every machine that runs this suite has; there they are left out of the
# collection (they are CPU tests: the GPU selection has nothing to skip).
try:
    import hypothesis  # noqa: F401
except ImportError:
    collect_ignore = ["test_config_rules.py"]


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built librlb.so")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    oracle.set_threads(min(16, os.cpu_count() or 1))
    return oracle
