import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def repo_root():
    return ROOT


def build_library():
    """Build libsip.so (if stale) and import the package."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2504_03573_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_sip_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2504_03573_gb300
    return paper_2504_03573_gb300
