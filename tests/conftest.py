import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libgsp")
    config.addinivalue_line("markers", "slow: full-size parity cases (minutes of oracle time)")


def build_gsp() -> str:
    """Build libgsp.so (load the build script by path: the package needs the library)."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2603_08661_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_gsp_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


@pytest.fixture(scope="session")
def gsp_lib():
    """The CUDA library binding; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_gsp()
    import paper_2603_08661_gb300 as gsp
    return gsp
