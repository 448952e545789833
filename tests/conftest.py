import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


@pytest.fixture(scope="session")
def fgml():
    """The CUDA library binding; built in-tree on first use."""
    from paper_2006_14970_gb300 import build as fbuild
    fbuild.build()
    from paper_2006_14970_gb300 import fgml as lib
    return lib
