import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def emulated_library(tmp_path_factory):
    """The test-only emulated library (tests/emulated_library.py), built once."""
    import emulated_library as el

    if not el.available():
        pytest.skip("g++ or the CUDA headers are missing")
    return el.build(str(tmp_path_factory.mktemp("library_emulation")))
